// k_bruteforce.cu -- exact top-k by (Gamma, id) over all objects (Def. 2 with the
// fusion distance of Eq. 6), and with exclude_self the exact candidate sets C(u)
// of Sec. 4.1 (every object is a query, itself excluded).
//
// Layout: a CTA owns a tile of 32 queries and scans one slice of the objects in
// tiles of 128.  Each tile's squared distances are register-tiled (2 queries x 8
// objects per thread) from shared-memory staged 32-wide dimension chunks; the
// epilogue turns them into Gamma with the packed-attribute chi and a warp per 4
// queries filters them against the query's current k-th record and inserts the
// survivors into a sorted per-query list in shared memory.  With several slices
// (small query batches) the per-slice lists go to scratch and a warp-per-query
// k-way merge writes the final rows.
#include <cmath>
#include <cstdio>
#include <mutex>

#include "nhq_internal.cuh"

namespace nhq {

namespace {

constexpr int TQ = 32;   // queries per CTA
constexpr int TN = 128;  // objects per tile
constexpr int DC = 32;   // dimensions per staged chunk
constexpr int DS = DC + 4;  // staged row stride: 16-byte aligned rows, read as float4
constexpr int NT = 256;  // threads per CTA
constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ bool rec_less(float ga, uint32_t ia, float gb, uint32_t ib) {
    return ga < gb || (ga == gb && ia < ib);
}

__global__ void __launch_bounds__(NT) topk_tile_kernel(TopkArgs a, int64_t per_split,
                                                       uint32_t *__restrict__ part_id,
                                                       float *__restrict__ part_g) {
    extern __shared__ __align__(16) unsigned char smem[];
    float(*Qs)[DS] = reinterpret_cast<float(*)[DS]>(smem);
    float(*Xs)[DS] = reinterpret_cast<float(*)[DS]>(smem + sizeof(float) * TQ * DS);
    float *G = reinterpret_cast<float *>(smem + sizeof(float) * (TQ + TN) * DS);
    float *Lg = G + TQ * TN;
    uint32_t *Li = reinterpret_cast<uint32_t *>(Lg + TQ * a.k);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ty = tid >> 4, tx = tid & 15;
    const int64_t q0 = (int64_t)blockIdx.x * TQ;
    const int split = blockIdx.y, S = gridDim.y;
    const int64_t n_begin = (int64_t)split * per_split;
    const int64_t n_end = min(a.N, n_begin + per_split);
    const int k = a.k;

    int cnt[4] = {0, 0, 0, 0};  // list lengths of this warp's 4 queries

    for (int64_t n0 = n_begin; n0 < n_end; n0 += TN) {
        float acc[2][8];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j)
                acc[i][j] = 0.f;

        for (int dk = 0; dk < a.d; dk += DC) {
            for (int idx = tid; idx < TQ * DC; idx += NT) {
                int r = idx / DC, c = idx % DC;
                int64_t q = q0 + r;
                int col = dk + c;
                Qs[r][c] = (q < a.nq && col < a.d) ? a.Q[q * a.qstride + col] : 0.f;
            }
            for (int idx = tid; idx < TN * (DC / 4); idx += NT) {
                int r = idx / (DC / 4), c4 = idx % (DC / 4);
                int64_t o = n0 + r;
                int col = dk + 4 * c4;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (o < n_end && col < a.xstride)
                    v = *reinterpret_cast<const float4 *>(a.X + o * a.xstride + col);
                *reinterpret_cast<float4 *>(&Xs[r][4 * c4]) = v;
            }
            __syncthreads();
            // four dimensions per shared-memory load; each pair still sums its squared
            // differences one dimension at a time, in dimension order
#pragma unroll 1
            for (int c = 0; c < DC; c += 4) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&Qs[ty][c]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&Qs[ty + 16][c]);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float4 b = *reinterpret_cast<const float4 *>(&Xs[tx + 16 * j][c]);
                    float t0 = a0.x - b.x, t1 = a1.x - b.x;
                    acc[0][j] = fmaf(t0, t0, acc[0][j]);
                    acc[1][j] = fmaf(t1, t1, acc[1][j]);
                    t0 = a0.y - b.y;
                    t1 = a1.y - b.y;
                    acc[0][j] = fmaf(t0, t0, acc[0][j]);
                    acc[1][j] = fmaf(t1, t1, acc[1][j]);
                    t0 = a0.z - b.z;
                    t1 = a1.z - b.z;
                    acc[0][j] = fmaf(t0, t0, acc[0][j]);
                    acc[1][j] = fmaf(t1, t1, acc[1][j]);
                    t0 = a0.w - b.w;
                    t1 = a1.w - b.w;
                    acc[0][j] = fmaf(t0, t0, acc[0][j]);
                    acc[1][j] = fmaf(t1, t1, acc[1][j]);
                }
            }
            __syncthreads();
        }

        // epilogue: Gamma for each (query, object) of the tile
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            int r = ty + 16 * i;
            int64_t q = q0 + r;
            uint32_t qa = q < a.nq ? a.qattr[q] : 0u;
            const uint32_t qh = a.qhi && q < a.nq ? a.qhi[q] : a.w.hi;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                int c = tx + 16 * j;
                int64_t o = n0 + c;
                float g = __int_as_float(0x7f800000);
                if (q < a.nq && o < n_end && !(a.exclude_self && o == q)) {
                    float delta = __fsqrt_rn(acc[i][j]);
                    g = fusion_gamma(delta, chi_packed(qa, a.attr[o], qh, a.w.lo), a.w);
                }
                G[r * TN + c] = g;
            }
        }
        __syncthreads();

        // selection: warp w keeps the lists of queries 4w..4w+3
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int r = warp * 4 + i;
            if (q0 + r >= a.nq)
                continue;
            float *lg = Lg + r * k;
            uint32_t *li = Li + r * k;
#pragma unroll
            for (int jj = 0; jj < TN / 32; ++jj) {
                int c = lane + 32 * jj;
                float g = G[r * TN + c];
                uint32_t id = (uint32_t)(n0 + c);
                float tg = cnt[i] == k ? lg[k - 1] : __int_as_float(0x7f800000);
                uint32_t ti = cnt[i] == k ? li[k - 1] : kNone;
                bool surv = g < __int_as_float(0x7f800000) && rec_less(g, id, tg, ti);
                unsigned mask = __ballot_sync(FULL, surv);
                while (mask) {
                    int src = __ffs(mask) - 1;
                    mask &= mask - 1;
                    float cg = __shfl_sync(FULL, g, src);
                    uint32_t cid = (uint32_t)(n0 + 32 * jj + src);
                    if (cnt[i] == k && !rec_less(cg, cid, lg[k - 1], li[k - 1]))
                        continue;  // the threshold tightened meanwhile
                    int below = 0;
                    for (int e = lane; e < cnt[i]; e += 32)
                        below += rec_less(lg[e], li[e], cg, cid) ? 1 : 0;
                    int pos = __reduce_add_sync(FULL, below);
                    int hi = min(cnt[i], k - 1);  // entries [pos, hi) move up by one
                    for (int base = (hi - 1) & ~31; base >= (pos & ~31); base -= 32) {
                        int e = base + lane;
                        bool mv = e >= pos && e < hi;
                        float vg = 0.f;
                        uint32_t vi = 0;
                        if (mv) {
                            vg = lg[e];
                            vi = li[e];
                        }
                        __syncwarp();
                        if (mv) {
                            lg[e + 1] = vg;
                            li[e + 1] = vi;
                        }
                        __syncwarp();
                    }
                    if (lane == 0) {
                        lg[pos] = cg;
                        li[pos] = cid;
                    }
                    cnt[i] = min(cnt[i] + 1, k);
                    __syncwarp();
                }
            }
        }
        __syncthreads();
    }

    // write this slice's lists
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int r = warp * 4 + i;
        int64_t q = q0 + r;
        if (q >= a.nq)
            continue;
        const float *lg = Lg + r * k;
        const uint32_t *li = Li + r * k;
        for (int e = lane; e < k; e += 32) {
            float g = e < cnt[i] ? lg[e] : __int_as_float(0x7f800000);
            uint32_t id = e < cnt[i] ? li[e] : kNone;
            if (S == 1) {
                a.ids[q * k + e] = id;
                if (a.dists)
                    a.dists[q * k + e] = g;
                if (a.chi)
                    a.chi[q * k + e] =
                        id == kNone ? (uint8_t)255
                                    : (uint8_t)chi_packed(a.qattr[q], a.attr[id],
                                                          a.qhi ? a.qhi[q] : a.w.hi, a.w.lo);
            } else {
                int64_t o = (q * S + split) * (int64_t)k + e;
                part_id[o] = id;
                part_g[o] = g;
            }
        }
    }
}

// k-way merge of the S sorted slice lists of each query (one warp per query).
__global__ void topk_merge_kernel(TopkArgs a, int S, const uint32_t *__restrict__ part_id,
                                  const float *__restrict__ part_g) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= a.nq)
        return;
    const int k = a.k;
    int head = 0;
    auto load = [&](int h) -> unsigned long long {
        if (lane >= S || h >= k)
            return ~0ull;
        int64_t o = (q * S + lane) * (int64_t)k + h;
        return ((unsigned long long)__float_as_uint(part_g[o]) << 32) | part_id[o];
    };
    unsigned long long cur = load(0);
    for (int e = 0; e < k; ++e) {
        unsigned long long best = cur;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            unsigned long long o = __shfl_xor_sync(FULL, best, off);
            best = o < best ? o : best;
        }
        uint32_t id = (uint32_t)best;
        float g = __uint_as_float((uint32_t)(best >> 32));
        if (lane == 0) {
            a.ids[q * k + e] = id;
            if (a.dists)
                a.dists[q * k + e] = g;
            if (a.chi)
                a.chi[q * k + e] = id == kNone
                                       ? (uint8_t)255
                                       : (uint8_t)chi_packed(a.qattr[q], a.attr[id],
                                                             a.qhi ? a.qhi[q] : a.w.hi, a.w.lo);
        }
        if (cur == best && best != ~0ull) {
            ++head;
            cur = load(head);
        }
    }
}

int choose_splits(const TopkArgs &a, int sm_count) {
    int64_t tiles = (a.nq + TQ - 1) / TQ;
    int64_t want = (2 * (int64_t)sm_count + tiles - 1) / tiles;
    int64_t max_by_n = (a.N + 8 * TN - 1) / (8 * TN);  // at least ~8 tiles per slice
    int64_t s = want < max_by_n ? want : max_by_n;
    if (s > 32)
        s = 32;
    if (s < 1)
        s = 1;
    return (int)s;
}

size_t tile_smem(int k) {
    return sizeof(float) * (TQ + TN) * DS + sizeof(float) * TQ * TN +
           (sizeof(float) + sizeof(uint32_t)) * (size_t)TQ * k;
}

}  // namespace

size_t topk_scratch_bytes(const TopkArgs &a, int sm_count) {
    int S = choose_splits(a, sm_count);
    if (S == 1)
        return 0;
    return (size_t)a.nq * S * a.k * (sizeof(uint32_t) + sizeof(float));
}

cudaError_t launch_topk(const TopkArgs &a, void *scratch, size_t scratch_bytes, int sm_count,
                        cudaStream_t s) {
    if (a.nq <= 0)
        return cudaSuccess;
    int S = choose_splits(a, sm_count);
    int64_t per = (a.N + S - 1) / S;
    per = (per + TN - 1) / TN * TN;
    uint32_t *pid = nullptr;
    float *pg = nullptr;
    if (S > 1) {
        size_t need = (size_t)a.nq * S * a.k * (sizeof(uint32_t) + sizeof(float));
        if (scratch == nullptr || scratch_bytes < need)
            return cudaErrorInvalidValue;
        pid = reinterpret_cast<uint32_t *>(scratch);
        pg = reinterpret_cast<float *>(pid + (size_t)a.nq * S * a.k);
    }
    size_t smem = tile_smem(a.k);
    cudaError_t e = cudaFuncSetAttribute(topk_tile_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    dim3 grid((unsigned)((a.nq + TQ - 1) / TQ), (unsigned)S);
    topk_tile_kernel<<<grid, NT, smem, s>>>(a, per, pid, pg);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    if (S > 1) {
        int wpb = 8;
        topk_merge_kernel<<<(unsigned)((a.nq + wpb - 1) / wpb), 32 * wpb, 0, s>>>(a, S, pid, pg);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace nhq

// ---------------------------------------------------------------------------
// Allocation-free variant of the brute-force top-k (nhq_brute_force_noalloc).
//
// Some callers cannot allocate device memory when they call the library: code
// that runs under a memory budget owned by another allocator (a framework's
// caching pool, an embedded or real-time service that reserves all memory at
// start-up), or code that must not touch the allocator on its hot path.  For
// them the split path's only scratch -- the per-slice sorted lists that
// topk_tile_kernel writes and topk_merge_kernel reads -- lives in the
// file-scope array below.  It is kNoAllocScratchBytes (16 MiB) of device memory
// on every GPU where this module is loaded, and stays there until the process
// exits.  Under CUDA's lazy module loading that happens on a device's first use
// of this file's code, possibly the first nhq_brute_force_noalloc call itself
// (its cudaGetSymbolAddress), so callers make a first call (Q = 0 suffices) at
// start-up, before their own allocator reserves the device's memory and before
// any stream capture.  Every call
// on a device shares it: each call fully rewrites the entries it later reads,
// so nothing has to start at zero, but calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on it.
// ---------------------------------------------------------------------------
namespace nhq {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

struct NoAllocDevice {
    bool ready = false;
    void *scratch = nullptr;  // device address of g_noalloc_scratch on this device
    int sm_count = 0;
};
constexpr int kNoAllocMaxDevices = 64;
NoAllocDevice g_noalloc_devices[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

bool is_device_pointer(const void *p) {
    cudaPointerAttributes at;
    if (p == nullptr || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Per-device set-up, done by the first call on the current device.  In host code
// g_noalloc_scratch names a host-side shadow, not device memory, so the device
// address is looked up with cudaGetSymbolAddress while this device is current.
nhq_status noalloc_setup(NoAllocDevice **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return report_error(NHQ_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return report_error(NHQ_ERR_ARG, "nhq_brute_force_noalloc: device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocDevice &d = g_noalloc_devices[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        if ((e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch)) != cudaSuccess)
            return report_error(NHQ_ERR_CUDA, cudaGetErrorString(e));
        int sms = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) !=
            cudaSuccess)
            return report_error(NHQ_ERR_CUDA, cudaGetErrorString(e));
        d.scratch = ptr;
        d.sm_count = sms;
        d.ready = true;
    }
    *out = &d;
    return NHQ_OK;
}

}  // namespace

}  // namespace nhq

extern "C" nhq_status nhq_brute_force_noalloc(const float *vectors,
                                              const uint32_t *packed_attributes, int64_t N,
                                              int32_t d, int32_t m, const float *queries,
                                              const uint32_t *packed_query_attributes,
                                              int64_t Q, int32_t k, nhq_weights w, uint32_t *ids,
                                              float *dists, uint8_t *chi, void *stream) {
    using namespace nhq;
    if (N < 1 || N > 0x7FFFFFFE || d < 1 || m < 1 || m > 4 || Q < 0 || k < 1 || k > kMaxK)
        return report_error(NHQ_ERR_ARG, "nhq_brute_force_noalloc: need N >= 1, d >= 1, m in "
                                         "1..4, Q >= 0, k in 1..256");
    if (d % 4 != 0)
        return report_error(NHQ_ERR_ARG, "nhq_brute_force_noalloc: d must be a multiple of 4");
    nhq_status st = validate_weights(w, true);  // the rules of nhq_brute_force
    if (st != NHQ_OK)
        return st;
    // the per-device set-up runs first, so that a call with Q = 0 can make it at start-up
    NoAllocDevice *dv = nullptr;
    if ((st = noalloc_setup(&dv)) != NHQ_OK)
        return st;
    if (Q == 0)
        return NHQ_OK;
    if (!is_device_pointer(vectors) || !is_device_pointer(packed_attributes) ||
        !is_device_pointer(queries) || !is_device_pointer(packed_query_attributes) ||
        !is_device_pointer(ids) || (dists && !is_device_pointer(dists)) ||
        (chi && !is_device_pointer(chi)))
        return report_error(NHQ_ERR_ARG, "nhq_brute_force_noalloc: every array must be device "
                                         "memory (NULL allowed for dists and chi)");
    if ((reinterpret_cast<uintptr_t>(vectors) & 15) != 0)
        return report_error(NHQ_ERR_ARG, "nhq_brute_force_noalloc: vectors must be 16-byte "
                                         "aligned");
    TopkArgs a;
    a.X = vectors;
    a.xstride = d;
    a.d = d;
    a.N = N;
    a.attr = packed_attributes;
    a.Q = queries;
    a.qstride = d;
    a.qattr = packed_query_attributes;
    a.qhi = nullptr;
    a.nq = Q;
    a.k = k;
    a.exclude_self = 0;
    a.w = make_fusion(w, m);
    a.ids = ids;
    a.dists = dists;
    a.chi = chi;
    const size_t need = topk_scratch_bytes(a, dv->sm_count);
    if (need > kNoAllocScratchBytes) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "nhq_brute_force_noalloc: Q = %lld, k = %d needs %zu scratch bytes, above the "
                 "fixed %zu (use nhq_brute_force, or fewer queries per call)",
                 (long long)Q, k, need, kNoAllocScratchBytes);
        return report_error(NHQ_ERR_ARG, msg);
    }
    cudaError_t e = launch_topk(a, dv->scratch, kNoAllocScratchBytes, dv->sm_count,
                                reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return report_error(NHQ_ERR_CUDA, cudaGetErrorString(e));
    return NHQ_OK;
}
