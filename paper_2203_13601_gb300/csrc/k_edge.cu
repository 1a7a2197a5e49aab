// k_edge.cu -- landing-zone edge selection (Sec. 4.1, Def. 6) for every vertex,
// and the reverse-candidate lists of the optional second selection pass.
//
// Edge selection: one CTA (4 warps) per vertex u.  The candidate rows (and u's)
// are staged in shared memory when they fit, so every later distance reads
// on-chip memory.  Gamma(p, u) of all candidates is computed by 16 teams of 8
// lanes, the records (Gamma, p) are bitonic-sorted, and the selection walks
// them in order: candidate p joins N(u) iff for every accepted j
//     Gamma(p, u) < Gamma(p, j)   and   Gamma(p, u) > Gamma(u, j),
// the 16 teams testing 16 accepted neighbours per pass (a CTA-wide vote).
#include <cub/cub.cuh>

#include "nhq_internal.cuh"

namespace nhq {

namespace {

constexpr int ES_THREADS = 128;
constexpr int TEAM = 8;
constexpr int TEAMS = ES_THREADS / TEAM;
constexpr unsigned FULL = 0xFFFFFFFFu;

struct EdgeArgs {
    const float *X;
    int xstride, d;
    int64_t N;
    const uint32_t *attr;
    Fusion w;
    const uint32_t *cand;
    int L, R;
    uint32_t *out;
    int staged;  // candidate rows live in shared memory
    int rstride; // floats per staged row
};

// squared distance between two rows, one team of 8 lanes; result in every team lane
__device__ __forceinline__ float team_dist2(const float *__restrict__ a,
                                            const float *__restrict__ b, int xs4, int tl) {
    float acc = 0.f;
    for (int c = tl; c < xs4; c += TEAM) {
        float4 x = reinterpret_cast<const float4 *>(a)[c];
        float4 y = reinterpret_cast<const float4 *>(b)[c];
        float t;
        t = x.x - y.x; acc = fmaf(t, t, acc);
        t = x.y - y.y; acc = fmaf(t, t, acc);
        t = x.z - y.z; acc = fmaf(t, t, acc);
        t = x.w - y.w; acc = fmaf(t, t, acc);
    }
    acc += __shfl_xor_sync(FULL, acc, 1);
    acc += __shfl_xor_sync(FULL, acc, 2);
    acc += __shfl_xor_sync(FULL, acc, 4);
    return acc;
}

__global__ void __launch_bounds__(ES_THREADS) edge_select_kernel(EdgeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem);  // [kMaxCand]
    uint32_t *cid = reinterpret_cast<uint32_t *>(keys + kMaxCand);           // [kMaxCand]
    uint32_t *acc_id = cid + kMaxCand;                                       // [kMaxDegree]
    int *acc_slot = reinterpret_cast<int *>(acc_id + kMaxDegree);            // [kMaxDegree]
    float *acc_g = reinterpret_cast<float *>(acc_slot + kMaxDegree);         // [kMaxDegree]
    int *misc = reinterpret_cast<int *>(acc_g + kMaxDegree);                 // [4]
    float *rows = reinterpret_cast<float *>(misc + 4);                       // [(L+1)][rstride]

    const int tid = threadIdx.x, team = tid / TEAM, tl = tid % TEAM;
    const int xs4 = a.xstride / 4;
    const int64_t u = blockIdx.x;
    const uint32_t au = a.attr[u];

    // 1. candidate ids (invalid, self and out-of-range dropped; repeats later)
    if (tid == 0)
        misc[0] = 0;
    __syncthreads();
    for (int s = tid; s < a.L; s += ES_THREADS) {
        uint32_t p = a.cand[u * a.L + s];
        bool ok = p != kNone && (int64_t)p < a.N && (int64_t)p != u;
        if (ok) {
            int slot = atomicAdd(&misc[0], 1);
            cid[slot] = p;
        }
    }
    __syncthreads();
    const int n = misc[0];  // staging slots are in arrival order; results do not depend on it

    const float *urow = a.X + u * a.xstride;
    if (a.staged) {
        float *dst = rows + (size_t)a.L * a.rstride;
        for (int c = tid; c < xs4; c += ES_THREADS)
            reinterpret_cast<float4 *>(dst)[c] = reinterpret_cast<const float4 *>(urow)[c];
        urow = dst;
        for (int idx = tid; idx < n * xs4; idx += ES_THREADS) {
            int i = idx / xs4, c = idx % xs4;
            reinterpret_cast<float4 *>(rows + (size_t)i * a.rstride)[c] =
                reinterpret_cast<const float4 *>(a.X + (int64_t)cid[i] * a.xstride)[c];
        }
        __syncthreads();
    }
    auto row_of_slot = [&](int i) -> const float * {
        return a.staged ? rows + (size_t)i * a.rstride : a.X + (int64_t)cid[i] * a.xstride;
    };

    // 2. Gamma(p, u) for every candidate; key = (Gamma, p) with the staging slot kept aside
    for (int base = 0; base < n; base += TEAMS) {
        int i = base + team;
        int ii = i < n ? i : 0;
        float dd = team_dist2(row_of_slot(ii), urow, xs4, tl);
        if (i < n && tl == 0) {
            uint32_t p = cid[i];
            float g = fusion_gamma(__fsqrt_rn(dd), chi_packed(a.attr[p], au, a.w.mask), a.w);
            // high 32 bits Gamma, then id (32 bits) -> order by (Gamma, id); the slot is
            // recovered after sorting by searching cid (ids are unique after dedup below)
            keys[i] = ((unsigned long long)__float_as_uint(g) << 32) | p;
        }
    }
    __syncthreads();
    for (int i = n + tid; i < kMaxCand; i += ES_THREADS)
        keys[i] = ~0ull;
    __syncthreads();

    // 3. bitonic sort of kMaxCand keys ascending
    for (int size = 2; size <= kMaxCand; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = tid; i < kMaxCand / 2; i += ES_THREADS) {
                int lo = 2 * stride * (i / stride) + (i % stride);
                int hi = lo + stride;
                bool up = ((lo & size) == 0);
                unsigned long long x = keys[lo], y = keys[hi];
                if ((x > y) == up) {
                    keys[lo] = y;
                    keys[hi] = x;
                }
            }
            __syncthreads();
        }
    }

    // 4. sequential landing-zone selection
    int deg = 0;
    const int R = a.R;
    for (int t = 0; t < n && deg < R; ++t) {
        unsigned long long kt = keys[t];
        if (t > 0 && kt == keys[t - 1])
            continue;  // repeated candidate
        uint32_t p = (uint32_t)kt;
        float gpu_ = __uint_as_float((uint32_t)(kt >> 32));
        // staging slot of p
        if (tid == 0)
            misc[1] = -1;
        __syncthreads();
        for (int i = tid; i < n; i += ES_THREADS)
            if (cid[i] == p)
                atomicMax(&misc[1], i);
        __syncthreads();
        int ps = misc[1];
        bool ok = true;
        if (deg > 0) {
            const float *prow = row_of_slot(ps);
            uint32_t ap = a.attr[p];
            int fail = 0;
            for (int base = 0; base < deg && !fail; base += TEAMS) {
                int j = base + team;
                int jj = j < deg ? j : 0;
                float dd = team_dist2(prow, row_of_slot(acc_slot[jj]), xs4, tl);
                bool bad = false;
                if (j < deg) {
                    float gpj = fusion_gamma(__fsqrt_rn(dd),
                                             chi_packed(ap, a.attr[acc_id[j]], a.w.mask), a.w);
                    bad = !(gpu_ < gpj && gpu_ > acc_g[j]);
                }
                fail = __syncthreads_or(bad ? 1 : 0);
            }
            ok = !fail;
        }
        if (ok) {
            if (tid == 0) {
                acc_id[deg] = p;
                acc_slot[deg] = ps;
                acc_g[deg] = gpu_;
            }
            ++deg;
            __syncthreads();
        }
    }
    for (int s = tid; s < R; s += ES_THREADS)
        a.out[u * R + s] = s < deg ? acc_id[s] : kNone;
}

// ---------------------------------------------------------------- reverse pass
__global__ void indeg_kernel(const uint32_t *__restrict__ nbr, int64_t total, int64_t N,
                             uint32_t *__restrict__ indeg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = nbr[i];
        if (v != kNone && (int64_t)v < N)
            atomicAdd(&indeg[v], 1u);
    }
}

__global__ void fill_sources_kernel(const uint32_t *__restrict__ nbr, int64_t N, int R,
                                    const uint32_t *__restrict__ off, uint32_t *__restrict__ cur,
                                    uint32_t *__restrict__ src) {
    int64_t total = N * (int64_t)R;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = nbr[i];
        if (v != kNone && (int64_t)v < N) {
            uint32_t pos = off[v] + atomicAdd(&cur[v], 1u);
            src[pos] = (uint32_t)(i / R);
        }
    }
}

// One warp per v: out[v] = N(v) (valid slots, in order) then the `cap` smallest
// sources u not already in N(v), ascending; kNone padding.
__global__ void reverse_rows_kernel(const uint32_t *__restrict__ nbr, int64_t N, int R, int cap,
                                    const uint32_t *__restrict__ off,
                                    const uint32_t *__restrict__ indeg,
                                    const uint32_t *__restrict__ src, uint32_t *__restrict__ out) {
    extern __shared__ uint32_t sh[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (v >= N)
        return;
    uint32_t *best = sh + wib * (kMaxDegree + kMaxDegree);  // sorted smallest sources
    uint32_t *fw = best + kMaxDegree;                        // forward list
    const int W = R + cap;
    // forward neighbours (valid slots, slot order)
    int nf = 0;
    for (int base = 0; base < R; base += 32) {
        int s = base + lane;
        uint32_t x = s < R ? nbr[v * R + s] : kNone;
        bool ok = x != kNone && (int64_t)x < N;
        unsigned b = __ballot_sync(FULL, ok);
        if (ok)
            fw[nf + __popc(b & ((1u << lane) - 1))] = x;
        nf += __popc(b);
    }
    __syncwarp();
    int nb = 0;
    const uint32_t beg = off[v], cnt = indeg[v];
    for (uint32_t base = 0; cap > 0 && base < cnt; base += 32) {
        uint32_t i = base + lane;
        uint32_t x = i < cnt ? src[beg + i] : kNone;
        bool ok = i < cnt;
        for (int f = 0; f < nf && ok; ++f)
            if (fw[f] == x)
                ok = false;
        unsigned b = __ballot_sync(FULL, ok);
        while (b) {
            int sl = __ffs(b) - 1;
            b &= b - 1;
            uint32_t c = __shfl_sync(FULL, x, sl);
            if (nb == cap && c >= best[cap - 1])
                continue;
            int below = 0, same = 0;
            for (int e = lane; e < nb; e += 32) {
                below += best[e] < c ? 1 : 0;
                same += best[e] == c ? 1 : 0;
            }
            if (__reduce_add_sync(FULL, same) > 0)
                continue;  // u listed v more than once
            int pos = __reduce_add_sync(FULL, below);
            int hi = min(nb, cap - 1);
            for (int bs = (hi - 1) & ~31; bs >= (pos & ~31); bs -= 32) {
                int e = bs + lane;
                bool mv = e >= pos && e < hi;
                uint32_t val = mv ? best[e] : 0u;
                __syncwarp();
                if (mv)
                    best[e + 1] = val;
                __syncwarp();
            }
            if (lane == 0)
                best[pos] = c;
            nb = min(nb + 1, cap);
            __syncwarp();
        }
    }
    for (int s = lane; s < W; s += 32) {
        uint32_t x = kNone;
        if (s < nf)
            x = fw[s];
        else if (s - nf < nb)
            x = best[s - nf];
        out[v * W + s] = x;
    }
}

inline int grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 8192 ? 8192 : g));
}

}  // namespace

cudaError_t launch_edge_select(const nhq_index *ix, const uint32_t *cand, int L, int R,
                               uint32_t *out, cudaStream_t s) {
    EdgeArgs a;
    a.X = ix->X;
    a.xstride = ix->xstride;
    a.d = ix->d;
    a.N = ix->N;
    a.attr = ix->attr;
    a.w = make_fusion(ix->w, ix->m);
    a.cand = cand;
    a.L = L;
    a.R = R;
    a.out = out;
    a.rstride = ix->xstride + 4;
    size_t fixed = sizeof(unsigned long long) * kMaxCand + sizeof(uint32_t) * kMaxCand +
                   (sizeof(uint32_t) + sizeof(int) + sizeof(float)) * kMaxDegree + 4 * sizeof(int);
    fixed = (fixed + 15) & ~(size_t)15;
    size_t staged = sizeof(float) * (size_t)(L + 1) * a.rstride;
    a.staged = fixed + staged <= 100 * 1024 ? 1 : 0;
    size_t smem = fixed + (a.staged ? staged : 0);
    cudaError_t e = cudaFuncSetAttribute(edge_select_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    if (ix->N > 0)
        edge_select_kernel<<<(unsigned)ix->N, ES_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

size_t reverse_scratch_bytes(int64_t N, int R) {
    size_t cub_bytes = 0;
    cub::DeviceScan::ExclusiveSum(nullptr, cub_bytes, (uint32_t *)nullptr, (uint32_t *)nullptr,
                                  (int)N);
    // indeg, off, cur [N] + src [N*R] + cub temp (+ alignment slack)
    return sizeof(uint32_t) * (3 * (size_t)N + (size_t)N * R) + cub_bytes + 1024;
}

cudaError_t launch_reverse_candidates(const uint32_t *nbr, int64_t N, int R, int cap,
                                      uint32_t *out, void *scratch, cudaStream_t s) {
    uint32_t *indeg = reinterpret_cast<uint32_t *>(scratch);
    uint32_t *off = indeg + N;
    uint32_t *cur = off + N;
    uint32_t *src = cur + N;
    uintptr_t t = reinterpret_cast<uintptr_t>(src + (size_t)N * R);
    t = (t + 255) & ~(uintptr_t)255;
    void *cub_tmp = reinterpret_cast<void *>(t);
    size_t cub_bytes = 0;
    cudaError_t e;
    if ((e = cub::DeviceScan::ExclusiveSum(nullptr, cub_bytes, indeg, off, (int)N)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(indeg, 0, sizeof(uint32_t) * N, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(cur, 0, sizeof(uint32_t) * N, s)) != cudaSuccess)
        return e;
    indeg_kernel<<<grid_for(N * R), 256, 0, s>>>(nbr, N * (int64_t)R, N, indeg);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    if ((e = cub::DeviceScan::ExclusiveSum(cub_tmp, cub_bytes, indeg, off, (int)N, s)) !=
        cudaSuccess)
        return e;
    fill_sources_kernel<<<grid_for(N * R), 256, 0, s>>>(nbr, N, R, off, cur, src);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    const int wpb = 4;
    size_t smem = sizeof(uint32_t) * wpb * 2 * kMaxDegree;
    reverse_rows_kernel<<<(unsigned)((N + wpb - 1) / wpb), 32 * wpb, smem, s>>>(
        nbr, N, R, cap, off, indeg, src, out);
    return cudaGetLastError();
}

}  // namespace nhq
