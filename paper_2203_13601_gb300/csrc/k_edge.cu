// k_edge.cu -- landing-zone edge selection (Sec. 4.1, Def. 6) for every vertex,
// and the reverse-candidate lists of the optional second selection pass.
//
// Edge selection: one CTA (4 warps) per vertex u.  The candidate rows (and u's)
// are copied into shared memory with cp.async when they fit, so every later
// distance reads on-chip memory.  Gamma(p, u) of all candidates is computed by 16
// teams of 8 lanes and the records (Gamma(p, u), p) are bitonic-sorted.  Def. 6
// admits p iff for every neighbour j accepted before it
//     Gamma(p, u) < Gamma(p, j)   and   Gamma(p, u) > Gamma(u, j).
// The walk applies it the other way round: when j is accepted, the teams test every
// later candidate that is still alive against j and reject those that fail, so the
// next alive candidate in order is accepted without further tests.  That takes one
// parallel round of distances per accepted neighbour instead of one test sequence
// per candidate, and gives the same neighbours as testing candidate by candidate.
#include <cub/cub.cuh>

#include "nhq_internal.cuh"

namespace nhq {

namespace {

constexpr int ES_THREADS = 128;
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
    const uint32_t *rows;  // vertex of block b: rows[b], or row0 + b when rows is null;
    int64_t row0;          // cand and out are indexed by b
};

// squared distance between two rows, one team of T lanes (T = 4 or 8); result in
// every lane of the team
template <int T>
__device__ __forceinline__ float team_dist2_t(const float *__restrict__ a,
                                              const float *__restrict__ b, int xs4, int tl) {
    float acc = 0.f;
    for (int c = tl; c < xs4; c += T) {
        const float4 x = reinterpret_cast<const float4 *>(a)[c];
        const float4 y = reinterpret_cast<const float4 *>(b)[c];
        float t;
        t = x.x - y.x; acc = fmaf(t, t, acc);
        t = x.y - y.y; acc = fmaf(t, t, acc);
        t = x.z - y.z; acc = fmaf(t, t, acc);
        t = x.w - y.w; acc = fmaf(t, t, acc);
    }
#pragma unroll
    for (int o = 1; o < T; o <<= 1)
        acc += __shfl_xor_sync(FULL, acc, o);
    return acc;
}

// stable block-wide compaction (128 threads): the values of the flagged threads, in
// thread order, into out[]; returns their count (every thread)
__device__ __forceinline__ int block_compact(bool flag, int value, int *out, int *cnt, int lane,
                                             int warp) {
    const unsigned bal = __ballot_sync(FULL, flag);
    if (lane == 0)
        cnt[warp] = __popc(bal);
    __syncthreads();
    int pos = __popc(bal & ((1u << lane) - 1u)), total = 0;
    for (int w = 0; w < 4; ++w) {
        pos += w < warp ? cnt[w] : 0;
        total += cnt[w];
    }
    if (flag)
        out[pos] = value;
    __syncthreads();
    return total;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__global__ void __launch_bounds__(ES_THREADS) edge_select_kernel(EdgeArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    unsigned long long *keys = reinterpret_cast<unsigned long long *>(smem);  // [kMaxCand]
    uint32_t *cid = reinterpret_cast<uint32_t *>(keys + kMaxCand);           // [kMaxCand] by slot
    int *order = reinterpret_cast<int *>(cid + kMaxCand);                     // [kMaxCand] slot of rank
    int *listA = order + kMaxCand;                                            // [kMaxCand] live ranks
    int *listB = listA + kMaxCand;                                            // [kMaxCand]
    int *keep = listB + kMaxCand;                                             // [kMaxCand]
    float *gpu = reinterpret_cast<float *>(keep + kMaxCand);                  // [kMaxCand] by slot
    uint32_t *acc_id = reinterpret_cast<uint32_t *>(gpu + kMaxCand);          // [kMaxDegree]
    uint32_t *sattr = acc_id + kMaxDegree;                                    // [kMaxCand] by slot
    int *misc = reinterpret_cast<int *>(sattr + kMaxCand);                    // [4]
    float *rows = reinterpret_cast<float *>(misc + 4);                        // [(L+1)][rstride]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int T4 = 4, TEAMS4 = ES_THREADS / T4;  // teams of 4 lanes
    const int team = tid / T4, tl = tid % T4;
    const int xs4 = a.xstride / 4;
    const int64_t b = blockIdx.x;
    const int64_t u = a.rows ? (int64_t)a.rows[b] : a.row0 + b;
    const uint32_t au = a.attr[u];

    // 1. candidate ids (invalid, self and out-of-range dropped) in list order
    {
        const uint32_t p = tid < a.L ? a.cand[b * a.L + tid] : kNone;
        const bool ok = p != kNone && (int64_t)p < a.N && (int64_t)p != u;
        const unsigned bal = __ballot_sync(FULL, ok);
        if (lane == 0)
            misc[warp] = __popc(bal);
        __syncthreads();
        int pos = __popc(bal & ((1u << lane) - 1u));
        for (int w = 0; w < warp; ++w)
            pos += misc[w];
        if (ok) {
            cid[pos] = p;
            sattr[pos] = a.attr[p];
        }
    }
    int n = 0;
    for (int w = 0; w < ES_THREADS / 32; ++w)
        n += misc[w];
    __syncthreads();

    // 2. rows of the candidates (slots 0..n-1) and of u (slot n) into shared memory
    if (a.staged) {
        const uint32_t rbase = (uint32_t)__cvta_generic_to_shared(rows);
        for (int idx = tid; idx < (n + 1) * xs4; idx += ES_THREADS) {
            const int r = idx / xs4, c = idx % xs4;
            const int64_t src = r < n ? (int64_t)cid[r] : u;
            cp_async16(rbase + (uint32_t)(r * a.rstride + 4 * c) * 4u,
                       a.X + src * a.xstride + 4 * c);
        }
        asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
    }
    auto row_of_slot = [&](int i) -> const float * {
        if (a.staged)
            return rows + (size_t)i * a.rstride;
        return a.X + (i < n ? (int64_t)cid[i] : u) * a.xstride;
    };

    // 3. Gamma(p, u) of every candidate and its record (Gamma, p)
    for (int base = 0; base < n; base += TEAMS4) {
        const int i = base + team;
        const float dd = team_dist2_t<T4>(row_of_slot(i < n ? i : 0), row_of_slot(n), xs4, tl);
        if (i < n && tl == 0) {
            const float g = fusion_gamma(__fsqrt_rn(dd), chi_packed(sattr[i], au, a.w.hi, a.w.lo), a.w);
            gpu[i] = g;
            keys[i] = ((unsigned long long)__float_as_uint(g) << 32) | cid[i];
        }
    }
    __syncthreads();

    // 4. rank of every record by counting (equal records, i.e. a repeated candidate,
    //    by slot; only the first of them is considered)
    bool first = false;
    if (tid < n) {
        const unsigned long long ki = keys[tid];
        int rk = 0;
        bool dup = false;
        for (int j = 0; j < n; ++j) {
            const unsigned long long kj = keys[j];
            const bool same_before = kj == ki && j < tid;
            rk += (kj < ki || same_before) ? 1 : 0;
            dup = dup || same_before;
        }
        order[rk] = tid;
        keep[rk] = dup ? 0 : 1;
    }
    __syncthreads();
    first = tid < n && keep[tid] != 0;
    int na = block_compact(first, tid, listA, misc, lane, warp);  // live ranks, ascending

    // 5. landing-zone walk (Def. 6): the first live record is accepted, the others are
    //    tested against it and the survivors stay live, in order
    int deg = 0;
    const int R = a.R;
    int *A = listA, *B = listB;
    while (na > 0) {
        const int sj = order[A[0]];
        const float gju = gpu[sj];
        if (tid == 0)
            acc_id[deg] = cid[sj];
        if (++deg >= R)
            break;
        const float *jrow = row_of_slot(sj);
        const uint32_t aj = sattr[sj];
        for (int base = 1; base < na; base += TEAMS4) {  // whole warps run every round
            const int k = base + team;
            const bool live = k < na;
            const int sq = order[A[live ? k : 0]];
            const float dd = team_dist2_t<T4>(row_of_slot(sq), jrow, xs4, tl);
            if (live && tl == 0) {
                const float g =
                    fusion_gamma(__fsqrt_rn(dd), chi_packed(sattr[sq], aj, a.w.hi, a.w.lo), a.w);
                const float gq = gpu[sq];
                keep[k] = (gq < g && gq > gju) ? 1 : 0;
            }
        }
        __syncthreads();
        const int k = tid + 1;
        const bool kept = k < na && keep[k] != 0;
        na = block_compact(kept, kept ? A[k] : 0, B, misc, lane, warp);
        int *tmp = A;
        A = B;
        B = tmp;
    }
    __syncthreads();
    for (int s2 = tid; s2 < R; s2 += ES_THREADS)
        a.out[b * R + s2] = s2 < deg ? acc_id[s2] : kNone;
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

cudaError_t launch_edge_select_rows(const nhq_index *ix, const uint32_t *cand, int L, int R,
                                    const uint32_t *rows, int64_t row0, int64_t count,
                                    uint32_t *out, cudaStream_t s) {
    EdgeArgs a;
    a.X = ix->X;
    a.xstride = ix->xstride;
    a.d = ix->d;
    a.N = ix->N;
    a.attr = ix->attr;
    a.w = make_fusion(ix->w, ix->layout);
    a.cand = cand;
    a.L = L;
    a.R = R;
    a.out = out;
    a.rstride = ix->xstride + 4;
    a.rows = rows;
    a.row0 = row0;
    size_t fixed = sizeof(unsigned long long) * kMaxCand +
                   (sizeof(uint32_t) + 4 * sizeof(int) + sizeof(float)) * kMaxCand +
                   sizeof(uint32_t) * (kMaxDegree + kMaxCand) + 4 * sizeof(int);
    fixed = (fixed + 15) & ~(size_t)15;
    size_t staged = sizeof(float) * (size_t)(L + 1) * a.rstride;
    a.staged = fixed + staged <= 100 * 1024 ? 1 : 0;
    size_t smem = fixed + (a.staged ? staged : 0);
    cudaError_t e = cudaFuncSetAttribute(edge_select_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    if (count > 0)
        edge_select_kernel<<<(unsigned)count, ES_THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_edge_select(const nhq_index *ix, const uint32_t *cand, int L, int R,
                               uint32_t *out, cudaStream_t s) {
    return launch_edge_select_rows(ix, cand, L, R, nullptr, 0, ix->N, out, s);
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
