// k_nsw.cu -- the per-wave steps of the incremental build (NPG_nsw of Sec. 4.3, in
// insertion waves; the search and the landing-zone selection are the kernels of
// k_search.cu and k_edge.cu):
//   seeds    entry points of each new vertex v in the graph of [0, s): min(32, s)
//            consecutive ids (h + j) mod s from h = splitmix64(seed ^ mix64(v))[0] mod s;
//            or (attribute entry) the earlier vertices whose attributes equal v's, at most
//            32 evenly spaced, from the index's sorted attribute table (ids ascending
//            within a tuple, so the earlier ones are a prefix of the tuple's run)
//   queries  the wave's rows as a contiguous query batch, attributes unpacked
//   pairs    every selected edge v -> u of the wave as the key u << 32 | v; after a
//            radix sort the keys of one u are contiguous and ascending in v
//   segments the first key of every u
//   reverse  the candidate row of such a u: N(u), then its new sources ascending (at
//            most cap)
//   install  rows written into the adjacency and their neighbours' attribute words
//            refreshed
#include <cub/cub.cuh>

#include "nhq_internal.cuh"

namespace nhq {

namespace {

constexpr int NSW_SEEDS = 32;

__global__ void nsw_seeds_kernel(int64_t s, int64_t B, uint64_t seed, uint32_t *seeds) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= B * NSW_SEEDS)
        return;
    const int64_t b = i / NSW_SEEDS;
    const int j = (int)(i % NSW_SEEDS);
    const uint64_t v = (uint64_t)(s + b);
    const uint64_t h = splitmix_at(seed ^ mix64(v), 0) % (uint64_t)s;
    seeds[i] = (int64_t)j < s ? (uint32_t)((h + (uint64_t)j) % (uint64_t)s) : kNone;
}

__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t *a, int64_t n, uint32_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__global__ void nsw_attr_seeds_kernel(int64_t s, int64_t B, uint64_t seed,
                                      const uint32_t *__restrict__ attr,
                                      const uint32_t *__restrict__ attr_sorted,
                                      const uint32_t *__restrict__ id_sorted, int64_t N,
                                      uint32_t *__restrict__ seeds) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= B)
        return;
    const int64_t v = s + b;
    const uint32_t av = attr[v];
    const int64_t lo = lower_bound_u32(attr_sorted, N, av);
    const int64_t hi = av == 0xFFFFFFFFu ? N : lower_bound_u32(attr_sorted, N, av + 1u);
    const int64_t c = lower_bound_u32(id_sorted + lo, hi - lo, (uint32_t)s);  // ids < s
    uint32_t *row = seeds + b * NSW_SEEDS;
    if (c > 0) {
        const int64_t S = c < NSW_SEEDS ? c : NSW_SEEDS;
        for (int j = 0; j < NSW_SEEDS; ++j)
            row[j] = j < S ? id_sorted[lo + ((int64_t)j * c) / S] : kNone;
    } else {
        const uint64_t h = splitmix_at(seed ^ mix64((uint64_t)v), 0) % (uint64_t)s;
        for (int j = 0; j < NSW_SEEDS; ++j)
            row[j] = (int64_t)j < s ? (uint32_t)((h + (uint64_t)j) % (uint64_t)s) : kNone;
    }
}

__global__ void nsw_queries_kernel(const float *__restrict__ X, int xstride, int d,
                                   const uint32_t *__restrict__ attr, AttrLayout L, int64_t s,
                                   int64_t B, float *__restrict__ q, uint8_t *__restrict__ qa) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < B * d) {
        const int64_t b = i / d;
        q[i] = X[(s + b) * xstride + (i % d)];
    }
    if (i < B * L.m) {
        const int64_t b = i / L.m;
        const int j = (int)(i % L.m);
        qa[i] = (uint8_t)((attr[s + b] >> L.shift[j]) & ((1u << L.width[j]) - 1u));
    }
}

__global__ void nsw_pairs_kernel(const uint32_t *__restrict__ rows, int R, int64_t s, int64_t B,
                                 unsigned long long *__restrict__ keys) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= B * R)
        return;
    const uint32_t u = rows[i];
    keys[i] = u == kNone ? ~0ull
                         : ((unsigned long long)u << 32) | (unsigned long long)(s + i / R);
}

__global__ void nsw_segments_kernel(const unsigned long long *__restrict__ keys, int64_t n,
                                    uint32_t *__restrict__ seg_start, int *__restrict__ nseg) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || keys[i] == ~0ull)
        return;
    if (i == 0 || (keys[i] >> 32) != (keys[i - 1] >> 32))
        seg_start[atomicAdd(nseg, 1)] = (uint32_t)i;
}

__global__ void nsw_reverse_kernel(const unsigned long long *__restrict__ keys, int64_t n,
                                   const uint32_t *__restrict__ seg_start, int nseg,
                                   const uint32_t *__restrict__ nbr, int R, int cap,
                                   uint32_t *__restrict__ U, uint32_t *__restrict__ cand) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nseg)
        return;
    const int64_t i0 = seg_start[j];
    const uint32_t u = (uint32_t)(keys[i0] >> 32);
    U[j] = u;
    uint32_t *row = cand + (int64_t)j * (R + cap);
    int w = 0;
    for (int t = 0; t < R; ++t) {
        const uint32_t x = nbr[(int64_t)u * R + t];
        if (x != kNone)
            row[w++] = x;
    }
    for (int64_t i = i0; i < n && i - i0 < cap && (keys[i] >> 32) == u && keys[i] != ~0ull; ++i)
        row[w++] = (uint32_t)keys[i];
    for (; w < R + cap; ++w)
        row[w] = kNone;
}

// rows[b] of `src` into adjacency row (list ? list[b] : row0 + b), with its attribute words
__global__ void nsw_install_kernel(const uint32_t *__restrict__ src, const uint32_t *list,
                                   int64_t row0, int64_t count, int R,
                                   const uint32_t *__restrict__ attr, uint32_t *__restrict__ nbr,
                                   uint32_t *__restrict__ nbr_attr) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count * R)
        return;
    const int64_t b = i / R;
    const int64_t u = list ? (int64_t)list[b] : row0 + b;
    const uint32_t v = src[i];
    nbr[u * R + i % R] = v;
    nbr_attr[u * R + i % R] = v == kNone ? 0u : attr[v];
}

inline unsigned blocks_for(int64_t n) { return (unsigned)((n + 255) / 256 > 0 ? (n + 255) / 256 : 1); }

}  // namespace

int nsw_seed_count() { return NSW_SEEDS; }

cudaError_t launch_nsw_seeds(int64_t s, int64_t B, uint64_t seed, uint32_t *seeds,
                             cudaStream_t st) {
    nsw_seeds_kernel<<<blocks_for(B * NSW_SEEDS), 256, 0, st>>>(s, B, seed, seeds);
    return cudaGetLastError();
}

cudaError_t launch_nsw_attr_seeds(const nhq_index *ix, int64_t s, int64_t B, uint64_t seed,
                                  uint32_t *seeds, cudaStream_t st) {
    nsw_attr_seeds_kernel<<<blocks_for(B), 256, 0, st>>>(s, B, seed, ix->attr, ix->attr_sorted,
                                                          ix->id_sorted, ix->N, seeds);
    return cudaGetLastError();
}

cudaError_t launch_nsw_queries(const nhq_index *ix, int64_t s, int64_t B, float *q, uint8_t *qa,
                               cudaStream_t st) {
    const int64_t n = B * (ix->d > ix->m ? ix->d : ix->m);
    nsw_queries_kernel<<<blocks_for(n), 256, 0, st>>>(ix->X, ix->xstride, ix->d, ix->attr,
                                                      ix->layout, s, B, q, qa);
    return cudaGetLastError();
}

size_t nsw_sort_scratch_bytes(int64_t n) {
    size_t b = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, b, (const unsigned long long *)nullptr,
                                   (unsigned long long *)nullptr, (int)n);
    return b;
}

// the wave's edges as sorted (u, v) keys, then the segment starts; *nseg_dev receives
// the number of distinct u
cudaError_t launch_nsw_pairs(const uint32_t *rows, int R, int64_t s, int64_t B,
                             unsigned long long *keys, unsigned long long *sorted, void *tmp,
                             size_t tmp_bytes, uint32_t *seg_start, int *nseg_dev,
                             cudaStream_t st) {
    const int64_t n = B * R;
    nsw_pairs_kernel<<<blocks_for(n), 256, 0, st>>>(rows, R, s, B, keys);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    size_t tb = tmp_bytes;
    if ((e = cub::DeviceRadixSort::SortKeys(tmp, tb, keys, sorted, (int)n, 0, 64, st)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(nseg_dev, 0, sizeof(int), st)) != cudaSuccess)
        return e;
    nsw_segments_kernel<<<blocks_for(n), 256, 0, st>>>(sorted, n, seg_start, nseg_dev);
    return cudaGetLastError();
}

cudaError_t launch_nsw_reverse(const unsigned long long *sorted, int64_t n,
                               const uint32_t *seg_start, int nseg, const uint32_t *nbr, int R,
                               int cap, uint32_t *U, uint32_t *cand, cudaStream_t st) {
    if (nseg <= 0)
        return cudaSuccess;
    nsw_reverse_kernel<<<blocks_for(nseg), 256, 0, st>>>(sorted, n, seg_start, nseg, nbr, R, cap,
                                                          U, cand);
    return cudaGetLastError();
}

cudaError_t launch_nsw_install(const uint32_t *src, const uint32_t *list, int64_t row0,
                               int64_t count, int R, const uint32_t *attr, uint32_t *nbr,
                               uint32_t *nbr_attr, cudaStream_t st) {
    if (count <= 0)
        return cudaSuccess;
    nsw_install_kernel<<<blocks_for(count * R), 256, 0, st>>>(src, list, row0, count, R, attr,
                                                               nbr, nbr_attr);
    return cudaGetLastError();
}

}  // namespace nhq
