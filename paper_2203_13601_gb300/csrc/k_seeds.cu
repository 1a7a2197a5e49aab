// k_seeds.cu -- seed sets B for Alg. 2 chosen by attributes.
//
// The index keeps its packed attribute words sorted ascending together with
// the object ids (a stable radix sort, so ids stay ascending within a tuple).
// For NHQ_SEED_ATTRIBUTE one thread per query binary-searches the run of
// objects whose attributes equal the query's, P (ascending ids), and takes
// S = min(ef, 32, |P|) of them evenly spaced: P[floor(j * |P| / S)], j < S.
// A query whose tuple does not occur falls back to the random stream of
// NHQ_SEED_RANDOM (first min(ef, 32) distinct ids of <= 64 splitmix64 draws).
//
// The same pass sorts the queries into cost buckets, 31 - bit length of (|P| + 1):
// under constant weights a query whose tuple is frequent expands more records (its
// pool fills with matching objects and keeps improving), so the search takes the
// queries with the largest |P| first and the batch does not end on a few long ones
// started last.  The order decides only which warp takes a query when; every
// query's result is the same.
#include <cub/cub.cuh>

#include "nhq_internal.cuh"

namespace nhq {

namespace {

__global__ void iota_kernel(uint32_t *out, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (uint32_t)i;
}

__device__ __forceinline__ int64_t lower_bound_u32(const uint32_t *a, int64_t n, uint32_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__global__ void attribute_seeds_kernel(SearchArgs a, const uint32_t *__restrict__ attr_sorted,
                                       const uint32_t *__restrict__ id_sorted,
                                       uint32_t *__restrict__ seeds,
                                       uint8_t *__restrict__ bucket) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= a.nq)
        return;
    uint32_t qa = 0;
    for (int j = 0; j < a.w.m; ++j)
        qa |= (uint32_t)a.qattr[q * a.w.m + j] << (8 * j);
    const int ef = a.ef_arr ? a.ef_arr[q] : a.ef;
    const int want = ef < 32 ? ef : 32;
    const int64_t lo = lower_bound_u32(attr_sorted, a.N, qa);
    const int64_t hi = qa == 0xFFFFFFFFu ? a.N : lower_bound_u32(attr_sorted, a.N, qa + 1u);
    const int64_t c = hi - lo;
    if (bucket != nullptr) {
        const int bits = 64 - __clzll((unsigned long long)c + 1ull);  // 1..
        bucket[q] = (uint8_t)(bits >= 32 ? 0 : 32 - bits);
    }
    uint32_t *row = seeds + q * 32;
    int j = 0;
    if (c > 0) {
        const int S = (int64_t)want < c ? want : (int)c;
        for (; j < S; ++j)
            row[j] = id_sorted[lo + ((int64_t)j * c) / S];
    } else {
        const uint64_t s0 = a.seed ^ mix64((uint64_t)q);
        for (int t = 0; t < 64 && j < want; ++t) {
            const uint32_t v = (uint32_t)(splitmix_at(s0, (uint64_t)t) % (unsigned long long)a.N);
            bool dup = false;
            for (int i = 0; i < j; ++i)
                dup = dup || row[i] == v;
            if (!dup)
                row[j++] = v;
        }
    }
    for (; j < 32; ++j)
        row[j] = kNone;
}

// counting sort of the query indices by bucket, one block
__global__ void query_order_kernel(const uint8_t *__restrict__ bucket, int64_t nq,
                                   uint32_t *__restrict__ order) {
    __shared__ unsigned int hist[32], base[32];
    if (threadIdx.x < 32)
        hist[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x)
        atomicAdd(&hist[bucket[q] & 31], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int sum = 0;
        for (int b = 0; b < 32; ++b) {
            base[b] = sum;
            sum += hist[b];
        }
    }
    __syncthreads();
    for (int64_t q = threadIdx.x; q < nq; q += blockDim.x)
        order[atomicAdd(&base[bucket[q] & 31], 1u)] = (uint32_t)q;
}

}  // namespace

size_t attribute_sort_scratch_bytes(int64_t N) {
    size_t cub_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, cub_bytes, (const uint32_t *)nullptr,
                                    (uint32_t *)nullptr, (const uint32_t *)nullptr,
                                    (uint32_t *)nullptr, (int)N);
    return sizeof(uint32_t) * (size_t)N + 256 + cub_bytes;
}

cudaError_t launch_attribute_sort(const uint32_t *attr, int64_t N, uint32_t *attr_sorted,
                                  uint32_t *id_sorted, void *scratch, size_t scratch_bytes,
                                  cudaStream_t s) {
    uint32_t *iota = reinterpret_cast<uint32_t *>(scratch);
    uintptr_t t = reinterpret_cast<uintptr_t>(iota + N);
    t = (t + 255) & ~(uintptr_t)255;
    void *tmp = reinterpret_cast<void *>(t);
    size_t cub_bytes = 0;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(nullptr, cub_bytes, attr, attr_sorted, iota,
                                                    id_sorted, (int)N);
    if (e != cudaSuccess)
        return e;
    if ((char *)tmp + cub_bytes > (char *)scratch + scratch_bytes)
        return cudaErrorInvalidValue;
    int64_t g = (N + 255) / 256;
    iota_kernel<<<(unsigned)(g > 8192 ? 8192 : g), 256, 0, s>>>(iota, N);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    return cub::DeviceRadixSort::SortPairs(tmp, cub_bytes, attr, attr_sorted, iota, id_sorted,
                                           (int)N, 0, 32, s);
}

cudaError_t launch_attribute_seeds(const SearchArgs &a, const uint32_t *attr_sorted,
                                   const uint32_t *id_sorted, uint32_t *seeds, uint8_t *bucket,
                                   cudaStream_t s) {
    if (a.nq <= 0)
        return cudaSuccess;
    attribute_seeds_kernel<<<(unsigned)((a.nq + 127) / 128), 128, 0, s>>>(a, attr_sorted,
                                                                            id_sorted, seeds,
                                                                            bucket);
    return cudaGetLastError();
}

cudaError_t launch_query_order(const uint8_t *bucket, int64_t nq, uint32_t *order,
                               cudaStream_t s) {
    if (nq <= 0)
        return cudaSuccess;
    query_order_kernel<<<1, 1024, 0, s>>>(bucket, nq, order);
    return cudaGetLastError();
}

}  // namespace nhq
