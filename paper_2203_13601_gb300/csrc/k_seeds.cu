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

constexpr int kMaxCompletions = 64;

// The run [*lo, *lo + count) of the packed word `word` in the sorted attribute table.
__device__ __forceinline__ int64_t tuple_run(const uint32_t *attr_sorted, int64_t N,
                                             uint32_t word, int64_t *lo) {
    const int64_t l = lower_bound_u32(attr_sorted, N, word);
    const int64_t h = word == 0xFFFFFFFFu ? N : lower_bound_u32(attr_sorted, N, word + 1u);
    *lo = l;
    return h - l;
}

// Completion t of an open query: its word with every open field j set to the digit of t
// in the mixed radix amax[j] + 1 over the open fields, the lowest field fastest.
__device__ __forceinline__ uint32_t completion_word(const Fusion &w, uint32_t qa, uint32_t qhi,
                                                    int64_t t) {
    uint32_t word = qa;
    for (int j = 0; j < w.m; ++j) {
        if ((field_hi(w, j) & ~qhi) == 0u)
            continue;
        const int64_t r = (int64_t)w.amax[j] + 1;
        word |= (uint32_t)(t % r) << w.shift[j];
        t /= r;
    }
    return word;
}

// The number of completions of an open query (-1 above kMaxCompletions).
__device__ __forceinline__ int64_t open_completions(const Fusion &w, uint32_t qhi) {
    int64_t T = 1;
    for (int j = 0; j < w.m; ++j)
        if ((field_hi(w, j) & ~qhi) != 0u) {
            T *= (int64_t)w.amax[j] + 1;
            if (T > kMaxCompletions)
                return -1;
        }
    return T;
}

// Seeds of an open query (a field left open by the wildcard) under the attribute seed
// modes: its completions fill each open field with 0..amax[j]; with at most 64 of them,
// P = their runs one after another in completion order and row[0..S) = P[floor(j c / S)],
// S = min(want, c), the rest kNone.  Returns c = |P| (row untouched when c = 0), or -1
// when there are more than 64 completions.
__device__ int64_t open_query_seeds(const Fusion &w, uint32_t qa, uint32_t qhi,
                                    const uint32_t *attr_sorted, const uint32_t *id_sorted,
                                    int64_t N, int want, uint32_t *row) {
    const int64_t T = open_completions(w, qhi);
    if (T < 0)
        return -1;
    int64_t c = 0, lo;
    for (int64_t t = 0; t < T; ++t)
        c += tuple_run(attr_sorted, N, completion_word(w, qa, qhi, t), &lo);
    if (c == 0)
        return 0;
    const int S = (int64_t)want < c ? want : (int)c;
    int j = 0;
    int64_t base = 0;
    for (int64_t t = 0; t < T && j < S; ++t) {
        const int64_t ct = tuple_run(attr_sorted, N, completion_word(w, qa, qhi, t), &lo);
        while (j < S) {
            const int64_t r = ((int64_t)j * c) / S;
            if (r >= base + ct)
                break;
            row[j++] = id_sorted[lo + (r - base)];
        }
        base += ct;
    }
    for (; j < 32; ++j)
        row[j] = kNone;
    return c;
}

__global__ void attribute_seeds_kernel(SearchArgs a, const uint32_t *__restrict__ attr_sorted,
                                       const uint32_t *__restrict__ id_sorted,
                                       uint32_t *__restrict__ seeds,
                                       uint8_t *__restrict__ bucket) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= a.nq)
        return;
    uint32_t qhi;
    const uint32_t qa = pack_query_word(a.qattr + q * a.w.m, a.w, &qhi);
    const int ef = a.ef_arr ? a.ef_arr[q] : a.ef;
    const int want = ef < 32 ? ef : 32;
    uint32_t *row = seeds + q * 32;
    // a query that leaves an attribute open takes its seeds from its completions' runs
    const bool open = qhi != a.w.hi;
    int64_t lo = 0, c = 0;
    if (open) {
        c = open_query_seeds(a.w, qa, qhi, attr_sorted, id_sorted, a.N, want, row);
        c = c < 0 ? 0 : c;
    } else {
        c = tuple_run(attr_sorted, a.N, qa, &lo);
    }
    if (bucket != nullptr) {
        const int bits = 64 - __clzll((unsigned long long)c + 1ull);  // 1..
        bucket[q] = (uint8_t)(bits >= 32 ? 0 : 32 - bits);
    }
    if (open && c > 0)
        return;  // row written
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

// NHQ_SEED_ATTRIBUTE_NEAR: one warp per query; lane l takes the sampled members
// l, l + 32, ... (at most 256 in all), computes delta^2 to the query in f32 in index order
// (separately rounded, as the canonical form), and the warp takes the smallest
// (delta^2, id) keys one at a time
__global__ void attribute_near_seeds_kernel(SearchArgs a, const uint32_t *__restrict__ attr_sorted,
                                            const uint32_t *__restrict__ id_sorted,
                                            uint32_t *__restrict__ seeds,
                                            uint8_t *__restrict__ bucket) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= a.nq)
        return;
    uint32_t qhi;
    const uint32_t qa = pack_query_word(a.qattr + q * a.w.m, a.w, &qhi);
    const int ef = a.ef_arr ? a.ef_arr[q] : a.ef;
    const int want = ef < 32 ? ef : 32;
    uint32_t *row = seeds + q * 32;
    // A query that leaves an attribute open: P = its completions' runs one after another
    // (lane l holds completions l and l + 32, at most 64); (base0, c0) and (base1, c1)
    // are those runs' offsets in P and sizes.
    const bool open = qhi != a.w.hi;
    int64_t lo = 0, c = 0;
    int64_t lo0 = 0, c0 = 0, base0 = 0, lo1 = 0, c1 = 0, base1 = 0;
    if (open) {
        const int64_t T = open_completions(a.w, qhi);
        if (T > 0) {
            if (lane < T)
                c0 = tuple_run(attr_sorted, a.N, completion_word(a.w, qa, qhi, lane), &lo0);
            if (lane + 32 < T)
                c1 = tuple_run(attr_sorted, a.N, completion_word(a.w, qa, qhi, lane + 32), &lo1);
            long long p0 = c0, p1 = c1;  // inclusive prefix sums over the lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const long long u0 = __shfl_up_sync(0xFFFFFFFFu, p0, o);
                const long long u1 = __shfl_up_sync(0xFFFFFFFFu, p1, o);
                if (lane >= o) {
                    p0 += u0;
                    p1 += u1;
                }
            }
            const long long tot0 = __shfl_sync(0xFFFFFFFFu, p0, 31);
            const long long tot1 = __shfl_sync(0xFFFFFFFFu, p1, 31);
            base0 = p0 - c0;
            base1 = tot0 + p1 - c1;
            c = tot0 + tot1;
        }
    } else {
        c = tuple_run(attr_sorted, a.N, qa, &lo);
    }
    if (lane == 0 && bucket != nullptr) {
        const int bits = 64 - __clzll((unsigned long long)c + 1ull);
        bucket[q] = (uint8_t)(bits >= 32 ? 0 : 32 - bits);
    }
    if (c == 0) {  // the random stream of NHQ_SEED_RANDOM
        if (lane == 0) {
            int j = 0;
            const uint64_t s0 = a.seed ^ mix64((uint64_t)q);
            for (int t = 0; t < 64 && j < want; ++t) {
                const uint32_t v = (uint32_t)(splitmix_at(s0, (uint64_t)t) % (unsigned long long)a.N);
                bool dup = false;
                for (int i = 0; i < j; ++i)
                    dup = dup || row[i] == v;
                if (!dup)
                    row[j++] = v;
            }
            for (; j < 32; ++j)
                row[j] = kNone;
        }
        return;
    }
    const int M = c < 256 ? (int)c : 256;
    const float *qv = a.Q + q * a.qstride;
    // rows start on 32-byte boundaries (xstride is a multiple of 8); the query row on a
    // 16-byte one when qstride is a multiple of 4 and the batch is 16-byte aligned
    const bool vec4 = (a.d & 3) == 0 && (a.qstride & 3) == 0 &&
                      ((reinterpret_cast<uintptr_t>(a.Q) & 15) == 0);
    // sampled member j = lane + 32 t is P[floor(j c / M)]
    uint32_t vid[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int j0 = lane + 32 * t;
        vid[t] = !open && j0 < M ? id_sorted[lo + ((int64_t)j0 * c) / M] : kNone;
        if (open) {  // the owner of each rank among the lanes' runs reads its id
            for (int l = 0; l < 32; ++l) {
                const int j = 32 * t + l;
                if (j >= M)
                    break;  // warp-uniform
                const int64_t r = ((int64_t)j * c) / M;
                const unsigned h0 = __ballot_sync(0xFFFFFFFFu, r >= base0 && r < base0 + c0);
                const unsigned h1 = __ballot_sync(0xFFFFFFFFu, r >= base1 && r < base1 + c1);
                const int src = h0 ? __ffs(h0) - 1 : __ffs(h1) - 1;
                uint32_t v = 0;
                if (lane == src)
                    v = id_sorted[h0 ? lo0 + (r - base0) : lo1 + (r - base1)];
                v = __shfl_sync(0xFFFFFFFFu, v, src);
                if (lane == l)
                    vid[t] = v;
            }
        }
    }
    unsigned long long key[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int j = lane + 32 * t;
        key[t] = ~0ull;
        if (j < M) {
            const uint32_t v = vid[t];
            const float *xv = a.X + (int64_t)v * a.xstride;
            float s = 0.f;
            if (vec4) {
                const float4 *x4 = reinterpret_cast<const float4 *>(xv);
                const float4 *q4 = reinterpret_cast<const float4 *>(qv);
                for (int i = 0; i < (a.d >> 2); ++i) {
                    const float4 xa = __ldg(x4 + i), qa4 = q4[i];
                    float dd = __fsub_rn(qa4.x, xa.x);
                    s = __fadd_rn(s, __fmul_rn(dd, dd));
                    dd = __fsub_rn(qa4.y, xa.y);
                    s = __fadd_rn(s, __fmul_rn(dd, dd));
                    dd = __fsub_rn(qa4.z, xa.z);
                    s = __fadd_rn(s, __fmul_rn(dd, dd));
                    dd = __fsub_rn(qa4.w, xa.w);
                    s = __fadd_rn(s, __fmul_rn(dd, dd));
                }
            } else {
                for (int i = 0; i < a.d; ++i) {
                    const float dd = __fsub_rn(qv[i], xv[i]);
                    s = __fadd_rn(s, __fmul_rn(dd, dd));
                }
            }
            key[t] = ((unsigned long long)__float_as_uint(s) << 32) | v;
        }
    }
    const int S = want < M ? want : M;
    for (int r = 0; r < 32; ++r) {
        unsigned long long best = ~0ull;
        int bt = -1;
        if (r < S) {
#pragma unroll
            for (int t = 0; t < 8; ++t)
                if (key[t] < best) {
                    best = key[t];
                    bt = t;
                }
        }
        unsigned long long m = best;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xFFFFFFFFu, m, o);
            m = other < m ? other : m;
        }
        if (r < S && bt >= 0 && best == m) {  // keys are unique: one owner
#pragma unroll
            for (int t = 0; t < 8; ++t)
                if (t == bt)
                    key[t] = ~0ull;
            row[r] = (uint32_t)m;
        }
        if (r >= S && lane == 0)
            row[r] = kNone;
    }
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

cudaError_t launch_attribute_near_seeds(const SearchArgs &a, const uint32_t *attr_sorted,
                                        const uint32_t *id_sorted, uint32_t *seeds,
                                        uint8_t *bucket, cudaStream_t s) {
    if (a.nq <= 0)
        return cudaSuccess;
    attribute_near_seeds_kernel<<<(unsigned)((a.nq + 7) / 8), 256, 0, s>>>(a, attr_sorted,
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
