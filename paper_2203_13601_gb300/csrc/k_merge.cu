// k_merge.cu -- operations on finished result lists:
//   * merge of per-shard top-k lists (the paper's parallel form: the object set
//     split into shards with one graph each, every shard searched for every
//     query, the lists combined by (Gamma, id));
//   * post-filter (the "search, then filter by attributes" strategy the paper
//     compares against): the records with chi = 0, in order;
//   * recall of result lists against ground-truth lists (Eq. 3), for the tuner.
//
// One warp per query.  Every shard's list is already sorted by (Gamma, local id),
// and adding the shard's offset keeps that order, so the merge only compares the
// heads: lane l owns the heads of shards l, l + 32, ...; each round the warp takes
// the smallest head key (Gamma bits << 32 | global id) and its owner advances.
#include "nhq_internal.cuh"

namespace nhq {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

struct MergeArgs {
    int P, k_in, k_out;
    int64_t Q;
    const uint32_t *ids;
    const float *dists;
    const uint8_t *chi;
    const uint32_t *offsets;
    uint32_t *out_ids;
    float *out_dists;
    uint8_t *out_chi;
};

__device__ __forceinline__ unsigned long long head_key(const MergeArgs &a, int p, int64_t q,
                                                       int h) {
    if (h >= a.k_in)
        return ~0ull;
    const int64_t o = ((int64_t)p * a.Q + q) * a.k_in + h;
    const uint32_t id = a.ids[o];
    if (id == kNone)
        return ~0ull;  // the rest of the row is padding
    return ((unsigned long long)__float_as_uint(a.dists[o]) << 32) | (uint32_t)(a.offsets[p] + id);
}

__global__ void merge_topk_kernel(MergeArgs a, int heads_per_lane) {
    extern __shared__ int head_pos[];  // [warps per block][32 * heads_per_lane]
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (q >= a.Q)
        return;
    int *pos = head_pos + wib * 32 * heads_per_lane;
    // best head of this lane's shards, kept with its shard index
    unsigned long long best = ~0ull;
    int best_p = -1;
    for (int i = 0; i < heads_per_lane; ++i) {
        const int p = lane + 32 * i;
        pos[lane * heads_per_lane + i] = 0;
        if (p < a.P) {
            const unsigned long long kk = head_key(a, p, q, 0);
            if (kk < best) {
                best = kk;
                best_p = p;
            }
        }
    }
    for (int r = 0; r < a.k_out; ++r) {
        unsigned long long m = best;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(FULL, m, o);
            m = other < m ? other : m;
        }
        const int64_t out = q * a.k_out + r;
        if (m == ~0ull) {  // every shard is exhausted
            if (lane == 0) {
                a.out_ids[out] = kNone;
                a.out_dists[out] = __int_as_float(0x7f800000);
                if (a.out_chi)
                    a.out_chi[out] = 255;
            }
            continue;
        }
        // keys are unique (global ids differ), so exactly one lane owns the minimum
        if (best == m) {
            const int p = best_p;
            const int slot = lane * heads_per_lane + p / 32;
            const int h = pos[slot];
            const int64_t o = ((int64_t)p * a.Q + q) * a.k_in + h;
            a.out_ids[out] = (uint32_t)m;
            a.out_dists[out] = __uint_as_float((uint32_t)(m >> 32));
            if (a.out_chi)
                a.out_chi[out] = a.chi[o];
            pos[slot] = h + 1;
            best = ~0ull;
            best_p = -1;
            for (int i = 0; i < heads_per_lane; ++i) {
                const int pp = lane + 32 * i;
                if (pp < a.P) {
                    const unsigned long long kk = head_key(a, pp, q, pos[lane * heads_per_lane + i]);
                    if (kk < best) {
                        best = kk;
                        best_p = pp;
                    }
                }
            }
        }
        __syncwarp();
    }
}

// one warp per query: stable compaction of the records with chi = 0
__global__ void postfilter_kernel(int64_t Q, int k_in, int k_out, const uint32_t *__restrict__ ids,
                                  const float *__restrict__ dists, const uint8_t *__restrict__ chi,
                                  uint32_t *__restrict__ out_ids, float *__restrict__ out_dists) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= Q)
        return;
    int got = 0;
    for (int base = 0; base < k_in && got < k_out; base += 32) {
        const int j = base + lane;
        const int64_t o = q * k_in + j;
        const bool keep = j < k_in && ids[o] != kNone && chi[o] == 0;
        const unsigned bal = __ballot_sync(FULL, keep);
        const int p = got + __popc(bal & ((1u << lane) - 1u));
        if (keep && p < k_out) {
            out_ids[q * k_out + p] = ids[o];
            out_dists[q * k_out + p] = dists[o];
        }
        got += __popc(bal);
    }
    for (int p = got + lane; p < k_out; p += 32) {
        out_ids[q * k_out + p] = kNone;
        out_dists[q * k_out + p] = __int_as_float(0x7f800000);
    }
}

}  // namespace

cudaError_t launch_postfilter(int64_t Q, int k_in, int k_out, const uint32_t *ids,
                              const float *dists, const uint8_t *chi, uint32_t *out_ids,
                              float *out_dists, cudaStream_t s) {
    if (Q <= 0)
        return cudaSuccess;
    const int wpb = 8;
    postfilter_kernel<<<(unsigned)((Q + wpb - 1) / wpb), 32 * wpb, 0, s>>>(
        Q, k_in, k_out, ids, dists, chi, out_ids, out_dists);
    return cudaGetLastError();
}

cudaError_t launch_merge_topk(int P, int64_t Q, int k_in, int k_out, const uint32_t *ids,
                              const float *dists, const uint8_t *chi, const uint32_t *offsets,
                              uint32_t *out_ids, float *out_dists, uint8_t *out_chi,
                              cudaStream_t s) {
    if (Q <= 0)
        return cudaSuccess;
    MergeArgs a;
    a.P = P;
    a.k_in = k_in;
    a.k_out = k_out;
    a.Q = Q;
    a.ids = ids;
    a.dists = dists;
    a.chi = chi;
    a.offsets = offsets;
    a.out_ids = out_ids;
    a.out_dists = out_dists;
    a.out_chi = out_chi;
    const int hpl = (P + 31) / 32;
    const int wpb = 4;
    const size_t smem = sizeof(int) * 32 * hpl * wpb;
    cudaError_t e = cudaFuncSetAttribute(merge_topk_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    merge_topk_kernel<<<(unsigned)((Q + wpb - 1) / wpb), 32 * wpb, smem, s>>>(a, hpl);
    return cudaGetLastError();
}

// Recall (Eq. 3) of one query per warp: hits = |ids_q[0..kt) & truth_q| over the valid
// truth entries; acc[0] += hits / valid and acc[1] += 1 for queries with a valid entry.
// Ids within a row are distinct (search and brute force never repeat one), so counting
// the found ids that occur in the truth row counts the intersection.
__global__ void recall_kernel(const uint32_t *__restrict__ ids, int k,
                              const uint32_t *__restrict__ truth, int kt, int64_t Q,
                              double *acc) {
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= Q)
        return;
    const uint32_t *t = truth + q * kt;
    const uint32_t *f = ids + q * k;
    int hits = 0, valid = 0;
    for (int j = lane; j < kt; j += 32) {
        const uint32_t v = t[j];
        if (v == kNone)
            continue;
        ++valid;
        for (int i = 0; i < kt; ++i)
            hits += f[i] == v ? 1 : 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        hits += __shfl_xor_sync(FULL, hits, o);
        valid += __shfl_xor_sync(FULL, valid, o);
    }
    if (lane == 0 && valid > 0) {
        atomicAdd(acc, (double)hits / (double)valid);
        atomicAdd(acc + 1, 1.0);
    }
}

cudaError_t launch_recall(const uint32_t *ids, int k, const uint32_t *truth, int kt, int64_t Q,
                          double *acc, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess || Q <= 0)
        return e;
    const int wpb = 8;
    recall_kernel<<<(unsigned)((Q + wpb - 1) / wpb), 32 * wpb, 0, s>>>(ids, k, truth, kt, Q, acc);
    return cudaGetLastError();
}

}  // namespace nhq
