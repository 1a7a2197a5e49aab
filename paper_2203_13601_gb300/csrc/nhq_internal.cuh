// nhq_internal.cuh -- device helpers and launch declarations shared by the
// library's translation units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "nhq.h"

namespace nhq {

constexpr uint32_t kNone = 0xFFFFFFFFu;                 // empty id / hash slot
constexpr unsigned long long kInfKey = ~0ull;           // key larger than any record
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;      // splitmix64 increment
constexpr int kMaxDegree = 64;
constexpr int kMaxK = 256;
constexpr int kMaxEf = 1024;
constexpr int kMaxCand = 128;

constexpr int kMaxAttr = 32;

// How the m attribute codes of an object share one u32 word: code j occupies bits
// [shift[j], shift[j] + width[j]).  Up to 4 attributes take a byte each (shift 8j, any
// code 0..255); more take the fewest bits that hold 0..maxc[j] + 1, where maxc[j] is the
// largest code of attribute j among the objects.  A query code above maxc[j] equals no
// object's code and is stored as maxc[j] + 1, so chi on words equals chi on codes.
struct AttrLayout {
    int m = 0;
    uint8_t shift[kMaxAttr] = {};
    uint8_t width[kMaxAttr] = {};
    uint8_t maxc[kMaxAttr] = {};
    uint8_t amax[kMaxAttr] = {};  // the largest code of each attribute among the objects
    uint32_t hi = 0;  // the top bit of every field
    uint32_t lo = 0;  // the other bits of every field
};

// Fusion-distance weights (Eq. 6) and the attribute layout, as the kernels see them.
struct Fusion {
    int mode;  // nhq_weight_mode
    float wv, wl;
    int m;
    uint32_t hi, lo;  // AttrLayout::hi / lo
    uint8_t shift[kMaxAttr], maxc[kMaxAttr], amax[kMaxAttr];
    int wild;  // 1: a query code 255 leaves its attribute unconstrained (queries only)
};

// ---- splitmix64 (Vigna): the finaliser and the j-th output of a stream ----
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t splitmix_at(uint64_t s0, uint64_t j) {
    return mix64(s0 + (j + 1) * kGolden);
}

// chi (Eq. 4-5) on packed attribute words: the number of fields in which a and b differ.
// In x = a ^ b, adding the low bits of a field to the field's low-bit mask carries into
// the field's top bit iff a low bit is set, and never past it; so the top bit of
// ((x & lo) + lo) | x is set exactly for the nonzero fields.
__host__ __device__ __forceinline__ int chi_packed(uint32_t a, uint32_t b, uint32_t hi,
                                                   uint32_t lo) {
    const uint32_t x = a ^ b;
#ifdef __CUDA_ARCH__
    return __popc((((x & lo) + lo) | x) & hi);
#else
    return __builtin_popcount((((x & lo) + lo) | x) & hi);
#endif
}

// the top bit of field j (w.hi has one bit per field, and field j ends where j + 1 starts)
__host__ __device__ __forceinline__ uint32_t field_hi(const Fusion &w, int j) {
    const uint32_t next = j + 1 < w.m ? w.shift[j + 1] : 32u;
    return w.hi & (next >= 32u ? 0xFFFFFFFFu : ((1u << next) - 1u)) & ~((1u << w.shift[j]) - 1u);
}

// A query's packed word under the layout in w (codes above maxc[j] become maxc[j] + 1);
// *hi = the top bits of the fields the query constrains (w.hi less the fields whose code
// is the wildcard 255 when w.wild is set), to pass to chi_packed in place of w.hi.
__host__ __device__ __forceinline__ uint32_t pack_query_word(const uint8_t *qa, const Fusion &w,
                                                            uint32_t *hi) {
    uint32_t word = 0, open = 0;
    for (int j = 0; j < w.m; ++j) {
        const uint32_t v = qa[j];
        if (w.wild && v == 255u) {
            open |= field_hi(w, j);
            continue;
        }
        const uint32_t c = v <= w.maxc[j] ? v : (uint32_t)w.maxc[j] + 1u;
        word |= c << w.shift[j];
    }
    *hi = w.hi & ~open;
    return word;
}

// Gamma (Eq. 6) from delta and chi, each operation rounded once (round-to-nearest),
// so it equals the canonical f32 evaluation of the formula.
__device__ __forceinline__ float fusion_gamma(float delta, int chi, const Fusion &w) {
    // chi = 0: the attribute term is +0 and delta >= 0, so the sum is the vector term
    // exactly (this skips the rounded division of the proportional form)
    if (chi == 0 && w.mode != NHQ_W_HARMONIC)
        return w.mode == NHQ_W_CONSTANT ? __fmul_rn(w.wv, delta) : delta;
    if (w.mode == NHQ_W_PROPORTIONAL) {
        float wl = __fdiv_rn(delta, (float)w.m);
        return __fadd_rn(delta, __fmul_rn(wl, (float)chi));
    }
    if (w.mode == NHQ_W_CONSTANT)
        return __fadd_rn(__fmul_rn(w.wv, delta), __fmul_rn(w.wl, (float)chi));
    if (w.mode == NHQ_W_HARMONIC) {  // Sec. 6.5 curves i (w.wl = 0) and ii (w.wl = c)
        const float h = w.wl > 0.f ? (chi == 0 ? 1.f : __fmul_rn(w.wl, (float)chi)) : (float)chi;
        const float den = __fadd_rn(delta, h);
        return den == 0.f ? 0.f : __fdiv_rn(__fmul_rn(__fmul_rn(2.f, delta), h), den);
    }
    return chi == 0 ? delta : __int_as_float(0x7f800000);  // NHQ_W_FILTER
}

// A record (Gamma, id) as one u64 whose unsigned order is the lexicographic
// order on (Gamma, id) for Gamma >= 0 (+inf included).  Bit 0 is a free flag.
__device__ __forceinline__ unsigned long long make_key(float g, uint32_t id) {
    return ((unsigned long long)__float_as_uint(g) << 32) | ((unsigned long long)id << 1);
}
__device__ __forceinline__ uint32_t key_id(unsigned long long k) {
    return (uint32_t)(k >> 1) & 0x7FFFFFFFu;
}
__device__ __forceinline__ float key_gamma(unsigned long long k) {
    return __uint_as_float((uint32_t)(k >> 32));
}

// Logit of the learned early-stop model for the warp-uniform features f (every
// lane passes the same f): lane owns hidden units lane and lane + 32; fp16
// weights, f32 accumulation, butterfly sum over the warp.
__device__ __forceinline__ float mlp_logit_warp(const __half *w, const float *f, int lane) {
    constexpr int I = NHQ_MLP_INPUTS, H = NHQ_MLP_HIDDEN;
    float acc = 0.f;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const int j = lane + 32 * hh;
        float z = __half2float(w[I * H + j]);
#pragma unroll
        for (int i = 0; i < I; ++i)
            z = fmaf(__half2float(w[i * H + j]), f[i], z);
        acc = fmaf(__half2float(w[I * H + H + j]), fmaxf(z, 0.f), acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    return acc + __half2float(w[I * H + 2 * H]);
}

}  // namespace nhq

// ---------------------------------------------------------------- host side
struct nhq_index {
    int64_t N = 0;
    int d = 0, m = 0, R = 0;
    int xstride = 0;  // elements per stored row (d rounded up to a multiple of 16)
    nhq_weights w{};
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;
    float *X = nullptr;            // [N][xstride] f32
    __nv_bfloat16 *Xh = nullptr;   // [N][xstride] bf16 copy (built on first BF16 search)
    __nv_fp8_e4m3 *X8 = nullptr;   // [N][xstride] fp8 e4m3 copy (built on first FP8 search)
    __half *Xf = nullptr;          // [N][xstride] f16 copy (built on first F16 search)
    nhq::AttrLayout layout;        // how attr packs the m codes
    uint32_t *attr = nullptr;      // [N] packed attributes
    uint32_t *nbr = nullptr;       // [N][R] adjacency, kNone padded
    uint32_t *nbr_attr = nullptr;  // [N][R] packed attributes of each neighbour
    __nv_bfloat16 *Xk = nullptr;  // [N][kpad] bf16 rows for the tensor-core candidate build
    float *normk = nullptr;       // [N] squared norms of those rows
    int kpad = 0;                 // d rounded up to a multiple of 64
    uint32_t *attr_sorted = nullptr;  // [N] packed attributes, ascending (stable radix sort)
    uint32_t *id_sorted = nullptr;    // [N] object ids in that order
    // entry cells (nhq_index_build_cells): E centroid rows, the cell of every object and
    // the objects sorted by (attribute word, cell)
    int E = 0;
    float *cent = nullptr;                   // [E][xstride]
    float *centT = nullptr;                  // [d][E] the centroids as columns
    float *cnh = nullptr;                    // [E] -|c|^2 / 2
    uint32_t *cell = nullptr;                // [N]
    unsigned long long *cell_key = nullptr;  // [N] (attribute word << 16 | cell), ascending
    uint32_t *cell_id = nullptr;             // [N] object ids in that order
    // scratch arena (grown on demand, owned by the index)
    void *scratch = nullptr;
    size_t scratch_bytes = 0;
};

namespace nhq {

// a byte per attribute (m <= 4), the layout of nhq_pack_attributes
AttrLayout byte_layout(int m);
// the layout of m attributes whose largest codes are maxc[0..m); false if the fields
// need more than 32 bits
bool compact_layout(int m, const uint8_t *maxc, AttrLayout *out);
nhq::Fusion make_fusion(const nhq_weights &w, const AttrLayout &L);
nhq::Fusion make_fusion(const nhq_weights &w, int m);  // byte layout
nhq_status report_error(nhq_status s, const char *message);  // nhq_api.cu
// NHQ_OK, or NHQ_ERR_ARG with the message set, by the weight rules of nhq_brute_force
nhq_status validate_weights(const nhq_weights &w, bool allow_filter);  // nhq_api.cu

// k_util.cu
cudaError_t launch_pack_attributes(const uint8_t *a, int64_t n, const AttrLayout &L,
                                   uint32_t *out, cudaStream_t s);
// query words under the layout in w and, when hi_out is not null, each query's chi mask
cudaError_t launch_pack_queries(const uint8_t *a, int64_t n, const Fusion &w, uint32_t *out,
                                uint32_t *hi_out, cudaStream_t s);
// out[0..kMaxAttr) = the largest code of each of the m attributes over n rows
cudaError_t launch_attr_max(const uint8_t *a, int64_t n, int m, unsigned int *out,
                            cudaStream_t s);
cudaError_t launch_copy_rows(const float *src, int64_t N, int d, int xstride, float *dst,
                             int *nonfinite_flag, cudaStream_t s);
cudaError_t launch_rows_to_bf16(const float *src, int64_t n_elems, __nv_bfloat16 *dst, cudaStream_t s);
cudaError_t launch_rows_to_fp8(const float *src, int64_t n_elems, __nv_fp8_e4m3 *dst, cudaStream_t s);
cudaError_t launch_rows_to_f16(const float *src, int64_t n_elems, __half *dst, cudaStream_t s);
// rows of f16 / bf16 (dtype NHQ_F16 / NHQ_BF16) widened into the padded f32 layout
cudaError_t launch_copy_rows_typed(const void *src, int dtype, int64_t N, int d, int xstride,
                                   float *dst, int *nonfinite_flag, cudaStream_t s);
cudaError_t launch_gather_nbr_attr(const uint32_t *nbr, const uint32_t *attr, int64_t N, int R,
                                   uint32_t *out, int *bad, cudaStream_t s);

// k_bruteforce.cu -- exact top-k by (Gamma, id); also the exact candidate sets
struct TopkArgs {
    const float *X;
    int xstride;
    int d;
    int64_t N;
    const uint32_t *attr;
    const float *Q;
    int qstride;
    const uint32_t *qattr;
    const uint32_t *qhi;  // [nq] per-query chi masks (wildcards), or null: w.hi
    int64_t nq;
    int k;
    int exclude_self;  // query q is object q (candidate sets)
    Fusion w;
    uint32_t *ids;     // [nq][k]
    float *dists;      // [nq][k] or null
    uint8_t *chi;      // [nq][k] or null
};
size_t topk_scratch_bytes(const TopkArgs &a, int sm_count);
cudaError_t launch_topk(const TopkArgs &a, void *scratch, size_t scratch_bytes, int sm_count,
                        cudaStream_t s);

// k_edge.cu
// landing-zone selection for the vertices rows[b] (or row0 + b), candidate row b -> out row b
cudaError_t launch_edge_select_rows(const nhq_index *ix, const uint32_t *cand, int L, int R,
                                    const uint32_t *rows, int64_t row0, int64_t count,
                                    uint32_t *out, cudaStream_t s);
// incremental build: the per-wave kernels of k_nsw.cu
int nsw_seed_count();
cudaError_t launch_nsw_seeds(int64_t s, int64_t B, uint64_t seed, uint32_t *seeds, cudaStream_t st);
cudaError_t launch_nsw_queries(const nhq_index *ix, int64_t s, int64_t B, float *q, uint8_t *qa,
                               cudaStream_t st);
cudaError_t launch_nsw_attr_seeds(const nhq_index *ix, int64_t s, int64_t B, uint64_t seed,
                                  uint32_t *seeds, cudaStream_t st);
size_t nsw_sort_scratch_bytes(int64_t n);
cudaError_t launch_nsw_pairs(const uint32_t *rows, int R, int64_t s, int64_t B,
                             unsigned long long *keys, unsigned long long *sorted, void *tmp,
                             size_t tmp_bytes, uint32_t *seg_start, int *nseg_dev,
                             cudaStream_t st);
cudaError_t launch_nsw_reverse(const unsigned long long *sorted, int64_t n,
                               const uint32_t *seg_start, int nseg, const uint32_t *nbr, int R,
                               int cap, uint32_t *U, uint32_t *cand, cudaStream_t st);
cudaError_t launch_nsw_install(const uint32_t *src, const uint32_t *list, int64_t row0,
                               int64_t count, int R, const uint32_t *attr, uint32_t *nbr,
                               uint32_t *nbr_attr, cudaStream_t st);
cudaError_t launch_edge_select(const nhq_index *ix, const uint32_t *cand, int L, int R,
                               uint32_t *out, cudaStream_t s);
size_t reverse_scratch_bytes(int64_t N, int R);
cudaError_t launch_reverse_candidates(const uint32_t *nbr, int64_t N, int R, int cap,
                                      uint32_t *out, void *scratch, cudaStream_t s);

// k_search.cu
struct SearchArgs {
    const float *X;
    const __nv_bfloat16 *Xh;
    const __nv_fp8_e4m3 *X8;
    const __half *Xf;
    int xstride;
    int d;
    int64_t N;
    const uint32_t *attr;
    const uint32_t *nbr;
    const uint32_t *nbr_attr;
    int R;
    Fusion w;
    const float *Q;
    int qstride;
    const uint8_t *qattr;  // [nq][m] u8
    int64_t nq;
    const int32_t *k_arr;  // per-query k or null
    const int32_t *ef_arr;
    int k, ef;             // uniform values (or maxima when arrays are given)
    int k_out;             // row width of the outputs
    int h;
    uint64_t seed;
    int max_iters;
    int vec_dtype;
    int rerank;
    uint32_t *ids;
    float *dists;
    uint8_t *chi;
    int32_t *status;
    int32_t *ndc;
    int32_t *expansions;
    const uint32_t *seeds;  // [nq][n_seeds] given seed ids or null (random stream)
    int n_seeds;
    const uint32_t *order;  // [nq] processing order of the queries, or null (index order)
    // learned early stop: fp16 weights (null = off), logit threshold, schedule
    const __half *stop_w16;
    float stop_logit;
    int stop_min, stop_every;  // stop_every == 0: neither model nor traces
    // traces (null = off): features [cap][8], top-k hash and query row per record
    float *tr_feat;
    unsigned long long *tr_hash;
    int32_t *tr_q;
    unsigned int *tr_count;
    int64_t tr_cap;
    unsigned long long *tr_final;  // [nq] top-k hash at the end of each query
    unsigned long long *counter;  // scratch work counter (zeroed by the launcher)
    int warps_per_block;
    int hash_bits;
    int wpq;  // warps per query (1, 2 or 4): the group shares each expansion's distance passes
    int tile_rows;  // rows per team of 8 lanes and distance pass (2 or 4)
};
size_t search_scratch_bytes(int64_t nq);
cudaError_t launch_attribute_sort(const uint32_t *attr, int64_t N, uint32_t *attr_sorted,
                                  uint32_t *id_sorted, void *scratch, size_t scratch_bytes,
                                  cudaStream_t s);
size_t attribute_sort_scratch_bytes(int64_t N);
// k_knn_tc.cu
int knn_tc_kmax();
// Xk/norms rows in the order perm (sorted position -> original id); the candidate
// kernel takes attributes in the same order and writes rows and ids in original ids
cudaError_t launch_knn_tc_prepare(const float *X, int xstride, int d, int64_t N, int kpad,
                                  const uint32_t *perm, __nv_bfloat16 *Xk, float *norms,
                                  cudaStream_t s);
cudaError_t launch_knn_tc(const __nv_bfloat16 *Xk, int kpad, const float *norms,
                          const uint32_t *attr, const uint32_t *perm, int64_t N, const Fusion &w,
                          int K, uint32_t *ids, float *dists, int *err, cudaStream_t s);

// k_mlp.cu
cudaError_t launch_mlp_to_half(const float *params, __half *w16, cudaStream_t s);
cudaError_t launch_trace_labels(const unsigned long long *hash, const int32_t *tq,
                                const unsigned long long *final_hash, int64_t n, uint8_t *lab,
                                cudaStream_t s);
cudaError_t mlp_forward(const float *params, const float *X, int64_t n, float *logits,
                        cudaStream_t s);
cudaError_t mlp_grad(const float *params, const float *X, const float *y, int64_t n,
                     int64_t total, float *g, float *loss, cudaStream_t s);
cudaError_t mlp_train(float *params, const float *X, const float *y, int64_t n, int epochs,
                      int batch, float lr, cudaStream_t s);

// Seeds of NHQ_SEED_ATTRIBUTE into seeds[nq][32] (rows padded with kNone).
cudaError_t launch_attribute_seeds(const SearchArgs &a, const uint32_t *attr_sorted,
                                   const uint32_t *id_sorted, uint32_t *seeds, uint8_t *bucket,
                                   cudaStream_t s);
// Seeds of NHQ_SEED_ATTRIBUTE_NEAR (one warp per query), with the same cost buckets.
cudaError_t launch_attribute_near_seeds(const SearchArgs &a, const uint32_t *attr_sorted,
                                        const uint32_t *id_sorted, uint32_t *seeds,
                                        uint8_t *bucket, cudaStream_t s);
// order[0..nq) = the queries by ascending bucket (each bucket in any order)
cudaError_t launch_query_order(const uint8_t *bucket, int64_t nq, uint32_t *order,
                               cudaStream_t s);
int nnd_kmax();
size_t nnd_scratch_bytes(int64_t N, int K);
cudaError_t launch_nndescent(const float *X, int xstride, int64_t N, const uint32_t *attr,
                             const Fusion &w, int K, int max_iters, double delta, uint64_t seed,
                             void *scratch, uint32_t *ids, float *dists, int *iters_done,
                             cudaStream_t s);
cudaError_t launch_postfilter(int64_t Q, int k_in, int k_out, const uint32_t *ids,
                              const float *dists, const uint8_t *chi, uint32_t *out_ids,
                              float *out_dists, cudaStream_t s);
cudaError_t launch_merge_topk(int P, int64_t Q, int k_in, int k_out, const uint32_t *ids,
                              const float *dists, const uint8_t *chi, const uint32_t *offsets,
                              uint32_t *out_ids, float *out_dists, uint8_t *out_chi,
                              cudaStream_t s);
cudaError_t launch_search(SearchArgs a, void *scratch, int sm_count, size_t smem_optin,
                          cudaStream_t s);
// the search launch for one scoring type (k_search_<type>.cu), sized by launch_search
cudaError_t launch_search_f32(const SearchArgs &a, int ef_cap, int wpb, size_t smem,
                              int sm_count, cudaStream_t s);
cudaError_t launch_search_bf16(const SearchArgs &a, int ef_cap, int wpb, size_t smem,
                               int sm_count, cudaStream_t s);
cudaError_t launch_search_fp8(const SearchArgs &a, int ef_cap, int wpb, size_t smem,
                              int sm_count, cudaStream_t s);
cudaError_t launch_search_f16(const SearchArgs &a, int ef_cap, int wpb, size_t smem,
                              int sm_count, cudaStream_t s);
// k_entry.cu -- entry cells and the entry model
int64_t entry_param_count(int d, int E);
cudaError_t launch_gather_centroids(const float *X, int xstride, int64_t N, int E,
                                    const uint32_t *attr, float *cent, uint32_t *cattr,
                                    cudaStream_t s);
size_t cell_sort_scratch_bytes(int64_t N);
cudaError_t launch_cell_sort(const uint32_t *attr, const uint32_t *cell, int64_t N,
                             unsigned long long *key_sorted, uint32_t *id_sorted, void *scratch,
                             size_t scratch_bytes, cudaStream_t s);
cudaError_t launch_entry_to_half(const float *params, int64_t n, __half *w16, cudaStream_t s);
cudaError_t launch_cell_seeds(const SearchArgs &a, const uint32_t *attr_sorted,
                              const uint32_t *id_sorted, const unsigned long long *cell_key,
                              const uint32_t *cell_id, int E, int T, const float *scores,
                              int32_t *cells_out, uint32_t *seeds, uint8_t *bucket,
                              cudaStream_t s);
// cT[d][E] = the centroid rows as columns, nh[E] = -|c|^2 / 2
cudaError_t launch_centroid_columns(const float *cent, int xstride, int d, int E, float *cT,
                                    float *nh, cudaStream_t s);
// out[n][E] = q.c - |c|^2 / 2 (largest for the nearest centroid)
cudaError_t launch_entry_scores_nearest(const float *cT, const float *nh, int d, int E,
                                        const float *Q, int64_t qstride, int64_t n, float *out,
                                        cudaStream_t s);
// out[n][E] = the entry model's logits (fp16 weights w16, the f32 scale params[0]);
// hidden[n][64] is working memory
cudaError_t launch_entry_scores_learned(const __half *w16, const float *params, int d, int E,
                                        const float *Q, int64_t qstride, int64_t n,
                                        float *hidden, float *out, cudaStream_t s);
cudaError_t launch_entry_labels(const uint32_t *ids, int k, int64_t n, const uint32_t *cell,
                                int64_t N, int32_t *labels, cudaStream_t s);
size_t entry_train_chunk_bytes(int B, int E);
cudaError_t entry_grad_accumulate(const float *P, int d, int E, const float *X,
                                  const int32_t *y, int64_t n, int64_t total, int B, float *G,
                                  float *loss, void *work, cudaStream_t s);
cudaError_t launch_entry_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr,
                              float c1, float c2, cudaStream_t s);
// acc[0] = sum over queries with a valid truth entry of |ids & truth| / valid, acc[1] = their count
cudaError_t launch_recall(const uint32_t *ids, int k, const uint32_t *truth, int kt, int64_t Q,
                          double *acc, cudaStream_t s);

}  // namespace nhq
