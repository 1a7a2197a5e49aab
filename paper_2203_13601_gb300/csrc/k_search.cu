// k_search.cu -- joint pruning (Alg. 2) on the composite index, ef-bounded,
// with the two-stage "random TOGG" routing of Sec. 4.2 / Sec. 5.2.
//
// One warp owns one query at a time; warps pull query indices from a global
// counter (persistent grid sized to the device).  Per warp, shared memory holds
//   pool  [ef]  u64 records (Gamma bits << 32 | id << 1 | expanded), sorted
//   cand  [64]  candidate records of the current expansion
//   hash  [H]   visited filter (open addressing)
//   qv    [d]   the query vector
// Each expansion: take the smallest unexpanded record, read the parent's
// neighbour ids and their attribute words (one coalesced row each, issued one
// expansion ahead), drop already-evaluated ids through the visited filter,
// prune by the attribute lower bound w_l * chi when the weights are constant
// (a candidate whose bound already exceeds the pool's last record cannot
// enter), accumulate squared distances with teams of 8 lanes (128-bit loads,
// shuffle reduction), finish every candidate's Gamma in one warp-wide step
// (lane j holds candidate j's record in a register), and merge the survivors
// into the pool (rank by broadcast compares for up to 8, warp bitonic sort
// beyond).
//
// The pool after every expansion equals the serial algorithm's: inserting a
// batch and keeping the ef smallest equals inserting the batch one record at a
// time.  When the visited filter fills it is rebuilt from the pool's ids; an
// id forgotten that way either is in the pool (and re-inserted) or was rejected
// or evicted while the pool was full, so re-evaluating it rejects it again (its
// record is above the pool's last record, which only decreases).
//
// The kernel templates live in k_search.cuh; k_search_<type>.cu instantiate them per
// scoring type, and this file sizes the launch and dispatches to them.
#include "k_search.cuh"

namespace nhq {

// work counter | seeds [nq][32] u32 | order [nq] u32 | buckets [nq] u8
size_t search_scratch_bytes(int64_t nq) {
    return 256 + sizeof(uint32_t) * 33 * (size_t)nq + (size_t)nq + 256;
}

cudaError_t launch_search(SearchArgs a, void *scratch, int sm_count, size_t smem_optin,
                          cudaStream_t s) {
    if (a.nq <= 0)
        return cudaSuccess;
    a.counter = reinterpret_cast<unsigned long long *>(scratch);
    cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess)
        return e;
    const int ef_cap = (a.ef + 31) & ~31;
    if (a.hash_bits <= 0)
        a.hash_bits = auto_hash_bits(ef_cap, a.R);
    if ((1 << a.hash_bits) < 2 * (ef_cap + a.R) + 64)
        return cudaErrorInvalidValue;
    const WarpLayout L = warp_layout(ef_cap, a.hash_bits, a.xstride);
    if (a.wpq < 1)
        a.wpq = 1;
    if (a.wpq != 1 && a.wpq != 2 && a.wpq != 4)
        return cudaErrorInvalidValue;
    int wpb = a.warps_per_block > 0 ? a.warps_per_block : 8;
    if (wpb < a.wpq)
        wpb = a.wpq;
    // one shared-memory area per group of wpq warps
    while (wpb > a.wpq && L.total * (wpb / a.wpq) + 2048 > smem_optin)
        wpb >>= 1;
    if (L.total * (wpb / a.wpq) + 2048 > smem_optin || wpb % a.wpq != 0)
        return cudaErrorInvalidValue;
    const size_t smem = L.total * (wpb / a.wpq) + (a.stop_w16 != nullptr ? 2 * 656 : 0);
    if (a.vec_dtype == NHQ_VEC_BF16)
        return launch_search_bf16(a, ef_cap, wpb, smem, sm_count, s);
    if (a.vec_dtype == NHQ_VEC_FP8E4M3)
        return launch_search_fp8(a, ef_cap, wpb, smem, sm_count, s);
    if (a.vec_dtype == NHQ_VEC_F16)
        return launch_search_f16(a, ef_cap, wpb, smem, sm_count, s);
    return launch_search_f32(a, ef_cap, wpb, smem, sm_count, s);
}

}  // namespace nhq
