// k_search_bf16.cu -- the search kernel with __nv_bfloat16 scoring rows (the templates of
// k_search.cuh instantiated in a translation unit of their own).
#include "k_search.cuh"

namespace nhq {

cudaError_t launch_search_bf16(const SearchArgs &a, int ef_cap, int wpb, size_t smem,
                              int sm_count, cudaStream_t s) {
    return launch_dtype<__nv_bfloat16>(a, a.Xh, ef_cap, wpb, smem, sm_count, s);
}

}  // namespace nhq
