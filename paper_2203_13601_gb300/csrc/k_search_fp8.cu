// k_search_fp8.cu -- the search kernel with __nv_fp8_e4m3 scoring rows (the templates of
// k_search.cuh instantiated in a translation unit of their own).
#include "k_search.cuh"

namespace nhq {

cudaError_t launch_search_fp8(const SearchArgs &a, int ef_cap, int wpb, size_t smem,
                              int sm_count, cudaStream_t s) {
    return launch_dtype<__nv_fp8_e4m3>(a, a.X8, ef_cap, wpb, smem, sm_count, s);
}

}  // namespace nhq
