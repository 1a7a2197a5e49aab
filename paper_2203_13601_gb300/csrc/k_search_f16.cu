// k_search_f16.cu -- the search kernel with __half scoring rows (the templates of
// k_search.cuh instantiated in a translation unit of their own).
#include "k_search.cuh"

namespace nhq {

cudaError_t launch_search_f16(const SearchArgs &a, int ef_cap, int wpb, size_t smem,
                              int sm_count, cudaStream_t s) {
    return launch_dtype<__half>(a, a.Xf, ef_cap, wpb, smem, sm_count, s);
}

}  // namespace nhq
