// k_search_f32.cu -- the search kernel with float scoring rows (the templates of
// k_search.cuh instantiated in a translation unit of their own).
#include "k_search.cuh"

namespace nhq {

cudaError_t launch_search_f32(const SearchArgs &a, int ef_cap, int wpb, size_t smem,
                              int sm_count, cudaStream_t s) {
    return launch_dtype<float>(a, a.X, ef_cap, wpb, smem, sm_count, s);
}

}  // namespace nhq
