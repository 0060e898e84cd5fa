// The kernels of cliffs_step.cu for grids with open (radiating) outer edges: the OPEN
// instantiations, in a translation unit of their own so that both compile in parallel and
// the reflecting-edge kernels carry none of the open-edge code.
#include "step_kernels.cuh"

namespace cliffs {

#define CLIFFS_V2O(K, ...) (const void*)K<false, false, __VA_ARGS__>, (const void*)K<true, false, __VA_ARGS__>, \
                           (const void*)K<false, true, __VA_ARGS__>, (const void*)K<true, true, __VA_ARGS__>

const void* fused_kernel_open(int v) {
    static const void* const t[16] = {CLIFFS_V2O(k_step_fused, false, false, true), CLIFFS_V2O(k_step_fused, true, false, true),
                                      CLIFFS_V2O(k_step_fused, false, true, true), CLIFFS_V2O(k_step_fused, true, true, true)};
    return t[v];
}
const void* batch_kernel_open(int v) {
    static const void* const t[8] = {CLIFFS_V2O(k_batch, false, true, false), CLIFFS_V2O(k_batch, true, true, false)};
    return t[v];
}
const void* xsweep_kernel_open(int v) {
    static const void* const t[8] = {CLIFFS_V2O(k_xsweep, false, true), CLIFFS_V2O(k_xsweep, true, true)};
    return t[v];
}
const void* ysweep_kernel_open(int v) {
    static const void* const t[8] = {CLIFFS_V2O(k_ysweep, false, true), CLIFFS_V2O(k_ysweep, true, true)};
    return t[v];
}

}  // namespace cliffs
