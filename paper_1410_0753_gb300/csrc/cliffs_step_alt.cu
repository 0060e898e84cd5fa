// The persistent batched kernel for the alternating sweep order (ALT: y first on the odd
// steps), with reflecting and with open outer edges; in a translation unit of its own so
// that it compiles in parallel with the others.
#include "step_kernels.cuh"

namespace cliffs {

#define CLIFFS_V2A(K, ...) (const void*)K<false, false, __VA_ARGS__>, (const void*)K<true, false, __VA_ARGS__>, \
                           (const void*)K<false, true, __VA_ARGS__>, (const void*)K<true, true, __VA_ARGS__>

// index: spherical +1, friction +2, eq. (solver1) +4, open edges +8
const void* batch_kernel_alt(int v) {
    static const void* const t[16] = {CLIFFS_V2A(k_batch, false, false, true), CLIFFS_V2A(k_batch, true, false, true),
                                      CLIFFS_V2A(k_batch, false, true, true), CLIFFS_V2A(k_batch, true, true, true)};
    return t[v];
}

}  // namespace cliffs
