// Batched sampling-kernel variants for coupled classes whose instances all have one uniform
// degree of 4, 5, 7 or 8 (degrees 3 and 6 are in mcpd_batch.cu): the degree is a compile-time
// constant (and, up to degree 6, thresholds are mask-indexed), as in the single-instance kernels.
// A separate translation unit so that the library builds in parallel.
#include "mcpd_pairs.cuh"

namespace mcpd {

PairsKernelFn pick_batch_degree(int udeg, bool wide) {
    switch (udeg) {
        case 4: return wide ? pairs_kernel<true, false, true, 4, true> : pairs_kernel<true, false, true, 4, false>;
        case 5: return wide ? pairs_kernel<true, false, true, 5, true> : pairs_kernel<true, false, true, 5, false>;
        case 7: return wide ? pairs_kernel<true, false, true, 7, true> : pairs_kernel<true, false, true, 7, false>;
        case 8: return wide ? pairs_kernel<true, false, true, 8, true> : pairs_kernel<true, false, true, 8, false>;
        default: return nullptr;
    }
}

}  // namespace mcpd
