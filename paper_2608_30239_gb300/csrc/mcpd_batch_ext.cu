// Batched sampling-kernel variants with the meeting cap and lags above 1 (EXT) for coupled
// classes whose instances all have one uniform degree from 3 to 8: the degree is a compile-time
// constant (and, up to degree 6, thresholds are mask-indexed).  A separate translation unit so
// that the library builds in parallel.
#include "mcpd_pairs.cuh"

namespace mcpd {

PairsKernelFn pick_batch_ext_degree(int udeg, bool wide) {
    switch (udeg) {
        case 3: return wide ? pairs_kernel<true, false, true, 3, true, true> : pairs_kernel<true, false, true, 3, false, true>;
        case 4: return wide ? pairs_kernel<true, false, true, 4, true, true> : pairs_kernel<true, false, true, 4, false, true>;
        case 5: return wide ? pairs_kernel<true, false, true, 5, true, true> : pairs_kernel<true, false, true, 5, false, true>;
        case 6: return wide ? pairs_kernel<true, false, true, 6, true, true> : pairs_kernel<true, false, true, 6, false, true>;
        case 7: return wide ? pairs_kernel<true, false, true, 7, true, true> : pairs_kernel<true, false, true, 7, false, true>;
        case 8: return wide ? pairs_kernel<true, false, true, 8, true, true> : pairs_kernel<true, false, true, 8, false, true>;
        default: return nullptr;
    }
}

}  // namespace mcpd
