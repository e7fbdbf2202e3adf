// The batched variants of the sampling kernel (mcpd_pairs.cuh with BATCH): many instances of
// uneven size in one persistent launch, tables read through the read-only cache from per-instance
// descriptors.  Compiled for any degree (rows padded to eight entries, thresholds indexed by
// (n+, n-)) and, for coupled classes whose instances all have uniform degree 3 or 6, with that
// degree as a compile-time constant and mask-indexed thresholds, as the single-instance kernels
// are.  A separate translation unit so that the library builds in parallel.
#include "mcpd_pairs.cuh"

namespace mcpd {

PairsKernelFn pick_batch(int coupled, int scan, int udeg, bool wide, bool ext) {
    if (coupled && ext)
        return wide ? pairs_kernel<true, false, true, 0, true, true> : pairs_kernel<true, false, true, 0, false, true>;
    if (coupled) {
        switch (udeg) {
            case 3: return wide ? pairs_kernel<true, false, true, 3, true> : pairs_kernel<true, false, true, 3, false>;
            case 6: return wide ? pairs_kernel<true, false, true, 6, true> : pairs_kernel<true, false, true, 6, false>;
            default: return wide ? pairs_kernel<true, false, true, 0, true> : pairs_kernel<true, false, true, 0, false>;
        }
    }
    if (scan == MCPD_SCAN_SYSTEMATIC)
        return wide ? pairs_kernel<false, true, true, 0, true> : pairs_kernel<false, true, true, 0, false>;
    return wide ? pairs_kernel<false, false, true, 0, true> : pairs_kernel<false, false, true, 0, false>;
}

int batch_kernel_degree(int coupled, int ext, int udeg) {
    return (coupled && !ext && (udeg == 3 || udeg == 6)) ? udeg : 0;
}

}  // namespace mcpd
