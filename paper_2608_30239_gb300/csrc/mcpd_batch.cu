// The batched variants of the sampling kernel (mcpd_pairs.cuh with BATCH): many instances of
// uneven size in one persistent launch, tables read through the read-only cache from per-instance
// descriptors.  Compiled for any degree (rows padded to eight entries, thresholds indexed by
// (n+, n-)) and, for coupled classes whose instances all have one uniform degree from 3 to 8,
// with that degree as a compile-time constant (mask-indexed thresholds up to degree 6), as the
// single-instance kernels are: degrees 3 and 6 here, 4, 5, 7 and 8 in mcpd_batch_deg.cu, and the
// variants with the meeting cap and lags in mcpd_batch_ext.cu.  Separate translation units so
// that the library builds in parallel.
#include "mcpd_pairs.cuh"

namespace mcpd {

PairsKernelFn pick_batch(int coupled, int scan, int udeg, bool wide, bool ext) {
    if (coupled && ext) {
        if (udeg >= 3 && udeg <= 8) return pick_batch_ext_degree(udeg, wide);
        return wide ? pairs_kernel<true, false, true, 0, true, true> : pairs_kernel<true, false, true, 0, false, true>;
    }
    if (coupled) {
        switch (udeg) {
            case 3: return wide ? pairs_kernel<true, false, true, 3, true> : pairs_kernel<true, false, true, 3, false>;
            case 6: return wide ? pairs_kernel<true, false, true, 6, true> : pairs_kernel<true, false, true, 6, false>;
            case 4: case 5: case 7: case 8: return pick_batch_degree(udeg, wide);
            default: return wide ? pairs_kernel<true, false, true, 0, true> : pairs_kernel<true, false, true, 0, false>;
        }
    }
    if (scan == MCPD_SCAN_SYSTEMATIC)
        return wide ? pairs_kernel<false, true, true, 0, true> : pairs_kernel<false, true, true, 0, false>;
    return wide ? pairs_kernel<false, false, true, 0, true> : pairs_kernel<false, false, true, 0, false>;
}

int batch_kernel_degree(int coupled, int ext, int udeg) {
    (void)ext;                        // the capped / lagged variants have the same degree builds
    return (coupled && udeg >= 3 && udeg <= 8) ? udeg : 0;
}

}  // namespace mcpd
