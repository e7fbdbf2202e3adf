// The recording variants of the sampling kernel: the single-instance kernel (mcpd_pairs.cuh),
// coupled and uncoupled, compiled with TRACE, which also writes, for the first replications of every
// traced slot, the meeting time, the completion time and per draw the site and which chains flipped
// (MCPD_FETCH_TRACE_REC).  They
// exist for the trajectory parity tests against the CPU oracle; a plan launches them only when
// params.trace_steps > 0, and the production variants compile none of the recording.  A separate
// translation unit so that the library builds in parallel.
#include "mcpd_pairs.cuh"

namespace mcpd {
namespace {

using TraceFn = void (*)(const KParams, const BParams);

TraceFn pick_trace(int coupled, int scan, int udeg, bool ext) {
    if (!coupled && scan == MCPD_SCAN_SYSTEMATIC) {
        switch (udeg) {
            case 3: return pairs_kernel<false, true, false, 3, false, false, true>;
            case 4: return pairs_kernel<false, true, false, 4, false, false, true>;
            case 5: return pairs_kernel<false, true, false, 5, false, false, true>;
            case 6: return pairs_kernel<false, true, false, 6, false, false, true>;
            default: return pairs_kernel<false, true, false, 0, false, false, true>;
        }
    }
    if (!coupled) {
        switch (udeg) {
            case 3: return pairs_kernel<false, false, false, 3, false, false, true>;
            case 4: return pairs_kernel<false, false, false, 4, false, false, true>;
            case 5: return pairs_kernel<false, false, false, 5, false, false, true>;
            case 6: return pairs_kernel<false, false, false, 6, false, false, true>;
            default: return pairs_kernel<false, false, false, 0, false, false, true>;
        }
    }
    if (ext) {
        switch (udeg) {
            case 3: return pairs_kernel<true, false, false, 3, false, true, true>;
            case 4: return pairs_kernel<true, false, false, 4, false, true, true>;
            case 5: return pairs_kernel<true, false, false, 5, false, true, true>;
            case 6: return pairs_kernel<true, false, false, 6, false, true, true>;
            case 7: return pairs_kernel<true, false, false, 7, false, true, true>;
            case 8: return pairs_kernel<true, false, false, 8, false, true, true>;
            default: return pairs_kernel<true, false, false, 0, false, true, true>;
        }
    }
    switch (udeg) {
        case 3: return pairs_kernel<true, false, false, 3, false, false, true>;
        case 4: return pairs_kernel<true, false, false, 4, false, false, true>;
        case 5: return pairs_kernel<true, false, false, 5, false, false, true>;
        case 6: return pairs_kernel<true, false, false, 6, false, false, true>;
        case 7: return pairs_kernel<true, false, false, 7, false, false, true>;
        case 8: return pairs_kernel<true, false, false, 8, false, false, true>;
        default: return pairs_kernel<true, false, false, 0, false, false, true>;
    }
}

}  // namespace

int set_trace_smem(size_t bytes) {
    for (int c = 0; c <= 1; ++c)
        for (int sc : {MCPD_SCAN_SCORE, MCPD_SCAN_SYSTEMATIC}) {
            if (c && sc == MCPD_SCAN_SYSTEMATIC) continue;
            for (int ext = 0; ext <= c; ++ext)
                for (int ud = 0; ud <= 8; ++ud) {
                    if (ud == 1 || ud == 2 || (!c && ud > kMaskDeg)) continue;
                    if (cudaFuncSetAttribute(pick_trace(c, sc, ud, ext != 0), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(bytes)) != cudaSuccess)
                        return MCPD_ECUDA;
                }
        }
    return MCPD_OK;
}

int launch_pairs_trace(const KParams &kp, int grid, int block, size_t smem, void *stream) {
    if (!kp.trace_rec || kp.trace_stride <= 0) return MCPD_EINVAL;
    const BParams none{};
    const bool ext = kp.coupled && (kp.capped != 0 || kp.lag > 1);
    pick_trace(kp.coupled, kp.scan, kp.udeg, ext)<<<grid, block, smem, static_cast<cudaStream_t>(stream)>>>(kp, none);
    return cudaGetLastError() == cudaSuccess ? MCPD_OK : MCPD_ECUDA;
}

}  // namespace mcpd
