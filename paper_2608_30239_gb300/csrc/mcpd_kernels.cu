// CUDA kernels (sm_103a) for coupled score-weighted Markov chain pool decoding.
//
// pairs_kernel: persistent; one block per SM (or several when the pair state is small); every
// thread owns one logical slot at a time and runs its coupled pairs (Algorithm 3) back to back
// under the fixed horizon B with slot refill (Algorithm 4).  Per pair, shared memory holds the
// two chains' clone bit sets and the per-pool positive counts of both chains (one byte each), laid
// out word-interleaved over the warp's 32 lanes so that the per-step loads of different pairs never
// share a bank.  The clone->pool rows, the alias table of the scan weights and the acceptance
// thresholds are staged once per block.  The hot loop is integer-only: a Philox4x32-10 block
// feeds two steps, the site comes from the alias table, the full conditional from a table lookup
// indexed by (n+, n-), and the update from a 64-bit integer comparison.  The estimator
// H_{k:l} is accumulated exactly in integers, only when a site flips (see wprefix below), and
// slot sums go to N*_p buckets with 64/128-bit integer atomics, so the result does not depend on
// the schedule.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mcpd_device.cuh"
#include "mcpd_internal.h"
#include "mcpd_pairs.cuh"

namespace mcpd {
namespace {

// theta_j = (sum_{n ascending} S1[n][j] / n) / (P L);  Q_j = (sum_n S2[n][j] / n^2) / L^2;
// se_j = sqrt(max(0, (Q_j - (P theta_j) theta_j) / (P (P - 1)))).  Every operation is an
// explicitly rounded IEEE double operation, in this order.
__device__ __forceinline__ void finalize_one(const unsigned long long *S1, const unsigned long long *S2lo,
                                             const unsigned long long *S2hi, int na, int nb, long long P,
                                             long long L, int j, double *est, double *se) {
    const double dP = static_cast<double>(P), dL = static_cast<double>(L);
    double s1 = 0.0, s2 = 0.0;
    for (int b = 0; b < nb; ++b) {
        const size_t idx = static_cast<size_t>(b) * na + j;
        const double n = static_cast<double>(b + 1);
        s1 = __dadd_rn(s1, __ddiv_rn(static_cast<double>(static_cast<long long>(S1[idx])), n));
        const double sq = __dadd_rn(__dmul_rn(static_cast<double>(S2hi[idx]), 18446744073709551616.0),
                                    static_cast<double>(S2lo[idx]));
        s2 = __dadd_rn(s2, __ddiv_rn(sq, __dmul_rn(n, n)));
    }
    const double th = __ddiv_rn(s1, __dmul_rn(dP, dL));
    *est = th;
    if (P < 2) { *se = __longlong_as_double(0x7FF8000000000000LL); return; }
    const double Q = __ddiv_rn(s2, __dmul_rn(dL, dL));
    const double var = __ddiv_rn(__dsub_rn(Q, __dmul_rn(__dmul_rn(dP, th), th)),
                                 __dmul_rn(dP, __dsub_rn(dP, 1.0)));
    *se = var > 0.0 ? __dsqrt_rn(var) : 0.0;
}

__global__ void finalize_kernel(const unsigned long long *S1, const unsigned long long *S2lo,
                                const unsigned long long *S2hi, int na, int nb, long long P,
                                long long L, double *est, double *se) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= na) return;
    finalize_one(S1, S2lo, S2hi, na, nb, P, L, j, &est[j], &se[j]);
}

// Batched finalize: one thread per (instance, clone), outputs concatenated in instance order.
__global__ void finalize_batch_kernel(const InstDesc *insts, const int32_t *clone_inst,
                                      const int32_t *clone_local, long long total, double *est,
                                      double *se) {
    const long long g = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (g >= total) return;
    const InstDesc &d = insts[clone_inst[g]];
    finalize_one(d.S1, d.S2lo, d.S2hi, d.na, d.nb, d.P_total, d.L, clone_local[g], &est[g], &se[g]);
}

__global__ void philox_kernel(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, long long n) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 o = philox10(c, k0, k1);
    out[4 * i] = o.x; out[4 * i + 1] = o.y; out[4 * i + 2] = o.z; out[4 * i + 3] = o.w;
}

using PairsFn = PairsKernelFn;

PairsFn pick(int coupled, int scan, bool batch, int udeg = 0, bool wide = false, bool ext = false, bool rnd = true) {
    if (batch) return pick_batch(coupled, scan, batch_kernel_degree(coupled, ext, udeg), wide, ext);
    if (coupled && !ext && !rnd) {   // the default all-negative start: no random-start check in the loop
        switch (udeg) {
            case 3: return pairs_kernel<true, false, false, 3, false, false, false, false>;
            case 4: return pairs_kernel<true, false, false, 4, false, false, false, false>;
            case 5: return pairs_kernel<true, false, false, 5, false, false, false, false>;
            case 6: return pairs_kernel<true, false, false, 6, false, false, false, false>;
            case 7: return pairs_kernel<true, false, false, 7, false, false, false, false>;
            case 8: return pairs_kernel<true, false, false, 8, false, false, false, false>;
            default: return pairs_kernel<true, false, false, 0, false, false, false, false>;
        }
    }
    if (coupled && ext) {
        switch (udeg) {
            case 3: return pairs_kernel<true, false, false, 3, false, true>;
            case 4: return pairs_kernel<true, false, false, 4, false, true>;
            case 5: return pairs_kernel<true, false, false, 5, false, true>;
            case 6: return pairs_kernel<true, false, false, 6, false, true>;
            case 7: return pairs_kernel<true, false, false, 7, false, true>;
            case 8: return pairs_kernel<true, false, false, 8, false, true>;
            default: return pairs_kernel<true, false, false, 0, false, true>;
        }
    }
    if (coupled) {
        switch (udeg) {
            case 3: return pairs_kernel<true, false, false, 3>;
            case 4: return pairs_kernel<true, false, false, 4>;
            case 5: return pairs_kernel<true, false, false, 5>;
            case 6: return pairs_kernel<true, false, false, 6>;
            case 7: return pairs_kernel<true, false, false, 7>;
            case 8: return pairs_kernel<true, false, false, 8>;
            default: return pairs_kernel<true, false, false, 0>;
        }
    }
    if (scan == MCPD_SCAN_SYSTEMATIC) {
        switch (udeg) {
            case 3: return pairs_kernel<false, true, false, 3>;
            case 4: return pairs_kernel<false, true, false, 4>;
            case 5: return pairs_kernel<false, true, false, 5>;
            case 6: return pairs_kernel<false, true, false, 6>;
            default: return pairs_kernel<false, true, false, 0>;
        }
    }
    switch (udeg) {
        case 3: return pairs_kernel<false, false, false, 3>;
        case 4: return pairs_kernel<false, false, false, 4>;
        case 5: return pairs_kernel<false, false, false, 5>;
        case 6: return pairs_kernel<false, false, false, 6>;
        default: return pairs_kernel<false, false, false, 0>;
    }
}

int set_smem(size_t bytes, bool batch) {
    for (int c = 0; c < 2; ++c)
        for (int sc : {MCPD_SCAN_SCORE, MCPD_SCAN_SYSTEMATIC}) {
            if (c && sc == MCPD_SCAN_SYSTEMATIC) continue;
            for (int ud = 0; ud <= 8; ++ud) {
                if (ud && (ud < 3 || (!c && ud > kMaskDeg))) continue;
                if (batch && ud != batch_kernel_degree(c, 0, ud)) continue;
                for (int wide = 0; wide <= (batch ? 1 : 0); ++wide)
                    for (int ext = 0; ext <= c; ++ext)
                        for (int rnd = 0; rnd <= 1; ++rnd)
                            if (cudaFuncSetAttribute(pick(c, sc, batch, ud, wide != 0, ext != 0, rnd != 0),
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     static_cast<int>(bytes)) != cudaSuccess)
                                return MCPD_ECUDA;
            }
        }
    return batch ? MCPD_OK : set_trace_smem(bytes);
}

}  // namespace

int pairs_max_smem(int device, size_t *bytes) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
        return MCPD_ECUDA;
    *bytes = static_cast<size_t>(v);
    return MCPD_OK;
}

int launch_pairs(const KParams &kp, int grid, int block, size_t smem, void *stream) {
    if (kp.trace_rec) return launch_pairs_trace(kp, grid, block, smem, stream);
    const BParams none{};
    const bool ext = kp.capped != 0 || kp.lag > 1;
    pick(kp.coupled, kp.scan, false, kp.udeg, false, ext, kp.Tnu != nullptr)<<<grid, block, smem,
                                                                           static_cast<cudaStream_t>(stream)>>>(kp, none);
    return cudaGetLastError() == cudaSuccess ? MCPD_OK : MCPD_ECUDA;
}

int launch_batch(const BParams &bp, int grid, int block, size_t smem, void *stream) {
    const KParams none{};
    pick(bp.coupled, bp.scan, true, bp.udeg, bp.wide != 0, bp.ext != 0)<<<grid, block, smem, static_cast<cudaStream_t>(stream)>>>(none, bp);
    return cudaGetLastError() == cudaSuccess ? MCPD_OK : MCPD_ECUDA;
}

int launch_finalize_batch(const InstDesc *insts, int n_inst, const int32_t *clone_inst,
                          const int32_t *clone_local, long long total_clones, double *est,
                          double *se, void *stream) {
    (void)n_inst;
    if (total_clones <= 0) return MCPD_OK;
    finalize_batch_kernel<<<static_cast<unsigned>((total_clones + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
        insts, clone_inst, clone_local, total_clones, est, se);
    return cudaGetLastError() == cudaSuccess ? MCPD_OK : MCPD_ECUDA;
}

int launch_finalize(const unsigned long long *S1, const unsigned long long *S2lo,
                    const unsigned long long *S2hi, int na, int nb, long long P, long long L,
                    double *est, double *se, void *stream) {
    finalize_kernel<<<(na + 127) / 128, 128, 0, static_cast<cudaStream_t>(stream)>>>(S1, S2lo, S2hi, na, nb, P, L, est, se);
    return cudaGetLastError() == cudaSuccess ? MCPD_OK : MCPD_ECUDA;
}

int launch_philox(const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out, long long n, void *stream) {
    if (n <= 0) return MCPD_OK;
    philox_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(ctr, k0, k1, out, n);
    return cudaGetLastError() == cudaSuccess ? MCPD_OK : MCPD_ECUDA;
}

int pairs_y_regions(int coupled, int warps) {
    return coupled ? (warps + kWarpsPerYRegion - 1) / kWarpsPerYRegion : 0;
}

size_t pairs_smem_bytes(size_t tables, int wpp, int warps, int y_regions) {
    const size_t b = tables + static_cast<size_t>(warps + y_regions) * static_cast<size_t>(wpp) * 128 +
                     static_cast<size_t>(y_regions) * 4;
    return (b + 15) / 16 * 16;
}

int pairs_shape(int coupled, int scan, int udeg, bool batch, size_t tables, int wpp, size_t smem_optin,
                long long P, int sm_count, int warps, bool ext, bool rnd, PairsShape *out) {
    // Batches: the wide variant when the pair state leaves room for more warps than the narrow one
    // is compiled for.  The thread cap and the occupancy query use the variant the run launches
    // (ext: the one with meeting caps and lags > 1; rnd: the one that draws random starts).
    ext = ext && coupled;
    bool wide = batch;
    int cap = pairs_max_threads(coupled, scan, udeg, batch, wide, ext, rnd) / 32;
    auto bytes = [&](int w) { return pairs_smem_bytes(tables, wpp, w, pairs_y_regions(coupled, w)); };
    auto most = [&](size_t budget) {
        int best = 0;
        for (int w = 1; w <= cap && bytes(w) <= budget; ++w) best = w;
        return best;
    };
    auto resident = [&](int w, int *per_sm) {
        *per_sm = 1;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, pick(coupled, scan, batch, udeg, wide, ext, rnd),
                                                             w * 32, bytes(w)) == cudaSuccess;
    };
    int w1 = most(smem_optin);
    if (w1 < 1) return MCPD_ETOO_LARGE;
    if (batch) {
        const int narrow = pairs_max_threads(coupled, scan, udeg, true, false, ext) / 32;
        const int target = warps > 0 ? std::min(warps, w1) : w1;
        if (target <= narrow) { wide = false; cap = narrow; w1 = most(smem_optin); }
    }
    // The attribute is a permission shared by every launch of the kernel (the classes of a batch
    // have different sizes): allow the device's opt-in maximum.
    if (set_smem(smem_optin, batch) != MCPD_OK) return MCPD_ECUDA;
    PairsShape s;
    if (warps > 0) {
        if (warps > w1) return MCPD_EINVAL;
        s.warps = warps;
        if (!resident(warps, &s.per_sm)) return MCPD_ECUDA;
    } else {
        s.warps = w1;
        if (!resident(w1, &s.per_sm)) return MCPD_ECUDA;
        if (!batch) {
            // Two blocks per SM (each with its own copy of the tables) when that holds more warps.
            const int w2 = most(smem_optin / 2);
            int per2 = 1;
            if (w2 >= 1 && resident(w2, &per2) && per2 * w2 > s.per_sm * s.warps) { s.warps = w2; s.per_sm = per2; }
            // Whole rounds of slots: slots run for about the same time, so the fewest warps that
            // need no more rounds per thread than the widest shape finish at the same time with
            // no partly filled last round.
            if (P > 0) {
                const long long blocks = static_cast<long long>(sm_count) * s.per_sm;
                const long long rounds = (P + blocks * s.warps * 32 - 1) / (blocks * s.warps * 32);
                const long long w = (P + rounds * blocks * 32 - 1) / (rounds * blocks * 32);
                if (w >= 1 && w < s.warps) s.warps = static_cast<int>(w);
            }
        }
    }
    s.y_regions = pairs_y_regions(coupled, s.warps);
    s.wide = wide;
    s.smem = bytes(s.warps);
    if (s.per_sm < 1) s.per_sm = 1;
    *out = s;
    return MCPD_OK;
}

int pairs_max_threads(int coupled, int scan, int udeg, bool batch, bool wide, bool ext, bool rnd) {
    cudaFuncAttributes a{};
    if (cudaFuncGetAttributes(&a, pick(coupled, scan, batch, udeg, wide, ext && coupled, rnd)) != cudaSuccess)
        return 512;
    return a.maxThreadsPerBlock;
}


}  // namespace mcpd
