// Lane-group sampling kernel: G lanes (8, 16 or 32; G = 32 is one warp per pair) cooperate on one
// coupled pair.  It computes the same spec as pairs_kernel (Philox keying, alias draw, thresholds,
// Algorithms 3 and 4, integer estimator) and gives bit-identical results; it differs in layout:
//   - lane l of a group handles pool l of the drawn site: it reads that pool's counts of both
//     chains, and warp ballots count the pools with no other positive (n+, n-);
//   - the two chains' bit sets and byte counts of a pair sit contiguously in shared memory (one
//     copy per pair, not per thread), so large instances still fit many pairs per SM;
//   - meeting is detected by XOR of the two chains' bit-set words and a ballot over the group,
//     evaluated on the steps where a chain flipped (no other step can change it);
//   - lane l holds the Philox block of the group's steps t + 2l and t + 2l + 1, so one warp-wide
//     batch of blocks covers the next 2G steps of every group; they are shuffled to the group.
// Tables are read through the read-only cache from the batch's instance descriptors (a single
// instance is a batch of one).
#include <cuda_runtime.h>
#include <stdint.h>

#include "mcpd_device.cuh"
#include "mcpd_internal.h"

namespace mcpd {
namespace {

template <int G>
__global__ void __launch_bounds__(768, 1) group_kernel(const BParams bp) {
    extern __shared__ __align__(16) uint32_t gsm[];
    constexpr unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31, gl = lane % G, gbase = lane - gl;
    const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1u) << gbase);
    const int gib = threadIdx.x / G;                                  // group in block
    const long long gid = static_cast<long long>(blockIdx.x) * (blockDim.x / G) + gib;
    const int wpp = bp.max_wpp;
    uint32_t *X = gsm + static_cast<size_t>(gib) * 2 * wpp;           // X chain: bits, then bytes
    uint32_t *Y = X + wpp;                                            // Y chain, same layout
    for (int w = gl; w < 2 * wpp; w += G) X[w] = 0u;
    __syncthreads();

    long long *const pb = bp.pair_scratch + gid * pair_words(bp.max_na, bp.max_W);   // see pair_words
    long long *racc = pb;
    long long *sacc = pb + bp.max_na;
    uint32_t *trep = reinterpret_cast<uint32_t *>(pb + 2 * bp.max_na + kPairStats);
    uint32_t *tslot = trep + bp.max_W;

    // per-instance values (group-uniform)
    const unsigned long long *gAlias = nullptr, *gT = nullptr, *Tnu = nullptr;
    const uint16_t *rowsP = nullptr;
    const uint32_t *init_pairs = nullptr;
    unsigned long long *bS1 = nullptr, *bS2lo = nullptr, *bS2hi = nullptr, *bCount = nullptr;
    int na = 0, n_init = 0;
    uint32_t W = 0, B = 0, ell = 0, step_limit = 0, instance = 0, k0 = 0, k1 = 0, gshift = 0;
    long long kk = 0, LL = 0, work_begin = 0, work_end = 0, slot_offset = 0, tau_audit = 0;
    bool capped = false;
    uint32_t lag = 1;
    int cur = -1;
    auto load_instance = [&](const InstDesc &d) {
        gAlias = reinterpret_cast<const unsigned long long *>(d.alias);
        gT = reinterpret_cast<const unsigned long long *>(d.T);
        Tnu = reinterpret_cast<const unsigned long long *>(d.Tnu);
        rowsP = d.rows_pool; init_pairs = d.init_pairs; n_init = d.n_init_pairs;
        bS1 = d.S1; bS2lo = d.S2lo; bS2hi = d.S2hi; bCount = d.bcount;
        na = d.na; W = d.W; B = static_cast<uint32_t>(d.B); ell = static_cast<uint32_t>(d.ell);
        step_limit = static_cast<uint32_t>(d.step_limit); instance = d.instance;
        tau_audit = d.tau_audit; capped = d.capped != 0; lag = static_cast<uint32_t>(d.lag);
        k0 = static_cast<uint32_t>(d.seed); k1 = static_cast<uint32_t>(d.seed >> 32);
        kk = d.k; LL = d.L; slot_offset = d.slot_offset;
        work_begin = d.work_begin; work_end = d.work_begin + d.P;
        gshift = 0;
        while (((W + (1u << gshift) - 1) >> gshift) > 64) ++gshift;
    };
    // W(u) = sum_{v<=u} w(v), w(v) the number of window indices r = v - jL (j >= 0); for L > 1,
    // sum_{r=k}^{min(l,u)} (floor((u - r) / L) + 1) through F(n) = sum_{d=0}^{n} floor(d / L).
    auto wpre = [&](long long u) -> long long {
        if (u < kk) return 0;
        if (lag == 1) {
            if (u <= static_cast<long long>(ell)) { const long long a = u - kk + 1; return a * (a + 1) / 2; }
            return LL * (LL + 1) / 2 + (u - static_cast<long long>(ell)) * LL;
        }
        const long long lg = lag, m = min(u, static_cast<long long>(ell));
        auto F = [&](long long n) -> long long {
            if (n < 0) return 0;
            const long long q = n / lg;
            return lg * q * (q - 1) / 2 + q * (n - q * lg + 1);
        };
        return (m - kk + 1) + F(u - kk) - F(u - m - 1);
    };
    auto xc = [&](int j) -> uint8_t * { return reinterpret_cast<uint8_t *>(X + W) + j; };
    auto yc = [&](int j) -> uint8_t * { return reinterpret_cast<uint8_t *>(Y + W) + j; };
    // Add d (+1 or -1) to the byte count of pool j in chain base (lanes may share a pool word).
    auto count_add = [&](uint32_t *base, int j, int d) {
        uint32_t *word = base + W + (j >> 2);
        const uint32_t v = 1u << (8 * (j & 3));
        if (d > 0) atomicAdd(word, v); else atomicSub(word, v);
    };

    bool alive = true, met = false;
    uint32_t slot_local = 0, slot_g = 0, r = 0, t = 0, S = 0, N = 0, tau = 0, abort_t = 0xFFFFFFFFu;
    unsigned long long rep_words = 0, slot_words = 0;
    unsigned long long c_prog = 0, c_started = 0, c_retained = 0, c_aborted = 0, c_zero = 0,
                       c_limit = 0, c_sumtau = 0, c_audit = 0, c_prelag = 0;
    uint32_t c_maxtau = 0;

    auto group_or64 = [&](unsigned long long v) -> unsigned long long {
        const uint32_t lo = __reduce_or_sync(gmask, static_cast<uint32_t>(v));
        const uint32_t hi = __reduce_or_sync(gmask, static_cast<uint32_t>(v >> 32));
        return (static_cast<unsigned long long>(hi) << 32) | lo;
    };

    auto start_rep = [&]() {
        t = 0; tau = 0; met = false;
        abort_t = r > 0 ? (B - S) : 0xFFFFFFFFu;
        ++c_started;
        c_prelag += lag;
        if (Tnu) {   // Z_0 ~ prod Bernoulli(nu_i), X_0 = Y_0 = Z_0: lanes share the listed pairs
            unsigned long long mark = 0;
            for (int e = gl; e < n_init; e += G) {
                const int a = static_cast<int>(init_pairs[e]);
                const uint4 b = philox10(make_uint4(static_cast<uint32_t>(a) >> 1, r, slot_g, instance | (1u << 24)), k0, k1);
                for (int h = 0; h < 2; ++h) {
                    const int c = a + h;
                    if (c >= na) break;
                    const unsigned long long u = h ? ((static_cast<unsigned long long>(b.z) << 32) | b.w)
                                                   : ((static_cast<unsigned long long>(b.x) << 32) | b.y);
                    if (u < Tnu[c]) {
                        const uint32_t q = c >> 5;
                        atomicOr(&X[q], 1u << (c & 31));
                        atomicOr(&Y[q], 1u << (c & 31));
                        for (int l = 0; l < kRow; ++l) {
                            const uint32_t ent = __ldg(rowsP + static_cast<size_t>(c) * kRow + l);
                            if (ent == 0xFFFFu) break;
                            count_add(X, ent & 0x7FFF, 1);
                            count_add(Y, ent & 0x7FFF, 1);
                        }
                        mark |= 1ull << (q >> gshift);
                    }
                }
            }
            rep_words |= group_or64(mark);
            __syncwarp(gmask);
        }
    };

    auto start_slot = [&]() {
        unsigned long long s = 0;
        if (gl == 0) s = atomicAdd(&bp.counters[kWork], 1ull);
        s = __shfl_sync(gmask, s, 0, G);
        if (s >= static_cast<unsigned long long>(bp.total_work)) { alive = false; return; }
        const long long w = static_cast<long long>(s);
        if (cur < 0 || w < work_begin || w >= work_end) {
            int lo = 0, hi = bp.n_inst - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (bp.insts[mid].work_begin <= w) lo = mid; else hi = mid - 1;
            }
            cur = lo;
            load_instance(bp.insts[cur]);
        }
        slot_local = static_cast<uint32_t>(w - work_begin);
        slot_g = static_cast<uint32_t>(slot_offset + static_cast<long long>(slot_local));
        S = 0; N = 0; r = 0;
        start_rep();
    };

    // End of a replication (cooperative over the group's lanes, one state word each).  `move`:
    // completed, so X_C = Y_{C-L}; close the intervals (W(C) - W(C-L) per bit set in X_C) and add
    // the replication's sums to the slot's.  `at_cap`: completed unmet at the meeting cap C, so X's
    // intervals close at C and Y's at C - L: +-W(C-L) more where X_C and Y_{C-L} differ.
    auto finish_rep = [&](bool move, uint32_t C, bool at_cap = false) {
        const long long wX = move ? wpre(C) - wpre(static_cast<long long>(C) - lag) : 0;
        const long long wc = at_cap ? wpre(static_cast<long long>(C) - lag) : 0;
        unsigned long long groups = rep_words, slot_mark = 0;
        while (groups) {
            const int g = __ffsll(static_cast<long long>(groups)) - 1;
            groups &= groups - 1;
            const uint32_t q0 = static_cast<uint32_t>(g) << gshift, q1 = min(W, q0 + (1u << gshift));
            for (uint32_t q = q0 + gl; q < q1; q += G) {
                const uint32_t xw = X[q], yw = Y[q], tw = trep[q];
                uint32_t m = tw | xw | yw, moved = 0;
                while (m) {
                    const int b = __ffs(m) - 1;
                    const uint32_t bit = 1u << b;
                    m &= m - 1;
                    const int j = static_cast<int>(q * 32 + b);
                    long long v = 0;
                    if (tw & bit) { v = racc[j]; racc[j] = 0; }
                    if (move && (xw & bit)) v += wX;
                    if (xw & bit) v += wc;
                    if (yw & bit) v -= wc;
                    if (move && v != 0) {
                        atomicAdd(reinterpret_cast<unsigned long long *>(&sacc[j]), static_cast<unsigned long long>(v));
                        moved |= bit;
                    }
                    if ((xw | yw) & bit) {
                        for (int l = 0; l < kRow; ++l) {
                            const uint32_t ent = __ldg(rowsP + static_cast<size_t>(j) * kRow + l);
                            if (ent == 0xFFFFu) break;
                            if (xw & bit) count_add(X, ent & 0x7FFF, -1);
                            if (yw & bit) count_add(Y, ent & 0x7FFF, -1);
                        }
                    }
                }
                if (tw) trep[q] = 0u;
                if (xw) X[q] = 0u;
                if (yw) Y[q] = 0u;
                if (moved) { atomicOr(&tslot[q], moved); slot_mark |= 1ull << g; }
            }
        }
        slot_words |= group_or64(slot_mark);
        rep_words = 0;
        __syncwarp(gmask);
    };

    auto end_slot = [&](bool valid) {
        const int bkt = static_cast<int>(N) - 1;
        unsigned long long groups = slot_words;
        while (groups) {
            const int g = __ffsll(static_cast<long long>(groups)) - 1;
            groups &= groups - 1;
            const uint32_t q0 = static_cast<uint32_t>(g) << gshift, q1 = min(W, q0 + (1u << gshift));
            for (uint32_t q = q0 + gl; q < q1; q += G) {
                uint32_t tw = tslot[q];
                if (!tw) continue;
                while (tw) {
                    const int b = __ffs(tw) - 1;
                    tw &= tw - 1;
                    const int j = static_cast<int>(q * 32 + b);
                    const long long gsum = sacc[j];
                    sacc[j] = 0;
                    if (valid && gsum != 0) bucket_add(bS1, bS2lo, bS2hi, na, bkt, j, gsum);
                }
                tslot[q] = 0u;
            }
        }
        slot_words = 0;
        if (valid && gl == 0) atomicAdd(&bCount[bkt], 1ull);
        __syncwarp(gmask);
        start_slot();
    };

    auto complete = [&]() {
        const uint32_t C = t;
        c_prog += C;
        c_sumtau += tau;
        c_maxtau = max(c_maxtau, tau);
        if (tau_audit > 0 && (tau > tau_audit || tau == 0)) ++c_audit;   // tau = 0: capped
        finish_rep(true, C, !met);
        S += C;
        N += 1;
        ++c_retained;
        if (S > B) ++c_zero;
        if (S < B && B - S >= max(ell, 1u)) { ++r; start_rep(); }
        else end_slot(true);
    };

    // One coupled step of every group of the warp (all lanes execute it: ballots use the whole
    // warp); active: this group is inside its batch; fast: every active group of the warp has met
    // or is at its pre-lag step, so Y reads are not needed.
    auto step = [&](uint32_t ws, uint32_t wu, bool active, bool fast) -> int {
        uint32_t I = 0;
        {
            const unsigned long long prod = static_cast<unsigned long long>(ws) * static_cast<uint32_t>(max(na, 1));
            const uint32_t col = static_cast<uint32_t>(prod >> 32), coin = static_cast<uint32_t>(prod);
            if (active) {
                const unsigned long long e = __ldg(gAlias + col);
                I = coin < static_cast<uint32_t>(e) ? col : static_cast<uint32_t>(e >> 32);
            }
        }
        const uint32_t q = I >> 5, bit = 1u << (I & 31);
        const uint32_t xw = active ? X[q] : 0u;
        const bool own_y = active && t > 0 && !met;
        const uint32_t yw = own_y ? Y[q] : xw;
        const uint32_t xI = (xw & bit) ? 1u : 0u, yI = (yw & bit) ? 1u : 0u;
        const uint32_t ent = (active && gl < kRow) ? __ldg(rowsP + static_cast<size_t>(I) * kRow + gl) : 0xFFFFu;
        const bool valid = ent != 0xFFFFu;
        const int j = static_cast<int>(ent & 0x7FFFu);
        const uint32_t cx = valid ? *xc(j) : 255u;
        const uint32_t cy = (valid && own_y) ? *yc(j) : cx;
        const unsigned bX = (__ballot_sync(FULL, valid && cx == xI) >> gbase) & (gmask >> gbase);
        const unsigned bY = (__ballot_sync(FULL, valid && cy == yI) >> gbase) & (gmask >> gbase);
        const unsigned bP = (__ballot_sync(FULL, valid && (ent >> 15)) >> gbase) & (gmask >> gbase);
        if (!active) return 0;
        const uint32_t ix = 8u * __popc(bX & bP) + __popc(bX), iy = 8u * __popc(bY & bP) + __popc(bY);
        const unsigned long long TX = __ldg(gT + ix), TY = __ldg(gT + iy);
        const uint32_t thx = static_cast<uint32_t>(TX >> 32), thy = static_cast<uint32_t>(TY >> 32);
        uint32_t nX = wu < thx ? 1u : 0u, nY = wu < thy ? 1u : 0u;
        if (wu == thx || wu == thy) {
            const uint32_t lo = philox10(make_uint4(t, r, slot_g, instance | (2u << 24)), k0, k1).x;
            if (wu == thx) nX = lo < static_cast<uint32_t>(TX) ? 1u : 0u;
            if (wu == thy) nY = lo < static_cast<uint32_t>(TY) ? 1u : 0u;
        }
        if (t < lag) nY = yI;                                   // pre-lag: X only, Y stays Y_0
        else if (!own_y) nY = nX;                               // met: Y_{t+1-L} = X_{t+1}
        const uint32_t fx = nX ^ xI, fy = nY ^ yI;
        if (fx | fy) {
            if (valid) {
                if (fx) count_add(X, j, nX ? 1 : -1);
                if (fy) count_add(Y, j, nY ? 1 : -1);
            }
            if (gl == 0) {
                if (fx) X[q] = xw ^ bit;
                if (fy) Y[q] = yw ^ bit;
                long long ev = 0;
                if (t > 0 && !own_y) {                          // met: X at t+1 and Y at t+1-L
                    // together (the one-lag count of window indices r <= t; on a pre-lag step X
                    // alone, whose W(t) is the same count)
                    const long long a = static_cast<long long>(t) - kk + 1;
                    const long long w = a < 0 ? 0 : (a > LL ? LL : a);
                    ev = nX ? -w : w;
                } else {
                    if (fx) { const long long w = wpre(t); ev += nX ? -w : w; }
                    if (fy) { const long long w = wpre(static_cast<long long>(t) - lag); ev += nY ? w : -w; }
                }
                if (ev != 0) {
                    atomicAdd(reinterpret_cast<unsigned long long *>(&racc[I]), static_cast<unsigned long long>(ev));
                    atomicOr(&trep[q], bit);
                }
            }
            rep_words |= 1ull << (q >> gshift);
            __syncwarp(gmask);
            if (t < lag && !own_y) {
                met = false;                                    // X_{t+1} differs from Y_0 = X_t at I
            } else if (own_y) {                                 // ballot over XOR of the bit sets
                bool diff = false;
                for (uint32_t w = gl; w < W; w += G) diff |= (X[w] ^ Y[w]) != 0u;
                met = !__any_sync(gmask, diff);
            }
        } else if (t == 0) {
            met = true;                                         // X_1 = Y_0
        }
        ++t;
        if (met && t >= lag) {                                  // tau = inf{t >= L : X_t = Y_{t-L}}
            if (tau == 0) tau = t;
            if (t >= ell) return 1;
        }
        if (capped && t >= step_limit) return 1;        // unmet at the meeting cap: completed (C = t)
        if (t >= abort_t) return 2;
        return t >= step_limit ? 3 : 0;
    };

    start_slot();
    while (__any_sync(FULL, alive)) {
        const uint4 blk = alive ? philox10(make_uint4((t >> 1) + static_cast<uint32_t>(gl), r, slot_g, instance), k0, k1)
                                : make_uint4(0, 0, 0, 0);
        bool in_batch = alive;
        for (int s = 0; s < 2 * G; ++s) {
            const uint32_t ws = __shfl_sync(FULL, (s & 1) ? blk.z : blk.x, s >> 1, G);
            const uint32_t wu = __shfl_sync(FULL, (s & 1) ? blk.w : blk.y, s >> 1, G);
            const bool fast = __all_sync(FULL, !in_batch || t == 0 || met);
            const int ended = step(ws, wu, in_batch, fast);
            if (ended) {
                in_batch = false;
                if (ended == 1) {
                    complete();
                } else {
                    c_prog += t;
                    if (ended == 2) ++c_aborted;
                    else { ++c_limit; if (gl == 0) atomicExch(bp.error, 1); }
                    finish_rep(false, 0);
                    end_slot(ended == 2);
                }
            }
        }
    }
    if (gl == 0) {
        if (c_prog) atomicAdd(&bp.counters[kProgress], c_prog);
        if (c_started) atomicAdd(&bp.counters[kRepsStarted], c_started);
        if (c_prog) atomicAdd(&bp.counters[kSiteUpdates], 2 * c_prog - c_prelag);
        if (c_retained) atomicAdd(&bp.counters[kRepsRetained], c_retained);
        if (c_aborted) atomicAdd(&bp.counters[kRepsAborted], c_aborted);
        if (c_zero) atomicAdd(&bp.counters[kZeroCompletion], c_zero);
        if (c_limit) atomicAdd(&bp.counters[kStepLimitHits], c_limit);
        if (c_sumtau) atomicAdd(&bp.counters[kSumTau], c_sumtau);
        if (c_audit) atomicAdd(&bp.counters[kTauOverAudit], c_audit);
        if (c_maxtau) atomicMax(&bp.counters[kMaxTau], static_cast<unsigned long long>(c_maxtau));
    }
}

using GroupFn = void (*)(const BParams);

GroupFn pick_group(int lanes) {
    switch (lanes) {
        case 8: return group_kernel<8>;
        case 16: return group_kernel<16>;
        default: return group_kernel<32>;
    }
}

}  // namespace

int set_group_smem(int lanes, size_t bytes) {
    return cudaFuncSetAttribute(pick_group(lanes), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(bytes)) == cudaSuccess ? MCPD_OK : MCPD_ECUDA;
}

int group_max_threads(int lanes) {
    cudaFuncAttributes a{};
    if (cudaFuncGetAttributes(&a, pick_group(lanes)) != cudaSuccess) return 256;
    return a.maxThreadsPerBlock;
}

int group_occupancy(int lanes, int block, size_t smem, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, pick_group(lanes), block, smem) == cudaSuccess
               ? MCPD_OK : MCPD_ECUDA;
}

int launch_group(const BParams &bp, int grid, int block, size_t smem, void *stream) {
    pick_group(bp.lanes)<<<grid, block, smem, static_cast<cudaStream_t>(stream)>>>(bp);
    return cudaGetLastError() == cudaSuccess ? MCPD_OK : MCPD_ECUDA;
}

}  // namespace mcpd
