// The persistent sampling kernel (template): one thread per coupled pair (Algorithm 3) running
// its slots under the fixed horizon with refill (Algorithm 4).  Included by the translation units
// that instantiate it: mcpd_kernels.cu (the production variants) and mcpd_trace.cu (the variants
// that also record per-replication trajectories for the parity tests).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mcpd_device.cuh"
#include "mcpd_internal.h"

namespace mcpd {
namespace {

// The estimator's integer bookkeeping.  Swapping the sums in
// L H_{k:l} = sum_{r=k}^{l} [X_r + sum_{s>=1} (X_{r+s} - Y_{r+s-1})] gives
//   G_j = sum_{t=0}^{C} w(t) X_t[j] - sum_{t=0}^{C-1} w(t) Y_t[j],  w(t) = clamp(t - k + 1, 0, L),
// so a chain whose bit j is 1 on the time interval [s, e] contributes +-(W(e) - W(s-1)) with
// W(u) = sum_{v<=u} w(v) (quadratic, then linear).  Uncoupled chains (Algorithms 1/2) use
// w(t) = 1{b <= t <= b + T - 1}.  The kernel adds -+W at every flip and closes the open intervals
// at the end of a replication.  Once a pair has met (X_t = Y_{t-1}), Y_t = X_{t+1}: a flip of X at
// step t is also the flip of Y at step t, and the two events add to -+(W(t) - W(t-1)) = -+w(t).
// The uncoupled flip event W(t) has the same clamp form, so both modes use
// wstep(u) = clamp(u - s + 1, 0, cap) with (s, cap) = (k, L) or (b, T).
// With lag L (Y_{t+1-L} moves with X_{t+1}), the weight of X_t and Y_t is the number of window
// indices r = t - jL (j >= 0), W is its prefix sum, a Y flip at step t adds +-W(t - L), and the
// met flip and the closing term keep the one-lag count wstep (see wpre and met_flip).

// One persistent kernel for a single instance (BATCH = false: tables staged in shared memory,
// parameters from KParams) or for many instances in one launch (BATCH = true: tables read through
// the read-only cache from per-instance descriptors, work items (instance, slot) handed out
// instance-major from one counter).
// DEG > 0: every clone of the (single) instance sits in exactly DEG pools, so the pool loops have
// a compile-time trip count and rows hold no padding entries; DEG = 0 handles any degree <= 8.
//
// Shared memory: [tables (single instance)] [one region per warp] [y_regions Y regions] [one
// free mask per Y region].  A region is 32 columns of wpp words, word w of column c at word
// 32 w + c, so the same byte offset (a row entry) addresses a pool's count in any column and the
// 32 lanes of a warp touch 32 different banks.  Lane l's X chain is column l of its warp's
// region.  A pair that has not met keeps its Y chain in a column of the Y regions (column l of
// some region first, so that it shares no bank with its warp's other lanes), else in its own
// column of the global fallback (same layout, one region per warp).  A free Y column is all zero
// except, for DEG = 0, the padding pool's count.
// WIDE (batches only): compiled for 20 warps per block (96 registers) rather than 12 (up to 168),
// for size classes whose pair state leaves room for more than 12 warps.
// EXT: the meeting cap and lags L > 1 (runs that use neither launch the variant without them, whose
// hot loop the completion path's code would otherwise perturb).
// TRACE (single instance): also record the first replications of every traced slot (meeting time,
// completion time, and per draw the site and which chains flipped; MCPD_FETCH_TRACE_REC), for the
// trajectory parity tests.  The production variants compile none of it.
// RND = false: the instance has no random start (Z_0 = 0), so the warp never draws one; the
// runs with a random start launch RND = true (the default), whose loop checks for pending starts.
template <bool COUPLED, bool SYSTEMATIC, bool BATCH, int DEG, bool WIDE = false, bool EXT = false, bool TRACE = false,
          bool RND = true>
__global__ void __launch_bounds__(BATCH ? (WIDE ? 640 : 384) : (DEG >= 6 ? 640 : 512), 1) pairs_kernel(const KParams p, const BParams bp) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    uint4 *sRows = reinterpret_cast<uint4 *>(smem);
    unsigned long long *sAlias = nullptr, *sT = nullptr;
    int wpp, nyr;
    uint32_t *regions;
    if constexpr (!BATCH) {
        sAlias = reinterpret_cast<unsigned long long *>(smem + static_cast<size_t>(p.na) * 16);
        sT = sAlias + p.na;
        for (int i = threadIdx.x; i < p.na; i += blockDim.x) {
            sRows[i] = reinterpret_cast<const uint4 *>(p.rows)[i];
            sAlias[i] = p.alias[i];
        }
        for (int i = threadIdx.x; i < p.nT; i += blockDim.x) sT[i] = p.T[i];
        wpp = p.wpp;
        nyr = p.y_regions;
        regions = reinterpret_cast<uint32_t *>(smem + p.smem_tables);
    } else {
        wpp = bp.max_wpp;
        nyr = bp.y_regions;
        regions = reinterpret_cast<uint32_t *>(smem);
    }
    const uint32_t region_words = 32u * static_cast<uint32_t>(wpp);
    uint32_t *const st = regions + warp * region_words + lane;        // word w of X: st[w * 32]
    unsigned char *const cbase = reinterpret_cast<unsigned char *>(st);
    uint32_t *const yreg = regions + nwarps * region_words;
    uint32_t *const ymask = yreg + nyr * region_words;
    for (int w = 0; w < wpp; ++w) st[w * 32] = 0u;
    for (uint32_t i = threadIdx.x; i < nyr * region_words; i += blockDim.x) yreg[i] = 0u;
    if (static_cast<int>(threadIdx.x) < nyr) ymask[threadIdx.x] = 0xFFFFFFFFu;
    if constexpr (!BATCH) st[p.dummy_word_index * 32] = p.dummy_word;
    __syncthreads();

    const uint32_t gpair = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride_na = BATCH ? bp.max_na : p.na, stride_W = BATCH ? bp.max_W : p.W;
    // This pair's scratch block (see pair_words): one base pointer, the parts at fixed offsets.
    long long *const pb = (BATCH ? bp.pair_scratch : p.pair_scratch) +
                          static_cast<size_t>(gpair) * static_cast<size_t>(pair_words(stride_na, stride_W));
    // Clone j's replication sum at pb[2j] and slot sum at pb[2j + 1]: a flip event reduces into
    // both from one address.
    auto racc = [&](uint32_t j) { return pb + 2 * static_cast<size_t>(j); };
    auto sacc = [&](uint32_t j) { return pb + 2 * static_cast<size_t>(j) + 1; };
    auto pst = [&]() { return reinterpret_cast<unsigned long long *>(pb + 2 * stride_na); };
    auto trep = [&]() { return reinterpret_cast<uint32_t *>(pb + 2 * stride_na + kPairStats); };
    auto tslot = [&]() { return reinterpret_cast<uint32_t *>(pb + 2 * stride_na + kPairStats) + stride_W; };
    unsigned long long *counters = BATCH ? bp.counters : p.counters;
    auto yglob = [&]() {
        return (BATCH ? bp.y_state : p.y_state) + static_cast<size_t>(gpair >> 5) * region_words + lane;
    };
    uint32_t *ycol = nullptr;         // the Y column in use (shared or global), while D != 0
    int yslot = -1;                   // its index in the Y regions, -1 for the global column
#pragma unroll
    for (int i = 0; i < kPairStats; ++i) pst()[i] = 0ull;

    // Per-instance values (fixed for a single instance, reloaded when a batched slot changes
    // instance).
    // Values the step uses live in registers; the others are read where needed, from the kernel
    // parameters (one instance) or from the instance's descriptor (batch, read-only, cached).
    const uint4 *gRows = nullptr;
    const unsigned long long *gAlias = nullptr, *gT = nullptr;
    int na = 0, deg = 0;
    uint32_t W = 0, ell = 0, instance = 0, k0 = 0, k1 = 0;
    uint32_t dummy_entry = 0, gshift = 0, ws0 = 0, wcap = 0;
    int cur = -1;
    auto desc = [&]() -> const InstDesc * { return bp.insts + cur; };
#define MCPD_FIELD(name, batch_expr, single_expr) \
    auto name = [&]() { if constexpr (BATCH) return batch_expr; else return single_expr; }
    MCPD_FIELD(v_B, static_cast<uint32_t>(__ldg(&desc()->B)), static_cast<uint32_t>(p.B));
    MCPD_FIELD(v_unit, static_cast<uint32_t>(__ldg(&desc()->unit)), static_cast<uint32_t>(p.unit));
    MCPD_FIELD(v_step_limit, static_cast<uint32_t>(__ldg(&desc()->step_limit)), static_cast<uint32_t>(p.step_limit));
    MCPD_FIELD(v_tau_audit, __ldg(&desc()->tau_audit), p.tau_audit);
    auto v_capped = [&]() -> bool {
        if constexpr (!EXT) return false;
        else if constexpr (BATCH) return __ldg(&desc()->capped) != 0;
        else return p.capped != 0;
    };
    auto v_lag = [&]() -> uint32_t {
        if constexpr (!EXT) return 1u;
        else if constexpr (BATCH) return static_cast<uint32_t>(__ldg(&desc()->lag));
        else return static_cast<uint32_t>(p.lag);
    };
    MCPD_FIELD(v_k, __ldg(&desc()->k), p.k);
    MCPD_FIELD(v_L, __ldg(&desc()->L), p.L);
    MCPD_FIELD(v_burn, __ldg(&desc()->burn), p.burn);
    MCPD_FIELD(v_length, __ldg(&desc()->length), p.length);
    MCPD_FIELD(v_P, __ldg(&desc()->P), p.P);
    MCPD_FIELD(v_slot_offset, __ldg(&desc()->slot_offset), p.slot_offset);
    MCPD_FIELD(v_work_begin, __ldg(&desc()->work_begin), 0ll);
    MCPD_FIELD(v_dwi, __ldg(&desc()->dummy_word_index), p.dummy_word_index);
    MCPD_FIELD(v_dw, __ldg(&desc()->dummy_word), p.dummy_word);
    MCPD_FIELD(v_wpp, static_cast<uint32_t>(__ldg(&desc()->wpp)), static_cast<uint32_t>(p.wpp));
    MCPD_FIELD(v_Tnu, reinterpret_cast<const unsigned long long *>(__ldg(reinterpret_cast<const unsigned long long *>(&desc()->Tnu))),
               reinterpret_cast<const unsigned long long *>(p.Tnu));
    MCPD_FIELD(v_S1, reinterpret_cast<unsigned long long *>(__ldg(reinterpret_cast<const unsigned long long *>(&desc()->S1))), p.S1);
    MCPD_FIELD(v_S2lo, reinterpret_cast<unsigned long long *>(__ldg(reinterpret_cast<const unsigned long long *>(&desc()->S2lo))), p.S2lo);
    MCPD_FIELD(v_S2hi, reinterpret_cast<unsigned long long *>(__ldg(reinterpret_cast<const unsigned long long *>(&desc()->S2hi))), p.S2hi);
    MCPD_FIELD(v_bcount, reinterpret_cast<unsigned long long *>(__ldg(reinterpret_cast<const unsigned long long *>(&desc()->bcount))), p.bcount);
#undef MCPD_FIELD
    auto clamp32 = [](long long v) -> uint32_t { return v < 0 ? 0u : (v > 0xFFFFFFFFll ? 0xFFFFFFFFu : static_cast<uint32_t>(v)); };
    auto derive = [&]() {
        gshift = 0;
        while (((W + (1u << gshift) - 1) >> gshift) > 32) ++gshift;
        ws0 = clamp32(COUPLED ? v_k() : v_burn());
        wcap = clamp32(COUPLED ? v_L() : v_length());
    };
    // Uniform degree 3..kMaskDeg (every clone of the instance, or of every instance of a batched
    // class, sits in exactly DEG pools): rows hold plain offsets with the clone's positive-outcome
    // pools first and their number in the last entry; thresholds are indexed
    // npos * 64 + (mask of deciding pools).
    constexpr bool MASKT = DEG >= 3 && DEG <= kMaskDeg;
    auto load_instance = [&](int c) {
        cur = c;
        const InstDesc &d = bp.insts[c];
        gRows = reinterpret_cast<const uint4 *>(MASKT ? d.rows_mask : d.rows);
        gAlias = reinterpret_cast<const unsigned long long *>(d.alias);
        gT = reinterpret_cast<const unsigned long long *>(MASKT ? d.T_mask : d.T);
        na = d.na; deg = d.deg; W = d.W;
        dummy_entry = d.dummy_entry;
        ell = static_cast<uint32_t>(d.ell);
        instance = d.instance;
        k0 = static_cast<uint32_t>(d.seed); k1 = static_cast<uint32_t>(d.seed >> 32);
        derive();
    };
    if constexpr (!BATCH) {
        na = p.na; deg = p.deg; W = p.W;
        dummy_entry = p.dummy_entry;
        ell = static_cast<uint32_t>(p.ell);
        instance = p.instance;
        k0 = static_cast<uint32_t>(p.seed); k1 = static_cast<uint32_t>(p.seed >> 32);
        derive();
    }
    constexpr int NE = DEG > 0 ? DEG : kRow;       // row entries visited per clone
    auto rowAt = [&](uint32_t c) -> uint4 {
        if constexpr (BATCH) return __ldg(gRows + c); else return sRows[c];
    };
    auto aliasAt = [&](uint32_t c) -> unsigned long long {
        if constexpr (BATCH) return __ldg(gAlias + c); else return sAlias[c];
    };
    auto tAt = [&](uint32_t i) -> unsigned long long {
        if constexpr (BATCH) return __ldg(gT + i); else return sT[i];
    };
    auto entries = [&](const uint4 &row, uint32_t *ent) {
        ent[0] = row.x & 0xFFFFu; ent[1] = row.x >> 16; ent[2] = row.y & 0xFFFFu; ent[3] = row.y >> 16;
        ent[4] = row.z & 0xFFFFu; ent[5] = row.z >> 16; ent[6] = row.w & 0xFFFFu; ent[7] = row.w >> 16;
    };
    // Entry l of a row is a real pool (not past the clone's degree, not the padding pool).
    auto real = [&](int l, const uint32_t *ent) -> bool {
        return l < NE && (DEG > 0 || (l < deg && ent[l] != dummy_entry));
    };
    // Prefix sums of the estimator's per-time weights (see the comment on wprefix).
    // Lag L > 1: W(u) = sum_{r=k}^{min(l,u)} (floor((u - r) / L) + 1), the weight of X_t and Y_t
    // being the number of window indices r = t - jL (j >= 0); with F(n) = sum_{d=0}^{n} floor(d / L)
    // = L q (q - 1) / 2 + q (n - q L + 1), q = floor(n / L), the floor sum is F(u - k) - F(u - m - 1).
    auto wpre = [&](long long u) -> long long {
        if (COUPLED) {
            const long long kk = v_k(), LL = v_L();
            if (u < kk) return 0;
            const long long lg = v_lag();
            if (lg == 1) {
                if (u <= static_cast<long long>(ell)) { const long long a = u - kk + 1; return a * (a + 1) / 2; }
                return LL * (LL + 1) / 2 + (u - static_cast<long long>(ell)) * LL;
            }
            const long long m = min(u, static_cast<long long>(ell));
            auto F = [&](long long n) -> long long {
                if (n < 0) return 0;
                const long long q = n / lg;
                return lg * q * (q - 1) / 2 + q * (n - q * lg + 1);
            };
            return (m - kk + 1) + F(u - kk) - F(u - m - 1);
        } else {
            const long long v = u - v_burn() + 1, length = v_length();
            return v < 0 ? 0 : (v > length ? length : v);
        }
    };
    auto wstep = [&](uint32_t u) -> uint32_t { return u < ws0 ? 0u : min(u - ws0 + 1u, wcap); };

    bool alive = true;
    bool init_pending = false;        // a random start waits for the warp's draw (coop_init)
    bool fin_pending = false;         // a completed replication's state waits for the warp (coop_finish)
    uint32_t fin_words = 0;           // its groups of bit words (rep_words at completion)
    long long fin_wX = 0;             // its closing weight w(C)
    uint32_t slot_local = 0, slot_g = 0, r = 0, t = 0, S = 0, N = 0, tau = 0, D = 0;
    uint32_t abort_t = 0xFFFFFFFFu, t_end = 0, stop_unmet = 0, sysI = 0, reps_in_slot = 0;
    uint32_t rep_words = 0, slot_words = 0;   // groups of 2^gshift bit words touched
    int32_t *trec = nullptr;                   // TRACE: the record of the current replication

    // A pair that stops being met takes a free Y column (column `lane` of a Y region first,
    // then any free one; bounded tries), else its global column.
    auto acquire_y = [&]() {
        yslot = -1;
        for (int g = 0; g < nyr && yslot < 0; ++g)
            if (atomicAnd(&ymask[g], ~(1u << lane)) & (1u << lane)) yslot = g * 32 + lane;
        for (int g = 0; g < nyr && yslot < 0; ++g) {
            for (int tries = 0; tries < 32; ++tries) {
                const uint32_t fm = *reinterpret_cast<volatile uint32_t *>(&ymask[g]);
                if (!fm) break;
                const int c = __ffs(fm) - 1;
                if (atomicAnd(&ymask[g], ~(1u << c)) & (1u << c)) { yslot = g * 32 + c; break; }
            }
        }
        __threadfence_block();
        ycol = yslot >= 0 ? yreg + (yslot >> 5) * region_words + (yslot & 31) : yglob();
        if (DEG == 0) ycol[v_dwi() * 32] = v_dw();
    };
    // Empty the Y column in use and return it: its bit words (every Y bit lies in a group marked in
    // rep_words) and all its count words (the padding pool's word among them) to zero.  Zeroing
    // the count words costs one store each, where taking each set bit's pools back down costs a
    // row load and deg count updates per bit (a random start leaves many bits set).
    auto release_y = [&]() {
        uint32_t groups = rep_words;
        while (groups) {
            const int g = __ffs(groups) - 1;
            groups &= groups - 1;
            const uint32_t q0 = static_cast<uint32_t>(g) << gshift, q1 = min(W, q0 + (1u << gshift));
            for (uint32_t q = q0; q < q1; ++q) ycol[q * 32] = 0u;
        }
        for (uint32_t w = W, e = v_wpp(); w < e; ++w) ycol[w * 32] = 0u;
        __threadfence_block();
        if (yslot >= 0) atomicOr(&ymask[yslot >> 5], 1u << (yslot & 31));
        yslot = -1;
        ycol = nullptr;
    };
    // A pre-lag update flipped site I of X_t = X_0 and the start was random: Y_0 = X_0 goes to the
    // (empty) Y column: X_{t+1}'s bit words with bit I restored, X_{t+1}'s count words, and the
    // counts of I's pools as they were before the flip (cx, loaded this step).
    auto copy_y0 = [&](uint32_t qI, uint32_t bitI, const uint32_t *ent, const uint32_t *cx) {
        uint32_t groups = rep_words;
        while (groups) {
            const int g = __ffs(groups) - 1;
            groups &= groups - 1;
            const uint32_t q0 = static_cast<uint32_t>(g) << gshift, q1 = min(W, q0 + (1u << gshift));
            for (uint32_t q = q0; q < q1; ++q) {
                const uint32_t yw = st[q * 32] ^ (q == qI ? bitI : 0u);
                if (yw) ycol[q * 32] = yw;
            }
        }
        for (uint32_t w = W, e = v_wpp(); w < e; ++w) ycol[w * 32] = st[w * 32];
        unsigned char *yb = reinterpret_cast<unsigned char *>(ycol);
#pragma unroll
        for (int l = 0; l < kRow; ++l)
            if (real(l, ent)) yb[ent[l] & 0x7FFFu] = static_cast<unsigned char>(cx[l]);
    };

    // A batched pair keeps the pre-lag updates of its replications (sum of L) in the high half of
    // the started record, split at exit; one instance needs only the count.
    auto start_rep = [&]() {
        const uint32_t lag = v_lag();
        t = 0; D = 0; tau = lag; sysI = 0;    // tau = L unless a pre-lag update moves X
        const uint32_t step_limit = v_step_limit();
        abort_t = (COUPLED && r > 0) ? (v_B() - S) : 0xFFFFFFFFu;
        stop_unmet = min(abort_t, step_limit);
        t_end = COUPLED ? min(max(ell, lag), stop_unmet) : min(v_unit(), step_limit);
        red_add(reinterpret_cast<long long *>(&pst()[kPsStarted]),
                BATCH && COUPLED && EXT ? 1 + (static_cast<long long>(lag) << 32) : 1ll);
        ++reps_in_slot;
        if constexpr (TRACE) {
            trec = nullptr;
            if (slot_local % static_cast<uint32_t>(p.trace_stride) == 0 && r < static_cast<uint32_t>(p.trace_reps)) {
                trec = p.trace_rec + (static_cast<size_t>(slot_local / static_cast<uint32_t>(p.trace_stride)) *
                                      static_cast<size_t>(p.trace_reps) + r) * (4 + static_cast<size_t>(p.trace_steps));
                trec[3] = static_cast<int32_t>(r);
            }
        }
        // Z_0 ~ prod Bernoulli(nu_i); X_0 = Y_0 = Z_0 (clones with nu_i = 0 stay 0): drawn by the
        // whole warp before this lane's next step (coop_init at the top of the loop)
        if constexpr (RND) {
            if (v_Tnu()) init_pending = true;
        }
    };

    auto start_slot = [&]() {
        const unsigned long long s = atomicAdd(&counters[kWork], 1ull);
        if constexpr (BATCH) {
            if (s >= static_cast<unsigned long long>(bp.total_work)) { alive = false; return; }
            const long long w = static_cast<long long>(s);
            if (cur < 0 || w < v_work_begin() || w >= v_work_begin() + v_P()) {
                int lo = 0, hi = bp.n_inst - 1;             // last instance with work_begin <= w
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (bp.insts[mid].work_begin <= w) lo = mid; else hi = mid - 1;
                }
                if (cur >= 0) st[v_dwi() * 32] = 0u;    // the old layout's padding pool
                load_instance(lo);
                st[v_dwi() * 32] = v_dw();
            }
            slot_local = static_cast<uint32_t>(w - v_work_begin());
        } else {
            if (s >= static_cast<unsigned long long>(v_P())) { alive = false; return; }
            slot_local = static_cast<uint32_t>(s);
        }
        slot_g = static_cast<uint32_t>(v_slot_offset() + static_cast<long long>(slot_local));
        S = 0; N = 0; r = 0; reps_in_slot = 0;
        start_rep();
    };

    // End of a replication: empty the pair's state and the replication's accumulators; when `move`
    // (completed, so X_C = Y_{C-1}), first close the open intervals at C, which for a bit set in
    // X_C adds W(C) - W(C-1) (coupled) or W(C) (uncoupled), both wstep(C), and add the
    // replication's G into the slot's sums.
    // Flip events go to both the replication's sums and the slot's sums, so a completed
    // replication only zeroes its own (stores) and adds its closing terms; the replication's sums
    // are read back only when it is discarded (doomed or at the step limit), to take its events
    // out of the slot's sums.
    // defer (a completed replication whose slot goes on): the Y column is returned here and the
    // rest is left to the whole warp at the top of the loop (coop_finish).
    auto finish_rep = [&](bool move, uint32_t C, bool defer) {
        const long long wX = move ? static_cast<long long>(wstep(C)) : 0;
        if (COUPLED && (EXT ? ycol != nullptr : D != 0)) release_y();
        if (defer) {
            fin_pending = true;
            fin_words = rep_words;
            fin_wX = wX;
            rep_words = 0;
            return;
        }
        uint32_t groups = rep_words;
        while (groups) {
            const int g = __ffs(groups) - 1;
            groups &= groups - 1;
            const uint32_t q0 = static_cast<uint32_t>(g) << gshift;
            const uint32_t q1 = min(W, q0 + (1u << gshift));
            for (uint32_t q = q0; q < q1; ++q) {
                const uint32_t xw = st[q * 32];
                const uint32_t tw = __ldcg(&trep()[q]);
                uint32_t tm = tw;
                while (tm) {
                    const int b = __ffs(tm) - 1;
                    tm &= tm - 1;
                    const uint32_t j = q * 32 + b;
                    if (!move) red_add(sacc(j), -__ldcg(racc(j)));   // discarded: its events leave the slot
                    *racc(j) = 0;
                }
                if (move && wX != 0) {          // closing terms of the sites set in X_C
                    uint32_t om = xw;
                    while (om) {
                        const int b = __ffs(om) - 1;
                        om &= om - 1;
                        red_add(sacc(q * 32 + b), wX);
                    }
                }
                const uint32_t touched = tw | (move && wX != 0 ? xw : 0u);
                if (tw) trep()[q] = 0u;
                if (xw) st[q * 32] = 0u;
                if (touched) { red_or(&tslot()[q], touched); slot_words |= 1u << g; }
            }
        }
        // X's counts back to zero (one store per count word), the padding pool's count kept
        for (uint32_t w = W, e = v_wpp(); w < e; ++w) st[w * 32] = 0u;
        st[v_dwi() * 32] = v_dw();
        rep_words = 0;
    };

    auto end_slot = [&](bool valid) {
        const int bkt = static_cast<int>(N) - 1;
        long long *tr = nullptr;
        if constexpr (!BATCH) {
            if (valid && p.trace_stride > 0 && (slot_local % p.trace_stride) == 0)
                tr = p.trace_G + (static_cast<long long>(slot_local) / p.trace_stride) * na;
        }
        uint32_t groups = slot_words;
        while (groups) {
            const int g = __ffs(groups) - 1;
            groups &= groups - 1;
            const uint32_t q0 = static_cast<uint32_t>(g) << gshift;
            const uint32_t q1 = min(W, q0 + (1u << gshift));
            for (uint32_t q = q0; q < q1; ++q) {
                uint32_t tw = __ldcg(&tslot()[q]);
                if (!tw) continue;
                while (tw) {
                    const int b = __ffs(tw) - 1;
                    tw &= tw - 1;
                    const uint32_t j = q * 32 + b;
                    const long long gsum = __ldcg(sacc(j));
                    *sacc(j) = 0;
                    if (valid && gsum != 0) {
                        bucket_add(v_S1(), v_S2lo(), v_S2hi(), na, bkt, static_cast<int>(j), gsum);
                        if (tr) tr[j] = gsum;
                    }
                }
                tslot()[q] = 0u;
            }
        }
        slot_words = 0;
        if (valid) atomicAdd(&v_bcount()[bkt], 1ull);
        if constexpr (!BATCH) {
            if (p.slot_nstar) {
                p.slot_nstar[slot_local] = valid ? static_cast<int32_t>(N) : 0;
                p.slot_S[slot_local] = S;
                p.slot_reps[slot_local] = static_cast<int32_t>(reps_in_slot);
            }
        }
        start_slot();
    };

    // Completed at C = t: every completed replication is retained (a later one that could not
    // finish within B is aborted before it completes); then refill or end the slot.
    // Stopped unmet at the meeting cap c = t: H_{k:l} keeps the terms up to c, so X's intervals
    // close at c (+W(c) per bit of X_c) and Y's at c - L (-W(c-L) per bit of Y_{c-L}).  The
    // closing in finish_rep adds W(c) - W(c-L) = w1(c) per bit of X_c (w1 the one-lag weight: the
    // window indices r <= c); the rest is +-W(c-L) at every site where X_c and Y_{c-L} differ,
    // added here while the Y column is still held.
    auto cap_close = [&]() {
        const long long wc = wpre(static_cast<long long>(t) - v_lag());
        if (wc == 0) return;
        uint32_t groups = rep_words;          // every X and Y bit lies in a marked group
        while (groups) {
            const int g = __ffs(groups) - 1;
            groups &= groups - 1;
            const uint32_t q0 = static_cast<uint32_t>(g) << gshift, q1 = min(W, q0 + (1u << gshift));
            for (uint32_t q = q0; q < q1; ++q) {
                const uint32_t xw = st[q * 32];
                uint32_t dm = xw ^ ycol[q * 32];
                if (!dm) continue;
                red_or(&tslot()[q], dm);
                slot_words |= 1u << g;
                while (dm) {
                    const int b = __ffs(dm) - 1;
                    dm &= dm - 1;
                    red_add(sacc(q * 32 + b), ((xw >> b) & 1u) ? wc : -wc);
                }
            }
        }
    };

    // The retained record's high half counts the completions whose meeting time exceeds the audit
    // length, capped pairs (tau = 0) included (one reduction per completion, not two; split at
    // exit).  A pair that reaches the meeting cap c = t unmet completes with C = c.
    // TRACE: the replication's meeting time, its clock at the end and how it ended.
    auto trace_end = [&](int how) {
        if constexpr (TRACE) {
            if (trec) {
                trec[0] = COUPLED ? static_cast<int32_t>(tau) : 0;
                trec[1] = static_cast<int32_t>(t);
                trec[2] = how;
            }
        }
    };
    auto complete = [&]() {
        const uint32_t C = t;
        long long over = 0;
        trace_end(1);
        if (COUPLED && EXT && D != 0) cap_close();
        red_add(reinterpret_cast<long long *>(&pst()[kPsProgress]), C);
        if (COUPLED) {
            red_add(reinterpret_cast<long long *>(&pst()[kPsSumTau]), tau);
            red_max(&pst()[kPsMaxTau], tau);
            const long long audit = v_tau_audit();
            over = (audit > 0 && (tau > audit || tau == 0u)) ? (1ll << 32) : 0ll;
        }
        const uint32_t B = v_B();
        const uint32_t S_next = S + C;
        const bool goes_on = S_next < B && B - S_next >= v_unit();
        // a slot's last replication ends before its flush (end_slot); the 12-warp batch build
        // (up to 168 registers) keeps the one-lane end, measured faster there
        finish_rep(true, C, goes_on && !(BATCH && !WIDE));
        S = S_next;
        N += 1;
        red_add(reinterpret_cast<long long *>(&pst()[kPsRetained]), 1 + over);
        if (S > B) red_add(reinterpret_cast<long long *>(&pst()[kPsZero]), 1);   // only a slot's first replication ends beyond B
        if (goes_on) { ++r; start_rep(); }
        else end_slot(true);
    };

    auto abort_rep = [&]() {                  // doomed: S_p(r) would exceed B; discard it
        trace_end(2);
        red_add(reinterpret_cast<long long *>(&pst()[kPsProgress]), t);
        red_add(reinterpret_cast<long long *>(&pst()[kPsAborted]), 1);
        finish_rep(false, 0, false);
        end_slot(true);
    };

    auto limit_hit = [&]() {
        trace_end(3);
        red_add(reinterpret_cast<long long *>(&pst()[kPsProgress]), t);
        red_add(reinterpret_cast<long long *>(&pst()[kPsLimit]), 1);
        atomicExch(BATCH ? bp.error : p.error, 1);
        finish_rep(false, 0, false);
        end_slot(false);
    };

    // The clock reached t_end: 0 = go on, 1 = completed (met, or unmet at the meeting cap),
    // 2 = doomed, 3 = step limit.  A pair at the cap completes with C = t, so it is kept even when
    // t is also the clock at which an unfinished replication is doomed (S + C = B).  With lag L > 1
    // a pair whose X came back to Y_0 during the pre-lag updates meets at tau = L if X_L = Y_0.
    auto classify = [&]() -> int {
        if (COUPLED) {
            if (EXT && D == 0 && ycol != nullptr) {
                release_y();
                tau = t;
                t_end = min(max(ell, tau), stop_unmet);
                if (t < t_end) return 0;
            }
            if (D == 0 && t >= ell) return 1;
            if (v_capped() && t >= v_step_limit()) return 1;
            return t >= abort_t ? 2 : 3;
        }
        return t >= v_unit() ? 1 : 3;
    };

    // X moved at site I on a step where Y_{t+1-L} = X_{t+1} (met), or on a pre-lag update t < L
    // where Y stays at Y_0 = X_t: the counts of I's pools (from the values loaded this step), the
    // event -+w1(t), the number of window indices r <= t (after meeting, X's -+W(t) and Y's
    // +-W(t-L) add to it; before t = L only X moves and W(t) is the same count, W(t-L) being 0)
    // and, on a pre-lag update, the start of an unmet stretch.
    auto met_flip = [&](uint32_t I, uint32_t q, uint32_t bit, uint32_t xw, uint32_t nX,
                        const uint32_t *ent, const uint32_t *cx) {
        st[q * 32] = xw ^ bit;
        const uint32_t delta = nX ? 1u : 0xFFu;
#pragma unroll
        for (int l = 0; l < kRow; ++l)
            if (real(l, ent)) cbase[ent[l] & 0x7FFFu] = static_cast<unsigned char>(cx[l] + delta);
        const uint32_t w = wstep(t);
        if (w) {
            const long long ev = nX ? -static_cast<long long>(w) : static_cast<long long>(w);
            red_add(racc(I), ev);
            red_add(sacc(I), ev);
            red_or(&trep()[q], bit);
        }
        rep_words |= 1u << (q >> gshift);
        if (COUPLED && t < v_lag()) {       // X_{t+1} differs from Y_0 = X_t in bit I
            D = 1; tau = 0; t_end = stop_unmet;
            if (!EXT || ycol == nullptr) {      // first move: Y_0 = X_t to the Y column
                acquire_y();
                if (v_Tnu()) copy_y0(q, bit, ent, cx);
            }
        }
    };

    // A pair that has not met: X and Y move separately (events -+W(t) and +-W(t-L)); D follows
    // the Hamming distance, and at D = 0 the pair has met at tau = t + 1 if t + 1 >= L.  Before
    // that (t < L) Y stays at Y_0, and D = 0 means X came back to Y_0: the pair goes on (met
    // path, Y column kept) and classify decides at t = L.
    auto unmet_flip = [&](uint32_t I, uint32_t q, uint32_t bit, uint32_t xw, uint32_t yw,
                          uint32_t xI, uint32_t yI, uint32_t nX, uint32_t nY, const uint32_t *ent,
                          const uint32_t *cx, const uint32_t *cy) {
        long long ev = 0;
        const uint32_t lag = v_lag();
        if (EXT && t < lag) nY = yI;
        if (nX != xI) {
            st[q * 32] = xw ^ bit;
            const uint32_t delta = nX ? 1u : 0xFFu;
#pragma unroll
            for (int l = 0; l < kRow; ++l)
                if (real(l, ent)) cbase[ent[l] & 0x7FFFu] = static_cast<unsigned char>(cx[l] + delta);
            const long long w = wpre(t);
            ev += nX ? -w : w;
        }
        if (nY != yI) {
            ycol[q * 32] = yw ^ bit;
            unsigned char *yb = reinterpret_cast<unsigned char *>(ycol);
            const uint32_t delta = nY ? 1u : 0xFFu;
#pragma unroll
            for (int l = 0; l < kRow; ++l)
                if (real(l, ent)) yb[ent[l] & 0x7FFFu] = static_cast<unsigned char>(cy[l] + delta);
            const long long w = wpre(static_cast<long long>(t) - lag);
            ev += nY ? w : -w;
        }
        if (ev != 0) {
            red_add(racc(I), ev);
            red_add(sacc(I), ev);
            red_or(&trep()[q], bit);
        }
        rep_words |= 1u << (q >> gshift);
        D = D + (nX ^ nY) - (xI ^ yI);
        if (D == 0) {
            if (!EXT || t + 1 >= lag) {
                release_y();
                tau = t + 1;
                t_end = min(max(ell, tau), stop_unmet);
            } else {
                t_end = lag;
            }
        }
    };

    // One step of the pair.  X's full conditional from its counts; when some lane of the warp
    // has not met, Y's from its own column (a met lane reads its X column there, so Y = X).
    // The uniform U = wu 2^32 + lo needs lo only when wu equals a threshold's high word.
    // The site a step word selects (alias draw).
    auto site_of = [&](uint32_t ws) -> uint32_t {
        const unsigned long long prod = static_cast<unsigned long long>(ws) * static_cast<uint32_t>(na);
        const uint32_t col = static_cast<uint32_t>(prod >> 32), coin = static_cast<uint32_t>(prod);
        const unsigned long long e = aliasAt(col);
        return coin < static_cast<uint32_t>(e) ? col : static_cast<uint32_t>(e >> 32);
    };
    // The site of the current step and its row, drawn ahead: they depend on the step words only,
    // so the next step's alias and row loads overlap this step's work.
    uint32_t I_cur = 0;
    uint4 row_cur = make_uint4(0u, 0u, 0u, 0u);
    auto step = [&](uint32_t ws_next, uint32_t wu) -> int {
        uint32_t I;
        uint4 row;
        if (SYSTEMATIC) {
            I = sysI;
            row = rowAt(I);
        } else {
            I = I_cur;
            row = row_cur;
            I_cur = site_of(ws_next);
            row_cur = rowAt(I_cur);
        }
        const uint32_t q = I >> 5, bit = 1u << (I & 31);
        const uint32_t xw = st[q * 32];
        const uint32_t xI = (xw & bit) ? 1u : 0u;
        uint32_t ent[8];
        entries(row, ent);
        uint32_t cx[kRow], cy[kRow];
        uint32_t ix = 0;
#pragma unroll
        for (int l = 0; l < kRow; ++l) {
            cx[l] = 0u;
            cy[l] = 0u;
            if (l < NE && (DEG > 0 || l < deg)) {
                if constexpr (MASKT) {     // plain offsets, positive-outcome pools first
                    cx[l] = cbase[ent[l]];
                    if (cx[l] == xI) ix |= 1u << l;                // c_j - x_I = 0: pool j decides
                } else {
                    cx[l] = cbase[ent[l] & 0x7FFFu];
                    if (cx[l] == xI) ix += (ent[l] >> 15) ? 9u : 1u;
                }
            }
        }
        if constexpr (MASKT) ix += ent[kRow - 1] << 6;           // row of the positive-pool count
        const unsigned long long TX = tAt(ix);
        unsigned long long TY = TX;
        uint32_t yw = xw, yI = xI;
        bool own = false;
        // Y's side, for the lanes that have not met (a met lane keeps Y = X).
        auto ypart = [&](const uint32_t *yp) {
            const unsigned char *yb = reinterpret_cast<const unsigned char *>(yp);
            yw = own ? yp[q * 32] : xw;
            yI = (yw & bit) ? 1u : 0u;
            uint32_t iy = 0;
#pragma unroll
            for (int l = 0; l < kRow; ++l) {
                if (l < NE && (DEG > 0 || l < deg)) {
                    if constexpr (MASKT) {
                        cy[l] = own ? static_cast<uint32_t>(yb[ent[l]]) : cx[l];
                        if (cy[l] == yI) iy |= 1u << l;
                    } else {
                        cy[l] = own ? static_cast<uint32_t>(yb[ent[l] & 0x7FFFu]) : cx[l];
                        if (cy[l] == yI) iy += (ent[l] >> 15) ? 9u : 1u;
                    }
                }
            }
            if constexpr (MASKT) iy += ent[kRow - 1] << 6;
            TY = tAt(iy);
        };
        if (COUPLED) {
            const bool ymode = __any_sync(__activemask(), D != 0);
            if (ymode) {
                own = D != 0;
                ypart(ycol);
            }
        }
        const uint32_t thx = static_cast<uint32_t>(TX >> 32), thy = static_cast<uint32_t>(TY >> 32);
        uint32_t nX = wu < thx ? 1u : 0u, nY = wu < thy ? 1u : 0u;
        if (wu == thx || wu == thy) {
            const uint32_t lo = philox_low_word(make_uint4(t, r, slot_g, instance | (2u << 24)), k0, k1);
            if (wu == thx) nX = lo < static_cast<uint32_t>(TX) ? 1u : 0u;
            if (wu == thy) nY = lo < static_cast<uint32_t>(TY) ? 1u : 0u;
        }
        if constexpr (TRACE) {
            // draw t moves X_{t+1} and, from t = L on, Y_{t+1-L}; a pair that has met moves both
            // alike, and before t = L Y stays at Y_0
            if (trec && t < static_cast<uint32_t>(p.trace_steps)) {
                const uint32_t xf = nX != xI ? 1u : 0u;
                const uint32_t yf = !COUPLED ? 0u
                                    : own ? ((nY != yI && !(EXT && t < v_lag())) ? 1u : 0u)
                                          : (xf && t >= v_lag() ? 1u : 0u);
                trec[4 + t] = static_cast<int32_t>(I | (xf << 16) | (yf << 17));
            }
        }
        if (COUPLED && own) {
            if ((nX ^ xI) | (nY ^ yI)) unmet_flip(I, q, bit, xw, yw, xI, yI, nX, nY, ent, cx, cy);
        } else if (nX != xI) {
            met_flip(I, q, bit, xw, nX, ent, cx);
        }
        ++t;
        if (SYSTEMATIC) { ++sysI; if (sysI == static_cast<uint32_t>(na)) sysI = 0; }
        return t < t_end ? 0 : classify();
    };

    // Step draws: one Philox block per pair of steps (for a single instance with the round keys
    // precomputed in the kernel parameters).
    auto draw = [&](uint32_t c0) -> uint4 {
        if constexpr (BATCH) return philox10(make_uint4(c0, r, slot_g, instance), k0, k1);
        else return philox10_rk(make_uint4(c0, r, slot_g, instance), p.rk);
    };
    // Random start Z_0 ~ prod Bernoulli(nu_i): the initial state of lane src's new replication
    // (batched: of src's instance), drawn by every lane of `act`.  Lane e of the group takes the clone pairs e,
    // e + |act|, ... of the clones with nu_i > 0 (one Philox block each, tag 1, counter
    // (a / 2, r, slot, instance)), and sets the bits and pool counts it draws in src's column with
    // shared-memory atomics (a count word holds four pools of one column, and a count never passes
    // 255, so adding 1 << 8 b touches only its own byte).  The same draws and the same state as one
    // lane drawing them all, in about 1/|act| of the time, and not divergent.
    auto coop_init = [&](int src, unsigned act) {
        if constexpr (BATCH) {
            // src's instance: its tables, seed and layout
            const int c_s = __shfl_sync(act, cur, src);
            const uint32_t r_s = __shfl_sync(act, r, src), slot_s = __shfl_sync(act, slot_g, src);
            const InstDesc &d = bp.insts[c_s];
            const uint32_t *ip = d.init_pairs;
            const unsigned long long *tnu = reinterpret_cast<const unsigned long long *>(d.Tnu);
            const int n_ip = d.n_init_pairs, na_s = d.na, deg_s = d.deg;
            const uint32_t dummy_s = d.dummy_entry, inst_s = d.instance, W_s = static_cast<uint32_t>(d.W);
            const uint32_t k0_s = static_cast<uint32_t>(d.seed), k1_s = static_cast<uint32_t>(d.seed >> 32);
            const uint4 *rows_s = reinterpret_cast<const uint4 *>(MASKT ? d.rows_mask : d.rows);
            uint32_t gsh = 0;
            while (((W_s + (1u << gsh) - 1) >> gsh) > 32) ++gsh;
            uint32_t *const st_s = regions + warp * region_words + src;
            unsigned char *const cb_s = reinterpret_cast<unsigned char *>(st_s);
            const int nthr = __popc(act), rank = __popc(act & ((1u << lane) - 1u));
            uint32_t groups = 0;
            for (int e = rank; e < n_ip; e += nthr) {
                const int a = static_cast<int>(ip[e]);
                const uint4 b = philox10(make_uint4(static_cast<uint32_t>(a) >> 1, r_s, slot_s, inst_s | (1u << 24)),
                                         k0_s, k1_s);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = a + h;
                    if (c >= na_s) break;
                    const unsigned long long u = h ? ((static_cast<unsigned long long>(b.z) << 32) | b.w)
                                                   : ((static_cast<unsigned long long>(b.x) << 32) | b.y);
                    if (u < tnu[c]) {
                        const uint32_t q = c >> 5;
                        atomicOr(&st_s[q * 32], 1u << (c & 31));
                        uint32_t ent[8];
                        entries(__ldg(rows_s + c), ent);
#pragma unroll
                        for (int l = 0; l < kRow; ++l) {
                            if (!(l < NE && (DEG > 0 || (l < deg_s && ent[l] != dummy_s)))) continue;
                            const uint32_t off = MASKT ? ent[l] : (ent[l] & 0x7FFFu);
                            atomicAdd(reinterpret_cast<uint32_t *>(cb_s + (off & ~3u)), 1u << (8u * (off & 3u)));
                        }
                        groups |= 1u << (q >> gsh);
                    }
                }
            }
            groups = __reduce_or_sync(act, groups);
            if (lane == src) rep_words |= groups;
            __syncwarp(act);
        } else {
            const uint32_t r_s = __shfl_sync(act, r, src), slot_s = __shfl_sync(act, slot_g, src);
            uint32_t *const st_s = regions + warp * region_words + src;
            unsigned char *const cb_s = reinterpret_cast<unsigned char *>(st_s);
            const int nthr = __popc(act), rank = __popc(act & ((1u << lane) - 1u));
            uint32_t groups = 0;
            for (int e = rank; e < p.n_init_pairs; e += nthr) {
                const int a = static_cast<int>(p.init_pairs[e]);
                const uint4 b = philox10_rk(make_uint4(static_cast<uint32_t>(a) >> 1, r_s, slot_s,
                                                       instance | (1u << 24)), p.rk);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = a + h;
                    if (c >= na) break;
                    const unsigned long long u = h ? ((static_cast<unsigned long long>(b.z) << 32) | b.w)
                                                   : ((static_cast<unsigned long long>(b.x) << 32) | b.y);
                    if (u < p.Tnu[c]) {
                        const uint32_t q = c >> 5;
                        atomicOr(&st_s[q * 32], 1u << (c & 31));
                        uint32_t ent[8];
                        entries(rowAt(c), ent);
#pragma unroll
                        for (int l = 0; l < kRow; ++l) {
                            if (!real(l, ent)) continue;
                            const uint32_t off = MASKT ? ent[l] : (ent[l] & 0x7FFFu);
                            atomicAdd(reinterpret_cast<uint32_t *>(cb_s + (off & ~3u)), 1u << (8u * (off & 3u)));
                        }
                        groups |= 1u << (q >> gshift);
                    }
                }
            }
            groups = __reduce_or_sync(act, groups);
            if (lane == src) rep_words |= groups;
            __syncwarp(act);
        }
    };

    // The end of lane src's completed replication (deferred by finish_rep), by every lane of act:
    // the lane of rank e in act takes the words e, e + |act|, ... of src's column that lie in
    // src's fin_words groups.
    // Each reads its word of the replication's touched bits (independent loads across the lanes,
    // where one lane alone would wait on a chain of dependent loads), zeroes the replication sums
    // of those clones, adds the closing term w(C) of every site set in X_C to the slot's sums,
    // marks the slot's touched bits, and clears the word in the touched set and in X_C; the lanes
    // also zero X_C's count words (the padding pool's word back to its value).  The same state and
    // the same sums as src doing it alone, once every lane's writes are fenced.
    const long long pw = pair_words(stride_na, stride_W);
    auto coop_finish = [&](int src, unsigned act) {
        const uint32_t words_s = __shfl_sync(act, fin_words, src);
        const long long wX_s = __shfl_sync(act, fin_wX, src);
        uint32_t W_s, gsh_s, wpp_s, dwi_s, dw_s;
        if constexpr (BATCH) {
            const InstDesc &d = bp.insts[__shfl_sync(act, cur, src)];
            W_s = static_cast<uint32_t>(__ldg(&d.W));
            wpp_s = static_cast<uint32_t>(__ldg(&d.wpp));
            dwi_s = static_cast<uint32_t>(__ldg(&d.dummy_word_index));
            dw_s = __ldg(&d.dummy_word);
            gsh_s = __shfl_sync(act, gshift, src);
        } else {
            W_s = W; gsh_s = gshift;
            wpp_s = static_cast<uint32_t>(p.wpp);
            dwi_s = static_cast<uint32_t>(p.dummy_word_index);
            dw_s = p.dummy_word;
        }
        long long *const pb_s = pb + static_cast<long long>(src - lane) * pw;
        uint32_t *const trep_s = reinterpret_cast<uint32_t *>(pb_s + 2 * stride_na + kPairStats);
        uint32_t *const tslot_s = trep_s + stride_W;
        uint32_t *const st_s = regions + warp * region_words + src;
        const uint32_t nthr = static_cast<uint32_t>(__popc(act));
        const uint32_t rank = static_cast<uint32_t>(__popc(act & ((1u << lane) - 1u)));
        uint32_t grp = 0;
        for (uint32_t q = rank; q < W_s; q += nthr) {
            const uint32_t g = q >> gsh_s;
            if (!((words_s >> g) & 1u)) continue;
            const uint32_t xw = st_s[q * 32];
            const uint32_t tw = __ldcg(&trep_s[q]);
            uint32_t tm = tw;
            while (tm) {
                const int b = __ffs(tm) - 1;
                tm &= tm - 1;
                pb_s[2 * static_cast<size_t>(q * 32 + b)] = 0;            // replication sum
            }
            if (wX_s != 0) {
                uint32_t om = xw;
                while (om) {
                    const int b = __ffs(om) - 1;
                    om &= om - 1;
                    red_add(pb_s + 2 * static_cast<size_t>(q * 32 + b) + 1, wX_s);   // slot sum
                }
            }
            const uint32_t touched = tw | (wX_s != 0 ? xw : 0u);
            if (tw) trep_s[q] = 0u;
            if (xw) st_s[q * 32] = 0u;
            if (touched) { red_or(&tslot_s[q], touched); grp |= 1u << g; }
        }
        for (uint32_t w = W_s + rank; w < wpp_s; w += nthr) st_s[w * 32] = w == dwi_s ? dw_s : 0u;
        grp = __reduce_or_sync(act, grp);
        if (lane == src) slot_words |= grp;
        // src's next replication reduces into the sums and touched words these lanes just stored
        // to, and its slot's flush reads the slot sums they reduced into: every lane's global
        // writes are performed (GPU scope) before the warp goes on.
        __threadfence();
        __syncwarp(act);
    };

    start_slot();
    uint4 blk = draw(t >> 1);
    auto first_site = [&]() {               // the first step of a block
        if (!SYSTEMATIC) { I_cur = site_of(blk.x); row_cur = rowAt(I_cur); }
    };
    // A batched thread that found no slot has loaded no instance (its table pointers are null):
    // only threads with a slot draw their first site.
    if (alive) first_site();
    // The lanes still in the loop (every lane of the warp runs the kernel to its end, so the first
    // ballot names all 32).  The warp meets at the bottom of each iteration, so that the end of a
    // replication, or a random start, that a lane reached in a divergent branch is worked by all
    // of them at the top of the next, not only by the lanes that reached it with that lane.
    const bool rnd_run = RND && (BATCH ? bp.any_init != 0 : p.Tnu != nullptr);
    unsigned live = __ballot_sync(0xFFFFFFFFu, alive);
    while (alive) {
        {
            unsigned pend = __ballot_sync(live, fin_pending);
            if (pend) {
                // An ending lane's last flip events (reductions into its touched words and sums,
                // some issued this iteration) are performed before the other lanes read or store
                // to those words.
                if (fin_pending) __threadfence();
                __syncwarp(live);
                while (pend) {
                    const int src = __ffs(pend) - 1;
                    pend &= pend - 1;
                    coop_finish(src, live);
                }
                fin_pending = false;
            }
        }
        if constexpr (RND) {
            if (rnd_run) {   // random starts of lanes that began a replication
                unsigned pend = __ballot_sync(live, init_pending);
                while (pend) {
                    const int src = __ffs(pend) - 1;
                    pend &= pend - 1;
                    coop_init(src, live);
                }
                init_pending = false;
            }
        }
        // words (0,1) at even t and (2,3) at odd t; the next block is computed ahead (its first
        // site word is the second step's prefetch) and discarded if the replication ends
        uint4 nxt;
        int ended = 0;
        if constexpr (!BATCH && DEG <= kMaskDeg) {
            // both steps of the block inlined, the next block drawn between them
            ended = step(blk.z, blk.y);
            if (!ended) {
                nxt = draw((t >> 1) + 1);
                ended = step(nxt.x, blk.w);
            }
        } else if constexpr (BATCH && !WIDE) {
            // both steps inlined, the next block drawn first (measured faster here)
            nxt = draw((t >> 1) + 1);
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (!ended) ended = step(h ? nxt.x : blk.z, h ? blk.w : blk.y);
        } else {
            // the 20-warp batch and degree-7/8 builds would spill with both steps inlined
            nxt = draw((t >> 1) + 1);
#pragma unroll 1
            for (int h = 0; h < 2 && !ended; ++h) ended = step(h ? nxt.x : blk.z, h ? blk.w : blk.y);
        }
        if (ended) {
            if (ended == 1) complete();
            else if (ended == 2) abort_rep();
            else limit_hit();
            blk = draw(t >> 1);
            first_site();
        } else {
            blk = nxt;
        }
        live = __ballot_sync(live, alive);
    }

    // Split the packed records.  Started: count (low half) and, batched, the pre-lag updates (high
    // half).  Every replication started has ended retained, aborted or at the step limit, so the
    // retained count is started - aborted - limit and the rest of the retained record is the audit
    // count times 2^32.  Both splits are exact while the pair ran fewer than 2^32 progress units
    // (every replication takes at least one, and every pre-lag update is one).
    {
        const unsigned long long progress = __ldcg(&pst()[kPsProgress]);
        const unsigned long long sp = __ldcg(&pst()[kPsStarted]);
        const unsigned long long started = sp & 0xFFFFFFFFull;
        const unsigned long long prelag = BATCH && EXT ? sp >> 32 : started * v_lag();
        const unsigned long long packed = __ldcg(&pst()[kPsRetained]);
        const unsigned long long kept = started - __ldcg(&pst()[kPsAborted]) - __ldcg(&pst()[kPsLimit]);
        pst()[kPsStarted] = started;
        pst()[kPsRetained] = kept;
        pst()[kPsTauAudit] = (packed - kept) >> 32;
        pst()[kPsSiteUpdates] = COUPLED ? 2 * progress - prelag : progress;
        if (progress >> 32) atomicAdd(&counters[kPackLost], 1ull);
    }

    // Every lane of the warp is here: sum (or max) the pairs' statistics over the warp.
    const int dst[kPairStats] = {kProgress, kRepsStarted, kRepsRetained, kRepsAborted,
                                 kZeroCompletion, kStepLimitHits, kSumTau, kMaxTau, kTauOverAudit,
                                 kSiteUpdates};
#pragma unroll
    for (int i = 0; i < kPairStats; ++i) {
        unsigned long long v = __ldcg(&pst()[i]);
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long u = __shfl_down_sync(0xFFFFFFFFu, v, o);
            v = i == kPsMaxTau ? max(v, u) : v + u;
        }
        if (lane == 0 && v) {
            if (i == kPsMaxTau) atomicMax(&counters[dst[i]], v);
            else atomicAdd(&counters[dst[i]], v);
        }
    }
}

}  // namespace
}  // namespace mcpd
