// Host-side set-up of the sampler tables: likelihood constants, naive scores and pruning, score
// weights, their integer alias table, the acceptance thresholds of the full conditional, and the
// shared-memory layout of one coupled pair.  Compiled with -ffp-contract=off: every double
// expression below is evaluated operation by operation in the order written, which is the order
// the written spec of the tables fixes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <numeric>

#include "mcpd_internal.h"

namespace mcpd {
namespace {

constexpr double kTwo32 = 4294967296.0;

// floor(p * 2^64) for p in [0, 1], saturating at 2^64 - 1.
uint64_t scaled_threshold(double p) {
    if (!(p < 1.0)) return UINT64_MAX;
    if (!(p > 0.0)) return 0;
    return static_cast<uint64_t>(std::ldexp(p, 64));
}

int64_t round_half_even(double x) { return static_cast<int64_t>(std::nearbyint(x)); }

int fail(std::string *err, const std::string &msg, int code) {
    if (err) *err = msg;
    return code;
}

}  // namespace

int build_tables(const mcpd_design *d, const uint8_t *y, const mcpd_params *prm, Tables *out,
                 std::string *err) {
    if (!d || !y || !prm || !out) return fail(err, "null argument", MCPD_EINVAL);
    const int32_t n = d->n_clones, m = d->n_pools;
    if (n < 1 || m < 0 || !d->clone_ptr || (!d->clone_pools && n > 0 && d->clone_ptr[n] > 0))
        return fail(err, "bad design sizes", MCPD_EINVAL);
    if (n > kMaxClones) return fail(err, "more than 65535 clones", MCPD_ETOO_LARGE);
    if (m > kMaxPools) return fail(err, "more than 1022 pools", MCPD_ETOO_LARGE);
    const double fp = prm->fp, fn = prm->fn, q = prm->prior_q;
    if (!(fp > 0.0 && fp < 1.0) || !(fn > 0.0 && fn < 1.0) || !(q > 0.0 && q < 1.0))
        return fail(err, "fp, fn and prior_q must lie in (0, 1)", MCPD_EINVAL);
    if (prm->scan < MCPD_SCAN_SCORE || prm->scan > MCPD_SCAN_CUSTOM)
        return fail(err, "unknown scan", MCPD_EINVAL);
    if (prm->coupled && prm->scan == MCPD_SCAN_SYSTEMATIC)
        return fail(err, "the systematic scan is time-inhomogeneous: uncoupled only", MCPD_EINVAL);
    if (prm->scan == MCPD_SCAN_CUSTOM && !prm->scan_weights)
        return fail(err, "custom scan without weights", MCPD_EINVAL);
    if (prm->lanes_per_pair != 0 && prm->lanes_per_pair != 1)
        return fail(err, "lanes_per_pair must be 0 or 1", MCPD_EINVAL);
    if (d->clone_ptr[0] != 0) return fail(err, "clone_ptr[0] must be 0", MCPD_EINVAL);
    for (int32_t i = 0; i < n; ++i) {
        if (d->clone_ptr[i + 1] < d->clone_ptr[i]) return fail(err, "clone_ptr decreases", MCPD_EINVAL);
        if (d->clone_ptr[i + 1] - d->clone_ptr[i] > kRow)
            return fail(err, "a clone sits in more than 8 pools", MCPD_ETOO_LARGE);
        for (int32_t e = d->clone_ptr[i]; e < d->clone_ptr[i + 1]; ++e) {
            int32_t j = d->clone_pools[e];
            if (j < 0 || j >= m) return fail(err, "pool id out of range", MCPD_EINVAL);
            if (e > d->clone_ptr[i] && j <= d->clone_pools[e - 1])
                return fail(err, "pools of a clone must be strictly increasing", MCPD_EINVAL);
        }
    }
    for (int32_t j = 0; j < m; ++j)
        if (y[j] > 1) return fail(err, "y must hold 0/1 bytes", MCPD_EINVAL);

    Tables &t = *out;
    t = Tables();
    t.n = n; t.m = m; t.scan = prm->scan; t.coupled = prm->coupled != 0;

    // Likelihood ratio terms: Pr{y=1|xi=1} = 1 - fn, Pr{y=1|xi=0} = fp.
    const double a_pos = std::log(1.0 - fn) - std::log(fp);
    const double a_neg = std::log(fn) - std::log(1.0 - fp);
    const double lam = std::log(q) - std::log(1.0 - q);
    auto a_of = [&](int32_t j) { return y[j] ? a_pos : a_neg; };

    // Naive log score eta_i = lambda + log R_i = (lambda + n+_i a+) + n-_i a- (R_i, the product of
    // the likelihood ratios of the pools holding i, depends on its positive and negative pool
    // counts only, so clones with equal counts tie exactly and go to the lower index), and
    // pruning to the top n_active.
    std::vector<double> eta(n);
    for (int32_t i = 0; i < n; ++i) {
        int32_t npos = 0, nneg = 0;
        for (int32_t e = d->clone_ptr[i]; e < d->clone_ptr[i + 1]; ++e) (y[d->clone_pools[e]] ? npos : nneg) += 1;
        eta[i] = (lam + static_cast<double>(npos) * a_pos) + static_cast<double>(nneg) * a_neg;
    }
    int32_t na = (prm->n_active <= 0 || prm->n_active >= n) ? n : prm->n_active;
    std::vector<char> keep(n, 1);
    if (na < n) {
        std::vector<int32_t> order(n);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return eta[a] > eta[b]; });
        std::fill(keep.begin(), keep.end(), 0);
        for (int32_t r = 0; r < na; ++r) keep[order[r]] = 1;
    }
    t.na = na;
    for (int32_t i = 0; i < n; ++i) if (keep[i]) t.active.push_back(i);

    // Pool sizes over the active clones, and the pool-size limit of byte counts.
    std::vector<int32_t> dA(m + 1, 0);
    for (int32_t a = 0; a < na; ++a) {
        int32_t i = t.active[a];
        int32_t deg = d->clone_ptr[i + 1] - d->clone_ptr[i];
        t.deg_max = std::max(t.deg_max, deg);
        for (int32_t e = d->clone_ptr[i]; e < d->clone_ptr[i + 1]; ++e) dA[d->clone_pools[e]]++;
    }
    t.udeg = t.deg_max;
    for (int32_t a = 0; a < na; ++a) {
        const int32_t i = t.active[a];
        if (d->clone_ptr[i + 1] - d->clone_ptr[i] != t.deg_max) { t.udeg = 0; break; }
    }
    for (int32_t j = 0; j < m; ++j)
        if (dA[j] > kMaxPoolSize) return fail(err, "a pool holds more than 255 active clones", MCPD_ETOO_LARGE);

    // Scan weights.
    t.w.assign(na, 0.0);
    if (prm->scan == MCPD_SCAN_SCORE) {
        std::vector<double> s(na);
        for (int32_t a = 0; a < na; ++a) {
            int32_t i = t.active[a];
            double acc = 0.0;
            for (int32_t e = d->clone_ptr[i]; e < d->clone_ptr[i + 1]; ++e) {
                int32_t j = d->clone_pools[e];
                acc = acc + static_cast<double>(dA[j]) * a_of(j);
            }
            s[a] = acc;
        }
        double smax = s[0], smin = s[0];
        for (int32_t a = 1; a < na; ++a) { smax = std::max(smax, s[a]); smin = std::min(smin, s[a]); }
        const double gamma = 100.0 * static_cast<double>(na);
        const double tau = (smax > smin) ? std::log(gamma) / (smax - smin) : 0.0;
        double total = 0.0;
        for (int32_t a = 0; a < na; ++a) { t.w[a] = std::exp(tau * (s[a] - smax)); total = total + t.w[a]; }
        for (int32_t a = 0; a < na; ++a) t.w[a] = 0.5 * (t.w[a] / total) + 0.5 / static_cast<double>(na);
    } else if (prm->scan == MCPD_SCAN_CUSTOM) {
        double total = 0.0;
        for (int32_t a = 0; a < na; ++a) {
            double v = prm->scan_weights[a];
            if (!(v > 0.0) || !std::isfinite(v)) return fail(err, "custom weights must be positive", MCPD_EINVAL);
            total = total + v;
        }
        for (int32_t a = 0; a < na; ++a) t.w[a] = prm->scan_weights[a] / total;
    } else {
        for (int32_t a = 0; a < na; ++a) t.w[a] = 1.0 / static_cast<double>(na);
    }

    // Integer weights V (sum n_a 2^32) and the integer alias table (columns of mass 2^32).
    const uint64_t K = uint64_t(1) << 32;
    std::vector<uint64_t> V(na);
    if (prm->scan == MCPD_SCAN_UNIFORM || prm->scan == MCPD_SCAN_SYSTEMATIC) {
        std::fill(V.begin(), V.end(), K);
    } else {
        const double scale = static_cast<double>(na) * kTwo32;
        uint64_t sum = 0;
        for (int32_t a = 0; a < na; ++a) {
            uint64_t v = static_cast<uint64_t>(std::floor(t.w[a] * scale));
            V[a] = std::max<uint64_t>(v, 1);
            sum += V[a];
        }
        const int64_t deficit = static_cast<int64_t>((static_cast<uint64_t>(na) << 32) - sum);
        int32_t top = static_cast<int32_t>(std::max_element(V.begin(), V.end()) - V.begin());
        V[top] = static_cast<uint64_t>(static_cast<int64_t>(V[top]) + deficit);
        for (int32_t a = 0; a < na; ++a)
            if (V[a] < (uint64_t(1) << 30))
                return fail(err, "a scan weight is below 0.25 / n_a", MCPD_EINVAL);
    }
    std::vector<uint32_t> prob(na, 0xFFFFFFFFu), alias(na);
    std::iota(alias.begin(), alias.end(), 0u);
    {
        std::deque<int32_t> small, large;
        std::vector<uint64_t> rem = V;
        for (int32_t a = 0; a < na; ++a) (rem[a] < K ? small : large).push_back(a);
        while (!small.empty() && !large.empty()) {
            int32_t s = small.front(); small.pop_front();
            int32_t g = large.front();
            prob[s] = static_cast<uint32_t>(rem[s]);
            alias[s] = static_cast<uint32_t>(g);
            rem[g] -= K - rem[s];
            if (rem[g] < K) { large.pop_front(); small.push_back(g); }
        }
    }
    t.alias.resize(na);
    for (int32_t a = 0; a < na; ++a) t.alias[a] = uint64_t(prob[a]) | (uint64_t(alias[a]) << 32);

    // Acceptance thresholds T[n+][n-] = floor(sigma(lambda + n+ a+ + n- a-) 2^64), at least 1.
    t.T.assign(kTSide * kTSide, 0);
    for (int32_t p = 0; p < kTSide; ++p)
        for (int32_t r = 0; r < kTSide; ++r) {
            const double z = (lam + static_cast<double>(p) * a_pos) + static_cast<double>(r) * a_neg;
            const double pr = 1.0 / (1.0 + std::exp(-z));
            uint64_t v = scaled_threshold(pr);
            t.T[p * kTSide + r] = v == 0 ? 1 : v;
        }
    if (prm->init_marginals) {
        t.Tnu.resize(na);
        for (int32_t a = 0; a < na; ++a) {
            double v = prm->init_marginals[a];
            if (!(v >= 0.0 && v <= 1.0)) return fail(err, "init marginals must lie in [0, 1]", MCPD_EINVAL);
            t.Tnu[a] = scaled_threshold(v);
        }
        for (int32_t a = 0; a < na; a += 2)
            if (t.Tnu[a] || (a + 1 < na && t.Tnu[a + 1])) t.init_pairs.push_back(static_cast<uint32_t>(a));
    }

    // Shared-memory layout of one pair (the X chain): W words of bits, then one count byte per
    // pool, the padding pool m last.  Word w of a pair lives at word (w * 32 + lane) of its warp's
    // region, so the byte of pool j sits at (W + j / 4) * 128 + j % 4 from the lane's base.  The Y
    // chain uses the same layout, contiguous, in global memory while the pair has not met.
    t.W = (na + 31) / 32;
    t.Mp = (m + 1 + 3) / 4;
    t.wpp = t.W + t.Mp;
    auto count_offset = [&](int32_t j) -> uint32_t {
        return static_cast<uint32_t>((t.W + (j >> 2)) * 128 + (j & 3));
    };
    if (count_offset(m) > 0x7FFFu) return fail(err, "pair state too large for 15-bit offsets", MCPD_ETOO_LARGE);
    t.dummy_entry = static_cast<uint16_t>(count_offset(m));
    t.dummy_word_index = t.W + (m >> 2);
    t.dummy_word = 2u << (8 * (m & 3));
    t.rows.assign(static_cast<size_t>(na) * kRow, t.dummy_entry);
    t.rows_pool.assign(static_cast<size_t>(na) * kRow, 0xFFFFu);
    for (int32_t a = 0; a < na; ++a) {
        int32_t i = t.active[a];
        int32_t l = 0;
        for (int32_t e = d->clone_ptr[i]; e < d->clone_ptr[i + 1]; ++e, ++l) {
            int32_t j = d->clone_pools[e];
            t.rows[static_cast<size_t>(a) * kRow + l] = static_cast<uint16_t>(count_offset(j) | (y[j] ? 0x8000u : 0u));
            t.rows_pool[static_cast<size_t>(a) * kRow + l] = static_cast<uint16_t>(j | (y[j] ? 0x8000u : 0u));
        }
    }
    // Runs with a uniform degree 3 <= d <= kMaskDeg (single-instance kernels compiled for d, coupled
    // or not): each row lists the clone's positive-outcome pools first, as plain count offsets,
    // with their number in entry kRow - 1; T_mask[npos][m] = T[9 n+ + n-] for the mask m of
    // deciding pools (n+ of them among the first npos entries, n- among the rest).  The same
    // thresholds, indexed without per-entry codes.
    t.rows_mask.clear();
    t.T_mask.clear();
    if (t.udeg >= 3 && t.udeg <= kMaskDeg) {                  // the kernels compiled for degree d
        t.rows_mask.assign(static_cast<size_t>(na) * kRow, 0);
        for (int32_t a = 0; a < na; ++a) {
            const uint16_t *src = &t.rows[static_cast<size_t>(a) * kRow];
            uint16_t *dst = &t.rows_mask[static_cast<size_t>(a) * kRow];
            int32_t fill = 0;
            for (int32_t l = 0; l < t.udeg; ++l) if (src[l] & 0x8000u) dst[fill++] = static_cast<uint16_t>(src[l] & 0x7FFFu);
            const int32_t npos = fill;
            for (int32_t l = 0; l < t.udeg; ++l) if (!(src[l] & 0x8000u)) dst[fill++] = src[l];
            dst[kRow - 1] = static_cast<uint16_t>(npos);
        }
        t.T_mask.assign(static_cast<size_t>(kMaskDeg + 1) * 64, 0);
        for (int32_t npos = 0; npos <= kMaskDeg; ++npos)
            for (int32_t mask = 0; mask < 64; ++mask) {
                int32_t np = 0, nn = 0;
                for (int32_t l = 0; l < 6; ++l)
                    if (mask >> l & 1) { if (l < npos) ++np; else ++nn; }
                t.T_mask[static_cast<size_t>(npos) * 64 + mask] = t.T[static_cast<size_t>(np) * kTSide + nn];
            }
    }

    // Window, horizon and bucket count.
    t.P = prm->slots;
    if (t.P < 1 || t.P > (int64_t(1) << 31)) return fail(err, "slots must be in [1, 2^31]", MCPD_EINVAL);
    if (prm->slot_offset < 0 || prm->slot_offset + t.P > (int64_t(1) << 32))
        return fail(err, "global slot ids must fit 32 bits", MCPD_EINVAL);
    if (t.coupled) {
        t.ell = prm->ell < 0 ? na : prm->ell;
        t.k = prm->k < 0 ? round_half_even(0.1 * static_cast<double>(na)) + 1 : prm->k;
        if (prm->k < 0 && t.k > t.ell) t.k = t.ell;
        if (t.k < 0 || t.k > t.ell) return fail(err, "need 0 <= k <= l", MCPD_EINVAL);
        t.L = t.ell - t.k + 1;
        t.lag = prm->lag > 1 ? prm->lag : 1;
        if (prm->lag < 0 || t.lag > (int64_t(1) << 20)) return fail(err, "lag must be in [0, 2^20]", MCPD_EINVAL);
        t.unit = std::max<int64_t>(std::max<int64_t>(t.ell, t.lag), 1);
    } else {
        t.burn = prm->burn < 0 ? round_half_even(0.1 * static_cast<double>(na)) : prm->burn;
        t.length = prm->length < 0 ? na - t.burn : prm->length;
        if (t.burn < 0 || t.length < 1 || t.burn + t.length < 2)
            return fail(err, "need b >= 0, T >= 1, b + T >= 2", MCPD_EINVAL);
        t.L = t.length;
        t.k = t.burn;
        t.ell = t.burn + t.length - 1;
        t.unit = t.burn + t.length - 1;
    }
    if (prm->budget_site_updates > 0.0) {
        const double per = prm->budget_site_updates / (static_cast<double>(t.P) * (t.coupled ? 2.0 : 1.0));
        t.B = static_cast<int64_t>(std::floor(per));
    } else {
        t.B = prm->horizon;
    }
    if (t.B < 0 || t.B > (int64_t(1) << 30)) return fail(err, "horizon must be in [0, 2^30]", MCPD_EINVAL);
    t.nb = std::max<int64_t>(1, t.B / t.unit);
    if (t.nb > kMaxBuckets) return fail(err, "too many N*_p buckets (horizon / l > 65536)", MCPD_ETOO_LARGE);
    if (prm->tau_audit < 0) return fail(err, "tau_audit must be >= 0", MCPD_EINVAL);
    t.tau_audit = t.coupled ? prm->tau_audit : 0;
    t.step_limit = prm->step_limit > 0 ? prm->step_limit : int64_t(10000) * na;
    if (t.step_limit > (int64_t(1) << 31)) return fail(err, "step_limit above 2^31", MCPD_EINVAL);
    if (!t.coupled) t.step_limit = std::max(t.step_limit, t.unit + 1);
    if (t.coupled && t.step_limit < t.lag) return fail(err, "step_limit below the lag", MCPD_EINVAL);
    if (prm->meeting_cap < 0) return fail(err, "meeting_cap must be >= 0", MCPD_EINVAL);
    if (t.coupled && prm->meeting_cap > 0) {
        if (prm->meeting_cap < t.unit)
            return fail(err, "meeting_cap must be >= max(l, lag, 1)", MCPD_EINVAL);
        if (prm->meeting_cap > (int64_t(1) << 31)) return fail(err, "meeting_cap above 2^31", MCPD_EINVAL);
        if (t.tau_audit > prm->meeting_cap) return fail(err, "tau_audit above meeting_cap", MCPD_EINVAL);
        t.capped = true;
        t.step_limit = prm->meeting_cap;
        if (t.tau_audit == 0) t.tau_audit = prm->meeting_cap;
    }
    // Integer bounds on a slot's sum G_p: coupled, |G| of one replication <= L (1 + 2 tau) and a
    // slot's retained replications cost at most B + step_limit draws in total; uncoupled, each
    // replication's G lies in [0, T] (T = L) and a slot keeps at most nb of them.
    const long double gmax = t.coupled ? static_cast<long double>(t.L) * (2.0L * (t.B + t.step_limit) + 1.0L)
                                       : static_cast<long double>(t.L) * static_cast<long double>(t.nb);
    if (gmax * t.P > 9.0e18L || gmax * gmax * t.P > 3.0e38L)
        return fail(err, "integer sums could overflow for this window, horizon and slot count", MCPD_EOVERFLOW);
    t.slot_offset = prm->slot_offset;
    t.trace_stride = prm->trace_stride > 0 ? prm->trace_stride : 0;
    if (prm->trace_steps < 0 || prm->trace_steps > (int64_t(1) << 20) || prm->trace_reps < 0 ||
        prm->trace_reps > 1024)
        return fail(err, "trace_steps must be in [0, 2^20] and trace_reps in [0, 1024]", MCPD_EINVAL);
    if (prm->trace_steps > 0 && t.trace_stride == 0)
        return fail(err, "trajectory records need trace_stride > 0", MCPD_EINVAL);
    t.trace_steps = prm->trace_steps;
    t.trace_reps = prm->trace_steps > 0 ? (prm->trace_reps > 0 ? prm->trace_reps : 8) : 0;
    t.record_slots = prm->record_slots != 0;
    t.seed = prm->seed;
    if (prm->instance_id >= (1u << 24)) return fail(err, "instance_id must be < 2^24", MCPD_EINVAL);
    t.instance = prm->instance_id;
    return MCPD_OK;
}

}  // namespace mcpd
