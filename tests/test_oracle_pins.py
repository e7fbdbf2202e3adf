"""Pins of the CPU oracle against things other than itself (runs without a GPU).

Each test names what fixes the expected value: a value the paper prints (Table S1), a published
known-answer vector (Philox), a closed form, an invariant the paper proves (Proposition 1,
Theorem 1), brute-force enumeration, or an identity between two different formulas.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _inst(n, m, deg, npos, fp, fn, q, dseed=11, oseed=12):
    return synth.make_instance(n, m, deg, npos, fp, fn, q, dseed, oseed)


# ---------------------------------------------------------------------------------------------
def test_philox_known_answers(oracle_lib):
    """Philox4x32-10 blocks equal the published known-answer vectors (Salmon et al., SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle_lib.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_window_rounding_matches_table_s1(oracle_lib):
    """b_s = round(0.1 s n_a) is half-to-even: Table S1 prints b = 166 at M = 1665 (n_a = 333, s = 5)
    and b = 124 at M = 1235; round-half-up would give 167 and 124."""
    for line in open(os.path.join(GOLDEN, "table_s1.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        left, right = line.split("|")
        f = left.split()
        na = int(f[1])
        bs = [int(x) for x in f[2:7]]
        rest = [int(x) for x in right.split()]
        for s, b, mb in zip((1, 3, 5, 10, 20), bs, rest):
            k, ell = oracle_lib.window_defaults(na, s)
            assert k - 1 == b, (na, s)
            assert ell - (k - 1) == mb
            assert ell - k + 1 == mb           # L = l - k + 1 = M_s - b_s terms


# ---------------------------------------------------------------------------------------------
def test_enumeration_no_pools_gives_prior():
    """With no pools the posterior is the product prior: p_j = q exactly (up to rounding)."""
    inst = synth.Instance(n=6, m=0, clone_ptr=np.zeros(7, np.int32),
                          clone_pools=np.zeros(0, np.int32), y=np.zeros(0, np.uint8),
                          positives=np.zeros(0, np.int32), fp=0.1, fn=0.2, q=0.03)
    _, p = exact.posterior(inst)
    assert np.allclose(p, 0.03, rtol=0, atol=1e-15)


def test_enumeration_closed_forms():
    """n = 1: p = sigma(log q/(1-q) + sum_j a_j).  Two clones sharing one positive pool:
    p_1 = q (1-fn) / [(1-q)^2 fp + 2 q (1-q)(1-fn) + q^2 (1-fn)] * ((1-q) + q)."""
    fp, fn, q = 0.07, 0.13, 0.2
    one = synth.Instance(n=1, m=3, clone_ptr=np.array([0, 3], np.int32),
                         clone_pools=np.array([0, 1, 2], np.int32), y=np.array([1, 0, 1], np.uint8),
                         positives=np.zeros(0, np.int32), fp=fp, fn=fn, q=q)
    _, p = exact.posterior(one)
    ap, am = math.log((1 - fn) / fp), math.log(fn / (1 - fp))
    z = math.log(q / (1 - q)) + 2 * ap + am
    assert p[0] == pytest.approx(1 / (1 + math.exp(-z)), rel=1e-13)
    two = synth.Instance(n=2, m=1, clone_ptr=np.array([0, 1, 2], np.int32),
                         clone_pools=np.array([0, 0], np.int32), y=np.array([1], np.uint8),
                         positives=np.zeros(0, np.int32), fp=fp, fn=fn, q=q)
    _, p = exact.posterior(two)
    Z = (1 - q) ** 2 * fp + 2 * q * (1 - q) * (1 - fn) + q * q * (1 - fn)
    assert p[0] == pytest.approx((q * (1 - q) * (1 - fn) + q * q * (1 - fn)) / Z, rel=1e-13)
    assert p[1] == pytest.approx(p[0], rel=1e-15)


def test_pruned_posterior_is_conditional(oracle_lib):
    """pi_A is the full posterior conditioned on Z_{A^c} = 0 (Section "Knill's Method")."""
    inst = _inst(12, 6, 2, 2, 0.08, 0.15, 0.1)
    M = oracle_lib.Model(inst, n_active=8)
    act = M.tables()["active"]
    eta = M.tables()["eta"]
    # the kept clones are the top 8 by eta (ties to the lower index) and are listed ascending
    order = sorted(range(inst.n), key=lambda i: (-eta[i], i))[:8]
    assert list(act) == sorted(order)
    pi_full, _ = exact.posterior(inst)
    states = np.arange(1 << inst.n)
    pruned = np.setdiff1d(np.arange(inst.n), act)
    keep = np.all(((states[:, None] >> pruned[None, :]) & 1) == 0, axis=1)
    cond = pi_full * keep
    cond /= cond.sum()
    bits = (states[:, None] >> act[None, :]) & 1
    _, p_pruned = exact.posterior(inst, act)
    assert np.allclose(cond @ bits, p_pruned, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------------------------------------
def _direct_conditional(inst, active, x_active, i):
    """p_i(1 | x_-i) straight from the unnormalised posterior at x^{i<-1} and x^{i<-0}."""
    A = exact._incidence(inst, active)
    x1 = x_active.astype(np.int64).copy(); x1[i] = 1
    x0 = x_active.astype(np.int64).copy(); x0[i] = 0
    y = inst.y.astype(bool)

    def loglik(x):
        xi = (x @ A) > 0
        return np.where(xi, np.where(y, np.log1p(-inst.fn), np.log(inst.fn)),
                        np.where(y, np.log(inst.fp), np.log1p(-inst.fp))).sum()
    d = math.log(inst.q) - math.log1p(-inst.q) + (loglik(x1) - loglik(x0))
    return 1.0 / (1.0 + math.exp(-d))


@pytest.mark.parametrize("which", ["tiny", "library"])
def test_full_conditional_matches_posterior_ratio(oracle_lib, which):
    """The oracle's (n+, n-) counting reproduces pi(x^{i<-1}) / (pi(x^{i<-1}) + pi(x^{i<-0}))."""
    inst = synth.tiny_config(3) if which == "tiny" else synth.high_noise_config()
    M = oracle_lib.Model(inst)
    act = M.tables()["active"]
    rng = np.random.default_rng(5)
    for trial in range(60 if which == "tiny" else 25):
        dens = [0.0, 0.05, 0.3][trial % 3] if which == "tiny" else [0.0, 0.004, 0.02][trial % 3]
        x = (rng.random(M.na) < dens).astype(np.uint8)
        i = int(rng.integers(M.na))
        np_, nn = M.conditional_counts(x, i)
        p_or = M.conditional_prob(np_, nn)
        p_dir = _direct_conditional(inst, act, x, i)
        assert p_or == pytest.approx(p_dir, rel=1e-12, abs=1e-300)


def test_threshold_is_floor_of_p_times_2_64(oracle_lib):
    """T(n+, n-) = floor(p * 2^64) of the double p, clamped to [1, 2^64 - 1]; p itself agrees with a
    50-digit evaluation of sigma(lambda + n+ a+ + n- a-) within the rounding of the exponent."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    inst = synth.high_noise_config()
    M = oracle_lib.Model(inst)
    T = M.tables()["T"]
    fp, fn, q = (mp.mpf(v) for v in (inst.fp, inst.fn, inst.q))
    ap = mp.log(1 - fn) - mp.log(fp)
    am = mp.log(fn) - mp.log(1 - fp)
    lam = mp.log(q) - mp.log(1 - q)
    for a in range(M.deg_max + 1):
        for b in range(M.deg_max + 1):
            p = M.conditional_prob(a, b)
            exact_p = 1 / (1 + mp.exp(-(lam + a * ap + b * am)))
            # z carries a few ulps of its terms' magnitude; sigma passes that on relatively
            mag = float(abs(lam) + a * abs(ap) + b * abs(am)) + 1.0
            assert abs(mp.mpf(p) - exact_p) <= 8 * 2.0 ** -52 * mag * exact_p
            expect = math.floor(Fraction(p) * 2 ** 64)
            expect = min(max(expect, 1), 2 ** 64 - 1)
            assert int(T[a, b]) == expect


# ---------------------------------------------------------------------------------------------
def test_alias_table_mass_is_exact(oracle_lib):
    """Each alias column carries 2^32 of mass; the mass that reaches clone i is exactly V_i."""
    for inst in (synth.tiny_config(2), synth.paper_shaped_config()):
        M = oracle_lib.Model(inst)
        t = M.tables()
        V, prob, alias = t["V"], t["prob"], t["alias"]
        na = M.na
        assert int(V.astype(object).sum()) == na << 32
        assert int(V.min()) >= 1 << 30
        mass = [0] * na
        for col in range(na):
            if int(prob[col]) == 0xFFFFFFFF and int(alias[col]) == col:
                mass[col] += 1 << 32
            else:
                mass[col] += int(prob[col])
                mass[int(alias[col])] += (1 << 32) - int(prob[col])
        assert mass == [int(v) for v in V]


def test_score_weights_span_gamma(oracle_lib):
    """w_i = 0.5 e_i / sum e + 0.5 / n_a with max(e) / min(e) = gamma = 100 n_a when s varies;
    weights sum to one and order like the scores s_i."""
    inst = synth.high_noise_config()
    M = oracle_lib.Model(inst)
    t = M.tables()
    w, s = t["w"], t["score"]
    na = M.na
    e = (w - 0.5 / na) / 0.5
    assert e.max() / e.min() == pytest.approx(100 * na, rel=1e-9)
    assert w.sum() == pytest.approx(1.0, abs=1e-12)
    assert np.all(np.diff(w[np.argsort(s, kind="stable")]) >= -1e-18)
    # s_i = sum_{j in P(i)} d_j^A a_j from the incidence matrix
    A = exact._incidence(inst, t["active"])
    dA = A.sum(axis=0)
    a = np.where(inst.y == 1, M.a_plus, M.a_minus)
    assert np.allclose(A @ (dA * a), s, rtol=1e-12, atol=1e-9)


def test_site_selection_frequencies(oracle_lib):
    """Drawn sites follow V / (n_a 2^32) (chi-square over 2^18 words spread over 2^32)."""
    inst = synth.tiny_config(4)
    M = oracle_lib.Model(inst)
    V = M.tables()["V"].astype(np.float64)
    words = (np.arange(1 << 18, dtype=np.uint64) * np.uint64(16411) * np.uint64(1 << 14)
             + np.uint64(12345)) % np.uint64(1 << 32)
    counts = np.bincount([M.select_site(int(w)) for w in words], minlength=M.na)
    expect = V / V.sum() * len(words)
    chi2 = ((counts - expect) ** 2 / expect).sum()
    assert chi2 < 60.0          # 19 degrees of freedom


# ---------------------------------------------------------------------------------------------
def _invariance_instance(n, m, deg, seed):
    return _inst(n, m, deg, 2, 0.1, 0.2, 0.15, dseed=seed, oseed=seed + 1)


@pytest.mark.parametrize("n,m,deg,seed", [(8, 5, 2, 3), (10, 6, 3, 5)])
def test_pi_P_equals_pi(oracle_lib, n, m, deg, seed):
    """Proposition 1: pi P_i = pi for every i, so pi P_w = pi and pi P_unif = pi; the systematic
    sweep Q = P_1 ... P_n also leaves pi invariant.  Rows of every matrix sum to one."""
    inst = _invariance_instance(n, m, deg, seed)
    M = oracle_lib.Model(inst)
    t = M.tables()
    pi, _ = exact.posterior(inst)

    def cond(s, i):
        x = ((s >> np.arange(n)) & 1).astype(np.uint8)
        return M.conditional_prob(*M.conditional_counts(x, i))

    Ps, Pw = exact.transition_matrices(cond, n, t["w"])
    assert np.max(np.abs(Pw.sum(axis=1) - 1)) < 1e-14
    assert np.max(np.abs(pi @ Pw - pi)) < 1e-14
    Pu = sum(Ps) / n
    assert np.max(np.abs(pi @ Pu - pi)) < 1e-14
    Q = Ps[0]
    for P_i in Ps[1:]:
        Q = Q @ P_i
    assert np.max(np.abs(pi @ Q - pi)) < 1e-13
    # the chain actually moves: P_w is irreducible (some power is strictly positive)
    R = np.linalg.matrix_power(Pw, 4 * n)
    assert R.min() > 0


def test_wrong_full_conditional_breaks_invariance(oracle_lib):
    """Control: the pi P = pi check rejects a plausible slip (pools with c^{-i} > 0 counted too)."""
    inst = _invariance_instance(8, 5, 2, 3)
    M = oracle_lib.Model(inst)
    pi, _ = exact.posterior(inst)

    def wrong(s, i):
        deg = inst.clone_ptr[i + 1] - inst.clone_ptr[i]
        pools = inst.clone_pools[inst.clone_ptr[i]:inst.clone_ptr[i + 1]]
        npos = int(inst.y[pools].sum())
        return M.conditional_prob(npos, deg - npos)

    _, Pw = exact.transition_matrices(wrong, 8, M.tables()["w"])
    assert np.max(np.abs(pi @ Pw - pi)) > 1e-4


# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("k,ell", [(3, 20), (0, 0), (0, 1), (5, 5), (1, 7)])
def test_estimator_literal_definition_equals_swapped_sum(oracle_lib, k, ell):
    """G = L H_{k:l} from the literal H_r = X_r + sum_s (X_{r+s} - Y_{r+s-1}) equals the swapped-sum
    form sum_{r=k}^{l} X_r + sum_{t>k} min(t-k, L)(X_t - Y_{t-1}) for every replication."""
    inst = _inst(20, 8, 3, 2, 0.05, 0.1, 0.03)
    M = oracle_lib.Model(inst)
    run = oracle_lib.coupled_run(k, ell, 0, seed=99, step_limit=200000)
    for slot in range(40):
        a = M.replication(run, slot, 0, literal=True)
        b = M.replication(run, slot, 0, literal=False)
        assert a["status"] == 0 and b["status"] == 0
        assert a["C"] == b["C"] and a["tau"] == b["tau"]
        assert np.array_equal(a["G"], b["G"])


def test_coupling_invariants(oracle_lib):
    """Theorem 1(d) faithfulness X_t = Y_{t-1} for t >= tau, tau is the first such t >= 1, the
    replication uses C = max(l, tau) draws, and |H_{k:l}| <= 1 + 2 tau (pathwise bound)."""
    inst = _inst(20, 8, 3, 2, 0.05, 0.1, 0.03)
    M = oracle_lib.Model(inst)
    k, ell = 3, 20
    run = oracle_lib.coupled_run(k, ell, 0, seed=7, step_limit=200000)
    L = ell - k + 1
    saw_late_meeting = False
    for slot in range(60):
        r = M.replication(run, slot, 0, traj_cap=5000)
        C, tau = r["C"], r["tau"]
        X, Y = r["X"], r["Y"]
        assert r["draws"] == C == max(ell, tau)
        eq = [np.array_equal(X[t], Y[t - 1]) for t in range(1, C + 1)]
        assert eq.index(True) + 1 == tau
        assert all(eq[tau - 1:])
        assert np.all(np.abs(r["G"]) <= L * (1 + 2 * tau))
        assert np.array_equal(X[0], Y[0])                     # X_0 = Y_0 = Z_0
        saw_late_meeting |= tau > ell
        if tau <= k + 1:   # all correction terms vanish: G is the plain window sum
            assert np.array_equal(r["G"], X[k:ell + 1].sum(axis=0).astype(np.int64))
    assert saw_late_meeting


@pytest.mark.parametrize("cap", [20, 24, 40])
def test_meeting_cap_follows_the_uncapped_paths(oracle_lib, cap):
    """With a meeting cap c the chains are the uncapped chains up to c: a pair that meets at
    tau <= c gives the uncapped replication exactly; one with tau > c stops at C = c, tau = 0,
    and its X, Y paths are the uncapped paths cut at c."""
    inst = _inst(20, 8, 3, 2, 0.05, 0.1, 0.03)
    M = oracle_lib.Model(inst)
    k, ell = 3, 20
    free = oracle_lib.coupled_run(k, ell, 0, seed=7, step_limit=200000)
    capd = oracle_lib.coupled_run(k, ell, 0, seed=7, step_limit=200000, meeting_cap=cap)
    n_capped = 0
    for slot in range(80):
        u = M.replication(free, slot, 0, traj_cap=5000)
        c = M.replication(capd, slot, 0, traj_cap=5000)
        assert u["status"] == 0 and c["status"] == 0
        if u["tau"] <= cap:
            assert c["capped"] == 0 and c["tau"] == u["tau"] and c["C"] == u["C"]
            assert np.array_equal(c["G"], u["G"])
        else:
            n_capped += 1
            assert c["capped"] == 1 and c["tau"] == 0 and c["C"] == c["draws"] == cap
            assert np.array_equal(c["X"][:cap + 1], u["X"][:cap + 1])
            assert np.array_equal(c["Y"][:cap], u["Y"][:cap])
            assert not np.array_equal(c["X"][cap], c["Y"][cap - 1])
    assert n_capped > 0


def test_meeting_cap_at_the_window_keeps_only_the_window_term(oracle_lib):
    """k = l = c: every correction term of H_k has r + s > c, so a capped pair gives G = X_k
    (closed form); the literal and the swapped-sum forms agree with the cap."""
    inst = _inst(20, 8, 3, 2, 0.05, 0.1, 0.03)
    M = oracle_lib.Model(inst)
    k = 6
    run = oracle_lib.coupled_run(k, k, 0, seed=31, step_limit=200000, meeting_cap=k)
    seen = 0
    for slot in range(200):
        r = M.replication(run, slot, 0, traj_cap=100)
        lit = M.replication(run, slot, 0, literal=True)
        assert np.array_equal(lit["G"], r["G"]) and lit["capped"] == r["capped"]
        if r["capped"]:
            seen += 1
            assert np.array_equal(r["G"], r["X"][k].astype(np.int64))
    assert seen > 0


@pytest.mark.parametrize("k,ell,cap", [(3, 20, 20), (3, 20, 33), (0, 1, 2)])
def test_meeting_cap_literal_definition_equals_swapped_sum(oracle_lib, k, ell, cap):
    """The truncated H_{k:l} (inner sums over r + s <= c) from the literal double sum equals the
    swapped-sum form for capped and uncapped replications alike."""
    inst = _inst(20, 8, 3, 2, 0.05, 0.1, 0.03)
    M = oracle_lib.Model(inst)
    run = oracle_lib.coupled_run(k, ell, 0, seed=5, step_limit=200000, meeting_cap=cap)
    for slot in range(60):
        a = M.replication(run, slot, 0, literal=True)
        b = M.replication(run, slot, 0, literal=False)
        assert a["status"] == 0 and b["status"] == 0
        assert (a["C"], a["tau"], a["capped"]) == (b["C"], b["tau"], b["capped"])
        assert np.array_equal(a["G"], b["G"])


def test_meeting_cap_slot_runs(oracle_lib):
    """A cap at or above every meeting time changes nothing; a cap below some counts those pairs
    as capped and charges each exactly c progress units; a cap below l is rejected."""
    inst = _inst(20, 8, 3, 2, 0.05, 0.1, 0.03)
    M = oracle_lib.Model(inst)
    free = M.run_slots(oracle_lib.coupled_run(3, 20, 0, seed=13), 0, 300, per_slot=True)
    big = M.run_slots(oracle_lib.coupled_run(3, 20, 0, seed=13, meeting_cap=free["stats"]["max_tau"]),
                      0, 300, per_slot=True)
    for key in ("S1", "S2_lo", "S2_hi", "count", "slot_S"):
        assert np.array_equal(free[key], big[key]), key
    assert big["stats"]["capped"] == 0
    cap = 21
    taus = np.array([M.replication(oracle_lib.coupled_run(3, 20, 0, seed=13), p, 0)["tau"] for p in range(300)])
    small = M.run_slots(oracle_lib.coupled_run(3, 20, 0, seed=13, meeting_cap=cap), 0, 300, per_slot=True)
    assert small["stats"]["capped"] == int((taus > cap).sum()) > 0
    assert np.all(small["slot_S"][taus > cap] == cap)
    bad = M.run_slots(oracle_lib.coupled_run(3, 20, 0, seed=13, meeting_cap=19), 0, 10)
    assert bad["status"] == oracle_lib.ORC_EINVAL


def test_phi_is_inverse_transform(oracle_lib):
    """Phi_i(x, u) = 1{u < T}: U just below T sets the bit, U = T clears it."""
    inst = synth.tiny_config(1)
    M = oracle_lib.Model(inst)
    x = np.zeros(M.na, np.uint8)
    T00 = M.threshold(*M.conditional_counts(x, 4))
    assert M.phi(x, 4, T00 - 1) == 1
    assert M.phi(x, 4, T00) == 0


# ---------------------------------------------------------------------------------------------
def _z_scores(est, se, p):
    return np.abs(est - p) / se


NOISY = dict(n=20, m=8, deg=3, npos=2, fp=0.1, fn=0.2, q=0.05)


def _noisy():
    return _inst(**NOISY, dseed=1001, oseed=2001)


@pytest.mark.parametrize("start", ["all-negative", "all-positive"])
def test_coupled_estimator_unbiased(oracle_lib, start):
    """Theorem 1: E H_{k:l} = pi(h_j) from any initial distribution; z-tests against the 2^20
    enumeration, Bonferroni over the 20 clones."""
    inst = _noisy()
    _, p = exact.posterior(inst)
    nu = None if start == "all-negative" else np.ones(inst.n)
    res = oracle_lib.decode(inst, 120000, 3, 20, 0, seed=31, init_marginals=nu)
    assert res["status"] == 0
    z = _z_scores(res["est"], res["se"], p)
    assert z.max() < 4.5, z


def test_uncoupled_short_average_is_biased(oracle_lib):
    """Control for the test above: the ordinary finite average of Algorithm 2 with the same short
    window keeps its initialisation bias and fails the same z-test."""
    inst = _noisy()
    _, p = exact.posterior(inst)
    res = oracle_lib.decode(inst, 120000, 0, 0, 19, seed=31, coupled=False, burn=2, length=18)
    z = _z_scores(res["est"], res["se"], p)
    assert z.max() > 10


@pytest.mark.parametrize("horizon", [10, 60, 200])
def test_completion_time_aggregate_unbiased(oracle_lib, horizon):
    """Theorem 2: theta_CT with slot refill is unbiased for any horizon B, including B < l where
    every slot takes the zero-completion branch."""
    inst = _noisy()
    _, p = exact.posterior(inst)
    res = oracle_lib.decode(inst, 60000, 3, 20, horizon, seed=17, per_slot=True)
    assert res["status"] == 0
    z = _z_scores(res["est"], res["se"], p)
    assert z.max() < 4.5, z
    ns = res["slot_nstar"]
    if horizon < 20:
        assert np.all(ns == 1) and res["stats"]["zero_completion"] == 60000
    else:
        assert ns.max() >= 2


def test_slot_loop_follows_algorithm_4(oracle_lib):
    """Per-slot N*_p, retained cost and G_p equal a restatement of Algorithm 4 driven by single
    replications: start r while S_p(r-1) < B, retain S_p(r) <= B, else keep only a first one."""
    inst = _noisy()
    M = oracle_lib.Model(inst)
    B = 70
    run = oracle_lib.coupled_run(3, 20, B, seed=23)
    res = M.run_slots(run, 0, 50, 1, per_slot=True, slot_G=True)
    for p in range(50):
        S, N, G, Sret = 0, 0, np.zeros(M.na, np.int64), 0
        r = 0
        while True:
            rr = M.replication(run, p, r)
            S += rr["C"]
            if S <= B:
                N += 1; G += rr["G"]; Sret += rr["C"]
            else:
                if N == 0:
                    N = 1; G += rr["G"]; Sret += rr["C"]
                break
            if not S < B:
                break
            r += 1
        assert res["slot_nstar"][p] == N
        assert res["slot_S"][p] == Sret
        assert np.array_equal(res["slot_G"][p], G)


def test_bucket_finalize_equals_mean_of_slot_means(oracle_lib):
    """(1/P) sum_p A_p(B) computed slot by slot equals the bucketed form to rounding."""
    inst = _noisy()
    P = 3000
    res = oracle_lib.decode(inst, P, 3, 20, 90, seed=3, per_slot=True, slot_G=True)
    L = 18
    A = res["slot_G"] / (L * res["slot_nstar"][:, None].astype(np.float64))
    assert np.allclose(A.mean(axis=0), res["est"], rtol=1e-12, atol=1e-15)
    sd = A.std(axis=0, ddof=1) / math.sqrt(P)
    assert np.allclose(sd, res["se"], rtol=1e-9, atol=1e-15)


def test_multithreaded_and_partitioned_runs_are_identical(oracle_lib):
    """Slots are keyed by their global id: thread count and slot_offset partitions do not change
    the integer bucket sums."""
    inst = _noisy()
    M = oracle_lib.Model(inst)
    run = oracle_lib.coupled_run(3, 20, 90, seed=8)
    a = M.run_slots(run, 0, 400, 1)
    b = M.run_slots(run, 0, 400, 7)
    run2 = oracle_lib.coupled_run(3, 20, 90, seed=8, slot_offset=250)
    c1 = M.run_slots(run, 0, 250, 3)
    c2 = M.run_slots(run2, 0, 150, 2)
    for key in ("S1", "S2_lo", "S2_hi", "count"):
        assert np.array_equal(a[key], b[key])
    assert np.array_equal(a["S1"], c1["S1"] + c2["S1"])
    assert np.array_equal(a["count"], c1["count"] + c2["count"])


# ---------------------------------------------------------------------------------------------
# Lag-L coupling (Jacob, O'Leary and Atchade 2020; the paper's estimator is the case L = 1).

def test_lag_weight_counts_window_indices(oracle_lib):
    """w(t) = #{r in k..l : r <= t, r = t mod L}, by brute-force enumeration of (r, j)."""
    for k, ell in [(0, 0), (3, 20), (5, 5), (2, 11), (7, 40)]:
        for lag in (1, 2, 3, 5, 8):
            for t in range(0, 70):
                brute = sum(1 for r in range(k, ell + 1) for j in range(0, 70) if r + j * lag == t)
                assert oracle_lib.lag_weight(k, ell, lag, t) == brute, (k, ell, lag, t)


@pytest.mark.parametrize("lag", [2, 3, 7])
@pytest.mark.parametrize("cap", [0, 26])
def test_lag_literal_definition_equals_swapped_sum(oracle_lib, lag, cap):
    """The lag-L estimator from the literal H_r = X_r + sum_j (X_{r+jL} - Y_{r+(j-1)L}) equals the
    swapped-sum form, uncapped and capped."""
    inst = _inst(20, 8, 3, 2, 0.05, 0.1, 0.03)
    M = oracle_lib.Model(inst)
    run = oracle_lib.coupled_run(3, 20, 0, seed=17, step_limit=200000, meeting_cap=cap, lag=lag)
    for slot in range(50):
        a = M.replication(run, slot, 0, literal=True)
        b = M.replication(run, slot, 0, literal=False)
        assert a["status"] == 0 and b["status"] == 0
        assert (a["C"], a["tau"], a["capped"]) == (b["C"], b["tau"], b["capped"])
        assert np.array_equal(a["G"], b["G"])


@pytest.mark.parametrize("lag", [2, 5])
def test_lag_coupling_invariants(oracle_lib, lag):
    """X's path does not depend on the lag (X_{t+1} = Phi_{I_t}(X_t, U_t) for every t); faithfulness
    X_t = Y_{t-L} for t >= tau, tau the first such t >= L; C = max(l, tau); if tau <= k + L every
    correction term vanishes and G is the plain window sum of X."""
    inst = _inst(20, 8, 3, 2, 0.05, 0.1, 0.03)
    M = oracle_lib.Model(inst)
    k, ell = 3, 20
    one = oracle_lib.coupled_run(k, ell, 0, seed=7, step_limit=200000)
    lagged = oracle_lib.coupled_run(k, ell, 0, seed=7, step_limit=200000, lag=lag)
    saw_late = saw_early = False
    for slot in range(60):
        a = M.replication(one, slot, 0, traj_cap=5000)
        r = M.replication(lagged, slot, 0, traj_cap=5000)
        C, tau, X, Y = r["C"], r["tau"], r["X"], r["Y"]
        n = min(C, a["C"]) + 1
        assert np.array_equal(X[:n], a["X"][:n])
        assert r["draws"] == C == max(ell, tau) and tau >= lag
        eq = [np.array_equal(X[t], Y[t - lag]) for t in range(lag, C + 1)]
        assert eq.index(True) + lag == tau and all(eq[tau - lag:])
        assert np.array_equal(X[0], Y[0])
        saw_late |= tau > ell
        if tau <= k + lag:
            saw_early = True
            assert np.array_equal(r["G"], X[k:ell + 1].sum(axis=0).astype(np.int64))
    assert saw_late and saw_early


@pytest.mark.parametrize("lag", [2, 5])
def test_lag_estimator_unbiased(oracle_lib, lag):
    """The lag-L estimator is unbiased too (the telescoping argument holds for any L): z-tests
    against the 2^20 enumeration, Bonferroni over the 20 clones."""
    inst = _noisy()
    _, p = exact.posterior(inst)
    res = oracle_lib.decode(inst, 120000, 3, 20, 0, seed=37 + lag, lag=lag)
    assert res["status"] == 0
    z = _z_scores(res["est"], res["se"], p)
    assert z.max() < 4.5, z


def test_lag_changes_the_estimates_and_the_cost(oracle_lib):
    """L = 1 and L = 3 draw the same X path but pair it with different Y times: the sums differ,
    every replication costs at least max(l, L), and a cap below L is rejected."""
    inst = _inst(20, 8, 3, 2, 0.05, 0.1, 0.03)
    M = oracle_lib.Model(inst)
    a = M.run_slots(oracle_lib.coupled_run(3, 4, 0, seed=13), 0, 400, per_slot=True)
    b = M.run_slots(oracle_lib.coupled_run(3, 4, 0, seed=13, lag=6), 0, 400, per_slot=True)
    assert not np.array_equal(a["S1"], b["S1"])
    assert b["slot_S"].min() >= 6 and a["slot_S"].min() >= 4
    bad = M.run_slots(oracle_lib.coupled_run(3, 4, 0, seed=13, lag=6, meeting_cap=5), 0, 10)
    assert bad["status"] == oracle_lib.ORC_EINVAL


# ---------------------------------------------------------------------------------------------
# The uncoupled comparators (Algorithms 1 and 2), step by step against their definition.
def _step_words(seed, instance, slot, rep, t, oracle_lib):
    """(w_site, U) of draw t: Philox4x32-10 (pinned by its known-answer vectors) at counter
    (floor(t/2), rep, slot, instance) gives the site word and the uniform's high word (words 0, 1
    at even t, 2, 3 at odd t); the low word is word 0 of the tag-2 block at counter t."""
    key = [seed & 0xFFFFFFFF, seed >> 32]
    b = [int(v) for v in oracle_lib.philox([t >> 1, rep, slot, instance], key)]
    lo = int(oracle_lib.philox([t, rep, slot, (2 << 24) | instance], key)[0])
    ws, wu = (b[2], b[3]) if t & 1 else (b[0], b[1])
    return ws, (wu << 32) | lo


def _site(ws, na, prob, alias):
    """Alias draw written out: column floor(ws n_a / 2^32), kept if the low 32 bits of ws n_a are
    below its probability word, else its alias."""
    prod = ws * na
    col, coin = prod >> 32, prod & 0xFFFFFFFF
    return col if coin < int(prob[col]) else int(alias[col])


@pytest.mark.parametrize("scan,burn,length,start", [
    ("systematic", 0, 5, "zero"), ("systematic", 7, 1, "zero"), ("score", 3, 12, "zero"),
    ("uniform", 20, 20, "random"), ("score", 0, 1, "random"), ("score", 4, 9, "random")])
def test_uncoupled_path_follows_algorithms_1_and_2(oracle_lib, scan, burn, length, start):
    """Against a restatement from the posterior itself, not the oracle's own update: the stored
    path X_0..X_C of one chain has C = b + T - 1 draws, G_j = sum_{t=b}^{b+T-1} X_t[j] summed from
    the path, the site I_t = t mod n_a (systematic) or the alias draw of the step word (score,
    uniform), X_{t+1} differs from X_t at most at I_t, and its new bit is 1{U_t / 2^64 < p} with
    p = sigmoid(log pi(x^{I<-1}) - log pi(x^{I<-0})) from the unnormalised posterior (draws within
    1e-9 of p are not checked).  A chain that averages X_{b+1}..X_{b+T}, charges b + T draws or
    visits I_t = (t + 1) mod n_a fails here."""
    inst = _noisy()
    sc = {"systematic": oracle_lib.SCAN_SYSTEMATIC, "score": oracle_lib.SCAN_SCORE,
          "uniform": oracle_lib.SCAN_UNIFORM}[scan]
    nu = np.random.default_rng(5).uniform(0.0, 0.6, inst.n) if start == "random" else None
    M = oracle_lib.Model(inst, scan=sc, init_marginals=nu)
    tab = M.tables()
    na, seed = M.na, 0xABCDEF0123
    active = np.arange(inst.n)
    run = oracle_lib.uncoupled_run(burn, length, 0, seed=seed)
    C = burn + length - 1
    checked = 0
    for slot in range(40):
        rr = M.replication(run, slot, 0, traj_cap=C + 1)
        assert rr["status"] == 0 and rr["C"] == C and rr["draws"] == C
        X = rr["X"][:C + 1].astype(np.int64)
        assert np.array_equal(rr["G"], X[burn:burn + length].sum(axis=0))
        for t in range(C):
            ws, U = _step_words(seed, 0, slot, 0, t, oracle_lib)
            I = t % na if scan == "systematic" else _site(ws, na, tab["prob"], tab["alias"])
            assert rr["sites"][t] == I, (slot, t)
            diff = np.flatnonzero(X[t + 1] != X[t])
            assert set(diff.tolist()) <= {I}
            hi, lo = X[t].copy(), X[t].copy()
            hi[I], lo[I] = 1, 0
            lp = exact.log_posterior(inst, active, np.stack([hi, lo]))
            p = 1.0 / (1.0 + math.exp(-(lp[0] - lp[1])))
            u = U / 2.0 ** 64
            if abs(u - p) > 1e-9:
                assert X[t + 1][I] == (1 if u < p else 0), (slot, t)
                checked += 1
    assert checked >= 40 * C * 0.99


def test_uncoupled_long_chain_agrees_with_enumeration(oracle_lib):
    """Algorithm 2 with a long burn-in: the average over X_b..X_{b+T-1} of a score-weighted chain
    started all-negative is, after 100 sweeps of burn-in, within sampling error of the exact
    marginals of the 2^20 enumeration (z-tests over the 20 clones; the short-window control
    above fails the same test)."""
    inst = _noisy()
    _, p = exact.posterior(inst)
    res = oracle_lib.decode(inst, 4000, 0, 0, 0, seed=77, coupled=False, burn=2000, length=2000)
    assert res["status"] == 0
    z = _z_scores(res["est"], res["se"], p)
    assert z.max() < 4.5, z


# ---------------------------------------------------------------------------------------------
# The naive score and the pruning of Knill's method.
@pytest.mark.parametrize("which", ["tiny", "noisy", "library"])
def test_naive_score_is_the_posterior_log_ratio(oracle_lib, which):
    """eta_i = log pi(e_i | y) - log pi(0 | y) from the unnormalised posterior (Section "Knill's
    Method": the naive ranking scores a clone by the posterior odds of it alone being positive),
    for every clone, to 1e-12 relative.  A swapped a+ / a- or a weight that belongs to s_i fails."""
    inst = {"tiny": lambda: synth.tiny_config(1), "noisy": _noisy,
            "library": synth.high_noise_config}[which]()
    eta = oracle_lib.Model(inst).tables()["eta"]
    active = np.arange(inst.n)
    Z = np.vstack([np.zeros((1, inst.n), np.int64), np.eye(inst.n, dtype=np.int64)])
    lp = exact.log_posterior(inst, active, Z)
    ref = lp[1:] - lp[0]
    assert np.allclose(eta, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("n_active", [1, 7, 333, 1297])
def test_pruning_keeps_the_top_clones_by_the_independent_score(oracle_lib, n_active):
    """The retained clones are the n_active largest by the posterior log ratio above (ties, which
    the score's few distinct values make common, to the lower original index), listed ascending."""
    inst = synth.high_noise_config()
    Z = np.vstack([np.zeros((1, inst.n), np.int64), np.eye(inst.n, dtype=np.int64)])
    lp = exact.log_posterior(inst, np.arange(inst.n), Z)
    ref = np.round(lp[1:] - lp[0], 9)                   # exact ties stay ties
    order = sorted(range(inst.n), key=lambda i: (-ref[i], i))
    want = np.sort(np.array(order[:n_active]))
    got = oracle_lib.Model(inst, n_active=n_active).tables()["active"]
    assert np.array_equal(got, want)
