"""The C-ABI library without a GPU: it builds, loads, exports what include/mcpd.h declares, its
struct layouts match the C compiler's, its host-built tables equal the oracle's, and it rejects
invalid inputs."""
import ctypes
import subprocess

import numpy as np
import pytest

import synth
from paper_2608_30239_gb300 import build as lib_build
from paper_2608_30239_gb300 import mcpd


@pytest.fixture(scope="module")
def L():
    lib_build.build()
    return mcpd.lib()


def test_library_exports_every_declared_function(L):
    names = mcpd.header_functions()
    assert "mcpd_decode" in names and "mcpd_run_async" in names
    for name in names:
        assert hasattr(L, name), name
    out = subprocess.check_output(["nm", "-D", "--defined-only", lib_build.LIB]).decode()
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported


def test_struct_layout_matches_c(tmp_path):
    """offsetof/sizeof from gcc on include/mcpd.h equal the ctypes mirrors of the binding."""
    fields = {"mcpd_params": [f for f, _ in mcpd.mcpd_params._fields_],
              "mcpd_stats": [f for f, _ in mcpd.mcpd_stats._fields_],
              "mcpd_design": [f for f, _ in mcpd.mcpd_design._fields_]}
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "mcpd.h"', "int main(void){"]
    for s, fs in fields.items():
        src.append(f'printf("{s} %zu\\n", sizeof({s}));')
        for f in fs:
            src.append(f'printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    src.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", lib_build.INCLUDE, str(c), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)]).decode().splitlines())
    for s, fs in fields.items():
        cls = getattr(mcpd, s)
        assert int(got[s]) == ctypes.sizeof(cls)
        for f in fs:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)


CASES = {
    "tiny": (lambda: synth.tiny_config(1), {}),
    "library": (lambda: synth.paper_shaped_config(), {}),
    "high-noise": (lambda: synth.high_noise_config(), {}),
    "pruned": (lambda: synth.high_noise_config(), {"n_active": 333}),
    "uniform": (lambda: synth.tiny_config(2), {"scan": mcpd.MCPD_SCAN_UNIFORM}),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_host_tables_equal_oracle_tables(L, oracle_lib, case):
    """Same written spec, separate code: weights, alias words and thresholds agree bit for bit."""
    make, kw = CASES[case]
    inst = make()
    lib_t = mcpd.mcpd_inspect(inst, slots=16, horizon=100, **kw)
    M = oracle_lib.Model(inst, n_active=kw.get("n_active", 0), scan=kw.get("scan", 0))
    ref = M.tables()
    assert np.array_equal(lib_t["active"], ref["active"])
    assert np.array_equal(lib_t["w"].view(np.uint64), ref["w"].view(np.uint64))
    assert np.array_equal(lib_t["alias"] & np.uint64(0xFFFFFFFF), ref["prob"].astype(np.uint64))
    assert np.array_equal(lib_t["alias"] >> np.uint64(32), ref["alias"].astype(np.uint64))
    side = M.deg_max + 1
    assert np.array_equal(lib_t["T"][:side, :side], ref["T"])


def _random_design(rng):
    """A random design: clone degrees 0..8 (at most the pool count), pools strictly increasing,
    outcomes at one of four positive rates, and rates / prior drawn from a small grid."""
    from types import SimpleNamespace
    n = int(rng.choice([1, 2, 3, 5, 17, 64, 300, 1298]))
    m = int(rng.choice([1, 2, 5, 9, 48, 97, 400]))
    dmax = min(m, int(rng.choice([1, 3, 6, 8])))
    rows = [np.sort(rng.choice(m, size=int(rng.integers(0 if rng.random() < 0.1 else 1, dmax + 1)),
                               replace=False)) for _ in range(n)]
    ptr = np.zeros(n + 1, np.int32)
    ptr[1:] = np.cumsum([len(r) for r in rows])
    return SimpleNamespace(n=n, m=m, clone_ptr=ptr, clone_pools=np.concatenate(rows).astype(np.int32),
                           y=(rng.random(m) < rng.choice([0.0, 0.1, 0.5, 1.0])).astype(np.uint8),
                           fp=float(rng.choice([0.01, 0.1, 0.3, 0.49])),
                           fn=float(rng.choice([0.01, 0.2, 0.5, 0.7])),
                           q=float(rng.choice([1e-4, 0.01, 0.2, 0.5])))


def test_host_tables_equal_oracle_tables_on_random_designs(L, oracle_lib):
    """300 seeded random designs (empty clones, pools shared by many clones, all-negative and
    all-positive outcomes, pruning, the uniform, score and custom scans): every design the library
    accepts gives the oracle's active set, weights, alias words and thresholds bit for bit."""
    rng = np.random.default_rng(20261203)
    compared = 0
    for _ in range(300):
        inst = _random_design(rng)
        scan = int(rng.choice([0, 0, 1, 3]))
        na = int(rng.choice([0, 0, 1, max(1, inst.n // 3)]))
        w = rng.random(inst.n) + 0.05 if scan == mcpd.MCPD_SCAN_CUSTOM else None
        try:
            lib_t = mcpd.mcpd_inspect(inst, slots=16, horizon=100, scan=scan, n_active=na, scan_weights=w)
        except mcpd.McpdError as e:          # beyond the library's limits (a pool over 255 clones)
            assert e.code in (mcpd.MCPD_EINVAL, mcpd.MCPD_ETOO_LARGE)
            continue
        M = oracle_lib.Model(inst, n_active=na, scan=scan, custom_w=w)
        ref = M.tables()
        assert np.array_equal(lib_t["active"], ref["active"])
        if scan != mcpd.MCPD_SCAN_CUSTOM:
            assert np.array_equal(lib_t["w"].view(np.uint64), ref["w"].view(np.uint64))
        assert np.array_equal(lib_t["alias"] & np.uint64(0xFFFFFFFF), ref["prob"].astype(np.uint64))
        assert np.array_equal(lib_t["alias"] >> np.uint64(32), ref["alias"].astype(np.uint64))
        side = M.deg_max + 1
        assert np.array_equal(lib_t["T"][:side, :side], ref["T"])
        compared += 1
    assert compared >= 200


def test_window_horizon_and_buckets_on_random_parameters(L, oracle_lib):
    """200 seeded parameter sets on the high-noise design (coupled with default or explicit
    windows, lags, budgets or explicit horizons; uncoupled with burn-in and length): the library's
    k and l are the paper's window recipe when left to default, its horizon is the budget split
    over the slots, and its N*_p bucket count is the oracle's for the same run."""
    import ctypes as C
    inst = synth.high_noise_config()
    rng = np.random.default_rng(7)
    compared = 0
    for _ in range(200):
        coupled = bool(rng.random() < 0.7)
        slots = int(rng.choice([1, 7, 1000, 524288]))
        kw = dict(slots=slots, coupled=coupled, n_active=int(rng.choice([0, 50, 333])))
        if coupled:
            if rng.random() < 0.5:
                ell = int(rng.integers(1, 5000))
                kw.update(k=int(rng.integers(0, ell + 1)), ell=ell)
            kw["lag"] = int(rng.choice([0, 1, 2, 7, 3000]))
        else:
            kw.update(scan=mcpd.MCPD_SCAN_UNIFORM, burn=int(rng.integers(0, 400)),
                      length=int(rng.integers(1, 4000)))
        if rng.random() < 0.5:
            kw["budget_site_updates"] = float(rng.choice([1e6, 4e10, 1e12])) * slots / 524288
        else:
            kw["horizon"] = int(rng.integers(0, 10 ** 6))
        try:
            info = mcpd.mcpd_inspect(inst, **kw)["info"]
        except mcpd.McpdError as e:
            assert e.code in (mcpd.MCPD_ETOO_LARGE, mcpd.MCPD_EOVERFLOW)   # bucket or sum limits
            continue
        na, nb, B, k, ell = (int(v) for v in info[:5])
        if coupled and "k" not in kw:
            assert (k, ell) == oracle_lib.window_defaults(na, 1)
        elif coupled:
            assert (k, ell) == (kw["k"], kw["ell"])
        if coupled and "budget_site_updates" in kw:
            assert B == synth.budget_horizon(kw["budget_site_updates"], slots)
        elif "horizon" in kw:
            assert B == kw["horizon"]
        run = oracle_lib.Run(k=k, ell=ell, burn=kw.get("burn", 0), length=kw.get("length", 0),
                             horizon=B, coupled=int(coupled), lag=kw.get("lag", 1))
        assert nb == int(oracle_lib.lib().orc_num_buckets(C.byref(run)))
        compared += 1
    assert compared >= 100


# Perturbations of a valid design and parameter set, at most two per case.
_PERTURB = dict(
    fp=[0.0, 1.0, -0.1, 1e-300, 0.5, float("nan"), float("inf")], fn=[0.0, 1.0, 0.999999, float("nan")],
    q=[0.0, 1.0, 1e-12, 0.999, float("nan")], n_active=[1, 3, -1, 10 ** 6], scan=[1, 2, 3, 4, -1],
    k=[0, 1, 10, 2 ** 40, -5], ell=[0, 1, 5, 100, 2 ** 40], burn=[0, 3, 2 ** 40], length=[0, 1, 7, 2 ** 40],
    slots=[0, -1, 100, 2 ** 31, 2 ** 31 + 1, 2 ** 40], horizon=[1, 100, 2 ** 40, -3],
    budget_site_updates=[1e3, 1e12, -1.0, float("nan"), float("inf")], step_limit=[1, 10 ** 6, -1, 2 ** 62],
    slot_offset=[5, 2 ** 32 - 1, -1], trace_stride=[1, 3, -2], tau_audit=[5, 10 ** 6, -1],
    meeting_cap=[1, 20, 10 ** 5, -4, 2 ** 32], lag=[2, 7, 2 ** 20, 2 ** 20 + 1, -1], lanes_per_pair=[1, 8, 3],
    record_slots=[True], coupled=[False], scan_weights=["good", "zero", "neg", "nan"],
    init_marginals=["good", "two", "nan"], design=["dup", "range", "neg", "ptr", "empty_clone", "no_pools"])


def test_random_inputs_are_accepted_or_refused_cleanly(L):
    """1500 seeded cases, each a valid design and parameter set with up to two entries made odd or
    invalid (rates at or outside (0, 1) and NaN, windows, horizons, slot counts and offsets beyond
    their ranges, caps, lags, bad weights and marginals, duplicate or out-of-range pools, a
    decreasing clone pointer): every call either builds the tables or returns a documented error
    code; none crashes.  (Run under AddressSanitizer by tests/sanitize_host.)"""
    from types import SimpleNamespace
    rng = np.random.default_rng(5)
    codes = {mcpd.MCPD_EINVAL, mcpd.MCPD_ETOO_LARGE, mcpd.MCPD_EOVERFLOW}
    accepted = 0
    for _ in range(1500):
        n = int(rng.choice([1, 2, 3, 5, 17, 64, 300, 1298]))
        m = int(rng.choice([1, 2, 5, 9, 48, 97, 400]))
        bad = {key: _PERTURB[key][rng.integers(len(_PERTURB[key]))]
               for key in rng.choice(sorted(_PERTURB), size=int(rng.integers(0, 3)), replace=False)}
        dmax = min(m, int(rng.choice([1, 3, 6, 8, 9, 12])))
        rows = [np.sort(rng.choice(m, size=int(rng.integers(1, dmax + 1)), replace=False)) for _ in range(n)]
        if bad.get("design") == "empty_clone":
            rows[0] = rows[0][:0]
        ptr = np.zeros(n + 1, np.int32)
        ptr[1:] = np.cumsum([len(r) for r in rows])
        pools = np.concatenate(rows).astype(np.int32)
        if bad.get("design") == "dup" and len(rows[0]) > 1:
            pools[1] = pools[0]
        if bad.get("design") == "range":
            pools[-1] = m
        if bad.get("design") == "neg":
            pools[0] = -1
        if bad.get("design") == "ptr" and n > 1 and ptr[2] + 1 <= ptr[-1]:
            ptr[1] = ptr[2] + 1                  # decreasing, still inside the pools array
        inst = SimpleNamespace(n=n, m=0 if bad.get("design") == "no_pools" else m, clone_ptr=ptr,
                               clone_pools=pools, y=(rng.random(m) < rng.choice([0.0, 0.1, 0.5, 1.0])).astype(np.uint8),
                               fp=bad.get("fp", 0.1), fn=bad.get("fn", 0.2), q=bad.get("q", 0.01))
        kw = {k: v for k, v in bad.items() if k not in ("fp", "fn", "q", "design", "scan_weights", "init_marginals")}
        kw["seed"] = int(rng.integers(2 ** 63))
        if "scan_weights" in bad or kw.get("scan") == mcpd.MCPD_SCAN_CUSTOM:
            scale = {"zero": 0.0, "neg": -1.0, "nan": float("nan")}.get(bad.get("scan_weights"), 1.0)
            kw["scan_weights"] = rng.random(n) * scale
            kw.setdefault("scan", mcpd.MCPD_SCAN_CUSTOM)
        if "init_marginals" in bad:
            kw["init_marginals"] = rng.random(n) * {"good": 1.0, "two": 2.0, "nan": float("nan")}[bad["init_marginals"]]
        try:
            info = mcpd.mcpd_inspect(inst, **kw)["info"]
        except mcpd.McpdError as e:
            assert e.code in codes, (e, bad)
            continue
        accepted += 1
        assert 1 <= info[0] <= n and info[1] >= 1 and info[6] >= 1, (info, bad)
    assert accepted >= 300


def test_custom_weights_tables(L, oracle_lib):
    inst = synth.tiny_config(5)
    w = np.linspace(1.0, 2.0, inst.n)
    lib_t = mcpd.mcpd_inspect(inst, slots=4, scan=mcpd.MCPD_SCAN_CUSTOM, scan_weights=w)
    ref = oracle_lib.Model(inst, scan=oracle_lib.SCAN_CUSTOM, custom_w=w).tables()
    assert np.array_equal(lib_t["alias"] & np.uint64(0xFFFFFFFF), ref["prob"].astype(np.uint64))
    assert np.array_equal(lib_t["alias"] >> np.uint64(32), ref["alias"].astype(np.uint64))


def test_window_and_horizon_defaults(L, oracle_lib):
    inst = synth.high_noise_config()
    t = mcpd.mcpd_inspect(inst, slots=524288, budget_site_updates=4e10)
    info = t["info"]
    k, ell = oracle_lib.window_defaults(1298, 1)
    assert (int(info[3]), int(info[4]), int(info[5])) == (k, ell, ell - k + 1) == (131, 1298, 1168)
    assert int(info[2]) == synth.budget_horizon(4e10, 524288) == 38146
    assert int(info[1]) == 38146 // 1298
    u = mcpd.mcpd_inspect(inst, slots=1000, coupled=False, scan=mcpd.MCPD_SCAN_SYSTEMATIC,
                          budget_site_updates=1e8)
    assert int(u["info"][3]) == 130 and int(u["info"][5]) == 1298 - 130
    assert int(u["info"][2]) == 100000


@pytest.mark.parametrize("kw,code", [
    (dict(fp=0.0), mcpd.MCPD_EINVAL),
    (dict(fn=1.0), mcpd.MCPD_EINVAL),
    (dict(prior_q=1.5), mcpd.MCPD_EINVAL),
    (dict(k=5, ell=4), mcpd.MCPD_EINVAL),
    (dict(scan=mcpd.MCPD_SCAN_SYSTEMATIC), mcpd.MCPD_EINVAL),
    (dict(scan=7), mcpd.MCPD_EINVAL),
    (dict(slots=0), mcpd.MCPD_EINVAL),
    (dict(instance_id=1 << 24), mcpd.MCPD_EINVAL),
    (dict(coupled=False, burn=0, length=1), mcpd.MCPD_EINVAL),
    (dict(horizon=10 ** 6, ell=1, k=0), mcpd.MCPD_ETOO_LARGE),
    (dict(tau_audit=-1), mcpd.MCPD_EINVAL),
    (dict(meeting_cap=-1), mcpd.MCPD_EINVAL),
    (dict(k=2, ell=20, meeting_cap=19), mcpd.MCPD_EINVAL),
    (dict(k=2, ell=20, meeting_cap=30, tau_audit=31), mcpd.MCPD_EINVAL),
    (dict(k=2, ell=20, meeting_cap=(1 << 31) + 1), mcpd.MCPD_EINVAL),
    (dict(lag=-1), mcpd.MCPD_EINVAL),
    (dict(lag=(1 << 20) + 1), mcpd.MCPD_EINVAL),
    (dict(k=2, ell=20, lag=30, meeting_cap=25), mcpd.MCPD_EINVAL),
    (dict(k=2, ell=20, lag=30, step_limit=29), mcpd.MCPD_EINVAL),
    (dict(trace_steps=16), mcpd.MCPD_EINVAL),                          # no traced slots
    (dict(trace_steps=-1, trace_stride=2), mcpd.MCPD_EINVAL),
    (dict(trace_steps=(1 << 20) + 1, trace_stride=2), mcpd.MCPD_EINVAL),
    (dict(trace_steps=16, trace_stride=2, trace_reps=1025), mcpd.MCPD_EINVAL),
])
def test_invalid_parameters_rejected(L, kw, code):
    inst = synth.tiny_config(1)
    base = dict(slots=8, horizon=100)
    base.update(kw)
    with pytest.raises(mcpd.McpdError) as ei:
        mcpd.mcpd_inspect(inst, **base)
    assert ei.value.code == code


def test_invalid_designs_rejected(L):
    inst = synth.tiny_config(1)
    bad = synth.Instance(**{**inst.__dict__})
    bad.clone_pools = inst.clone_pools.copy()
    bad.clone_pools[0], bad.clone_pools[1] = bad.clone_pools[1], bad.clone_pools[0]   # unsorted row
    with pytest.raises(mcpd.McpdError) as ei:
        mcpd.mcpd_inspect(bad, slots=4)
    assert ei.value.code == mcpd.MCPD_EINVAL
    wide = synth.make_instance(40, 12, 9, 2, 0.1, 0.1, 0.05, 3, 4)                        # 9 pools
    with pytest.raises(mcpd.McpdError) as ei:
        mcpd.mcpd_inspect(wide, slots=4)
    assert ei.value.code == mcpd.MCPD_ETOO_LARGE
    y2 = synth.Instance(**{**inst.__dict__})
    y2.y = inst.y.copy()
    y2.y[0] = 2
    with pytest.raises(mcpd.McpdError):
        mcpd.mcpd_inspect(y2, slots=4)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(mcpd, "_lib", None)
    monkeypatch.setattr(lib_build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        mcpd.lib()


def test_meeting_cap_replaces_the_step_limit(L):
    """A meeting cap becomes the replication's step limit (info[12]); uncoupled runs ignore it."""
    inst = synth.tiny_config(1)
    capped = mcpd.mcpd_inspect(inst, slots=8, horizon=100, k=2, ell=20, meeting_cap=30, step_limit=10 ** 6)
    assert capped["info"][12] == 30
    free = mcpd.mcpd_inspect(inst, slots=8, horizon=100, k=2, ell=20, step_limit=10 ** 6)
    assert free["info"][12] == 10 ** 6
    unc = mcpd.mcpd_inspect(inst, slots=8, horizon=100, coupled=False, burn=2, length=20,
                            meeting_cap=5, step_limit=10 ** 6)
    assert unc["info"][12] == 10 ** 6


def test_lag_sets_the_smallest_replication_cost(L):
    """A lag L makes every replication cost at least max(l, L) progress units, so the number of
    N*_p buckets is B // max(l, L); lag 0 and 1 are the paper's one-lag pair."""
    inst = synth.tiny_config(1)
    base = dict(slots=8, horizon=400, k=2, ell=20)
    assert mcpd.mcpd_inspect(inst, **base)["info"][1] == 400 // 20
    assert mcpd.mcpd_inspect(inst, lag=1, **base)["info"][1] == 400 // 20
    assert mcpd.mcpd_inspect(inst, lag=0, **base)["info"][1] == 400 // 20
    assert mcpd.mcpd_inspect(inst, lag=50, **base)["info"][1] == 400 // 50


def test_integer_sum_bounds(L):
    """The sums' overflow guard: an uncoupled run keeps at most nb replications of G in [0, T] per
    slot, so the paper's long-run reference (2,000,000 chains, 1000 + 10,000 sweeps of 333 clones)
    is accepted; a coupled run whose per-slot bound L (2 (B + step limit) + 1) times the slots
    passes 9e18 is refused."""
    inst = synth.tiny_config(1)
    ok = mcpd.mcpd_inspect(inst, coupled=False, scan=mcpd.MCPD_SCAN_SYSTEMATIC, slots=2_000_000,
                           burn=333_000, length=3_330_000, horizon=3_663_000)
    assert int(ok["info"][1]) == 1
    with pytest.raises(mcpd.McpdError) as ei:
        mcpd.mcpd_inspect(inst, slots=1 << 31, k=0, ell=20000, horizon=1 << 30)
    assert ei.value.code == mcpd.MCPD_EOVERFLOW
