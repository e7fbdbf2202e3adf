"""CPU oracle for coupled score-weighted MCPD: test infrastructure only.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py` may import this
package.  It shares no code with the CUDA library (`paper_2608_30239_gb300`): the sampler lives in
plain C (`mcpd_oracle.c`, built with gcc, IEEE double, no fused multiply-add) and the exact
posterior by enumeration in numpy (`exact.py`).  Each function cites the part of the paper it
restates; the pins that tie it to something other than itself are in `tests/test_oracle_pins.py`.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mcpd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SCAN_SCORE, SCAN_UNIFORM, SCAN_SYSTEMATIC, SCAN_CUSTOM = 0, 1, 2, 3
ORC_OK, ORC_EINVAL, ORC_ENOMEM, ORC_ESTEP_LIMIT, ORC_EFAITHFUL = 0, -1, -2, -3, -4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off keeps every double operation separate).

    With MCPD_ORACLE_SANITIZE=1 in the environment a separate copy is built and loaded under
    AddressSanitizer and UndefinedBehaviorSanitizer (the process needs both runtimes preloaded:
    LD_PRELOAD="$(gcc -print-file-name=libasan.so):$(gcc -print-file-name=libubsan.so)")."""
    os.makedirs(_BUILD, exist_ok=True)
    sanitize = os.environ.get("MCPD_ORACLE_SANITIZE") == "1"
    lib_path = os.path.join(_BUILD, "liboracle_san.so") if sanitize else _LIB
    if force or not os.path.exists(lib_path) or os.path.getmtime(lib_path) < os.path.getmtime(_SRC):
        tmp = lib_path + f".tmp{os.getpid()}"
        opt = (["-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
                "-fno-sanitize-recover=undefined"] if sanitize else ["-O2"])
        cmd = ["gcc", *opt, "-std=gnu11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
               "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, lib_path)
    return lib_path


class Run(C.Structure):
    """Mirror of `orc_run` in mcpd_oracle.c."""
    _fields_ = [("k", C.c_int64), ("ell", C.c_int64), ("burn", C.c_int64), ("length", C.c_int64),
                ("horizon", C.c_int64), ("step_limit", C.c_int64), ("seed", C.c_uint64),
                ("slot_offset", C.c_int64), ("instance", C.c_int32), ("coupled", C.c_int32),
                ("pad", C.c_int32), ("meeting_cap", C.c_int64), ("lag", C.c_int64)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.c_void_p
            L.orc_philox.argtypes = [P, P, P]
            L.orc_model_new.argtypes = [C.c_int32, C.c_int32, P, P, P, C.c_double, C.c_double,
                                        C.c_double, C.c_int32, C.c_int32, P, P, C.POINTER(P)]
            L.orc_model_new.restype = C.c_int
            L.orc_model_free.argtypes = [P]
            L.orc_model_dims.argtypes = [P, P]
            L.orc_model_constants.argtypes = [P, P]
            L.orc_model_tables.argtypes = [P] + [P] * 8
            L.orc_conditional_counts.argtypes = [P, P, C.c_int32, P, P]
            L.orc_conditional_prob.argtypes = [P, C.c_int32, C.c_int32]
            L.orc_conditional_prob.restype = C.c_double
            L.orc_threshold.argtypes = [P, C.c_int32, C.c_int32]
            L.orc_threshold.restype = C.c_uint64
            L.orc_select_site.argtypes = [P, C.c_uint32]
            L.orc_select_site.restype = C.c_int32
            L.orc_phi.argtypes = [P, P, C.c_int32, C.c_uint64]
            L.orc_phi.restype = C.c_int32
            L.orc_num_buckets.argtypes = [C.POINTER(Run)]
            L.orc_num_buckets.restype = C.c_int64
            L.orc_run_slots.argtypes = [P, C.POINTER(Run), C.c_int64, C.c_int64, C.c_int32,
                                        P, P, P, P, P, P, P, P, P]
            L.orc_run_slots.restype = C.c_int
            L.orc_replication.argtypes = [P, C.POINTER(Run), C.c_int64, C.c_int32, C.c_int32, P,
                                          P, P, P, P, C.c_int64]
            L.orc_replication.restype = C.c_int
            L.orc_lag_weight.argtypes = [C.c_int64] * 4
            L.orc_lag_weight.restype = C.c_int64
            L.orc_finalize.argtypes = [C.c_int32, C.c_int64, P, P, P, C.c_int64, C.c_int64, P, P]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and 2-word key."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c), _p(k), _p(out))
    return out


def window_defaults(n_active: int, sweeps: int = 1):
    """The paper's window recipe (Experimental Setup): M_s = s n_a updates, b_s = round(0.1 M_s),
    k = b_s + 1, l = M_s.  round() is half-to-even, which Table S1 fixes (b = 166 at M = 1665)."""
    M = sweeps * n_active
    b = round_half_even(0.1 * M)
    return b + 1, M


def round_half_even(x: float) -> int:
    return int(round(x))   # Python's round is half-to-even


class Model:
    """Sampler tables built by the oracle for one instance (pruning, weights, alias, thresholds)."""

    def __init__(self, inst, n_active=0, scan=SCAN_SCORE, custom_w=None, init_marginals=None):
        L = lib()
        self._keep = []
        cp = np.ascontiguousarray(inst.clone_ptr, dtype=np.int32)
        pools = np.ascontiguousarray(inst.clone_pools, dtype=np.int32)
        y = np.ascontiguousarray(inst.y, dtype=np.uint8)
        cw = None if custom_w is None else np.ascontiguousarray(custom_w, dtype=np.float64)
        nu = None if init_marginals is None else np.ascontiguousarray(init_marginals, dtype=np.float64)
        h = C.c_void_p()
        rc = L.orc_model_new(int(inst.n), int(inst.m), _p(cp), _p(pools), _p(y), float(inst.fp),
                             float(inst.fn), float(inst.q), int(n_active), int(scan), _p(cw), _p(nu),
                             C.byref(h))
        if rc != ORC_OK:
            raise ValueError(f"orc_model_new failed: {rc}")
        self.h = h
        self.inst = inst
        d = np.zeros(4, dtype=np.int32)
        L.orc_model_dims(h, _p(d))
        self.na, self.m, self.deg_max, self.nnz = (int(v) for v in d)
        c3 = np.zeros(3)
        L.orc_model_constants(h, _p(c3))
        self.a_plus, self.a_minus, self.lam = (float(v) for v in c3)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().orc_model_free(self.h)
                self.h = None
        except Exception:
            pass

    def tables(self) -> dict:
        na, side = self.na, self.deg_max + 1
        out = dict(eta=np.zeros(self.inst.n), active=np.zeros(na, np.int32), score=np.zeros(na),
                   w=np.zeros(na), V=np.zeros(na, np.uint64), prob=np.zeros(na, np.uint32),
                   alias=np.zeros(na, np.uint32), T=np.zeros(side * side, np.uint64))
        lib().orc_model_tables(self.h, *(_p(out[k]) for k in
                                         ("eta", "active", "score", "w", "V", "prob", "alias", "T")))
        out["T"] = out["T"].reshape(side, side)
        return out

    def conditional_counts(self, x, i):
        xx = np.ascontiguousarray(x, dtype=np.uint8)
        a, b = C.c_int32(), C.c_int32()
        lib().orc_conditional_counts(self.h, _p(xx), int(i), C.byref(a), C.byref(b))
        return a.value, b.value

    def conditional_prob(self, np_, nn):
        return lib().orc_conditional_prob(self.h, int(np_), int(nn))

    def threshold(self, np_, nn) -> int:
        return int(lib().orc_threshold(self.h, int(np_), int(nn)))

    def select_site(self, w) -> int:
        return int(lib().orc_select_site(self.h, int(w)))

    def phi(self, x, i, U) -> int:
        """Apply Phi_i(x, U) in place to a uint8 state array; returns the new bit."""
        return int(lib().orc_phi(self.h, _p(x), int(i), int(U)))

    def replication(self, run: Run, slot: int, rep: int = 0, literal: bool = False,
                    traj_cap: int = 0):
        G = np.zeros(self.na, dtype=np.int64)
        o3 = np.zeros(4, dtype=np.int64)
        tx = ty = sites = None
        if traj_cap:
            tx = np.zeros((traj_cap, self.na), dtype=np.uint8)
            ty = np.zeros((traj_cap, self.na), dtype=np.uint8)
            sites = np.full(traj_cap, -1, dtype=np.int32)
        rc = lib().orc_replication(self.h, C.byref(run), int(slot), int(rep), int(literal), _p(G),
                                   _p(o3), _p(tx), _p(ty), _p(sites), int(traj_cap))
        res = dict(status=rc, G=G, C=int(o3[0]), tau=int(o3[1]), draws=int(o3[2]), capped=int(o3[3]))
        if traj_cap:
            res.update(X=tx, Y=ty, sites=sites)
        return res

    def run_slots(self, run: Run, p_begin: int, p_end: int, threads: int = 1,
                  per_slot: bool = False, slot_G: bool = False) -> dict:
        nb = int(lib().orc_num_buckets(C.byref(run)))
        na = self.na
        S1 = np.zeros((nb, na), np.int64)
        lo = np.zeros((nb, na), np.uint64)
        hi = np.zeros((nb, na), np.uint64)
        cnt = np.zeros(nb, np.int64)
        P = p_end - p_begin
        ns = np.zeros(P, np.int32) if per_slot else None
        sS = np.zeros(P, np.int64) if per_slot else None
        sr = np.zeros(P, np.int32) if per_slot else None
        sG = np.zeros((P, na), np.int64) if slot_G else None
        st = np.zeros(7, np.int64)
        rc = lib().orc_run_slots(self.h, C.byref(run), int(p_begin), int(p_end), int(threads),
                                 _p(S1), _p(lo), _p(hi), _p(cnt), _p(ns), _p(sS), _p(sr), _p(sG),
                                 _p(st))
        return dict(status=rc, nb=nb, S1=S1, S2_lo=lo, S2_hi=hi, count=cnt, slot_nstar=ns,
                    slot_S=sS, slot_reps=sr, slot_G=sG,
                    stats=dict(draws=int(st[0]), reps=int(st[1]), max_tau=int(st[2]),
                               sum_tau=int(st[3]), step_limit_hits=int(st[4]),
                               zero_completion=int(st[5]), capped=int(st[6])))

    def finalize(self, res: dict, P: int, L: int):
        est = np.zeros(self.na)
        se = np.zeros(self.na)
        lib().orc_finalize(self.na, res["nb"], _p(res["S1"]), _p(res["S2_lo"]), _p(res["S2_hi"]),
                           int(P), int(L), _p(est), _p(se))
        return est, se


def lag_weight(k, ell, lag, t) -> int:
    """Weight of X_t and Y_t in G = L H_{k:l} for the lag-L estimator (mcpd_oracle.c)."""
    return int(lib().orc_lag_weight(int(k), int(ell), int(lag), int(t)))


def coupled_run(k, ell, horizon, seed=1, step_limit=10_000_000, slot_offset=0, instance=0,
                meeting_cap=0, lag=1) -> Run:
    return Run(k=k, ell=ell, burn=0, length=1, horizon=horizon, step_limit=step_limit, seed=seed,
               slot_offset=slot_offset, instance=instance, coupled=1, meeting_cap=meeting_cap, lag=lag)


def uncoupled_run(burn, length, horizon, seed=1, slot_offset=0, instance=0) -> Run:
    return Run(k=0, ell=0, burn=burn, length=length, horizon=horizon, step_limit=0, seed=seed,
               slot_offset=slot_offset, instance=instance, coupled=0)


def decode(inst, P, k, ell, horizon, seed=1, threads=None, n_active=0, scan=SCAN_SCORE,
           custom_w=None, init_marginals=None, per_slot=False, slot_G=False, coupled=True,
           burn=0, length=1, slot_offset=0, instance=0, step_limit=10_000_000, meeting_cap=0, lag=1):
    """Whole decode on the CPU: per-clone theta_CT estimates and standard errors (active order)."""
    M = Model(inst, n_active=n_active, scan=scan, custom_w=custom_w, init_marginals=init_marginals)
    run = (coupled_run(k, ell, horizon, seed, step_limit, slot_offset, instance, meeting_cap, lag) if coupled
           else uncoupled_run(burn, length, horizon, seed, slot_offset, instance))
    res = M.run_slots(run, 0, P, threads or os.cpu_count() or 1, per_slot=per_slot, slot_G=slot_G)
    L = (ell - k + 1) if coupled else length
    est, se = M.finalize(res, P, L)
    res.update(est=est, se=se, model=M, L=L)
    return res
