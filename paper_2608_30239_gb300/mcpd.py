"""Thin ctypes binding of the C ABI in include/mcpd.h (argument marshalling only).

Every call goes to `_build/libmcpd.so`; nothing here computes any step of the method.  If the
library is missing the import fails loudly: there is no CPU fallback.  PyTorch is used only for
device buffers and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from . import build as _build

MCPD_OK, MCPD_EINVAL, MCPD_ETOO_LARGE, MCPD_ENOMEM, MCPD_ECUDA, MCPD_ESTEP_LIMIT, MCPD_EOVERFLOW = \
    0, -1, -2, -3, -4, -5, -6
MCPD_SCAN_SCORE, MCPD_SCAN_UNIFORM, MCPD_SCAN_SYSTEMATIC, MCPD_SCAN_CUSTOM = 0, 1, 2, 3
(MCPD_FETCH_S1, MCPD_FETCH_S2_LO, MCPD_FETCH_S2_HI, MCPD_FETCH_COUNT, MCPD_FETCH_SLOT_NSTAR,
 MCPD_FETCH_SLOT_S, MCPD_FETCH_SLOT_REPS, MCPD_FETCH_TRACE_G, MCPD_FETCH_TRACE_REC) = range(9)

_ERRNAMES = {0: "MCPD_OK", -1: "MCPD_EINVAL", -2: "MCPD_ETOO_LARGE", -3: "MCPD_ENOMEM",
             -4: "MCPD_ECUDA", -5: "MCPD_ESTEP_LIMIT", -6: "MCPD_EOVERFLOW"}


class McpdError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class mcpd_design(C.Structure):
    _fields_ = [("n_clones", C.c_int32), ("n_pools", C.c_int32),
                ("clone_ptr", C.c_void_p), ("clone_pools", C.c_void_p)]


class mcpd_params(C.Structure):
    _fields_ = [("fp", C.c_double), ("fn", C.c_double), ("prior_q", C.c_double),
                ("n_active", C.c_int32), ("scan", C.c_int32), ("coupled", C.c_int32),
                ("lanes_per_pair", C.c_int32), ("scan_weights", C.c_void_p),
                ("init_marginals", C.c_void_p), ("k", C.c_int64), ("ell", C.c_int64),
                ("burn", C.c_int64), ("length", C.c_int64), ("slots", C.c_int64),
                ("horizon", C.c_int64), ("budget_site_updates", C.c_double),
                ("step_limit", C.c_int64), ("seed", C.c_uint64), ("instance_id", C.c_uint32),
                ("record_slots", C.c_int32), ("slot_offset", C.c_int64),
                ("trace_stride", C.c_int64), ("tau_audit", C.c_int64), ("meeting_cap", C.c_int64),
                ("lag", C.c_int64), ("trace_steps", C.c_int64), ("trace_reps", C.c_int64)]


class mcpd_stats(C.Structure):
    _fields_ = [(name, C.c_int64) for name in
                ("progress_units", "site_updates", "reps_started", "reps_retained", "reps_aborted",
                 "zero_completion_slots", "step_limit_hits", "max_tau", "sum_tau", "n_buckets",
                 "n_active")] + [("kernel_ms", C.c_double), ("tau_over_audit", C.c_int64),
                                 ("resident_pairs", C.c_int64), ("h2d_bytes", C.c_int64),
                                 ("d2h_bytes", C.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


HEADER = os.path.join(_build.INCLUDE, "mcpd.h")
_lib = None


def header_functions():
    """Names of the functions include/mcpd.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mcpd_[a-z_]+)\s*\(", text)))


def lib(build_if_missing: bool = False):
    global _lib
    if _lib is None:
        if build_if_missing:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"CUDA library not built: {_build.LIB} (run __graft_entry__.build())")
        L = C.CDLL(_build.LIB)
        P, I64 = C.c_void_p, C.c_int64
        sig = {
            "mcpd_ctx_create": (C.c_int, [C.c_int, P, C.POINTER(P)]),
            "mcpd_ctx_destroy": (None, [P]),
            "mcpd_last_error": (C.c_char_p, [P]),
            "mcpd_plan_create": (C.c_int, [P, C.POINTER(mcpd_design), P, C.POINTER(mcpd_params),
                                           C.POINTER(P)]),
            "mcpd_plan_destroy": (None, [P]),
            "mcpd_plan_info": (C.c_int, [P, P]),
            "mcpd_plan_active": (C.c_int, [P, P]),
            "mcpd_run_async": (C.c_int, [P, P, P, P]),
            "mcpd_run_slots_async": (C.c_int, [P, P, C.c_int64, C.c_int32, P, P]),
            "mcpd_collect": (C.c_int, [P, P, C.POINTER(mcpd_stats)]),
            "mcpd_fetch_bytes": (C.c_size_t, [P, C.c_int]),
            "mcpd_fetch": (C.c_int, [P, P, C.c_int, P, C.c_size_t]),
            "mcpd_decode": (C.c_int, [P, C.POINTER(mcpd_design), P, C.POINTER(mcpd_params), P, P,
                                      P, C.POINTER(mcpd_stats)]),
            "mcpd_inspect": (C.c_int, [C.POINTER(mcpd_design), P, C.POINTER(mcpd_params), P, P,
                                       P, P, P]),
            "mcpd_philox_device": (C.c_int, [P, P, C.c_uint32, C.c_uint32, P, I64]),
            "mcpd_decode_noalloc": (C.c_int, [P, C.POINTER(mcpd_design), P, C.POINTER(mcpd_params),
                                              P, P, C.POINTER(mcpd_stats)]),
            "mcpd_batch_create": (C.c_int, [P, C.c_int32, P, P, P, C.c_int32, C.POINTER(P)]),
            "mcpd_batch_destroy": (None, [P]),
            "mcpd_batch_classes": (C.c_int, [C.c_int32, P, P, P, C.c_int32, C.c_int32, P, P]),
            "mcpd_batch_info": (C.c_int, [P, P]),
            "mcpd_batch_offsets": (C.c_int, [P, P]),
            "mcpd_batch_set_shape": (C.c_int, [P, P, C.c_int32, C.c_int32]),
            "mcpd_batch_run_async": (C.c_int, [P, P, P, P]),
            "mcpd_batch_capture_graph": (C.c_int, [P, P, P, P]),
            "mcpd_batch_launch_graph": (C.c_int, [P, P]),
            "mcpd_batch_collect": (C.c_int, [P, P, C.POINTER(mcpd_stats)]),
            "mcpd_batch_extend_async": (C.c_int, [P, P, P, P, P]),
            "mcpd_batch_fetch": (C.c_int, [P, P, C.c_int32, C.c_int, P, C.c_size_t]),
            "mcpd_batch_autotune": (C.c_int, [P, P, P, P, C.c_int32, C.c_int32, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def _check_out(est, se, need, device):
    """Refuses output buffers the kernels could write past: each must be a contiguous float64 CUDA
    tensor on the context's device with at least `need` elements (one per active clone)."""
    import torch
    for name, a in (("est", est), ("se", se)):
        if not isinstance(a, torch.Tensor):
            raise TypeError(f"{name}: a torch tensor is required, got {type(a).__name__}")
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError(f"{name}: a contiguous float64 tensor is required, got {a.dtype}")
        if a.numel() < need:
            raise ValueError(f"{name}: {a.numel()} elements, {need} needed")
        if not a.is_cuda or a.device.index != device:
            raise ValueError(f"{name}: on {a.device}, the context is on cuda:{device}")


class _Keep:
    """Holds the numpy arrays a ctypes struct points into."""

    def __init__(self):
        self.items = []

    def arr(self, a, dtype):
        if a is None:
            return None
        a = np.ascontiguousarray(a, dtype=dtype)
        self.items.append(a)
        return a


def make_design(inst, keep: _Keep):
    cp = keep.arr(inst.clone_ptr, np.int32)
    pools = keep.arr(inst.clone_pools, np.int32)
    y = keep.arr(inst.y, np.uint8)
    d = mcpd_design(int(inst.n), int(inst.m), _ptr(cp).value, _ptr(pools).value if len(pools) else None)
    return d, y


def make_params(inst=None, keep: _Keep | None = None, *, fp=None, fn=None, prior_q=None,
                n_active=0, scan=MCPD_SCAN_SCORE, coupled=True, scan_weights=None,
                init_marginals=None, k=-1, ell=-1, burn=-1, length=-1, slots=1, horizon=0,
                budget_site_updates=0.0, step_limit=0, seed=1, instance_id=0, record_slots=False,
                slot_offset=0, trace_stride=0, lanes_per_pair=0, tau_audit=0, meeting_cap=0, lag=0,
                trace_steps=0, trace_reps=0):
    keep = keep or _Keep()
    sw = keep.arr(scan_weights, np.float64)
    nu = keep.arr(init_marginals, np.float64)
    return mcpd_params(
        fp=float(inst.fp if fp is None else fp), fn=float(inst.fn if fn is None else fn),
        prior_q=float(inst.q if prior_q is None else prior_q), n_active=int(n_active),
        scan=int(scan), coupled=int(bool(coupled)), lanes_per_pair=int(lanes_per_pair),
        scan_weights=None if sw is None else _ptr(sw).value,
        init_marginals=None if nu is None else _ptr(nu).value, k=int(k), ell=int(ell),
        burn=int(burn), length=int(length), slots=int(slots), horizon=int(horizon),
        budget_site_updates=float(budget_site_updates), step_limit=int(step_limit),
        seed=int(seed) & 0xFFFFFFFFFFFFFFFF, instance_id=int(instance_id),
        record_slots=int(bool(record_slots)), slot_offset=int(slot_offset),
        trace_stride=int(trace_stride), tau_audit=int(tau_audit), meeting_cap=int(meeting_cap),
        lag=int(lag), trace_steps=int(trace_steps), trace_reps=int(trace_reps))


def mcpd_inspect(inst, **params):
    """Host-built tables of the library (no GPU): info, active ids, weights, alias words, T."""
    L = lib()
    keep = _Keep()
    d, y = make_design(inst, keep)
    prm = make_params(inst, keep, **params)
    info = np.zeros(16, np.int64)
    rc = L.mcpd_inspect(C.byref(d), _ptr(y), C.byref(prm), _ptr(info), None, None, None, None)
    if rc != MCPD_OK:
        raise McpdError(rc, "mcpd_inspect")
    na = int(info[0])
    active = np.zeros(na, np.int32)
    w = np.zeros(na)
    alias = np.zeros(na, np.uint64)
    T = np.zeros(81, np.uint64)
    rc = L.mcpd_inspect(C.byref(d), _ptr(y), C.byref(prm), _ptr(info), _ptr(active), _ptr(w),
                        _ptr(alias), _ptr(T))
    if rc != MCPD_OK:
        raise McpdError(rc, "mcpd_inspect")
    return dict(info=info, active=active, w=w, alias=alias, T=T.reshape(9, 9))


class Context:
    """mcpd_ctx on one device and one stream (default: torch's current stream on that device)."""

    def __init__(self, device: int = 0, stream=None):
        L = lib()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        h = C.c_void_p()
        rc = L.mcpd_ctx_create(int(device), C.c_void_p(stream), C.byref(h))
        if rc != MCPD_OK:
            raise McpdError(rc, "mcpd_ctx_create")
        self.h = h
        self.device = int(device)

    def error(self) -> str:
        return lib().mcpd_last_error(self.h).decode()

    def check(self, rc, what):
        if rc != MCPD_OK:
            raise McpdError(rc, f"{what}: {self.error()}")

    def close(self):
        if getattr(self, "h", None):
            lib().mcpd_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def philox(self, ctr_dev, key0, key1, out_dev, n):
        self.check(lib().mcpd_philox_device(self.h, _ptr(ctr_dev), key0, key1, _ptr(out_dev), n),
                   "mcpd_philox_device")

    def decode(self, inst, **params):
        """mcpd_decode: host arrays in, host arrays out (original clone order)."""
        keep = _Keep()
        d, y = make_design(inst, keep)
        prm = make_params(inst, keep, **params)
        est = np.zeros(inst.n)
        se = np.zeros(inst.n)
        act = np.zeros(inst.n, np.int32)
        st = mcpd_stats()
        rc = lib().mcpd_decode(self.h, C.byref(d), _ptr(y), C.byref(prm), _ptr(est), _ptr(se),
                               _ptr(act), C.byref(st))
        if rc not in (MCPD_OK, MCPD_ESTEP_LIMIT):
            self.check(rc, "mcpd_decode")
        return dict(status=rc, est=est, se=se, active=act, stats=st.as_dict())


    def decode_noalloc(self, inst, est_dev, se_dev, **params):
        """mcpd_decode_noalloc: host inputs, caller-owned device outputs [n_active], and no device
        allocation by the library (its scratch is a fixed 64 MiB array inside the library)."""
        keep = _Keep()
        d, y = make_design(inst, keep)
        prm = make_params(inst, keep, **params)
        st = mcpd_stats()
        rc = lib().mcpd_decode_noalloc(self.h, C.byref(d), _ptr(y), C.byref(prm), _ptr(est_dev),
                                       _ptr(se_dev), C.byref(st))
        if rc not in (MCPD_OK, MCPD_ESTEP_LIMIT):
            self.check(rc, "mcpd_decode_noalloc")
        out = st.as_dict()
        out["status"] = rc
        return out


class Plan:
    """mcpd_plan: tables on the device plus scratch; run many times."""

    def __init__(self, ctx: Context, inst, **params):
        self.ctx = ctx
        keep = _Keep()
        d, y = make_design(inst, keep)
        prm = make_params(inst, keep, **params)
        h = C.c_void_p()
        ctx.check(lib().mcpd_plan_create(ctx.h, C.byref(d), _ptr(y), C.byref(prm), C.byref(h)),
                  "mcpd_plan_create")
        self.h = h
        info = np.zeros(16, np.int64)
        lib().mcpd_plan_info(h, _ptr(info))
        self.info = info
        self.n_active = int(info[0])
        self.n_buckets = int(info[1])
        self.horizon, self.k, self.ell, self.L, self.slots = (int(v) for v in info[2:7])
        self.active = np.zeros(self.n_active, np.int32)
        lib().mcpd_plan_active(h, _ptr(self.active))
        self.trace_steps = int(params.get("trace_steps", 0))
        self.trace_reps = (int(params.get("trace_reps", 0)) or 8) if self.trace_steps > 0 else 0

    def run_async(self, est_dev, se_dev):
        _check_out(est_dev, se_dev, self.n_active, self.ctx.device)
        self.ctx.check(lib().mcpd_run_async(self.ctx.h, self.h, _ptr(est_dev), _ptr(se_dev)),
                       "mcpd_run_async")

    def run_slots_async(self, slots, est_dev, se_dev, accumulate=False):
        """mcpd_run_slots_async: `slots` slots with the plan's horizon; accumulate=True adds them
        to the slots already run (the next global slot ids) and finalizes over all of them."""
        _check_out(est_dev, se_dev, self.n_active, self.ctx.device)
        self.ctx.check(lib().mcpd_run_slots_async(self.ctx.h, self.h, int(slots), int(bool(accumulate)),
                                                  _ptr(est_dev), _ptr(se_dev)), "mcpd_run_slots_async")

    def collect(self, allow_step_limit=False):
        st = mcpd_stats()
        rc = lib().mcpd_collect(self.ctx.h, self.h, C.byref(st))
        if rc != MCPD_OK and not (allow_step_limit and rc == MCPD_ESTEP_LIMIT):
            self.ctx.check(rc, "mcpd_collect")
        out = st.as_dict()
        out["status"] = rc
        return out

    def fetch(self, what):
        dt = {MCPD_FETCH_S1: np.int64, MCPD_FETCH_S2_LO: np.uint64, MCPD_FETCH_S2_HI: np.uint64,
              MCPD_FETCH_COUNT: np.int64, MCPD_FETCH_SLOT_NSTAR: np.int32,
              MCPD_FETCH_SLOT_S: np.int64, MCPD_FETCH_SLOT_REPS: np.int32,
              MCPD_FETCH_TRACE_G: np.int64, MCPD_FETCH_TRACE_REC: np.int32}[what]
        nbytes = lib().mcpd_fetch_bytes(self.h, what)
        out = np.zeros(nbytes // np.dtype(dt).itemsize, dtype=dt)
        self.ctx.check(lib().mcpd_fetch(self.ctx.h, self.h, what, _ptr(out), nbytes), "mcpd_fetch")
        if what in (MCPD_FETCH_S1, MCPD_FETCH_S2_LO, MCPD_FETCH_S2_HI):
            out = out.reshape(self.n_buckets, self.n_active)
        if what == MCPD_FETCH_TRACE_G:
            out = out.reshape(-1, self.n_active)
        if what == MCPD_FETCH_TRACE_REC:
            out = out.reshape(-1, self.trace_reps, 4 + self.trace_steps)
        return out

    def buckets(self):
        return dict(S1=self.fetch(MCPD_FETCH_S1), S2_lo=self.fetch(MCPD_FETCH_S2_LO),
                    S2_hi=self.fetch(MCPD_FETCH_S2_HI), count=self.fetch(MCPD_FETCH_COUNT))

    def close(self):
        if getattr(self, "h", None):
            lib().mcpd_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_classes(instances, params, order_mode=0, classes=0, sm_count=152):
    """mcpd_batch_classes: the classes a Batch of these instances would form on a GPU with
    `sm_count` multiprocessors, computed on the host.  Returns (class of each instance, number of
    classes)."""
    n = len(instances)
    if isinstance(params, dict):
        params = [params] * n
    keep = _Keep()
    designs = (mcpd_design * n)()
    ys = (C.c_void_p * n)()
    prms = (mcpd_params * n)()
    for i, (inst, kw) in enumerate(zip(instances, params)):
        d, y = make_design(inst, keep)
        designs[i] = d
        ys[i] = _ptr(y).value
        prms[i] = make_params(inst, keep, **kw)
    cls = np.zeros(n, np.int32)
    nc = C.c_int32(0)
    rc = lib().mcpd_batch_classes(n, designs, ys, prms, int(order_mode) | (int(classes) << 8), int(sm_count),
                                  _ptr(cls), C.byref(nc))
    if rc != MCPD_OK:
        raise McpdError(rc, "mcpd_batch_classes")
    return cls, int(nc.value)


class Batch:
    """mcpd_batch: many instances (each with its own parameters) decoded in one persistent launch
    per class.

    `instances` is a list of synth-like instances; `params` a list of keyword dicts (one per
    instance) or one dict for all.  `order_mode` 0 (input order) or 1 (longest slots first);
    `classes` 0 (automatic: coupled instances grouped by uniform degree, then cut by size) or 1..8
    size classes.  Outputs of run()/fetch are concatenated in
    input order; `offsets[i]:offsets[i+1]` belong to instance i."""

    def __init__(self, ctx: Context, instances, params, order_mode=0, classes=0):
        self.ctx = ctx
        n = len(instances)
        if isinstance(params, dict):
            params = [params] * n
        self._keep = _Keep()
        designs = (mcpd_design * n)()
        ys = (C.c_void_p * n)()
        prms = (mcpd_params * n)()
        for i, (inst, kw) in enumerate(zip(instances, params)):
            d, y = make_design(inst, self._keep)
            designs[i] = d
            ys[i] = _ptr(y).value
            prms[i] = make_params(inst, self._keep, **kw)
        h = C.c_void_p()
        ctx.check(lib().mcpd_batch_create(ctx.h, n, designs, ys, prms, int(order_mode) | (int(classes) << 8),
                                          C.byref(h)), "mcpd_batch_create")
        self.h = h
        self.n_inst = n
        self.info = self._info()
        self.classes = int(self.info[9])
        self.total_active = int(self.info[0])
        self.offsets = np.zeros(n + 1, np.int64)
        lib().mcpd_batch_offsets(h, _ptr(self.offsets))
        self.nb = [int(mcpd_inspect(inst, **kw)["info"][1]) for inst, kw in zip(instances, params)]
        self.na = [int(v) for v in np.diff(self.offsets)]

    def _info(self):
        info = np.zeros(16, np.int64)
        lib().mcpd_batch_info(self.h, _ptr(info))
        return info

    def set_shape(self, warps_per_block=0, lanes_per_pair=1):
        self.ctx.check(lib().mcpd_batch_set_shape(self.ctx.h, self.h, int(lanes_per_pair),
                                                  int(warps_per_block)), "mcpd_batch_set_shape")
        self.info = self._info()

    def run_async(self, est_dev, se_dev):
        _check_out(est_dev, se_dev, self.total_active, self.ctx.device)
        self.ctx.check(lib().mcpd_batch_run_async(self.ctx.h, self.h, _ptr(est_dev), _ptr(se_dev)),
                       "mcpd_batch_run_async")

    def extend_async(self, est_dev, se_dev, mask=None):
        """mcpd_batch_extend_async: every instance (or those with mask[i]) runs its next P_i slots
        into the same buckets; est/se are finalized over all slots so far."""
        _check_out(est_dev, se_dev, self.total_active, self.ctx.device)
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.int32)
        if m is not None and len(m) != self.n_inst:
            raise ValueError("mask needs one entry per instance")
        self.ctx.check(lib().mcpd_batch_extend_async(self.ctx.h, self.h, _ptr(m), _ptr(est_dev), _ptr(se_dev)),
                       "mcpd_batch_extend_async")

    def capture_graph(self, est_dev, se_dev):
        _check_out(est_dev, se_dev, self.total_active, self.ctx.device)
        self.ctx.check(lib().mcpd_batch_capture_graph(self.ctx.h, self.h, _ptr(est_dev), _ptr(se_dev)),
                       "mcpd_batch_capture_graph")

    def launch_graph(self):
        self.ctx.check(lib().mcpd_batch_launch_graph(self.ctx.h, self.h), "mcpd_batch_launch_graph")

    def collect(self, allow_step_limit=False):
        st = mcpd_stats()
        rc = lib().mcpd_batch_collect(self.ctx.h, self.h, C.byref(st))
        if rc != MCPD_OK and not (allow_step_limit and rc == MCPD_ESTEP_LIMIT):
            self.ctx.check(rc, "mcpd_batch_collect")
        out = st.as_dict()
        out["status"] = rc
        return out

    def buckets(self, i):
        out = {}
        for key, what, dt in (("S1", MCPD_FETCH_S1, np.int64), ("S2_lo", MCPD_FETCH_S2_LO, np.uint64),
                              ("S2_hi", MCPD_FETCH_S2_HI, np.uint64), ("count", MCPD_FETCH_COUNT, np.int64)):
            n = self.nb[i] * (1 if what == MCPD_FETCH_COUNT else self.na[i])
            a = np.zeros(n, dt)
            self.ctx.check(lib().mcpd_batch_fetch(self.ctx.h, self.h, i, what, _ptr(a), a.nbytes),
                           "mcpd_batch_fetch")
            out[key] = a if what == MCPD_FETCH_COUNT else a.reshape(self.nb[i], self.na[i])
        return out

    def autotune(self, est_dev, se_dev, candidates=((1, 0), (8, 0), (16, 0), (32, 0)), reps=1):
        """candidates: (lanes per pair, warps per block) pairs (0 warps: as many as fit).  Returns
        the chosen pair and {pair: mean ms} (-1 where a candidate does not fit)."""
        _check_out(est_dev, se_dev, self.total_active, self.ctx.device)
        cand = [(int(a), int(b)) for a, b in candidates]
        lanes = np.asarray([c[0] for c in cand], np.int32)
        warps = np.asarray([c[1] for c in cand], np.int32)
        times = np.zeros(len(cand))
        best = C.c_int32()
        self.ctx.check(lib().mcpd_batch_autotune(self.ctx.h, self.h, _ptr(lanes), _ptr(warps), len(cand),
                                                 int(reps), _ptr(est_dev), _ptr(se_dev), C.byref(best),
                                                 _ptr(times)), "mcpd_batch_autotune")
        self.info = self._info()
        return cand[int(best.value)], dict(zip(cand, (float(t) for t in times)))

    def close(self):
        if getattr(self, "h", None):
            lib().mcpd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
