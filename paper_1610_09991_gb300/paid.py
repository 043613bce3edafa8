"""Thin ctypes binding of libpaid (include/paid.h) with the same names.

Only argument marshalling happens here: device buffers come from torch
tensors (``data_ptr()``), the stream from ``torch.cuda.current_stream()``,
and every step of the cubature runs in the library's CUDA kernels.  There is
no CPU fallback: without libpaid.so (see ``build.py``) or without a CUDA
device every call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpaid.so")

PH, PP, MONOMIAL, OVERLAP, FLOW_PH, FLOW_PP = 0, 1, 2, 3, 4, 5
FF_SHELL1, FF_SHELL12 = 5, 9
OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_POOL, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
# kernels one paid_mlp_forward call launches: the weight cast and the fused
# five-layer forward pass
MLP_FORWARD_LAUNCHES = 2
CONVERGED, BUDGET, NONFINITE, ROUNDCAP, POOL = 0, 1, 2, 3, 4
GROUP_NONE, GROUP_PER_PAIR, GROUP_GLOBAL = 0, 1, 2       # options.group_mode

#: every entry point declared in include/paid.h
EXPORTS = ("paid_options_default", "paid_create", "paid_destroy", "paid_workspace_size",
           "paid_pool_capacity", "paid_integrate_batch", "paid_integrate_multi",
           "paid_integrate_multi_seeded", "paid_cell_errors", "paid_last_stats",
           "paid_error_string", "paid_last_error", "paid_mlp_param_count",
           "paid_mlp_workspace_size", "paid_mlp_init", "paid_mlp_features", "paid_mlp_forward",
           "paid_mlp_grad", "paid_mlp_adamw", "paid_rule_regions", "paid_check_math",
           "paid_get_options", "paid_autotune", "paid_tu_flow_rhs", "paid_integrate_batch_static",
           "paid_set_trace_buffer", "paid_mlp_group_features", "paid_proposal_train",
           "paid_proposal_train_workspace_size", "paid_proposal_save", "paid_proposal_load",
           "paid_wait")


class paid_options(ctypes.Structure):
    _fields_ = [("rule_n", ctypes.c_int), ("init_level", ctypes.c_int),
                ("eval_fp32", ctypes.c_int), ("max_rounds", ctypes.c_int),
                ("cover", ctypes.c_double), ("pool_capacity", ctypes.c_int64),
                ("timing", ctypes.c_int), ("device_loop", ctypes.c_int),
                ("group_mode", ctypes.c_int), ("eval_blocks", ctypes.c_int),
                ("trace", ctypes.c_int)]


class paid_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int), ("region_evals", ctypes.c_int64),
                ("node_evals", ctypes.c_int64), ("peak_pool", ctypes.c_int64),
                ("pool_capacity", ctypes.c_int64), ("n_integrals", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("eval_launches", ctypes.c_int64),
                ("eval_ms", ctypes.c_double), ("reduce_ms", ctypes.c_double),
                ("scan_ms", ctypes.c_double), ("split_ms", ctypes.c_double),
                ("escalated", ctypes.c_int64), ("df_regions", ctypes.c_int64),
                ("df_ms", ctypes.c_double), ("throttled_rounds", ctypes.c_int64),
                ("graph_launches", ctypes.c_int64)]


class paid_batch(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("T", ctypes.c_double), ("nq", ctypes.c_int),
                ("q", ctypes.c_void_p), ("npairs", ctypes.c_int), ("lm", ctypes.c_void_p),
                ("rel_tol", ctypes.c_double), ("abs_tol", ctypes.c_double),
                ("max_regions", ctypes.c_int64), ("values", ctypes.c_void_p),
                ("errors", ctypes.c_void_p), ("regions", ctypes.c_void_p),
                ("status", ctypes.c_void_p), ("tu_v", ctypes.c_void_p * 2),
                ("tu_out", ctypes.c_void_p * 2)]


_lock = threading.Lock()
_lib = None


class PaidError(RuntimeError):
    def __init__(self, rc, msg):
        super().__init__("libpaid error %d (%s): %s" % (rc, error_string(rc) if _lib else "?", msg))
        self.rc = rc


def load(path: str = LIB_PATH):
    """Load libpaid.so and declare its signatures; raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError("libpaid.so not built (%s); run paper_1610_09991_gb300/build.py "
                               "or __graft_entry__.build()" % path)
        lib = ctypes.CDLL(path)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.paid_options_default.argtypes = [ctypes.POINTER(paid_options)]
        lib.paid_create.argtypes = [ctypes.POINTER(P), D, D, D, I, ctypes.POINTER(paid_options), I]
        lib.paid_destroy.argtypes = [P]
        lib.paid_destroy.restype = None
        lib.paid_workspace_size.argtypes = [P, I64, I64, ctypes.POINTER(ctypes.c_size_t)]
        lib.paid_pool_capacity.argtypes = [P, I64, ctypes.c_size_t, ctypes.POINTER(I64)]
        lib.paid_integrate_batch.argtypes = [P, I, I, P, I, P, D, D, D, I64, P, P, P, P, P,
                                             ctypes.c_size_t, P]
        lib.paid_integrate_multi.argtypes = [P, ctypes.POINTER(paid_batch), I, P,
                                             ctypes.c_size_t, P]
        lib.paid_last_stats.argtypes = [P, ctypes.POINTER(paid_stats)]
        lib.paid_error_string.argtypes = [I]
        lib.paid_error_string.restype = ctypes.c_char_p
        lib.paid_last_error.argtypes = [P]
        lib.paid_last_error.restype = ctypes.c_char_p
        lib.paid_integrate_multi_seeded.argtypes = [P, ctypes.POINTER(paid_batch), I, P, D, P,
                                                    ctypes.c_size_t, P]
        lib.paid_cell_errors.argtypes = [P, I, I, P, I, P, D, P, P, ctypes.c_size_t, P]
        lib.paid_rule_regions.argtypes = [P, I, D, P, I, P, I, P, P, P, P, ctypes.c_size_t, P]
        lib.paid_check_math.argtypes = [P, I, I64, P, P, P, P]
        lib.paid_get_options.argtypes = [P, ctypes.POINTER(paid_options)]
        lib.paid_tu_flow_rhs.argtypes = [P, I, I, P, P, P, P, P, P, P, P, P]
        lib.paid_autotune.argtypes = [P, ctypes.POINTER(paid_batch), I, ctypes.c_char_p, P,
                                      ctypes.c_size_t, P]
        lib.paid_mlp_param_count.argtypes = [ctypes.POINTER(I64)]
        lib.paid_mlp_workspace_size.argtypes = [I64, ctypes.POINTER(ctypes.c_size_t)]
        lib.paid_mlp_init.argtypes = [P, ctypes.c_uint64, P]
        lib.paid_mlp_features.argtypes = [P, I, I, P, I, P, D, P, P]
        lib.paid_mlp_forward.argtypes = [P, P, I64, P, P, ctypes.c_size_t, P]
        lib.paid_mlp_grad.argtypes = [P, P, P, I64, P, P, P, ctypes.c_size_t, P]
        lib.paid_mlp_adamw.argtypes = [P, P, P, P, I, ctypes.c_float, ctypes.c_float, P]
        lib.paid_set_trace_buffer.argtypes = [P, P, I64]
        lib.paid_wait.argtypes = [P, ctypes.POINTER(I)]
        lib.paid_mlp_group_features.argtypes = [P, I, I, P, D, P, P]
        lib.paid_proposal_train_workspace_size.argtypes = [I64, I64, ctypes.POINTER(ctypes.c_size_t)]
        lib.paid_proposal_train.argtypes = [P, P, P, P, P, I64, I, I64, ctypes.c_float,
                                            ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(I),
                                            P, P, ctypes.c_size_t, P]
        lib.paid_proposal_save.argtypes = [P, ctypes.c_char_p, P]
        lib.paid_proposal_load.argtypes = [P, ctypes.c_char_p, P]
        lib.paid_integrate_batch_static.argtypes = [P, I, I, P, I, P, D, D, D, I64, P, P, P, P, P]
        _lib = lib
        return lib


def error_string(rc: int) -> str:
    return load().paid_error_string(rc).decode()


def options_default() -> paid_options:
    o = paid_options()
    load().paid_options_default(ctypes.byref(o))
    return o


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libpaid needs a CUDA device; none is available")
    return torch


@dataclass
class Result:
    values: object
    errors: object
    regions: object
    status: object


class Context:
    """One paid_ctx: lattice (t, t', mu), form-factor set and options."""

    def __init__(self, t=1.0, tp=-0.25, mu=-1.0, ffset=FF_SHELL12, device=0, **options):
        self._lib = load()
        torch = _torch()
        self.device = device
        self.torch_device = torch.device("cuda", device)
        o = options_default()
        for k, v in options.items():
            if not hasattr(o, k):
                raise TypeError("unknown option %r" % k)
            setattr(o, k, v)
        self.options = o
        h = ctypes.c_void_p()
        rc = self._lib.paid_create(ctypes.byref(h), t, tp, mu, ffset, ctypes.byref(o), device)
        if rc != OK:
            raise PaidError(rc, "paid_create")
        self._h = h
        self.lattice = (t, tp, mu)
        self.ffset = ffset
        self._ws = None

    def close(self):
        if getattr(self, "_h", None):
            self._lib.paid_destroy(self._h)
            self._h = None
        self._ws = None

    def release_workspace(self):
        """Drop the cached workspace (results already returned stay valid) and
        hand the memory back to the device for other allocations."""
        self._ws = None
        _torch().cuda.empty_cache()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        return self._lib.paid_last_error(self._h).decode()

    def workspace_size(self, n_integrals: int, pool_capacity: int) -> int:
        b = ctypes.c_size_t()
        rc = self._lib.paid_workspace_size(self._h, n_integrals, pool_capacity, ctypes.byref(b))
        if rc != OK:
            raise PaidError(rc, self.last_error())
        return b.value

    def pool_capacity(self, n_integrals: int, ws_bytes: int) -> int:
        c = ctypes.c_int64()
        rc = self._lib.paid_pool_capacity(self._h, n_integrals, ws_bytes, ctypes.byref(c))
        if rc != OK:
            raise PaidError(rc, self.last_error())
        return c.value

    def last_stats(self) -> dict:
        s = paid_stats()
        self._lib.paid_last_stats(self._h, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in paid_stats._fields_}

    def workspace(self, n_integrals: int, pool_capacity: int):
        """A device byte tensor large enough for n integrals and the capacity
        (kept and reused across calls while it is big enough)."""
        torch = _torch()
        need = self.workspace_size(n_integrals, pool_capacity)
        if self._ws is None or self._ws.numel() < need:
            # hand cached blocks back first: one large block is needed, and the
            # cache may hold the memory in pieces
            self._ws = None
            torch.cuda.empty_cache()
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.torch_device)
        return self._ws

    #: regions per unit the default pool is sized for: an integral's regions
    #: take 64 bytes, a (kind, q) group's ~2 KB (every pair's values); the pool
    #: streams units in when it holds fewer, and a call that cannot progress
    #: grows it
    DEFAULT_REGIONS_PER_UNIT = 8192
    DEFAULT_GROUP_REGIONS_PER_UNIT = 2048

    def default_capacity(self, n_units: int, max_regions: int) -> int:
        """Pool capacity used when none is given: every unit at min(its budget,
        8192 regions per integral or 2048 per (kind, q) group), or the capacity
        an earlier call had to grow to, bounded by 70 % of the device's free
        memory."""
        torch = _torch()
        free, _ = torch.cuda.mem_get_info(self.device)
        # memory torch holds in its cache is available to this allocation too
        cached = torch.cuda.memory_reserved(self.device) - torch.cuda.memory_allocated(self.device)
        n0 = 4 ** self.options.init_level
        per = (self.DEFAULT_GROUP_REGIONS_PER_UNIT if self.options.group_mode
               else self.DEFAULT_REGIONS_PER_UNIT)
        want = max(n_units * n0, n_units * min(max_regions, per),
                   getattr(self, "_grown_capacity", 0))
        held = self._ws.numel() if self._ws is not None else 0
        limit = self.pool_capacity(n_units, int(0.7 * (free + cached + held)))
        return int(max(n_units * n0, min(want, limit, 2 ** 32 - 1)))

    def integrate_multi(self, batches, pool_capacity=None, stream=None, asynchronous=False):
        """Device-resident batches: a list of dicts with keys kind, T, q (cuda
        float64 [nq, 2]), lm (cuda int32 [npairs, 2]), rel_tol, abs_tol,
        max_regions.  Returns one Result of cuda tensors per batch.  With
        asynchronous=True (device loop only) the call returns once the work is
        queued: wait() gives its outcome, and a full pool is not retried."""
        return self._integrate(batches, pool_capacity, stream, None, asynchronous)

    def wait(self) -> int:
        """paid_wait: the outcome code of the last integrate call."""
        out = ctypes.c_int(OK)
        rc = self._lib.paid_wait(self._h, ctypes.byref(out))
        if rc != OK:
            raise PaidError(rc, self.last_error())
        self.last_rc = out.value
        return out.value

    def integrate_multi_seeded(self, batches, proposal=None, margin=1.0, pool_capacity=None,
                               stream=None):
        """As integrate_multi, with the initial partition from level maps
        (cuda float32 [units, 256], global unit order: (kind, q) groups in
        group mode, else integrals; None = uniform level 4): cell c starts at
        level floor(map[c] - margin)."""
        return self._integrate(batches, pool_capacity, stream, (proposal, float(margin)))

    def set_trace_buffer(self, maps):
        """Give the integrate calls a buffer for the trace maps (options.trace):
        cuda float32 [units, 256] (None clears it); it is kept referenced here."""
        torch = _torch()
        if maps is None:
            rc = self._lib.paid_set_trace_buffer(self._h, None, 0)
        else:
            if (maps.dtype != torch.float32 or maps.dim() != 2 or maps.shape[1] != 256
                    or not maps.is_contiguous() or maps.device != self.torch_device):
                raise ValueError("trace maps must be contiguous float32 [units, 256] on %s"
                                 % self.torch_device)
            rc = self._lib.paid_set_trace_buffer(self._h, maps.data_ptr(), maps.shape[0])
        if rc != OK:
            raise PaidError(rc, "paid_set_trace_buffer")
        self._trace = maps

    def group_features(self, kind, q, T, stream=None):
        """Proposal inputs with one row per (kind, q) group: cuda bfloat16 [nq, 32]."""
        torch = _torch()
        x = torch.empty((q.shape[0], 32), dtype=torch.bfloat16, device=self.torch_device)
        if stream is None:
            stream = torch.cuda.current_stream(self.torch_device)
        rc = self._lib.paid_mlp_group_features(self._h, int(kind), q.shape[0], q.data_ptr(),
                                               float(T), x.data_ptr(),
                                               ctypes.c_void_p(stream.cuda_stream))
        if rc != OK:
            raise PaidError(rc, "paid_mlp_group_features")
        return x

    def rule_regions(self, kind, q, lm, T, regions, stream=None):
        """The nested rule on given regions for every pair of one (kind, q).

        q: cuda float64 [2]; lm: cuda int32 [npairs, 2]; regions: cuda int32
        [nreg, 3] = (level, ix, iy).  Returns (q2N, dq), cuda float64
        [nreg, npairs]: Q_2N and Q_N - Q_2N times the region's Jacobian."""
        torch = _torch()
        nreg, npairs = regions.shape[0], lm.shape[0]
        q2 = torch.empty((nreg, npairs), dtype=torch.float64, device=self.torch_device)
        dq = torch.empty_like(q2)
        if stream is None:
            stream = torch.cuda.current_stream(self.torch_device)
        # (a group-mode context reports a larger layout: still enough)
        need = self.workspace_size(1, max(nreg, 16))
        ws = self._ws if self._ws is not None and self._ws.numel() >= need else \
            torch.empty(need, dtype=torch.uint8, device=self.torch_device)
        rc = self._lib.paid_rule_regions(self._h, int(kind), float(T), q.data_ptr(), npairs,
                                         lm.data_ptr(), nreg, regions.data_ptr(), q2.data_ptr(),
                                         dq.data_ptr(), ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                         ctypes.c_void_p(stream.cuda_stream))
        if rc != OK:
            raise PaidError(rc, self.last_error())
        return q2, dq

    def check_math(self, which, x, y=None):
        """paid_check_math on cuda float64 tensors: 0 = exp(-x), 1 = x / y (FP64),
        2 = exp(-x) in float-float, 3 / 4 = 2T F(x, y) of the bubbles in
        float-float / FP64, 5 / 6 = the flow kernel at Omega = 0.1."""
        torch = _torch()
        out = torch.empty_like(x)
        stream = torch.cuda.current_stream(self.torch_device)
        rc = self._lib.paid_check_math(self._h, int(which), x.numel(), x.data_ptr(),
                                       y.data_ptr() if y is not None else None, out.data_ptr(),
                                       ctypes.c_void_p(stream.cuda_stream))
        if rc != OK:
            raise PaidError(rc, self.last_error())
        return out

    def tu_flow_rhs(self, VP, VC, VD, Xpp, Xph, stream=None):
        """paid_tu_flow_rhs on cuda float64 [nq, nff, nff] tensors; returns
        (dP, dC, dD)."""
        torch = _torch()
        for a in (VP, VC, VD, Xpp, Xph):
            if a.dtype != torch.float64 or not a.is_contiguous() or a.shape != VP.shape:
                raise ValueError("contiguous float64 [nq, nff, nff] tensors expected")
        nq, nff = VP.shape[0], VP.shape[1]
        dP, dC, dD = (torch.empty_like(VP) for _ in range(3))
        if stream is None:
            stream = torch.cuda.current_stream(self.torch_device)
        rc = self._lib.paid_tu_flow_rhs(self._h, nq, nff, VP.data_ptr(), VC.data_ptr(),
                                        VD.data_ptr(), Xpp.data_ptr(), Xph.data_ptr(),
                                        dP.data_ptr(), dC.data_ptr(), dD.data_ptr(),
                                        ctypes.c_void_p(stream.cuda_stream))
        if rc != OK:
            raise PaidError(rc, self.last_error())
        return dP, dC, dD

    def cell_errors(self, kind, q, lm, T, stream=None):
        """Relative log10 error maps of the uniform level-4 grid: cuda float32 [n, 256]."""
        torch = _torch()
        n = q.shape[0] * lm.shape[0]
        out = torch.empty((n, 256), dtype=torch.float32, device=self.torch_device)
        if stream is None:
            stream = torch.cuda.current_stream(self.torch_device)
        ws = self.workspace(n, n * 256)
        rc = self._lib.paid_cell_errors(self._h, int(kind), q.shape[0], q.data_ptr(), lm.shape[0],
                                        lm.data_ptr(), float(T), out.data_ptr(),
                                        ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                        ctypes.c_void_p(stream.cuda_stream))
        if rc != OK:
            raise PaidError(rc, self.last_error())
        return out

    def features(self, kind, q, lm, T, stream=None):
        """Proposal inputs of one batch: cuda bfloat16 [n, 32]."""
        torch = _torch()
        n = q.shape[0] * lm.shape[0]
        x = torch.empty((n, 32), dtype=torch.bfloat16, device=self.torch_device)
        if stream is None:
            stream = torch.cuda.current_stream(self.torch_device)
        rc = self._lib.paid_mlp_features(self._h, int(kind), q.shape[0], q.data_ptr(), lm.shape[0],
                                         lm.data_ptr(), float(T), x.data_ptr(),
                                         ctypes.c_void_p(stream.cuda_stream))
        if rc != OK:
            raise PaidError(rc, "paid_mlp_features")
        return x

    def get_options(self) -> paid_options:
        """The context's current options (paid_get_options)."""
        o = paid_options()
        self._lib.paid_get_options(self._h, ctypes.byref(o))
        self.options = o
        return o

    def autotune(self, batches, cache_path=None, stream=None):
        """paid_autotune on device-resident sample batches (dicts as for
        integrate_multi; their outputs are scratch).  With cache_path, an entry
        for this GPU and mode is applied without timing.  Returns the tuned
        options."""
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream(self.torch_device)
        path = cache_path.encode() if cache_path else None
        arr, outs, n_int, maxr = self._batch_array(batches or [])
        n = self.units(batches or [])
        cap = self.default_capacity(n, maxr) if n else 0
        while True:
            nbytes = 0
            ws = None
            if n:
                ws = self.workspace(n, cap)
                nbytes = self.workspace_size(n, cap)
            rc = self._lib.paid_autotune(self._h, arr if batches else None, len(batches or []),
                                         path,
                                         ctypes.c_void_p(ws.data_ptr()) if ws is not None else None,
                                         nbytes, ctypes.c_void_p(stream.cuda_stream))
            if rc == ERR_CUDA and n:
                # no candidate completed: a pool too small for the sample
                # stops every one of them; grow it while memory allows
                del ws
                self.release_workspace()
                free, _ = torch.cuda.mem_get_info(self.device)
                bigger = min(4 * cap, self.pool_capacity(n, int(0.9 * free)), 2 ** 32 - 1)
                if bigger > cap:
                    cap = bigger
                    self._grown_capacity = max(getattr(self, "_grown_capacity", 0), cap)
                    continue
            if rc != OK:
                raise PaidError(rc, self.last_error())
            return self.get_options()

    def _batch_array(self, batches):
        """ctypes paid_batch array and fresh output tensors for dict batches."""
        torch = _torch()
        dev = self.torch_device
        arr = (paid_batch * max(1, len(batches)))()
        outs = []
        n = 0
        maxr = 1
        for i, b in enumerate(batches):
            q, lm = b["q"], b["lm"]
            for t_, dt in ((q, torch.float64), (lm, torch.int32)):
                if t_.device != dev or t_.dtype != dt or not t_.is_contiguous():
                    raise ValueError("q must be contiguous float64 and lm int32 on %s" % dev)
            nq, npairs = q.shape[0], lm.shape[0]
            r = Result(torch.empty(nq * npairs, dtype=torch.float64, device=dev),
                       torch.empty(nq * npairs, dtype=torch.float64, device=dev),
                       torch.empty(nq * npairs, dtype=torch.int64, device=dev),
                       torch.empty(nq * npairs, dtype=torch.int32, device=dev))
            outs.append(r)
            a = arr[i]
            a.kind, a.T, a.nq, a.q, a.npairs, a.lm = (int(b["kind"]), float(b["T"]), nq,
                                                     q.data_ptr(), npairs, lm.data_ptr())
            a.rel_tol = float(b.get("rel_tol", 1e-6))
            a.abs_tol = float(b.get("abs_tol", 1e-10))
            a.max_regions = int(b.get("max_regions", 100000))
            a.values, a.errors = r.values.data_ptr(), r.errors.data_ptr()
            a.regions, a.status = r.regions.data_ptr(), r.status.data_ptr()
            # flow kinds, group mode: truncated-unity products formed in the
            # call (tu_v: couplings, tu_out: outputs; cuda float64 [nq, nff, nff])
            for f in ("tu_v", "tu_out"):
                ts = b.get(f) or ()
                for j, t_ in enumerate(ts):
                    if t_ is None:
                        continue
                    if (t_.device != dev or t_.dtype != torch.float64 or not t_.is_contiguous()
                            or t_.numel() != nq * npairs):
                        raise ValueError("%s tensors must be contiguous float64 [nq, nff, nff] "
                                         "on %s" % (f, dev))
                    getattr(a, f)[j] = t_.data_ptr()
            n += nq * npairs
            maxr = max(maxr, a.max_regions)
        return arr, outs, n, maxr

    def _integrate(self, batches, pool_capacity, stream, seeded, asynchronous=False):
        torch = _torch()
        arr, outs, n_int, maxr = self._batch_array(batches)
        # workspace and pool are sized per unit: a (kind, q) group in group
        # mode, else an integral
        n = self.units(batches)
        if stream is None:
            stream = torch.cuda.current_stream(self.torch_device)
        cap = pool_capacity or self.default_capacity(n, maxr)
        while True:
            ws = self.workspace(n, cap)
            # the library sizes its pool from the bytes it is given: pass the
            # size for `cap`, not the (possibly larger) cached workspace
            nbytes = self.workspace_size(n, cap)
            if seeded is None:
                rc = self._lib.paid_integrate_multi(self._h, arr, len(batches),
                                                    ctypes.c_void_p(ws.data_ptr()), nbytes,
                                                    ctypes.c_void_p(stream.cuda_stream))
            else:
                prop, margin = seeded
                if prop is not None and (prop.dtype != torch.float32
                                         or tuple(prop.shape) != (n, 256)
                                         or not prop.is_contiguous()
                                         or prop.device != self.torch_device):
                    raise ValueError("proposal must be contiguous float32 [%d, 256]" % n)
                rc = self._lib.paid_integrate_multi_seeded(
                    self._h, arr, len(batches), prop.data_ptr() if prop is not None else None,
                    margin, ctypes.c_void_p(ws.data_ptr()), nbytes,
                    ctypes.c_void_p(stream.cuda_stream))
            if rc == OK and not asynchronous:
                # the device-loop calls return at once: their outcome (pool,
                # round cap) comes from paid_wait
                out = ctypes.c_int(OK)
                rc = self._lib.paid_wait(self._h, ctypes.byref(out))
                rc = out.value if rc == OK else rc
            # a pool that could not progress, or (seeded start) one too small
            # for the seed: grow it and run again
            grow = rc == ERR_POOL or (rc == ERR_OOM and seeded is not None)
            if grow and pool_capacity is None and cap < 2 ** 32 - 1:
                # drop every reference to the old workspace before sizing the next
                del ws
                self.release_workspace()
                free, _ = torch.cuda.mem_get_info(self.device)
                bigger = min(4 * cap, self.pool_capacity(n, int(0.9 * free)), 2 ** 32 - 1)
                if bigger > cap:
                    cap = bigger
                    self._grown_capacity = cap
                    continue
                ws = None
            if rc not in (OK, ERR_TIMEOUT, ERR_POOL):
                raise PaidError(rc, self.last_error())
            self.last_rc = rc
            return outs

    def units(self, batches) -> int:
        """Units of a call: (kind, q) groups in group mode, else integrals."""
        if self.options.group_mode:
            return sum(int(b["q"].shape[0]) for b in batches)
        return sum(int(b["q"].shape[0]) * int(b["lm"].shape[0]) for b in batches)

    def integrate_batch(self, kind, q, lm, T, rel_tol=1e-6, abs_tol=1e-10, max_regions=100000,
                        pool_capacity=None, stream=None) -> Result:
        """One batch (device tensors in, device tensors out), idx = iq * npairs + ip."""
        return self.integrate_multi([dict(kind=kind, T=T, q=q, lm=lm, rel_tol=rel_tol,
                                          abs_tol=abs_tol, max_regions=max_regions)],
                                    pool_capacity=pool_capacity, stream=stream)[0]

    def integrate_host(self, batches, pool_capacity=None, proposal=None, margin=1.0):
        """End-to-end call on host (numpy) inputs: copies q and lm from pinned
        host memory to the device, integrates (seeded from `proposal`, a
        Proposal network, with `margin` -- a number, or a function of the
        batch temperature giving a margin or None for the uniform start -- when
        given), and copies the results back.
        Returns (list of numpy Result, bytes host->device, bytes device->host)."""
        torch = _torch()
        dev = self.torch_device
        stream = torch.cuda.current_stream(dev)
        dbs, h2d = [], 0
        for b in batches:
            qh = torch.from_numpy(np.ascontiguousarray(b["q"], dtype=np.float64)).pin_memory()
            lh = torch.from_numpy(np.ascontiguousarray(b["lm"], dtype=np.int32)).pin_memory()
            d = dict(b)
            d["q"] = qh.to(dev, non_blocking=True)
            d["lm"] = lh.to(dev, non_blocking=True)
            h2d += qh.numel() * 8 + lh.numel() * 4
            dbs.append(d)
        if proposal is None:
            outs = self.integrate_multi(dbs, pool_capacity=pool_capacity, stream=stream)
        elif callable(margin):
            # a margin per batch temperature (None: the uniform start)
            from . import proposal as PR
            outs = PR.integrate(proposal, self, dbs, margin, stream=stream,
                                pool_capacity=pool_capacity)
        else:
            maps = proposal.predict(self, dbs, stream)
            outs = self.integrate_multi_seeded(dbs, maps, margin, pool_capacity=pool_capacity,
                                               stream=stream)
        # results into pinned host buffers (torch caches them), one wait
        hosts, d2h = [], 0
        for r in outs:
            hb = []
            for t in (r.values, r.errors, r.regions, r.status):
                h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
                h.copy_(t, non_blocking=True)
                hb.append(h)
                d2h += h.numel() * h.element_size()
            hosts.append(hb)
        stream.synchronize()
        return [Result(*(h.numpy() for h in hb)) for hb in hosts], h2d, d2h

    def integrate_batch_static(self, kind, q, lm, T, rel_tol=1e-6, abs_tol=1e-10,
                               max_regions=100000, stream=None) -> Result:
        """paid_integrate_batch_static: like integrate_batch, but the library
        keeps the region pool in a fixed 64 MiB device array of its own, so the
        call needs no workspace (for callers that cannot allocate device
        memory when they integrate; at most 4096 integrals per call, and calls
        must not overlap on the GPU because they share that array).  The output
        tensors here are made by torch before the call; a caller that cannot
        allocate passes buffers it already holds to the C function."""
        torch = _torch()
        lib = self._lib
        dev = self.torch_device
        for t_, dt, what in ((q, torch.float64, "q"), (lm, torch.int32, "lm")):
            if (t_.device != dev or t_.dtype != dt or not t_.is_contiguous() or t_.dim() != 2
                    or t_.shape[1] != 2):
                raise ValueError("%s must be a contiguous %s [n, 2] tensor on %s"
                                 % (what, dt, dev))
        nq, npairs = q.shape[0], lm.shape[0]
        r = Result(torch.empty(nq * npairs, dtype=torch.float64, device=dev),
                   torch.empty(nq * npairs, dtype=torch.float64, device=dev),
                   torch.empty(nq * npairs, dtype=torch.int64, device=dev),
                   torch.empty(nq * npairs, dtype=torch.int32, device=dev))
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        rc = lib.paid_integrate_batch_static(self._h, int(kind), nq, q.data_ptr(), npairs,
                                             lm.data_ptr(), float(T), float(rel_tol),
                                             float(abs_tol), int(max_regions),
                                             r.values.data_ptr(), r.errors.data_ptr(),
                                             r.regions.data_ptr(), r.status.data_ptr(),
                                             ctypes.c_void_p(stream.cuda_stream))
        self.last_rc = rc
        if rc not in (OK, ERR_TIMEOUT, ERR_POOL):
            raise PaidError(rc, error_string(rc))
        return r


class Proposal:
    """The refinement-proposal network on the device: FP32 master parameters,
    AdamW moments, and the library's BF16 tensor-core kernels for the forward
    pass, the MSE gradient and the update."""

    def __init__(self, device=0, seed=0, params=None):
        torch = _torch()
        self._lib = load()
        self.device = torch.device("cuda", device)
        n = ctypes.c_int64()
        self._lib.paid_mlp_param_count(ctypes.byref(n))
        self.n = n.value
        self.params = torch.empty(self.n, dtype=torch.float32, device=self.device)
        if params is None:
            rc = self._lib.paid_mlp_init(self.params.data_ptr(), int(seed), None)
            if rc != OK:
                raise PaidError(rc, "paid_mlp_init")
        else:
            self.params.copy_(torch.as_tensor(params, dtype=torch.float32))
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad_buf = torch.zeros_like(self.params)
        self.loss_buf = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.step_count = 0
        self._ws = None
        # kernels this object has launched for inference (features + forward)
        self.launches = 0

    def _workspace(self, M):
        torch = _torch()
        b = ctypes.c_size_t()
        self._lib.paid_mlp_workspace_size(int(M), ctypes.byref(b))
        if self._ws is None or self._ws.numel() < b.value:
            self._ws = None
            self._ws = torch.empty(b.value, dtype=torch.uint8, device=self.device)
        return self._ws

    def forward(self, x, stream=None):
        torch = _torch()
        M = x.shape[0]
        out = torch.empty((M, 256), dtype=torch.float32, device=self.device)
        if M == 0:
            return out
        ws = self._workspace(M)
        s = stream or torch.cuda.current_stream(self.device)
        rc = self._lib.paid_mlp_forward(self.params.data_ptr(), x.data_ptr(), M, out.data_ptr(),
                                        ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                        ctypes.c_void_p(s.cuda_stream))
        if rc != OK:
            raise PaidError(rc, "paid_mlp_forward")
        self.launches += MLP_FORWARD_LAUNCHES
        return out

    def grad(self, x, target, stream=None):
        """(grad FP32 [n_params], loss FP32 [1]) of the MSE over the rows of x."""
        torch = _torch()
        ws = self._workspace(x.shape[0])
        s = stream or torch.cuda.current_stream(self.device)
        rc = self._lib.paid_mlp_grad(self.params.data_ptr(), x.data_ptr(), target.data_ptr(),
                                     x.shape[0], self.grad_buf.data_ptr(),
                                     self.loss_buf.data_ptr(), ctypes.c_void_p(ws.data_ptr()),
                                     ws.numel(), ctypes.c_void_p(s.cuda_stream))
        if rc != OK:
            raise PaidError(rc, "paid_mlp_grad")
        return self.grad_buf, self.loss_buf

    def step(self, x, target, lr=1e-3, weight_decay=1e-4, stream=None):
        torch = _torch()
        self.grad(x, target, stream)
        self.step_count += 1
        s = stream or torch.cuda.current_stream(self.device)
        rc = self._lib.paid_mlp_adamw(self.params.data_ptr(), self.grad_buf.data_ptr(),
                                      self.m.data_ptr(), self.v.data_ptr(), self.step_count,
                                      float(lr), float(weight_decay), ctypes.c_void_p(s.cuda_stream))
        if rc != OK:
            raise PaidError(rc, "paid_mlp_adamw")
        return self.loss_buf

    def train(self, x, target, epochs=10, batch=4096, lr=2e-3, weight_decay=1e-4, seed=0,
              stream=None):
        """paid_proposal_train: minibatch AdamW on the device over the rows of
        x (BF16 [M, 32]) and target (FP32 [M, 256]) with a cosine-decayed
        learning rate; returns the mean loss per epoch."""
        torch = _torch()
        M = x.shape[0]
        b = ctypes.c_size_t()
        rc = self._lib.paid_proposal_train_workspace_size(M, int(batch), ctypes.byref(b))
        if rc != OK:
            raise PaidError(rc, "paid_proposal_train_workspace_size")
        ws = torch.empty(b.value, dtype=torch.uint8, device=self.device)
        step = ctypes.c_int(self.step_count)
        hist = (ctypes.c_float * max(1, epochs))()
        s = stream or torch.cuda.current_stream(self.device)
        rc = self._lib.paid_proposal_train(self.params.data_ptr(), self.m.data_ptr(),
                                           self.v.data_ptr(), x.contiguous().data_ptr(),
                                           target.contiguous().data_ptr(), M, int(epochs),
                                           int(batch), float(lr), float(weight_decay), int(seed),
                                           ctypes.byref(step), hist, ctypes.c_void_p(ws.data_ptr()),
                                           ws.numel(), ctypes.c_void_p(s.cuda_stream))
        if rc != OK:
            raise PaidError(rc, "paid_proposal_train")
        self.step_count = step.value
        return [float(hist[i]) for i in range(epochs)]

    def save(self, path, stream=None):
        """paid_proposal_save: the FP32 parameters to a file."""
        torch = _torch()
        s = stream or torch.cuda.current_stream(self.device)
        rc = self._lib.paid_proposal_save(self.params.data_ptr(), str(path).encode(),
                                          ctypes.c_void_p(s.cuda_stream))
        if rc != OK:
            raise PaidError(rc, "paid_proposal_save")

    @classmethod
    def load(cls, path, device=0, stream=None):
        """paid_proposal_load: a network from a file written by save()."""
        torch = _torch()
        p = cls(device=device)
        s = stream or torch.cuda.current_stream(p.device)
        rc = p._lib.paid_proposal_load(p.params.data_ptr(), str(path).encode(),
                                       ctypes.c_void_p(s.cuda_stream))
        if rc != OK:
            raise PaidError(rc, "paid_proposal_load")
        return p

    def predict(self, ctx, batches, stream=None):
        """Level maps for ctx's units of these batches (group mode: one row per
        (kind, q) group; else one per integral), FP32 [units, 256]."""
        torch = _torch()
        self.launches += sum(1 for b in batches if int(b["q"].shape[0]) > 0)
        if ctx.options.group_mode:
            x = torch.cat([ctx.group_features(b["kind"], b["q"], b["T"], stream) for b in batches])
        else:
            x = torch.cat([ctx.features(b["kind"], b["q"], b["lm"], b["T"], stream)
                           for b in batches])
        return self.forward(x, stream)

    def state(self):
        return self.params.detach().cpu().numpy().copy()
