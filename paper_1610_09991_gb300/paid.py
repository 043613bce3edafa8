"""Thin ctypes binding of libpaid (include/paid.h) with the same names.

Only argument marshalling happens here: device buffers come from torch
tensors (``data_ptr()``), the stream from ``torch.cuda.current_stream()``,
and every step of the cubature runs in the library's CUDA kernels.  There is
no CPU fallback: without libpaid.so (see ``build.py``) or without a CUDA
device every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpaid.so")

PH, PP, MONOMIAL, OVERLAP = 0, 1, 2, 3
FF_SHELL1, FF_SHELL12 = 5, 9
OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_POOL, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
CONVERGED, BUDGET, NONFINITE, ROUNDCAP, POOL = 0, 1, 2, 3, 4

#: every entry point declared in include/paid.h
EXPORTS = ("paid_options_default", "paid_create", "paid_destroy", "paid_workspace_size",
           "paid_pool_capacity", "paid_integrate_batch", "paid_integrate_multi",
           "paid_last_stats", "paid_error_string", "paid_last_error")


class paid_options(ctypes.Structure):
    _fields_ = [("rule_n", ctypes.c_int), ("init_level", ctypes.c_int),
                ("eval_fp32", ctypes.c_int), ("max_rounds", ctypes.c_int),
                ("cover", ctypes.c_double), ("pool_capacity", ctypes.c_int64),
                ("timing", ctypes.c_int)]


class paid_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int), ("region_evals", ctypes.c_int64),
                ("node_evals", ctypes.c_int64), ("peak_pool", ctypes.c_int64),
                ("pool_capacity", ctypes.c_int64), ("n_integrals", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("eval_launches", ctypes.c_int64),
                ("eval_ms", ctypes.c_double), ("reduce_ms", ctypes.c_double),
                ("scan_ms", ctypes.c_double), ("split_ms", ctypes.c_double),
                ("escalated", ctypes.c_int64)]


class paid_batch(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("T", ctypes.c_double), ("nq", ctypes.c_int),
                ("q", ctypes.c_void_p), ("npairs", ctypes.c_int), ("lm", ctypes.c_void_p),
                ("rel_tol", ctypes.c_double), ("abs_tol", ctypes.c_double),
                ("max_regions", ctypes.c_int64), ("values", ctypes.c_void_p),
                ("errors", ctypes.c_void_p), ("regions", ctypes.c_void_p),
                ("status", ctypes.c_void_p)]


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
            self._ws = None
            self._ws = torch.empty(need, dtype=torch.uint8, device=self.torch_device)
        return self._ws

    def default_capacity(self, n_integrals: int, max_regions: int) -> int:
        """Pool capacity used when none is given: every integral at its budget,
        bounded by 70 % of the device's free memory."""
        torch = _torch()
        free, _ = torch.cuda.mem_get_info(self.device)
        n0 = 4 ** self.options.init_level
        want = max(n_integrals * n0, n_integrals * max_regions)
        held = self._ws.numel() if self._ws is not None else 0
        limit = self.pool_capacity(n_integrals, int(0.7 * (free + held)))
        return int(max(n_integrals * n0, min(want, limit, 2 ** 32 - 1)))

    def integrate_multi(self, batches, pool_capacity=None, stream=None):
        """Device-resident batches: a list of dicts with keys kind, T, q (cuda
        float64 [nq, 2]), lm (cuda int32 [npairs, 2]), rel_tol, abs_tol,
        max_regions.  Returns one Result of cuda tensors per batch."""
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
            n += nq * npairs
            maxr = max(maxr, a.max_regions)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        cap = pool_capacity or self.default_capacity(n, maxr)
        while True:
            ws = self.workspace(n, cap)
            rc = self._lib.paid_integrate_multi(self._h, arr, len(batches),
                                                ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                                ctypes.c_void_p(stream.cuda_stream))
            if rc == ERR_POOL and pool_capacity is None and cap < 2 ** 32 - 1:
                free, _ = torch.cuda.mem_get_info(self.device)
                bigger = min(4 * cap, self.pool_capacity(n, int(0.9 * (free + ws.numel()))),
                             2 ** 32 - 1)
                if bigger > cap:
                    cap = bigger
                    continue
            if rc not in (OK, ERR_TIMEOUT, ERR_POOL):
                raise PaidError(rc, self.last_error())
            self.last_rc = rc
            return outs

    def integrate_batch(self, kind, q, lm, T, rel_tol=1e-6, abs_tol=1e-10, max_regions=100000,
                        pool_capacity=None, stream=None) -> Result:
        """One batch (device tensors in, device tensors out), idx = iq * npairs + ip."""
        return self.integrate_multi([dict(kind=kind, T=T, q=q, lm=lm, rel_tol=rel_tol,
                                          abs_tol=abs_tol, max_regions=max_regions)],
                                    pool_capacity=pool_capacity, stream=stream)[0]

    def integrate_host(self, batches, pool_capacity=None):
        """End-to-end call on host (numpy) inputs: copies q and lm from pinned
        host memory to the device, integrates, and copies the results back.
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
        outs = self.integrate_multi(dbs, pool_capacity=pool_capacity, stream=stream)
        res, d2h = [], 0
        for r in outs:
            hv = [t.to("cpu", non_blocking=False).numpy() for t in
                  (r.values, r.errors, r.regions, r.status)]
            d2h += sum(x.nbytes for x in hv)
            res.append(Result(*hv))
        return res, h2d, d2h

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
        P_, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.paid_integrate_batch_static.argtypes = [P_, I, I, P_, I, P_, D, D, D, I64, P_, P_,
                                                    P_, P_, P_]
        dev = self.torch_device
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
