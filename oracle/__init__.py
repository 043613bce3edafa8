"""Python loader for the FP64 CPU oracle (``oracle/oracle.c``).

Test infrastructure only: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  The product library never imports
it, and it imports nothing from the product.

Every function follows the paper section named in ``oracle.c``:
the dispersion and form factors (Sec. 2), the Matsubara-summed bubble kernels
of Eq. chi_ph / chi_pp in temperature form, the nested Clenshaw-Curtis pair
(Sec. 3), the greedy adaptive loop of Algorithm 1 with the 4-way split of
Algorithm 2, and Algorithm 2's group form (one heap and one global error sum
over all (l, m) pairs of a (kind, q), Sec. 4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PH, PP, MONOMIAL, OVERLAP, FLOW_PH, FLOW_PP = 0, 1, 2, 3, 4, 5
CONVERGED, BUDGET, NONFINITE = 0, 1, 2
MAX_LEVEL = 29

_d = ctypes.c_double
_i = ctypes.c_int
_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.oracle_cc_rule.argtypes = [_i, _p, _p]
            lib.oracle_dispersion.argtypes = [_d] * 5
            lib.oracle_dispersion.restype = _d
            lib.oracle_form_factor.argtypes = [_i, _d, _d]
            lib.oracle_form_factor.restype = _d
            lib.oracle_kernel_ph.argtypes = [_d, _d, _d]
            lib.oracle_kernel_ph.restype = _d
            lib.oracle_kernel_pp.argtypes = [_d, _d, _d]
            lib.oracle_kernel_pp.restype = _d
            lib.oracle_kernel_flow_ph.argtypes = [_d, _d, _d]
            lib.oracle_kernel_flow_ph.restype = _d
            lib.oracle_kernel_flow_pp.argtypes = [_d, _d, _d]
            lib.oracle_kernel_flow_pp.restype = _d
            lib.oracle_integrand_point.argtypes = [_i, _d, _d, _i, _i, _d, _d, _d, _d, _d, _d]
            lib.oracle_integrand_point.restype = _d
            lib.oracle_region_eval.argtypes = [_i, _d, _d, _i, _i, _d, _d, _d, _d, _i,
                                               _i, _i64, _i64, _p, _p]
            lib.oracle_integrate_batch.argtypes = [_i, _i, _p, _i, _p, _d, _d, _d, _d,
                                                   _d, _d, _i64, _i, _i, _i, _p, _p, _p, _p]
            lib.oracle_integrate_group_global.argtypes = [_i, _i, _p, _i, _p, _d, _d, _d, _d,
                                                          _d, _d, _i64, _i, _i, _i,
                                                          _p, _p, _p, _p]
            lib.oracle_integrate_list.argtypes = [_i64, _p, _p, _p, _p, _d, _d, _d,
                                                  _d, _d, _i64, _i, _i, _i, _p, _p, _p, _p]
            lib.oracle_integrate_trace.argtypes = [_i, _d, _d, _i, _i, _d, _d, _d, _d,
                                                   _d, _d, _i64, _i, _i, _p, _p, _p,
                                                   _i64, _p, _p, _p, _p, _p, _p]
            lib.oracle_max_threads.restype = _i
            lib.oracle_trapezoid.argtypes = [_i, _d, _d, _i, _i, _d, _d, _d, _d, _i, _i]
            lib.oracle_trapezoid.restype = _d
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def trapezoid(kind, q, l, m, T, lat, M, nthreads=0):
    """The integral on an M x M periodic trapezoid grid (the definition, no adaptivity)."""
    t, tp, mu = lat
    return float(_load().oracle_trapezoid(kind, q[0], q[1], l, m, T, t, tp, mu, M, nthreads))


def brute_force(kind, q, l, m, T, lat, M0=1024, Mmax=8192, tol=1e-13):
    """Converged dense trapezoid: M doubled from M0 until two successive values
    agree within tol (absolute).  Returns (value, M) or (nan, Mmax).

    The flow kinds go to brute_force_h4: their kernel is not analytic on the
    Fermi surface and the trapezoid converges like h^4 there, never to 1e-13."""
    if kind in (FLOW_PH, FLOW_PP):
        return brute_force_h4(kind, q, l, m, T, lat)
    prev = trapezoid(kind, q, l, m, T, lat, M0)
    M = M0
    while M < Mmax:
        M *= 2
        cur = trapezoid(kind, q, l, m, T, lat, M)
        if abs(cur - prev) <= tol:
            return cur, M
        prev = cur
    return float("nan"), M


def brute_force_h4(kind, q, l, m, T, lat, M0=1024, Mmax=16384, tol=1e-11):
    """Dense trapezoid for an integrand whose fourth derivative jumps on a curve
    (the Omega-regulated flow kernels: |e| enters H(e), Sec. 2): the error
    falls like h^4, so every doubling of M is followed by one Richardson step
    R(M) = T(M) + (T(M) - T(M/2)) / 15, and two successive R must agree within
    tol.  Returns (value, M) or (nan, Mmax)."""
    prev = trapezoid(kind, q, l, m, T, lat, M0)
    prevR = None
    M = M0
    while M < Mmax:
        M *= 2
        cur = trapezoid(kind, q, l, m, T, lat, M)
        R = cur + (cur - prev) / 15.0
        if prevR is not None and abs(R - prevR) <= tol:
            return R, M
        prev, prevR = cur, R
    return float("nan"), M


def cc_rule(N: int):
    """Nodes and weights of the N-interval Clenshaw-Curtis rule on [-1, 1]."""
    x = np.zeros(N + 1)
    w = np.zeros(N + 1)
    if _load().oracle_cc_rule(N, _ptr(x), _ptr(w)) != 0:
        raise ValueError("invalid rule size %d" % N)
    return x, w


def dispersion(kx, ky, t, tp, mu):
    return _load().oracle_dispersion(kx, ky, t, tp, mu)


def form_factor(n, kx, ky):
    return _load().oracle_form_factor(n, kx, ky)


def kernel_ph(e1, e2, T):
    return _load().oracle_kernel_ph(e1, e2, T)


def kernel_pp(e1, e2, T):
    return _load().oracle_kernel_pp(e1, e2, T)


def kernel_flow_ph(e1, e2, omega):
    """d/dOmega of the ph frequency integral with the Omega regulator (Sec. 2)."""
    return _load().oracle_kernel_flow_ph(e1, e2, omega)


def kernel_flow_pp(e1, e2, omega):
    """d/dOmega of the pp frequency integral with the Omega regulator (Sec. 2)."""
    return _load().oracle_kernel_flow_pp(e1, e2, omega)


def integrand_point(kind, q, l, m, T, lat, kx, ky):
    t, tp, mu = lat
    return _load().oracle_integrand_point(kind, q[0], q[1], l, m, T, t, tp, mu, kx, ky)


def region_eval(kind, q, l, m, T, lat, L, ix, iy, rule_n=4):
    """(Q_N, Q_2N) of the level-L region with corner index (ix, iy)."""
    t, tp, mu = lat
    qN = np.zeros(1)
    q2N = np.zeros(1)
    rc = _load().oracle_region_eval(kind, q[0], q[1], l, m, T, t, tp, mu, rule_n,
                                    L, ix, iy, _ptr(qN), _ptr(q2N))
    if rc != 0:
        raise ValueError("invalid rule size")
    return float(qN[0]), float(q2N[0])


def integrate_batch(kind, q, lm, T, lat, rel_tol, abs_tol, max_regions,
                    rule_n=4, init_level=2, nthreads=0):
    """Adaptive integrals for every (q, pair); output index iq * npairs + ip.

    Returns (values, errors, regions, status) as numpy arrays."""
    t, tp, mu = lat
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 2)
    lm = np.ascontiguousarray(lm, dtype=np.int32).reshape(-1, 2)
    n = q.shape[0] * lm.shape[0]
    v = np.zeros(n)
    e = np.zeros(n)
    r = np.zeros(n, dtype=np.int64)
    s = np.zeros(n, dtype=np.int32)
    rc = _load().oracle_integrate_batch(kind, q.shape[0], _ptr(q), lm.shape[0], _ptr(lm),
                                        T, t, tp, mu, rel_tol, abs_tol, int(max_regions),
                                        rule_n, init_level, nthreads,
                                        _ptr(v), _ptr(e), _ptr(r), _ptr(s))
    if rc != 0:
        raise ValueError("oracle_integrate_batch: invalid argument")
    return v, e, r, s


def integrate_group_global(kind, q, lm, T, lat, rel_tol, abs_tol, max_regions,
                           rule_n=4, init_level=2, nthreads=0):
    """Algorithm 2 with the global error of Sec. 4: one group per q row (all
    of lm's pairs), one heap and one error sum per group; a group is done when
    sum_c E_c <= max(abs_tol, rel_tol * sum_c |V_c|).  Output index
    iq * npairs + ip: every pair's own value, error and leaf count, the
    group's status.  Returns (values, errors, regions, status)."""
    t, tp, mu = lat
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 2)
    lm = np.ascontiguousarray(lm, dtype=np.int32).reshape(-1, 2)
    n = q.shape[0] * lm.shape[0]
    v = np.zeros(n)
    e = np.zeros(n)
    r = np.zeros(n, dtype=np.int64)
    s = np.zeros(n, dtype=np.int32)
    rc = _load().oracle_integrate_group_global(kind, q.shape[0], _ptr(q), lm.shape[0], _ptr(lm),
                                               T, t, tp, mu, rel_tol, abs_tol, int(max_regions),
                                               rule_n, init_level, nthreads,
                                               _ptr(v), _ptr(e), _ptr(r), _ptr(s))
    if rc != 0:
        raise ValueError("oracle_integrate_group_global: invalid argument")
    return v, e, r, s


def integrate_list(kind, q, lm, T, lat, rel_tol, abs_tol, max_regions,
                   rule_n=4, init_level=2, nthreads=0):
    """Adaptive integrals over a flat list: kind[i], q[i], lm[i], T[i]."""
    t, tp, mu = lat
    kind = np.ascontiguousarray(kind, dtype=np.int32).reshape(-1)
    n = kind.shape[0]
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(n, 2)
    lm = np.ascontiguousarray(lm, dtype=np.int32).reshape(n, 2)
    T = np.ascontiguousarray(np.broadcast_to(np.asarray(T, dtype=np.float64), (n,)))
    v = np.zeros(n)
    e = np.zeros(n)
    r = np.zeros(n, dtype=np.int64)
    s = np.zeros(n, dtype=np.int32)
    rc = _load().oracle_integrate_list(n, _ptr(kind), _ptr(q), _ptr(lm), _ptr(T), t, tp, mu,
                                       rel_tol, abs_tol, int(max_regions), rule_n,
                                       init_level, nthreads, _ptr(v), _ptr(e), _ptr(r), _ptr(s))
    if rc != 0:
        raise ValueError("oracle_integrate_list: invalid argument")
    return v, e, r, s


def integrate_trace(kind, q, l, m, T, lat, rel_tol, abs_tol, max_regions,
                    rule_n=4, init_level=2, trace_cap=1 << 16):
    """One integral plus its final leaves.

    Returns dict(value, error, regions, status, level, ix, iy, valN, val2N, err)."""
    t, tp, mu = lat
    v = np.zeros(1)
    e = np.zeros(1)
    nl = np.zeros(1, dtype=np.int64)
    lev = np.zeros(trace_cap, dtype=np.int32)
    ix = np.zeros(trace_cap, dtype=np.int64)
    iy = np.zeros(trace_cap, dtype=np.int64)
    vN = np.zeros(trace_cap)
    v2N = np.zeros(trace_cap)
    er = np.zeros(trace_cap)
    st = _load().oracle_integrate_trace(kind, q[0], q[1], l, m, T, t, tp, mu, rel_tol, abs_tol,
                                        int(max_regions), rule_n, init_level, _ptr(v), _ptr(e),
                                        _ptr(nl), trace_cap, _ptr(lev), _ptr(ix), _ptr(iy),
                                        _ptr(vN), _ptr(v2N), _ptr(er))
    if st < 0:
        raise ValueError("oracle_integrate_trace: invalid argument")
    k = min(int(nl[0]), trace_cap)
    return dict(value=float(v[0]), error=float(e[0]), regions=int(nl[0]), status=int(st),
                level=lev[:k].copy(), ix=ix[:k].copy(), iy=iy[:k].copy(),
                valN=vN[:k].copy(), val2N=v2N[:k].copy(), err=er[:k].copy())


def tu_flow_rhs(VP, VC, VD, Xpp, Xph):
    """Right-hand sides of the truncated-unity flow equations for every transfer
    momentum (Eqs. matmul-P, matmul-C, matmul-D of Sec. 2):

        dP = V^P X^pp V^P,  dC = -V^C X^ph V^C,
        dD = 2 V^D X^ph V^D - V^C X^ph V^D - V^D X^ph V^C,

    with X the scale derivatives of the form-factor bubbles.  All arrays are
    [nq, nff, nff] float64; the products are plain matrix products per q."""
    VP, VC, VD, Xpp, Xph = (np.asarray(a, dtype=np.float64) for a in (VP, VC, VD, Xpp, Xph))
    dP = VP @ Xpp @ VP
    dC = -(VC @ Xph @ VC)
    dD = 2.0 * (VD @ Xph @ VD) - VC @ Xph @ VD - VD @ Xph @ VC
    return dP, dC, dD
