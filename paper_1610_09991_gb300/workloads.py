"""Seeded synthetic workloads: q grids, form-factor pairs, temperatures and
lattice parameters of the bubble-integral batches.

This module holds none of the method's arithmetic (no dispersion, no kernel,
no rule); it only builds the inputs that both the CUDA library and the CPU
oracle receive.  The paper prints no workload of its own for these integrands
(its figures are stripped and its TUfRG parameters are not stated), so the
batches below are the synthetic stand-ins: lattice t = 1, t' = -0.25,
mu = -1.0 (the t-t' Hubbard dispersion of Sec. 2), form-factor sets of one and
two bond shells, and q grids over the Brillouin zone.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PH, PP, MONOMIAL, OVERLAP, FLOW_PH, FLOW_PP = 0, 1, 2, 3, 4, 5
LATTICE = (1.0, -0.25, -1.0)  # (t, t', mu)


def q_grid_quadrant(n: int) -> np.ndarray:
    """n x n grid of [0, pi]^2 with both endpoints: q_i = i pi / (n-1).
    Order: qx-major, [iq] = (qx_i, qy_j) with iq = i*n + j."""
    g = np.array([i * math.pi / (n - 1) for i in range(n)])
    return np.array([(a, b) for a in g for b in g], dtype=np.float64)


def q_grid_bz(n: int) -> np.ndarray:
    """n x n periodic grid of the full zone: q_i = -pi + 2 pi i / n, i < n
    (closed under the C4v point group).  Order as q_grid_quadrant."""
    g = np.array([-math.pi + 2.0 * math.pi * i / n for i in range(n)])
    return np.array([(a, b) for a in g for b in g], dtype=np.float64)


def all_pairs(nff: int) -> np.ndarray:
    """Every (l, m) with l, m < nff, l-major."""
    return np.array([(l, m) for l in range(nff) for m in range(nff)], dtype=np.int32)


def log_temperatures(n: int = 12, t_hi: float = 1.0, t_lo: float = 0.005) -> np.ndarray:
    """n temperatures log-spaced from t_hi down to t_lo (T_j = t_lo^(j/(n-1)) for t_hi=1)."""
    return np.array([t_hi * (t_lo / t_hi) ** (j / (n - 1)) for j in range(n)])


@dataclass
class Batch:
    """One (kind, T) batch: nq * npairs integrals, index iq * npairs + ip."""
    kind: int
    T: float
    q: np.ndarray
    lm: np.ndarray
    rel_tol: float = 1e-6
    abs_tol: float = 1e-10
    max_regions: int = 100000

    @property
    def n(self) -> int:
        return int(self.q.shape[0] * self.lm.shape[0])


@dataclass
class Workload:
    name: str
    lattice: tuple
    ffset: int
    batches: list = field(default_factory=list)

    @property
    def n(self) -> int:
        return sum(b.n for b in self.batches)


def config_first_shell() -> Workload:
    """400 ph integrals at T = 0.5: q on a 4x4 grid of [0, pi]^2, all 25 pairs of
    the 5 first-shell form factors; rel tol 1e-6, abs tol 1e-10, <= 1e4 regions."""
    b = Batch(PH, 0.5, q_grid_quadrant(4), all_pairs(5), 1e-6, 1e-10, 10000)
    return Workload("ph_T0.5_q4x4_ff5_400", LATTICE, 5, [b])


def config_flow_step(T: float = 0.05, rel_tol: float = 1e-6, nq: int = 24) -> Workload:
    """One flow-step batch: ph + pp at temperature T, q on an nq x nq grid of the
    full zone, all 81 pairs of the 9 two-shell form factors
    (2 * 576 * 81 = 93,312 integrals at nq = 24)."""
    q = q_grid_bz(nq)
    lm = all_pairs(9)
    bs = [Batch(PH, T, q, lm, rel_tol, 1e-10, 100000),
          Batch(PP, T, q, lm, rel_tol, 1e-10, 100000)]
    return Workload("phpp_T%g_q%dx%d_ff9_%d" % (T, nq, nq, 2 * nq * nq * 81), LATTICE, 9, bs)


def config_flow_omega(omega: float = 0.1, rel_tol: float = 1e-6, nq: int = 24) -> Workload:
    """One flow step of the Omega-regulated scheme: the scale derivatives of the
    ph and pp bubbles of the flow equations at regulator scale Omega (carried in
    the batches' T field), l on an nq x nq grid of the full zone, all 81 pairs
    (2 * 576 * 81 = 93,312 integrals at nq = 24)."""
    q = q_grid_bz(nq)
    lm = all_pairs(9)
    bs = [Batch(FLOW_PH, omega, q, lm, rel_tol, 1e-10, 100000),
          Batch(FLOW_PP, omega, q, lm, rel_tol, 1e-10, 100000)]
    return Workload("flow_ph_pp_Omega%g_q%dx%d_ff9_%d" % (omega, nq, nq, 2 * nq * nq * 81),
                    LATTICE, 9, bs)


def config_temperature_sweep(nT: int = 12, nq: int = 16, rel_tol: float = 1e-6) -> Workload:
    """nT log-spaced temperatures from 1.0 to 0.005 x q on an nq x nq zone grid
    x 81 pairs x {ph, pp} (497,664 integrals at the defaults)."""
    q = q_grid_bz(nq)
    lm = all_pairs(9)
    bs = []
    for T in log_temperatures(nT):
        for kind in (PH, PP):
            bs.append(Batch(kind, float(T), q, lm, rel_tol, 1e-10, 100000))
    n = nT * nq * nq * 81 * 2
    return Workload("phpp_T12_q%dx%d_ff9_%d" % (nq, nq, n), LATTICE, 9, bs)


def sample_indices(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct indices of range(n), sorted, from a seeded generator."""
    rng = np.random.default_rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False))


def flatten(w: Workload):
    """Flat per-integral arrays (kind, q, lm, T, batch, local index) in the
    batch order of w, each batch in its own iq * npairs + ip order."""
    kinds, qs, lms, Ts, bid, loc = [], [], [], [], [], []
    for j, b in enumerate(w.batches):
        nq, npair = b.q.shape[0], b.lm.shape[0]
        iq = np.repeat(np.arange(nq), npair)
        ip = np.tile(np.arange(npair), nq)
        kinds.append(np.full(b.n, b.kind, dtype=np.int32))
        qs.append(b.q[iq])
        lms.append(b.lm[ip])
        Ts.append(np.full(b.n, b.T))
        bid.append(np.full(b.n, j, dtype=np.int32))
        loc.append(np.arange(b.n))
    return dict(kind=np.concatenate(kinds), q=np.concatenate(qs), lm=np.concatenate(lms),
                T=np.concatenate(Ts), batch=np.concatenate(bid), local=np.concatenate(loc))


def config_heldout(seed: int = 10000, nq: int = 24, rel_tol: float = 1e-6) -> Workload:
    """A flow-step batch (ph + pp, all 81 pairs, nq x nq zone grid) at a seeded
    held-out parameter draw (t', mu, T) of parameter_draws (seeds 10000+ are never
    used for training)."""
    tp, mu, T = parameter_draws(1, seed)[0]
    q = q_grid_bz(nq)
    lm = all_pairs(9)
    bs = [Batch(PH, T, q, lm, rel_tol, 1e-10, 100000), Batch(PP, T, q, lm, rel_tol, 1e-10, 100000)]
    return Workload("heldout%d_tp%.4f_mu%.4f_T%.4g_q%dx%d_ff9_%d" % (seed, tp, mu, T, nq, nq,
                                                                    2 * nq * nq * 81),
                    (1.0, tp, mu), 9, bs)


def parameter_draws(k: int, seed0: int):
    """k seeded parameter draws (t', mu, T) with t' ~ U[-0.35, 0],
    mu ~ U[-1.4, 0], T log-uniform on [0.005, 1]; draw j uses seed seed0 + j."""
    out = []
    for j in range(k):
        rng = np.random.default_rng(seed0 + j)
        tp = rng.uniform(-0.35, 0.0)
        mu = rng.uniform(-1.4, 0.0)
        T = math.exp(rng.uniform(math.log(0.005), math.log(1.0)))
        out.append((float(tp), float(mu), float(T)))
    return out
