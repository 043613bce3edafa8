"""Host logic of the benchmark's accuracy statements, on the CPU: the checkers
must count a planted deviation as a parity failure, and a disagreement that
is the reference's own false convergence must be decided by the brute-force
value in favour of the checked result."""
import importlib.util
import os

import numpy as np
import pytest

import oracle
from paper_1610_09991_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _first_shell_sample():
    (b,) = W.config_first_shell().batches
    q = b.q[:2]
    v, e, r, s = oracle.integrate_batch(b.kind, q, b.lm, b.T, W.LATTICE, b.rel_tol, b.abs_tol,
                                        b.max_regions)
    P = b.lm.shape[0]
    ident = lambda i: (b.kind, q[i // P], int(b.lm[i % P][0]), int(b.lm[i % P][1]), b.T)
    return b, v, s, ident


def test_accuracy_counts_a_planted_error(bench):
    b, v, s, ident = _first_shell_sample()
    ok = bench.accuracy(v.copy(), s, v, s, b.rel_tol, b.abs_tol, "self", ident, W.LATTICE)
    assert ok["parity_failures"] == 0 and ok["max_err_over_tol"] == 0.0
    bad = v.copy()
    i = int(np.argmax(np.abs(v)))
    bad[i] += 5 * max(b.rel_tol * abs(v[i]), b.abs_tol)
    got = bench.accuracy(bad, s, v, s, b.rel_tol, b.abs_tol, "planted", ident, W.LATTICE)
    assert got["parity_failures"] == 1
    assert got["disagreements_decided_by_brute_force"][0]["integral"] == i


def test_accuracy_sides_with_the_brute_force(bench):
    # the reference off by 5 tol (a false convergence): the checked values
    # match the brute force, so the disagreement is not a parity failure
    b, v, s, ident = _first_shell_sample()
    ref = v.copy()
    i = int(np.argmax(np.abs(v)))
    ref[i] += 5 * max(b.rel_tol * abs(v[i]), b.abs_tol)
    got = bench.accuracy(v, s, ref, s, b.rel_tol, b.abs_tol, "planted", ident, W.LATTICE)
    assert got["parity_failures"] == 0
    d = got["disagreements_decided_by_brute_force"]
    assert len(d) == 1 and d[0]["value_within_2tol_of_brute_force"]


def test_accuracy_counts_integrals_left_unconverged(bench):
    # the reference converged, the checked side stopped on its budget, the
    # round cap or a full pool with a value that may look right: each one is a
    # parity failure
    b, v, s, ident = _first_shell_sample()
    for status in (1, 3, 4):
        st = s.copy()
        st[[3, 7]] = status
        got = bench.accuracy(v.copy(), st, v, s, b.rel_tol, b.abs_tol, "planted", ident,
                             W.LATTICE)
        assert got["unconverged_where_reference_converged"] == 2
        assert got["parity_failures"] == 2
    # the reverse (the reference stopped, the checked side converged) is not
    st = s.copy()
    st[5] = 1
    got = bench.accuracy(v.copy(), s, v, st, b.rel_tol, b.abs_tol, "planted", ident, W.LATTICE)
    assert got["parity_failures"] == 0


def test_group_global_check(bench):
    w = W.config_flow_step(T=0.5, nq=2)
    vals, stats = [], []
    for b in w.batches:
        v, e, r, s = oracle.integrate_group_global(b.kind, b.q, b.lm, b.T, W.LATTICE, b.rel_tol,
                                                   b.abs_tol, b.max_regions, rule_n=12)
        vals.append(v)
        stats.append(s)
    gv, gs = np.concatenate(vals), np.concatenate(stats)
    ok = bench.group_global_check(w, gv, gs, 12, rows_per_batch=4)
    assert ok["parity_failures"] == 0 and ok["max_dev_over_group_tol"] == 0.0
    # 3 group tolerances spread over one group's pairs: one failure
    b = w.batches[0]
    P = b.lm.shape[0]
    tol_g = max(b.abs_tol, b.rel_tol * np.abs(gv[:P]).sum())
    bad = gv.copy()
    bad[:P] += 3 * tol_g / P
    got = bench.group_global_check(w, bad, gs, 12, rows_per_batch=4)
    assert got["parity_failures"] == 1
    assert abs(got["max_dev_over_group_tol"] - 3.0) < 1e-6
    # an unconverged group counts as a failure too
    st = gs.copy()
    st[P] = 1
    assert bench.group_global_check(w, gv, st, 12, rows_per_batch=4)["parity_failures"] == 1


class _DoneProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_keeps_only_the_timed_window(bench, tmp_path):
    """Only samples stamped inside the marked window count, and a throttle
    reason seen there is reported; samples before and after are dropped."""
    import datetime
    cs = bench.ClockSampler(0)
    base = datetime.datetime(2026, 1, 2, 3, 4, 5)
    rows = []
    for k, (mhz, hw) in enumerate([(1200, "Active"), (2070, "Not Active"), (2070, "Not Active"),
                                   (1980, "Active"), (900, "Not Active")]):
        ts = (base + datetime.timedelta(milliseconds=100 * k)).strftime("%Y/%m/%d %H:%M:%S.%f")
        rows.append(f"{ts[:-3]}, 0, {mhz}, 2070, 500.0, 0x0, Not Active, {hw}, Not Active, "
                    "Not Active")
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    cs.path, cs.proc = str(path), _DoneProc()
    cs.window = [(base + datetime.timedelta(milliseconds=100)).timestamp(),
                 (base + datetime.timedelta(milliseconds=300)).timestamp()]
    out = cs.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["hw_thermal_slowdown"]


def test_cpu_baseline_reports_all_threads_and_one_core(bench):
    """The oracle baseline: a seeded sample on every host thread and its first
    integrals on one thread, both as converged integrals per second."""
    cb, (idx, v, s) = bench.cpu_baseline(W.config_first_shell(), 8, one_core=3)
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0
    assert cb["converged"] == 8 and len(idx) == 8 and np.all(s == 0)
    assert cb["one_core"]["cores"] == 1 and cb["one_core"]["value"] > 0
