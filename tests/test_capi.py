"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/paid.h declares; host-side argument checks
answer without touching a device."""
import ctypes
import os
import re

import pytest

from paper_1610_09991_gb300 import build as B
from paper_1610_09991_gb300 import paid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return paid.load()


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(paid_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"paid_create", "paid_integrate_batch", "paid_integrate_multi"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert set(paid.EXPORTS) <= names


def test_binding_constants_match_the_header():
    txt = open(os.path.join(ROOT, "include", "paid.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"\bPAID_(\w+)\s*=\s*(-?\d+)", txt)}
    for name in ("PH", "PP", "MONOMIAL", "OVERLAP", "FLOW_PH", "FLOW_PP", "OK", "ERR_ARG",
                 "ERR_OOM", "ERR_CUDA", "ERR_POOL", "ERR_TIMEOUT", "CONVERGED", "BUDGET",
                 "NONFINITE", "ROUNDCAP", "POOL", "GROUP_NONE", "GROUP_PER_PAIR",
                 "GROUP_GLOBAL", "FF_SHELL1", "FF_SHELL12"):
        assert getattr(paid, name) == consts[name], name


def test_host_side_calls_without_gpu(lib):
    assert paid.error_string(paid.ERR_POOL) == "region pool full"
    o = paid.options_default()
    assert (o.rule_n, o.init_level, o.eval_fp32, o.max_rounds) == (4, 2, 0, 4096)
    assert (o.timing, o.device_loop) == (0, 1)
    assert lib.paid_options_default(None) == paid.ERR_ARG
    assert lib.paid_workspace_size(None, 10, 1000, None) == paid.ERR_ARG
    h = ctypes.c_void_p()
    # invalid arguments are rejected before any device is touched
    assert lib.paid_create(ctypes.byref(h), 1.0, -0.25, -1.0, 7, None, 0) == paid.ERR_ARG
    assert lib.paid_create(ctypes.byref(h), float("nan"), -0.25, -1.0, 9, None, 0) == paid.ERR_ARG
    bad = paid.options_default()
    bad.rule_n = 5
    assert lib.paid_create(ctypes.byref(h), 1.0, -0.25, -1.0, 9, ctypes.byref(bad), 0) == paid.ERR_ARG
    bad.rule_n = 8   # N = 8, 10, 12 only with the shared-partition kernel
    assert lib.paid_create(ctypes.byref(h), 1.0, -0.25, -1.0, 9, ctypes.byref(bad), 0) == paid.ERR_ARG
    bad.rule_n, bad.eval_fp32 = 4, 2       # precision modes are 0 (FP64) and 1 (FP32 pipe)
    assert lib.paid_create(ctypes.byref(h), 1.0, -0.25, -1.0, 9, ctypes.byref(bad), 0) == paid.ERR_ARG
    bad.group_mode, bad.eval_fp32 = 3, 0   # modes are 0, 1, 2
    assert lib.paid_create(ctypes.byref(h), 1.0, -0.25, -1.0, 9, ctypes.byref(bad), 0) == paid.ERR_ARG
    assert lib.paid_integrate_multi(None, None, 0, None, 0, None) == paid.ERR_ARG
    # the proposal's forward pass needs a 16-byte aligned output and a
    # 256-byte aligned workspace (checked before anything is launched)
    n = ctypes.c_int64()
    assert lib.paid_mlp_param_count(ctypes.byref(n)) == paid.OK and n.value == 271616
    P_, X_, WS = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000), 1 << 30
    fwd = lib.paid_mlp_forward
    fwd.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                    ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    assert fwd(P_, X_, 4, ctypes.c_void_p(0x30004), ctypes.c_void_p(0x40000), WS,
               None) == paid.ERR_ARG
    assert fwd(P_, X_, 4, ctypes.c_void_p(0x30000), ctypes.c_void_p(0x40010), WS,
               None) == paid.ERR_ARG
    assert fwd(P_, X_, 0, None, None, 0, None) == paid.OK


def test_no_cpu_fallback_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        paid.Context()
