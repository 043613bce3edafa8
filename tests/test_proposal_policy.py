"""Host logic of the learned proposal's margin policy, on the CPU: the band
lookup, the maps a policy makes from predicted levels, and which library call
a policy leads to (the uniform start with no inference when no batch is
seeded, the seeded call otherwise)."""
import types

import numpy as np
import torch

from paper_1610_09991_gb300 import proposal as PR


class _Prop:
    def __init__(self, levels):
        self.levels = levels
        self.calls = 0

    def predict(self, ctx, batches):
        self.calls += 1
        return self.levels.clone()


class _Ctx:
    def __init__(self, group_mode=1, init_level=3):
        self.options = types.SimpleNamespace(group_mode=group_mode, init_level=init_level)
        self.calls = []

    def integrate_multi(self, batches, pool_capacity=None, stream=None):
        self.calls.append(("uniform", None, None))
        return "uniform"

    def integrate_multi_seeded(self, batches, maps, margin, pool_capacity=None, stream=None):
        self.calls.append(("seeded", maps, margin))
        return "seeded"


def _batches(Ts, nq=3):
    q = torch.zeros((nq, 2), dtype=torch.float64)
    lm = torch.zeros((81, 2), dtype=torch.int32)
    return [dict(kind=k, T=T, q=q, lm=lm) for k, T in zip(range(len(Ts)), Ts)]


def test_band_lookup_uses_upper_edges():
    pol = PR.MarginPolicy((None, 1.0, 0.0), bands=(0.01, 0.1, float("inf")))
    assert pol(0.005) is None and pol(0.01) is None
    assert pol(0.05) == 1.0 and pol(0.1) == 1.0
    assert pol(0.5) == 0.0 and pol(50.0) == 0.0
    assert pol.as_dict() == {"T <= 0.01": None, "T <= 0.1": 1.0, "T <= inf": 0.0}


def test_seed_maps_apply_each_batch_margin():
    pol = PR.MarginPolicy((None, 0.5, 0.0), bands=(0.01, 0.1, float("inf")))
    bs = _batches([0.005, 0.05, 0.5])            # 3 units each in group mode
    levels = torch.full((9, 256), 6.0)
    ctx = _Ctx(init_level=3)
    maps = PR.seed_maps(_Prop(levels), ctx, bs, pol).numpy()
    assert np.all(maps[0:3] == 3.0)               # no seed: the start level
    assert np.all(maps[3:6] == 5.5)               # margin 0.5
    assert np.all(maps[6:9] == 6.0)               # margin 0
    # one unit per integral outside group mode: 3 q x 81 pairs per batch
    ctx1 = _Ctx(group_mode=0, init_level=2)
    lv = torch.full((3 * 3 * 81, 256), 5.0)
    maps1 = PR.seed_maps(_Prop(lv), ctx1, bs, pol).numpy()
    assert np.all(maps1[:243] == 2.0) and np.all(maps1[243:486] == 4.5)
    assert np.all(maps1[486:] == 5.0)


def test_integrate_routes_by_policy():
    levels = torch.full((6, 256), 6.0)
    nosed = PR.MarginPolicy((None, None), bands=(0.1, float("inf")))
    prop, ctx = _Prop(levels), _Ctx()
    assert PR.integrate(prop, ctx, _batches([0.01, 0.5]), nosed) == "uniform"
    assert prop.calls == 0 and ctx.calls[0][0] == "uniform"
    mixed = PR.MarginPolicy((None, 0.0), bands=(0.1, float("inf")))
    prop, ctx = _Prop(levels), _Ctx(init_level=2)
    assert PR.integrate(prop, ctx, _batches([0.01, 0.5]), mixed) == "seeded"
    kind, maps, margin = ctx.calls[0]
    assert prop.calls == 1 and kind == "seeded" and margin == 0.0
    assert np.all(maps[:3].numpy() == 2.0) and np.all(maps[3:].numpy() == 6.0)
