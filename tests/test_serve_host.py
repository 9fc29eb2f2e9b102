"""Host logic of the serving layer (no GPU): the engine plan that prepare()
makes for a request stream in batched mode."""
import types

import numpy as np

from paper_1312_1476_gb300 import serve


def _shell(budget, nslots_max=64):
    # a Server without its device state: prepare()'s planning part only
    s = serve.Server.__new__(serve.Server)
    s.budget = int(budget)
    s.nslots_max = nslots_max
    s.precision = "fp32"
    s.mode = "batched"
    s.plan = {}
    s.engines = {}
    s.created = []
    s.fields = types.SimpleNamespace(get=lambda *a: None)
    s.torch = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))
    s._engine_for = lambda r: s.created.append((r.shape, r.field_id))
    return s


def test_plan_fits_the_budget_and_follows_demand():
    reqs = serve.make_mix(400, rate=1e6, seed=4)
    s = _shell(60e9)
    s.prepare(reqs, tune=False)
    keys = {(r.shape, r.field_id) for r in reqs if r.kind != "solve"}
    assert set(s.plan) == keys and sorted(s.created) == sorted(keys)
    assert sum(v * s._slot_bytes(k[0]) for k, v in s.plan.items()) <= s.budget
    assert all(4 <= v <= 64 for v in s.plan.values())
    demand = {}
    for r in reqs:
        if r.kind != "solve":
            demand[(r.shape, r.field_id)] = demand.get((r.shape, r.field_id), 0) + r.count
    # among the expensive grids (no floor, no cap) slots grow with requested vectors
    big = [k for k in keys if len(k[0]) == 3 and k[0][0] == 128]
    big.sort(key=lambda k: demand[k])
    assert [s.plan[k] for k in big] == sorted(s.plan[k] for k in big)
    # cheap grids get their floor: an eighth of an equal share of the budget
    floor = s.budget // (8 * len(keys))
    for k in keys:
        if len(k[0]) == 2 and k[0][0] == 128:
            assert s.plan[k] >= min(64, floor // s._slot_bytes(k[0]))


def test_plan_keeps_earlier_engines():
    s = _shell(60e9)
    first = serve.make_mix(100, rate=1e6, seed=1, sizes2d=(256,), sizes3d=(64,), nfields=1)
    s.prepare(first, tune=False)
    plan1 = dict(s.plan)
    more = serve.make_mix(100, rate=1e6, seed=2, sizes2d=(256, 512), sizes3d=(64,), nfields=1)
    s.prepare(more, tune=False)
    assert all(s.plan[k] == v for k, v in plan1.items())
    assert sum(v * s._slot_bytes(k[0]) for k, v in s.plan.items()) <= s.budget
    assert len(s.plan) == len({(r.shape, r.field_id) for r in first + more if r.kind != "solve"})
