"""GPU tests of the serving layer: a request gives the same result alone and
in a concurrent mix, and admission keeps the in-flight memory estimate inside
the budget."""
import numpy as np
import pytest

from paper_1312_1476_gb300 import serve

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _mix():
    reqs = serve.make_mix(12, rate=1e6, seed=9, sizes2d=(128, 256), sizes3d=(32, 48), nfields=2,
                          max_samples=6, probes=(4, 8), p_logdet=0.3, p_solve=0.3)
    for r in reqs:
        r.arrival = 0.0
    return reqs


@pytest.mark.parametrize("tune", [False, True])
def test_alone_equals_mix(tune):
    torch.cuda.synchronize()
    srv = serve.Server(max_inflight=8)
    reqs = _mix()
    srv.prepare(reqs, tune=tune)
    if tune:
        assert srv.tuning and all(t["block_width"] >= 1 for t in srv.tuning.values())
    mixed, metrics = srv.serve(reqs, realtime=False)
    assert metrics["requests"] == len(reqs)
    assert all(r.status == 0 for r in mixed), [(r.rid, r.kind, r.shape, r.status) for r in mixed if r.status]
    kinds = {r.kind for r in reqs}
    assert kinds == {"sample", "logdet", "solve"}
    targets = sorted({0, 5, 11} | {min(i for i, r in enumerate(reqs) if r.kind == k) for k in kinds})
    for target in targets:
        one = serve.Server(max_inflight=1)
        one.tuning = dict(srv.tuning)
        alone, _ = one.serve([reqs[target]], realtime=False)
        a, b = alone[0], mixed[target]
        if a.kind in ("sample", "solve"):
            assert torch.equal(a.x, b.x)
        else:
            assert a.logdet == b.logdet and a.std_err == b.std_err
        assert a.m_used == b.m_used


def test_admission_respects_budget():
    reqs = _mix()
    probe = serve.Server(max_inflight=8)
    budget = 3 * max(probe.need(r) for r in reqs)
    srv = serve.Server(mem_budget=budget, max_inflight=8)
    peak = [0]
    orig = srv._run

    def run(req, t0):
        peak[0] = max(peak[0], srv.used)
        return orig(req, t0)

    srv._run = run
    out, metrics = srv.serve(reqs, realtime=False)
    assert len(out) == len(reqs)
    assert peak[0] <= budget
    assert metrics["p99_ms"] >= metrics["p50_ms"] > 0
