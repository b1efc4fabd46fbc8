"""Served execution on the GPU: each result is the same alone and in the mix.

Requests arrive over time while others are running; they are prepared on host
threads, join the running batch between rounds and share its launches, under
a memory budget small enough that some must wait for others to be retired.
Every job's observations must equal, bit for bit, the same job run alone.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1710_05155_gb300 as K  # noqa: E402
from paper_1710_05155_gb300 import serve, workloads  # noqa: E402


def _jobs():
    W = workloads
    spec = [
        # (params, sweeps, every, arrival)
        (dict(topo=W.CUBIC, d=3, L=32, m=3, replicas=64), 6000, 500, 0.0),
        (dict(topo=W.CUBIC, d=3, L=16, m=3, replicas=64), 300, 50, 0.005),
        (dict(topo=W.RRG, N=4096, z=4, m=2, replicas=64, graph_seed=11), 250, 25, 0.01),
        (dict(topo=W.CUBIC, d=3, L=24, m=2, replicas=128), 200, 40, 0.02),
        (dict(topo=W.RRG, N=2048, z=4, m=3, replicas=192, graph_seed=12), 120, 30, 0.03),
        (dict(topo=W.CUBIC, d=3, L=32, m=3, replicas=256), 90, 9, 0.04),
        (dict(topo=W.CUBIC, d=3, L=20, m=3, replicas=64), 400, 100, 0.05),
        (dict(topo=W.RRG, N=1 << 14, z=4, m=2, replicas=64, graph_seed=13), 60, 6, 0.06),
        (dict(topo=W.CUBIC, d=3, L=16, m=3, replicas=192), 77, 7, 0.08),
        (dict(topo=W.CUBIC, d=3, L=48, m=3, replicas=64), 40, 10, 0.10),
    ]
    return [W.Job(p, s, e, 100 + i, 0.72 + 0.01 * i, a, {"index": i})
            for i, (p, s, e, a) in enumerate(spec)]


def _alone(job):
    sim = K.Simulation(**job.params)
    sim.init(job.seed, job.rho)
    sweeps, counts = [], []
    t, c = sim.observe()
    sweeps.append(t)
    counts.append(c.copy())
    while t < job.sweeps:
        sim.sweep(min(job.every - t % job.every, job.sweeps - t))
        t, c = sim.observe()
        sweeps.append(t)
        counts.append(c.copy())
    sim.close()
    return np.array(sweeps), np.stack(counts)


@pytest.mark.parametrize("graph", [True, False])
def test_served_results_equal_solo_runs(graph):
    jobs = _jobs()
    # room for about three of the larger jobs at a time
    budget = 3 * max(serve.job_bytes(j) for j in jobs)
    be = serve.DeviceBackend(0, budget, graph, prepare_threads=3)
    try:
        srv = serve.Server(be, round_sweeps=0, keep_results=True, tune_at=3)
        rep = srv.run(jobs)
    finally:
        be.close()
    assert rep["done"] == len(jobs), [(r.status, r.error) for r in srv.records]
    assert rep["max_running"] >= 2
    for r in srv.records:
        sw, cnt = _alone(r.job)
        assert (r.sweeps == sw).all(), f"job {r.index}: observation sweeps differ"
        assert (r.counts == cnt).all(), f"job {r.index}: served result differs from its solo run"
    # the budget was respected and some jobs waited for memory
    assert rep["latency_p99_s"] >= rep["latency_p50_s"] > 0
