"""Served execution on the GPU: each result is the oracle's, alone and in the mix.

Requests arrive over time while others are running; they are prepared on host
threads, join the running batch between rounds and share its launches, under
a memory budget small enough that some must wait for others to be retired.
Every job's observations and final state planes must equal, bit for bit, the
oracle's run of that job alone; the plain single-context path is checked
against the same oracle runs.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle_runs  # noqa: E402
import paper_1710_05155_gb300 as K  # noqa: E402
from paper_1710_05155_gb300 import serve, workloads  # noqa: E402


def _jobs():
    W = workloads
    spec = [
        # (params, sweeps, every, arrival); the first job runs while the others arrive
        (dict(topo=W.CUBIC, d=3, L=16, m=3, replicas=64), 1000, 250, 0.0),
        (dict(topo=W.CUBIC, d=3, L=16, m=3, replicas=64), 300, 50, 0.005),
        (dict(topo=W.RRG, N=4096, z=4, m=2, replicas=64, graph_seed=11), 250, 25, 0.01),
        (dict(topo=W.CUBIC, d=3, L=24, m=2, replicas=128), 100, 20, 0.02),
        (dict(topo=W.RRG, N=2048, z=4, m=3, replicas=192, graph_seed=12), 120, 30, 0.03),
        (dict(topo=W.CUBIC, d=3, L=32, m=3, replicas=256), 20, 5, 0.04),
        (dict(topo=W.CUBIC, d=3, L=20, m=3, replicas=64), 200, 50, 0.05),
        (dict(topo=W.RRG, N=1 << 14, z=4, m=2, replicas=64, graph_seed=13), 60, 6, 0.06),
        (dict(topo=W.CUBIC, d=3, L=16, m=3, replicas=192), 77, 7, 0.08),
        (dict(topo=W.CUBIC, d=3, L=48, m=3, replicas=64), 20, 5, 0.10),
    ]
    return [W.Job(p, s, e, 100 + i, 0.72 + 0.01 * i, a, {"index": i})
            for i, (p, s, e, a) in enumerate(spec)]


@pytest.fixture(scope="module")
def oracle_results():
    return oracle_runs.run_jobs([(j.params, j.sweeps, j.every, j.seed, j.rho) for j in _jobs()])


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
def test_served_results_match_the_oracle(graph, oracle_results):
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
        w_sw, w_cnt, w_n, w_n0, w_p = oracle_results[r.index]
        assert (r.sweeps == w_sw).all(), f"job {r.index}: observation sweeps differ"
        assert (r.counts == w_cnt).all(), f"job {r.index}: served counts differ from the oracle's"
        n, n0, p = r.state
        assert (n == w_n).all() and (n0 == w_n0).all() and (p == w_p).all(), \
            f"job {r.index}: served final state differs from the oracle's"
    # the budget was respected and some jobs waited for memory
    assert rep["latency_p99_s"] >= rep["latency_p50_s"] > 0


def test_solo_runs_match_the_oracle(oracle_results):
    for job, want in zip(_jobs(), oracle_results):
        sw, cnt = _alone(job)
        assert (sw == want[0]).all() and (cnt == want[1]).all(), f"job {job.tag['index']}"
