"""Batched execution: every job in the mix gives the oracle's result.

A batch advances many jobs of uneven size and type together (one launch per
bond-class group for all cubic jobs of a shape class, one per colour class for
all graph jobs); the random streams are keyed by each job's own seed, sweep,
class and site, so each job's observations and final state planes must equal,
bit for bit, those of the oracle running that job alone.  Also: admission by
memory budget, removal, autotuning, adoption of a running context.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle_runs  # noqa: E402
import paper_1710_05155_gb300 as K  # noqa: E402

JOBS = [
    dict(params=dict(topo=K.KA_CUBIC, d=3, L=16, m=3, replicas=64), sweeps=37, every=10, seed=5, rho=0.75),
    dict(params=dict(topo=K.KA_CUBIC, d=3, L=24, m=3, replicas=64), sweeps=20, every=7, seed=6, rho=0.80),
    dict(params=dict(topo=K.KA_CUBIC, d=3, L=32, m=3, replicas=256), sweeps=25, every=25, seed=7, rho=0.85),
    dict(params=dict(topo=K.KA_CUBIC, d=3, L=20, m=2, replicas=128), sweeps=12, every=5, seed=8, rho=0.6),
    dict(params=dict(topo=K.KA_CUBIC, d=2, L=16, m=1, replicas=192), sweeps=9, every=4, seed=9, rho=0.5),
    dict(params=dict(topo=K.KA_RRG, N=4096, z=4, m=2, replicas=64, graph_seed=1), sweeps=30, every=10, seed=10, rho=0.78),
    dict(params=dict(topo=K.KA_RRG, N=2048, z=4, m=2, replicas=128, graph_seed=2), sweeps=17, every=6, seed=11, rho=0.82),
    dict(params=dict(topo=K.KA_RRG, N=1000, z=3, m=1, replicas=64, graph_seed=3), sweeps=14, every=14, seed=12, rho=0.7),
    dict(params=dict(topo=K.KA_RRG, N=3000, z=4, m=2, replicas=256, graph_seed=4), sweeps=13, every=5, seed=14, rho=0.8),
    dict(params=dict(topo=K.KA_CUBIC, d=3, L=8, m=3, replicas=64, flags=K.KA_FLAG_GENERIC), sweeps=11, every=3, seed=13, rho=0.7),
    # a caller-supplied graph: the layered random graph of section 5.2
    dict(params=dict(topo=K.KA_GRAPH, N=4 * 4 ** 3, z=6, m=3, replicas=128,
                     nbr=K.ka_layered_graph(3, 4, 4, 9)), sweeps=16, every=4, seed=15, rho=0.72),
    # a cubic lattice large enough to run with its own launches inside the rounds
    dict(params=dict(topo=K.KA_CUBIC, d=3, L=64, m=3, replicas=64), sweeps=6, every=3, seed=16, rho=0.8),
]


def _alone(job):
    sim = K.Simulation(**job["params"])
    sim.init(job["seed"], job["rho"])
    sweeps, counts = [], []
    t, c = sim.observe()
    sweeps.append(t)
    counts.append(c.copy())
    while t < job["sweeps"]:
        step = min(job["every"] - t % job["every"], job["sweeps"] - t)
        sim.sweep(step)
        t, c = sim.observe()
        sweeps.append(t)
        counts.append(c.copy())
    sim.close()
    return np.array(sweeps), np.stack(counts)


@pytest.fixture(scope="module")
def oracle_results():
    """The oracle's run of every job of JOBS: sweeps, counts, n, n0, p."""
    return oracle_runs.run_jobs([(j["params"], j["sweeps"], j["every"], j["seed"], j["rho"])
                                 for j in JOBS])


def _sites(params):
    return params["L"] ** params["d"] if params["topo"] == K.KA_CUBIC else params["N"]


def _check_job(b, jid, job, want):
    sw, cnt = b.observations(jid, job["params"]["replicas"])
    w_sw, w_cnt, w_n, w_n0, w_p = want
    assert (sw == w_sw).all(), f"job {jid}: observation sweeps differ"
    assert (cnt == w_cnt).all(), f"job {jid}: counts differ from the oracle's"
    n, n0, p = b.state(jid, job["params"]["replicas"] // 64, _sites(job["params"]))
    assert (n == w_n).all() and (n0 == w_n0).all() and (p == w_p).all(), \
        f"job {jid}: final state differs from the oracle's"


@pytest.mark.parametrize("flags,k", [(K.KA_BATCH_GRAPH, 8), (0, 5), (K.KA_BATCH_PLAIN, 6),
                                     (K.KA_BATCH_GRAPH, 1)])
def test_batched_jobs_match_the_oracle(flags, k, oracle_results):
    with K.Batch(flags=flags) as b:
        ids = [b.add(j["sweeps"], j["every"], j["seed"], j["rho"], **j["params"]) for j in JOBS]
        for _ in range(1000):
            if b.info()["active"] == 0:
                break
            b.step(k)
        assert b.info()["active"] == 0
        for jid, job, want in zip(ids, JOBS, oracle_results):
            t, done = b.poll(jid)
            assert done and t == job["sweeps"]
            _check_job(b, jid, job, want)


def test_jobs_joining_a_running_batch(oracle_results):
    # continuous batching: a job admitted while others are mid-run still
    # gives the oracle's result
    with K.Batch() as b:
        first = [b.add(j["sweeps"], j["every"], j["seed"], j["rho"], **j["params"]) for j in JOBS[:4]]
        b.step(6)
        b.step(6)
        late = [b.add(j["sweeps"], j["every"], j["seed"], j["rho"], **j["params"]) for j in JOBS[4:]]
        while b.info()["active"]:
            b.step(4)
        for jid, job, want in zip(first + late, JOBS, oracle_results):
            _check_job(b, jid, job, want)


def test_solo_runs_match_the_oracle(oracle_results):
    # the plain (single-context) path of the same jobs, observation by observation
    for job, want in zip(JOBS, oracle_results):
        sw, cnt = _alone(job)
        assert (sw == want[0]).all() and (cnt == want[1]).all()


def test_job_state_of_an_unknown_job_is_rejected():
    with K.Batch() as b:
        with pytest.raises(K.KaError) as e:
            b.state(12345, 1, 64)
        assert e.value.status == K.KA_EINVAL


def test_budget_admission_and_release():
    p = dict(topo=K.KA_CUBIC, d=3, L=32, m=3, replicas=64)
    one = K.ka_required_bytes(K.make_params(**p)[0])
    with K.Batch(hbm_budget=2 * one + one // 2) as b:
        a = b.add(10, 5, 1, 0.7, **p)
        b.add(10, 5, 2, 0.7, **p)
        with pytest.raises(K.KaError) as e:
            b.add(10, 5, 3, 0.7, **p)
        assert e.value.status == K.KA_EBUSY
        used = b.info()["used_bytes"]
        b.remove(a)
        assert b.info()["used_bytes"] < used
        b.add(10, 5, 3, 0.7, **p)
        while b.info()["active"]:
            b.step(10)


def test_autotune_picks_a_candidate():
    with K.Batch() as b:
        k0, t0 = b.tuning()
        assert k0 == 16 and t0 > 0  # before tuning: one wave of tiles
        for j in JOBS[:6]:
            b.add(200, 100, j["seed"], j["rho"], **j["params"])
        k = b.autotune()
        assert k in (4, 16, 64)
        kt, t = b.tuning()
        assert kt == k and t in (t0, t0 // 2, t0 // 4, t0 // 8, 2 ** 63 - 1)
        while b.info()["active"]:
            b.step()


def test_autotuned_mix_matches_the_oracle(oracle_results):
    # tuning moves cubic jobs between their own and the shared launches
    # mid-run; every job still ends with the oracle's observations and planes
    with K.Batch() as b:
        ids = [b.add(j["sweeps"], j["every"], j["seed"], j["rho"], **j["params"]) for j in JOBS]
        b.step(2)
        b.autotune()
        while b.info()["active"]:
            b.step()
        for jid, job, want in zip(ids, JOBS, oracle_results):
            _check_job(b, jid, job, want)


def test_adopt_rules():
    p = dict(topo=K.KA_CUBIC, d=3, L=16, m=3, replicas=64)
    with K.Batch() as b:
        params, keep = K.make_params(**p)
        fresh = K.ka_create(params, keep)
        with pytest.raises(K.KaError) as e:  # not initialised
            b.adopt(fresh, 10, 5)
        assert e.value.status == K.KA_ESTATE
        K.ka_init(fresh, 3, 0.7)
        K.ka_sweep(fresh, 4)  # adopted mid-run: observations continue from sweep 4
        jid = b.adopt(fresh, 12, 5)
        assert not fresh  # the batch owns it now
        sim = K.Simulation(**p)  # caller-owned buffer: cannot be handed over
        sim.init(3, 0.7)
        with pytest.raises(K.KaError) as e:
            b.adopt(sim.ctx, 10, 5)
        assert e.value.status == K.KA_EINVAL
        while b.info()["active"]:
            b.step(3)
        sw, cnt = b.observations(jid, 64)
        assert list(sw) == [4, 5, 10, 12]
        for t, c in zip(sw, cnt):
            if t == 4:
                continue
            sim.sweep(int(t) - sim.observe()[0])
            assert (sim.observe()[1] == c).all()
        sim.close()


def test_out_of_memory_is_reported_and_harmless():
    # about 2 TB of state: the allocation fails on the host side and nothing is left behind
    big = dict(topo=K.KA_CUBIC, d=3, L=1024, m=3, replicas=4096)
    params, keep = K.make_params(**big)
    assert K.ka_required_bytes(params) > (1 << 40)
    with pytest.raises(K.KaError) as e:
        K.ka_create(params, keep)
    assert e.value.status == K.KA_ENOMEM
    with K.Batch(hbm_budget=1 << 62) as b:
        with pytest.raises(K.KaError) as e:
            b.add(10, 5, 1, 0.7, **big)
        assert e.value.status == K.KA_ENOMEM
        assert b.info()["jobs"] == 0 and b.info()["used_bytes"] == 0
        jid = b.add(10, 5, 1, 0.7, topo=K.KA_CUBIC, d=3, L=16, m=3, replicas=64)
        while b.info()["active"]:
            b.step(5)
        assert b.poll(jid) == (10, True)
