"""Host logic of the request loop and the seeded workload generators (no GPU).

The server is driven through a fake backend with a fake clock: each round
costs one time unit and advances every running job by up to k sweeps, which
is enough to check admission order, the memory budget, continuous batching,
failure isolation and the latency accounting.
"""
import concurrent.futures as cf

import numpy as np
import pytest

from paper_1710_05155_gb300 import serve, workloads


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-3)


class FakeBackend:
    def __init__(self, clock, budget=100, k=10, fail=()):
        self.clock, self.budget, self.k, self.fail = clock, budget, k, set(fail)
        self.jobs = {}
        self.next_id = 1
        self.log = []  # (event, job index, time)
        self.max_used = 0

    def job_bytes(self, job):
        return job.tag["bytes"]

    def prepare(self, job):
        f = cf.Future()
        if job.tag["index"] in self.fail:
            f.set_exception(RuntimeError("topology failed"))
        else:
            f.set_result(job)
        return f

    def discard(self, handle):
        pass

    def adopt(self, job, _job):
        jid = self.next_id
        self.next_id += 1
        self.jobs[jid] = [job, 0]
        self.log.append(("adopt", job.tag["index"], self.clock.t))
        self.max_used = max(self.max_used, self.used())
        return jid

    def used(self):
        return sum(j.tag["bytes"] for j, _ in self.jobs.values())

    def autotune(self):
        return self.step(0)

    def step(self, k):
        k = k or self.k
        self.clock.t += 1.0
        for j in self.jobs.values():
            j[1] = min(j[0].sweeps, j[1] + k)
        return k

    def finished(self, jid):
        job, t = self.jobs[jid]
        return t >= job.sweeps

    def observations(self, jid, replicas):
        job, t = self.jobs[jid]
        return np.array([0, t]), np.zeros((2, replicas, 4), np.int64)

    def remove(self, jid):
        job, _ = self.jobs.pop(jid)
        self.log.append(("remove", job.tag["index"], self.clock.t))


def job(i, arrival, sweeps, nbytes, L=16):
    return workloads.Job(dict(topo=0, d=3, L=L, m=3, replicas=64), sweeps, 10, 1 + i, 0.7,
                         arrival, {"index": i, "bytes": nbytes})


def run(jobs, **kw):
    clock = FakeClock()
    be = FakeBackend(clock, **{k: v for k, v in kw.items() if k in ("budget", "k", "fail")})
    srv = serve.Server(be, clock=clock, sleep=clock.sleep, autotune=False,
                       keep_results=True)
    rep = srv.run(jobs)
    return srv, be, rep


def test_budget_bounds_resident_memory_and_admission_is_fifo():
    jobs = [job(i, 0.0, 50, 40) for i in range(6)]
    srv, be, rep = run(jobs, budget=100)
    assert rep["done"] == 6
    assert be.max_used <= 100
    adopted = [i for e, i, _ in be.log if e == "adopt"]
    assert adopted == sorted(adopted)  # first come, first served
    # two fit at a time: the third waits for the first to be retired
    t_adopt = {i: t for e, i, t in be.log if e == "adopt"}
    t_remove = {i: t for e, i, t in be.log if e == "remove"}
    assert t_adopt[2] >= t_remove[0]


def test_oversized_job_is_rejected_and_the_rest_run():
    jobs = [job(0, 0.0, 20, 10), job(1, 0.0, 20, 1000), job(2, 0.0, 20, 10)]
    srv, be, rep = run(jobs, budget=100)
    assert rep["done"] == 2 and rep["rejected"] == 1
    assert srv.records[1].status == "rejected"


def test_failed_preparation_fails_one_job_only():
    jobs = [job(i, 0.0, 20, 10) for i in range(3)]
    srv, be, rep = run(jobs, budget=100, fail={1})
    assert [r.status for r in srv.records] == ["done", "failed", "done"]
    assert rep["failed"] == 1


def test_late_arrival_joins_while_others_run():
    # job 0 is long; job 1 arrives later, is admitted at once and finishes first
    jobs = [job(0, 0.0, 1000, 10), job(1, 5.0, 20, 10)]
    srv, be, rep = run(jobs, budget=100)
    r0, r1 = srv.records
    assert r1.admitted < r0.finished
    assert r1.finished < r0.finished
    assert rep["max_running"] == 2


def test_latency_and_throughput_accounting():
    jobs = [job(0, 0.0, 30, 10), job(1, 2.0, 30, 10)]
    srv, be, rep = run(jobs, budget=100, k=10)
    r0, r1 = srv.records
    # 3 rounds of 10 sweeps each, one time unit per round
    assert r0.finished - r0.arrival == pytest.approx(3.0)
    lat = [r.finished - r.arrival for r in srv.records]
    assert rep["latency_p50_s"] == pytest.approx(np.percentile(lat, 50))
    work = sum(j.work for j in jobs)
    assert rep["moves_per_s"] == pytest.approx(work / rep["makespan_s"])
    assert r0.counts.shape == (2, 64, 4)


def test_instance_mix_recipe():
    jobs = workloads.instance_mix(512, master=1)
    assert len(jobs) == 512
    assert jobs[0].params == workloads.instance_mix(1, master=1)[0].params
    cubic = [j for j in jobs if j.params["topo"] == workloads.CUBIC]
    graphs = [j for j in jobs if j.params["topo"] == workloads.RRG]
    assert 200 < len(cubic) < 312
    assert {j.params["L"] for j in cubic} <= {16, 24, 32, 48, 64, 96}
    assert all(j.params["m"] == 3 and j.params["d"] == 3 for j in cubic)
    assert {j.params["N"] for j in graphs} <= {1 << u for u in range(12, 19)}
    assert all(j.params["z"] == 4 and j.params["m"] == 2 for j in graphs)
    assert all(0.75 <= j.rho <= 0.88 and 1000 <= j.sweeps <= 20000 for j in jobs)
    assert all(j.params["replicas"] == 64 and j.every == 100 for j in jobs)
    assert len({j.seed for j in jobs}) == 512


def test_request_trace_recipe():
    a = workloads.request_trace(2000, 200.0, master=1)
    b = workloads.request_trace(2000, 100.0, master=1)
    arr = np.array([j.arrival for j in a])
    assert (np.diff(arr) > 0).all()
    assert np.mean(np.diff(arr)) == pytest.approx(1 / 200.0, rel=0.1)
    # another rate: the same jobs, arrivals stretched
    assert [j.params for j in a] == [j.params for j in b]
    assert b[-1].arrival == pytest.approx(2 * a[-1].arrival)
    for j in a:
        p = j.params
        if p["topo"] == workloads.CUBIC:
            assert p["L"] % 4 == 0 and 32 <= p["L"] <= 128
        else:
            assert p["N"] in {1 << u for u in range(14, 21)} and p["z"] == 4
        assert p["m"] in (2, 3) and p["replicas"] in (64, 128, 192, 256)
        assert 0.70 <= j.rho <= 0.90 and 1000 <= j.sweeps <= 100000
        assert j.every == max(1, j.sweeps // 100)
    s = np.log([j.sweeps for j in a])
    assert np.mean(s) == pytest.approx((np.log(1e3) + np.log(1e5)) / 2, rel=0.05)


def test_scaled_sample():
    a = workloads.request_trace(10, 200.0, master=3)
    s = workloads.scaled(a, sweep_scale=0.1, rate_scale=2.0)
    for x, y in zip(a, s):
        assert y.sweeps == max(1, round(x.sweeps * 0.1))
        assert y.arrival == pytest.approx(x.arrival / 2)
        assert y.params == x.params and y.seed == x.seed


def test_contexts_in_preparation_are_released_on_failure():
    import threading

    class Failing(FakeBackend):
        def __init__(self, clock):
            super().__init__(clock, budget=1000)
            self.discarded = []

        def prepare(self, job):
            f = cf.Future()
            if job.tag["index"] == 0:
                f.set_result(job)  # ready at once: adopted, then the round fails
            else:
                threading.Timer(0.05, f.set_result, args=(job,)).start()
            return f

        def discard(self, handle):
            self.discarded.append(handle.tag["index"])

        def step(self, k):
            raise RuntimeError("device lost")

    clock = FakeClock()
    be = Failing(clock)
    srv = serve.Server(be, clock=clock, sleep=clock.sleep, autotune=False)
    with pytest.raises(RuntimeError):
        srv.run([job(i, 0.0, 10, 10) for i in range(3)])
    assert sorted(be.discarded) == [1, 2]
