"""Served execution: a request loop over one device-resident batch.

Requests (``workloads.Job``) arrive over time.  The server keeps every
admitted job's bit planes resident on the device and advances all of them
together, one batch round (``ka_batch_step``) at a time, so that jobs that
arrive while others are running join the very next round (continuous
batching).  Admission is first come, first served against a device-memory
budget: the head of the queue is admitted once its context plus observation
buffer (``ka_job_bytes``) fits beside what is resident or being prepared;
memory comes back as finished jobs are retired.  Topologies and initial
states are prepared on host threads, each with its own CUDA stream, while the
device runs rounds; a prepared context is handed to the batch with
``ka_batch_adopt``.  Each job's result is the same as running it alone: its
random streams depend only on its own seed, sweep, class and site.

The loop reports per-job latency (arrival to completion, split into queueing
and service) and the aggregate rate of attempted site-replica moves.

    python -m paper_1710_05155_gb300.serve --jobs 200 --rate 200
"""
from __future__ import annotations

import argparse
import collections
import concurrent.futures as cf
import json
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import workloads


@dataclass
class Record:
    job: object
    index: int
    arrival: float = 0.0
    reserved: float = -1.0   # admission: memory reserved, preparation started
    admitted: float = -1.0   # context handed to the batch
    finished: float = -1.0
    job_id: int = -1
    status: str = "waiting"  # waiting, preparing, running, done, rejected, failed
    error: str = ""
    sweeps: np.ndarray | None = None
    counts: np.ndarray | None = None
    state: tuple | None = None  # (n, n0, p) at the end, when the backend reports it


def job_bytes(job, device: int = 0) -> int:
    """Device bytes a job takes from the budget: context plus observation buffer."""
    from . import ka_job_bytes, make_params

    p, _ = make_params(device=device, **job.params)
    return ka_job_bytes(p, job.sweeps, job.every)


class DeviceBackend:
    """The batch runtime of the C library on one device."""

    def __init__(self, device: int = 0, hbm_budget: int = 150 << 30, graph: bool = True,
                 prepare_threads: int = 4):
        from . import KA_BATCH_GRAPH, Batch
        import torch

        self.device = device
        self.budget = hbm_budget
        self.batch = Batch(device=device, hbm_budget=hbm_budget,
                           flags=KA_BATCH_GRAPH if graph else 0)
        self._local = threading.local()
        self._torch = torch
        self.pool = cf.ThreadPoolExecutor(max_workers=prepare_threads)

    # --- host side -------------------------------------------------------
    def job_bytes(self, job) -> int:
        return job_bytes(job, self.device)

    def _prepare(self, job):
        from . import ka_create, ka_init, make_params

        st = getattr(self._local, "stream", None)
        if st is None:
            st = self._torch.cuda.Stream(device=self.device)
            self._local.stream = st
        p, keep = make_params(device=self.device, stream=st.cuda_stream, **job.params)
        ctx = ka_create(p, keep)
        ka_init(ctx, job.seed, job.rho)
        return ctx

    def prepare(self, job) -> cf.Future:
        return self.pool.submit(self._prepare, job)

    def discard(self, handle) -> None:
        from . import ka_destroy

        ka_destroy(handle)

    # --- device side -----------------------------------------------------
    def adopt(self, handle, job) -> int:
        return self.batch.adopt(handle, job.sweeps, job.every)

    def used(self) -> int:
        return self.batch.info()["used_bytes"]

    def active(self) -> int:
        return self.batch.info()["active"]

    def autotune(self) -> int:
        return self.batch.autotune()

    def step(self, k: int) -> int:
        return self.batch.step(k)

    def finished(self, job_id: int) -> bool:
        return self.batch.poll(job_id)[1]

    def observations(self, job_id: int, replicas: int):
        return self.batch.observations(job_id, replicas)

    def state(self, job_id: int, job):
        """Final (n, n0, p) of a job, canonical [R/64, N] uint64 each."""
        return self.batch.state(job_id, job.params["replicas"] // 64, job.sites)

    def remove(self, job_id: int) -> None:
        self.batch.remove(job_id)

    def close(self) -> None:
        self.pool.shutdown(wait=True)
        self.batch.close()


@dataclass
class Server:
    """First-come-first-served admission and continuous batching over a backend.

    ``round_sweeps`` = 0 takes the batch's autotuned round length (tuned once,
    on the live batch, when ``tune_at`` jobs are first running together)."""

    backend: object
    round_sweeps: int = 0
    autotune: bool = True
    tune_at: int = 4
    max_preparing: int = 8
    keep_results: bool = False
    clock: object = time.perf_counter
    sleep: object = time.sleep
    records: list = field(default_factory=list)

    def run(self, jobs) -> dict:
        be = self.backend
        recs = [Record(j, i, float(j.arrival)) for i, j in enumerate(jobs)]
        self.records = recs
        pending = collections.deque(sorted(range(len(recs)), key=lambda i: (recs[i].arrival, i)))
        waiting: collections.deque = collections.deque()
        preparing: dict = {}
        running: dict = {}
        reserved = 0
        tuned = not self.autotune
        rounds = 0
        busy = 0.0
        max_running = 0
        t0 = self.clock()

        def now() -> float:
            return self.clock() - t0

        try:
            while pending or waiting or preparing or running:
                t = now()
                while pending and recs[pending[0]].arrival <= t:
                    waiting.append(pending.popleft())
                # admission, in arrival order, against the memory budget
                while waiting and len(preparing) < self.max_preparing:
                    r = recs[waiting[0]]
                    need = be.job_bytes(r.job)
                    if need > be.budget:
                        waiting.popleft()
                        r.status, r.error, r.finished = "rejected", "larger than the budget", now()
                        continue
                    if be.used() + reserved + need > be.budget:
                        break
                    waiting.popleft()
                    reserved += need
                    r.reserved, r.status = now(), "preparing"
                    preparing[be.prepare(r.job)] = (r, need)
                # prepared contexts join the batch before its next round
                for fut in [f for f in preparing if f.done()]:
                    r, need = preparing.pop(fut)
                    reserved -= need
                    try:
                        handle = fut.result()
                    except Exception as e:  # a job that cannot be built fails alone
                        r.status, r.error, r.finished = "failed", str(e), now()
                        continue
                    try:
                        r.job_id = be.adopt(handle, r.job)
                    except Exception as e:
                        be.discard(handle)
                        r.status, r.error, r.finished = "failed", str(e), now()
                        continue
                    r.admitted, r.status = now(), "running"
                    running[r.job_id] = r
                if running:
                    max_running = max(max_running, len(running))
                    s = self.clock()
                    if not tuned and len(running) >= self.tune_at:
                        be.autotune()
                        tuned = True
                    else:
                        be.step(self.round_sweeps)
                    busy += self.clock() - s
                    rounds += 1
                    for jid in [j for j in running if be.finished(j)]:
                        r = running.pop(jid)
                        r.finished, r.status = now(), "done"
                        if self.keep_results:
                            r.sweeps, r.counts = be.observations(jid, r.job.params["replicas"])
                            if hasattr(be, "state"):
                                r.state = be.state(jid, r.job)
                        be.remove(jid)
                elif preparing:
                    cf.wait(list(preparing), timeout=0.01, return_when=cf.FIRST_COMPLETED)
                elif pending and not waiting:
                    self.sleep(min(0.01, max(0.0, recs[pending[0]].arrival - now())))
        finally:
            # on an early exit, contexts still being prepared are never adopted:
            # release them (the batch frees its own jobs when it is closed)
            for fut in preparing:
                try:
                    be.discard(fut.result())
                except Exception:
                    pass
        return self.report(busy, rounds, max_running)

    def report(self, busy: float, rounds: int, max_running: int) -> dict:
        done = [r for r in self.records if r.status == "done"]
        out = {"jobs": len(self.records), "done": len(done),
               "rejected": sum(r.status == "rejected" for r in self.records),
               "failed": sum(r.status == "failed" for r in self.records),
               "rounds": rounds, "max_running": max_running}
        if not done:
            return out
        lat = np.array([r.finished - r.arrival for r in done])
        queue = np.array([r.admitted - r.arrival for r in done])
        service = np.array([r.finished - r.admitted for r in done])
        first = min(r.arrival for r in self.records)
        makespan = max(r.finished for r in done) - first
        work = float(sum(r.job.work for r in done))
        out.update({
            "makespan_s": makespan,
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "latency_mean_s": float(lat.mean()),
            "queue_p50_s": float(np.percentile(queue, 50)),
            "service_p50_s": float(np.percentile(service, 50)),
            "moves_per_s": work / makespan if makespan > 0 else None,
            "device_round_frac": busy / makespan if makespan > 0 else None,
            "site_replica_moves": work,
        })
        return out


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description="Serve a seeded request trace on one GPU.")
    ap.add_argument("--jobs", type=int, default=200)
    ap.add_argument("--rate", type=float, default=200.0, help="arrivals per second")
    ap.add_argument("--master", type=int, default=1)
    ap.add_argument("--sweep-scale", type=float, default=1.0,
                    help="multiply every job's sweeps (a bounded sample of the trace)")
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--round", type=int, default=0, help="sweeps per round (0: autotuned)")
    ap.add_argument("--no-graph", action="store_true", help="launch rounds directly")
    ap.add_argument("--threads", type=int, default=4, help="host threads preparing jobs")
    ap.add_argument("--load", type=float, default=0.0,
                    help="also serve the trace at this fraction of the capacity measured "
                         "by the first run (e.g. 0.7)")
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)

    def serve(rate: float) -> dict:
        jobs = workloads.scaled(workloads.request_trace(a.jobs, rate, a.master), a.sweep_scale)
        be = DeviceBackend(a.device, int(a.budget_gb * (1 << 30)), not a.no_graph, a.threads)
        try:
            rep = Server(be, round_sweeps=a.round).run(jobs)
        finally:
            be.close()
        rep.update({"rate_per_s": rate, "sweep_scale": a.sweep_scale,
                    "mean_job_moves": float(np.mean([j.work for j in jobs]))})
        return rep

    first = serve(a.rate)
    print(json.dumps({"trace": "offered", **first}))
    if a.load > 0 and first.get("moves_per_s"):
        capacity = first["moves_per_s"] / first["mean_job_moves"]  # jobs per second
        second = serve(a.load * capacity)
        print(json.dumps({"trace": f"{a.load:.2f} of capacity", "capacity_jobs_per_s": capacity,
                          **second}))


if __name__ == "__main__":
    main()
