"""Seeded synthetic job mixes for batched and served execution.

The paper's own workloads are uniform random configurations at fixed density
on generated lattices and random regular graphs (sections 2 and 4), so every
input here is drawn from a seeded generator; nothing is read from disk.  This
module holds no arithmetic of the method: it only says which instances to
run (topology, size, m, density, replicas, sweeps, seeds, arrival times).

* ``instance_mix``: many independent instances of uneven size, half cubic
  (d=3, z=6, m=3, L uniform in {16, 24, 32, 48, 64, 96}) and half random
  regular graphs (z=4, m=2, N=2^u, u uniform in 12..18); rho uniform in
  [0.75, 0.88]; 64 replicas; sweeps uniform in [1000, 20000]; observed every
  100 sweeps.
* ``request_trace``: a finite stream of requests with Poisson arrivals: cubic
  L uniform over the multiples of 4 in [32, 128] or graphs N=2^u, u in
  14..20 (z=4); m in {2, 3}; rho uniform in [0.70, 0.90]; replicas in
  {64, 128, 192, 256}; sweeps log-uniform in [1e3, 1e5]; observed every
  max(1, sweeps // 100) sweeps.

Both draw from numpy's Philox generator keyed by a master seed; each job
gets its own dynamics seed and graph seed from the same stream.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CUBIC, RRG = 0, 1  # the topology codes of the C ABI (KA_CUBIC, KA_RRG)


@dataclass
class Job:
    """One simulation request: keyword arguments of ``make_params`` plus the run."""

    params: dict
    sweeps: int
    every: int
    seed: int
    rho: float
    arrival: float = 0.0  # seconds after the start of the trace
    tag: dict = field(default_factory=dict)

    @property
    def sites(self) -> int:
        p = self.params
        return p["L"] ** p["d"] if p["topo"] == CUBIC else p["N"]

    @property
    def work(self) -> int:
        """Attempted site-replica moves of the whole job (sites x replicas x sweeps)."""
        return self.sites * self.params["replicas"] * self.sweeps


def _rng(master: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=master))


def instance_mix(count: int = 512, master: int = 1, sweep_range=(1000, 20000),
                 every: int = 100) -> list[Job]:
    """Independent instances of uneven extent, all available at time 0."""
    g = _rng(master)
    jobs = []
    for i in range(count):
        rho = float(g.uniform(0.75, 0.88))
        if g.random() < 0.5:
            L = int(g.choice([16, 24, 32, 48, 64, 96]))
            params = dict(topo=CUBIC, d=3, L=L, m=3, replicas=64)
        else:
            u = int(g.integers(12, 19))
            params = dict(topo=RRG, N=1 << u, z=4, m=2, replicas=64,
                          graph_seed=int(g.integers(1, 1 << 62)))
        sweeps = int(g.integers(sweep_range[0], sweep_range[1] + 1))
        seed = int(g.integers(1, 1 << 62))
        jobs.append(Job(params, sweeps, every, seed, rho, 0.0, {"index": i}))
    return jobs


def request_trace(count: int = 2000, rate: float = 200.0, master: int = 1,
                  sweep_range=(1e3, 1e5)) -> list[Job]:
    """Requests with exponential inter-arrival times of mean 1/rate seconds."""
    g = _rng(master)
    jobs = []
    t = 0.0
    lo, hi = np.log(sweep_range[0]), np.log(sweep_range[1])
    for i in range(count):
        t += float(g.exponential(1.0 / rate))
        m = int(g.integers(2, 4))
        R = int(g.choice([64, 128, 192, 256]))
        rho = float(g.uniform(0.70, 0.90))
        if g.random() < 0.5:
            L = 4 * int(g.integers(8, 33))
            params = dict(topo=CUBIC, d=3, L=L, m=m, replicas=R)
        else:
            u = int(g.integers(14, 21))
            params = dict(topo=RRG, N=1 << u, z=4, m=m, replicas=R,
                          graph_seed=int(g.integers(1, 1 << 62)))
        sweeps = max(1, int(round(float(np.exp(g.uniform(lo, hi))))))
        every = max(1, sweeps // 100)
        seed = int(g.integers(1, 1 << 62))
        jobs.append(Job(params, sweeps, every, seed, rho, t, {"index": i}))
    return jobs


def scaled(jobs: list[Job], sweep_scale: float = 1.0, rate_scale: float = 1.0) -> list[Job]:
    """The same jobs with sweep counts (and observation intervals) and arrival
    times rescaled -- a bounded sample of a long trace."""
    out = []
    for j in jobs:
        sweeps = max(1, int(round(j.sweeps * sweep_scale)))
        every = max(1, int(round(j.every * sweep_scale)))
        out.append(Job(dict(j.params), sweeps, every, j.seed, j.rho, j.arrival / rate_scale,
                       dict(j.tag)))
    return out
