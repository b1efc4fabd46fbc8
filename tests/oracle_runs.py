"""Whole jobs run by the oracle, for the tests of batched and served execution.

A job is what the batch API takes: a topology (cubic d, L; random regular
graph N, z, graph seed; or a caller-supplied neighbour list), m, replicas,
seed, density, a sweep target and an observation interval.  ``run_job``
runs it on the oracle alone and returns what the batch reports for it: the
sweep of every observation (0, then every multiple of the interval, then the
target), the counts at each, and the final state planes packed as the
library's canonical words.  ``run_jobs`` spreads the jobs over processes
started with spawn (the oracle is serial C; jobs are independent).
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp

import numpy as np

import oracle as O

CUBIC, RRG, GRAPH = 0, 1, 2  # the topology codes of the C ABI


def topology(params: dict) -> O.Topology:
    if params["topo"] == CUBIC:
        return O.cubic(params["d"], params["L"])
    if params["topo"] == RRG:
        return O.rrg(params["N"], params["z"], params["graph_seed"])
    return O.graph(params["N"], params["z"], np.asarray(params["nbr"], np.int32).reshape(-1))


def run_job(params: dict, sweeps: int, every: int, seed: int, rho: float):
    """(observation sweeps [n_obs], counts [n_obs, R, 4], n, n0, p [R/64, N])."""
    topo = topology(params)
    st = O.init(topo.N, params["replicas"], seed, rho)
    obs_t, obs = [0], [O.observe(st)]
    t = 0
    while t < sweeps:
        k = min(every - t % every, sweeps - t)
        O.sweeps(topo, params["m"], st, seed, k)
        t += k
        obs_t.append(t)
        obs.append(O.observe(st))
    return (np.array(obs_t, np.int64), np.stack(obs), O.pack_words(st.n), O.pack_words(st.n0),
            O.pack_words(st.p))


def _run(args):
    return run_job(*args)


def run_jobs(jobs, workers: int = 8):
    """run_job over a list of (params, sweeps, every, seed, rho), in parallel."""
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as pool:
        return list(pool.map(_run, jobs))
