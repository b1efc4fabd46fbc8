"""Run one simulation from the command line and print its observables as JSON.

    python -m paper_1710_05155_gb300.cli --topo cubic --d 3 --L 16 --m 3 --replicas 64 \
        --rho 0.7 --sweeps 1000 --every 10
    python -m paper_1710_05155_gb300.cli --topo rrg --N 1048576 --z 4 --m 2 --rho 0.8 --sweeps 100

One JSON line per observation: the sweep, the persistence phi(t), the
density autocorrelation C(t) averaged over replicas and the dynamical
susceptibility chi_4(t) (sections 2.2 and 3.3 of the paper; see
``correlation``, ``persistence`` and ``susceptibility``), the mean particle count,
and a final line with the device time of the sweeps.
"""
from __future__ import annotations

import argparse
import json
import time

from . import KA_CUBIC, KA_RRG, Simulation, correlation, ka_info, persistence, susceptibility


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--topo", choices=["cubic", "rrg"], default="cubic")
    ap.add_argument("--d", type=int, default=3)
    ap.add_argument("--L", type=int, default=16)
    ap.add_argument("--N", type=int, default=4096)
    ap.add_argument("--z", type=int, default=4)
    ap.add_argument("--m", type=int, default=3)
    ap.add_argument("--replicas", type=int, default=64)
    ap.add_argument("--graph-seed", type=int, default=1)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--rho", type=float, default=0.7)
    ap.add_argument("--sweeps", type=int, default=100)
    ap.add_argument("--every", type=int, default=0, help="observe every this many sweeps "
                                                          "(0: only at the start and the end)")
    ap.add_argument("--device", type=int, default=0)
    a = ap.parse_args(argv)

    import torch

    if a.topo == "cubic":
        sim = Simulation(device=a.device, topo=KA_CUBIC, d=a.d, L=a.L, m=a.m, replicas=a.replicas)
    else:
        sim = Simulation(device=a.device, topo=KA_RRG, N=a.N, z=a.z, m=a.m, replicas=a.replicas,
                         graph_seed=a.graph_seed)
    sim.init(a.seed, a.rho)
    info = ka_info(sim.ctx)
    N, K = info["N"], info["K"]
    stream = sim.stream
    sweep_ms = 0.0

    def emit(t, counts):
        print(json.dumps({"sweep": int(t), "phi": persistence(counts, K),
                          "C": correlation(counts, N, K), "chi4": susceptibility(counts, N, K),
                          "particles": float(counts[:, 0].mean())}), flush=True)

    t, counts = sim.observe()
    emit(t, counts)
    every = a.every if a.every > 0 else max(a.sweeps, 1)
    t0 = time.perf_counter()
    while t < a.sweeps:
        n = min(every - t % every, a.sweeps - t)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.sweep(n)
        e1.record(stream)
        e1.synchronize()
        sweep_ms += e0.elapsed_time(e1)
        t, counts = sim.observe()
        emit(t, counts)
    print(json.dumps({"sweeps": a.sweeps, "N": N, "replicas": a.replicas,
                      "sweep_device_ms": sweep_ms, "wall_s": time.perf_counter() - t0,
                      "site_replica_moves_per_s": N * a.replicas * a.sweeps / (sweep_ms / 1e3)
                      if sweep_ms > 0 else None}), flush=True)
    sim.close()


if __name__ == "__main__":
    main()
