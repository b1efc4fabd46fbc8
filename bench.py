"""Benchmark of the multispin Kob-Andersen sweep on one or more GB300s.

Workload (one bench step): the periodic cubic lattice d=3, L=128
(2,097,152 sites), z=6, m=3, 256 replicas (4 uint64 words per site), at the
three densities rho = 0.80, 0.85, 0.88 (one context each, Philox seed 1):
S sweeps of every context followed by one device-side observation.  The
state of one context is 192 MiB (n, n0, p); the three together, 576 MiB,
exceed the 126 MB L2, so no L2 flush is needed between steps.

Metric: attempted KA moves per second counted per site x replica
(N * R * sweeps / time), whole job.  Printed as one JSON line on rank 0,
which also carries (one GPU):

* ``roofline``: the dominant kernel (k_pencils, the group launches along y
  and z: four of the six launches of a sweep) at 32 algorithmic bytes per
  site-word-sweep, beside the whole group-kernel path;
* ``rrg``: the random regular graph workload N=2^20, z=4, m=2, 64 replicas,
  rho = 0.55 .. 0.90 (the densities as the words of one context; one context
  per density beside it), with its own roofline at 48 bytes per
  site-word-sweep;
* ``batched``: a bounded sample of the 512-instance mix run batched and with
  per-job launches on the same GPU (``batched_over_plain``);
* ``served``: a bounded sample of the request trace through the serving loop
  (moves/s, p50/p99 latency at 200 requests/s and at 0.7 of the capacity);
* ``cpu_baseline``: the CPU oracle on one core and on every host core
  (processes over replica blocks), with the core count and CPU model;
* ``small``: the small configuration (d=3, L=16, m=3, 64 replicas, 1000
  sweeps observed every 10) in full on the GPU, and the oracle on 8 host
  processes for the same whole run; the ``rrg`` key carries the oracle on the
  random regular graph as its own ``cpu_baseline``.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--sweeps S] [--impl native|reference]

--impl reference times the CPU oracle (the serial restatement of the paper
used by the tests) on every host core, on a bounded sample of the same
workload.

Two more workloads, each printing its own JSON line (one GPU):

  python bench.py --workload batched   # 512-instance mix: batched rounds vs per-job launches
  python bench.py --workload served    # Poisson request trace through the serving loop
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

D, L, M, R, SEED = 3, 128, 3, 256, 1
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e, nominal (the measured copy peak is the roofline's)
RHOS = (0.80, 0.85, 0.88)
N_SITES = L ** D
WORDS = R // 64
GROUPS = 2 * D  # group launches per sweep and plane set: (mu, parity)
BYTES_PER_SITE_WORD_SWEEP = 32  # read + write of n and p, 8 bytes each
METRIC = "attempted KA moves/s (site x replica)"
UNIT = "site-replica moves/s"
WORKLOAD = ("cubic d=3 L=128 z=6 m=3, 256 replicas, rho in {0.80,0.85,0.88}, "
            "Philox seed 1, periodic")
# random regular graphs: N=2^20, z=4, m=2, 64 replicas, rho 0.55 .. 0.90
RRG_N, RRG_Z, RRG_M, RRG_R, RRG_GRAPH_SEED = 1 << 20, 4, 2, 64, 1
RRG_RHOS = tuple(round(0.55 + 0.05 * k, 2) for k in range(8))
RRG_BYTES_PER_SITE_WORD_SWEEP = 32 + 4 * RRG_Z  # + the int32 neighbour row of every site
PROFILE_STREAM = os.path.join("profiles", "k_pencils_L128_R256.md")
SRC_STREAM = os.path.join("paper_1710_05155_gb300", "csrc", "ka_cubic_stream.cuh")
PROFILE_GRAPH = os.path.join("profiles", "k_graph_class_rrg_N2p20_R64.md")
SRC_GRAPH = os.path.join("paper_1710_05155_gb300", "csrc", "ka_sweep_graph.cu")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_traffic(profile: str, source: str):
    """DRAM bytes per launch from a committed ncu summary, or None when the
    kernel source changed since that capture (its hash is in the summary)."""
    import hashlib

    try:
        fields = {}
        for line in open(os.path.join(ROOT, profile)):
            if ":" in line:
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        digest = hashlib.sha256(open(os.path.join(ROOT, source), "rb").read()).hexdigest()[:16]
        if fields.get("kernel_source_sha256_16") != digest:
            return None
        return float(fields["traffic_bytes_per_launch"])
    except Exception:
        return None


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


# the workloads the oracle is timed on: (topology, parameters, m)
ORACLE_CUBIC = ("cubic", (D, L), M)
ORACLE_SMALL = ("cubic", (3, 16), 3)                         # d=3 L=16 m=3 (the small config)
ORACLE_RRG = ("rrg", (RRG_N, RRG_Z, RRG_GRAPH_SEED), RRG_M)  # N=2^20 z=4 m=2


def _oracle_worker(conn, r0: int, n_rep: int, rho: float, spec=ORACLE_CUBIC) -> None:
    """One oracle process: replicas r0 .. r0 + n_rep - 1 of a workload; answers
    every (k, observe) message with the seconds its k sweeps (and, if asked,
    one observation) took."""
    import oracle as O

    kind, prm, m = spec
    topo = O.cubic(*prm) if kind == "cubic" else O.rrg(*prm)
    st = O.init(topo.N, n_rep, SEED, rho, r0=r0)
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg is None:
            break
        k, obs = msg
        t0 = time.perf_counter()
        O.sweeps(topo, m, st, SEED, k)
        if obs:
            O.observe(st)
        conn.send(time.perf_counter() - t0)
    conn.close()


class OracleBlocks:
    """The CPU oracle over `workers` processes (spawned), each holding its own
    block of replicas of a workload: replicas are independent, so the blocks
    sweep in parallel.  step(k) runs k sweeps on every block and returns the
    wall time until the last block is done."""

    def __init__(self, workers: int, n_rep: int, rho: float = RHOS[0], spec=ORACLE_CUBIC):
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for w in range(workers):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, w * n_rep, n_rep, rho, spec),
                            daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            assert c.recv() == "ready"
        self.workers, self.n_rep = workers, n_rep

    def step(self, k: int, observe: bool = False) -> float:
        t0 = time.perf_counter()
        for c in self.conns:
            c.send((k, observe))
        for c in self.conns:
            c.recv()
        return time.perf_counter() - t0

    def close(self) -> None:
        for c in self.conns:
            c.send(None)
        for p in self.procs:
            p.join(timeout=30)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(n_rep: int = 8, sweeps: int = 4) -> dict:
    """The oracle on one core and on every host core (n_rep replicas per
    process, `sweeps` sweeps after an untimed initial state)."""
    cores = host_cores()
    out = {"unit": UNIT, "kind": "oracle", "cpu_model": cpu_model(), "nproc": cores}
    for key, workers in (("one_core", 1), ("all_cores", cores)):
        blocks = OracleBlocks(workers, n_rep)
        dt = blocks.step(sweeps)
        blocks.close()
        out[key] = {"value": N_SITES * n_rep * workers * sweeps / dt, "cores": workers,
                    "seconds": dt,
                    "sample": f"L=128 d=3 m=3 rho=0.80, {n_rep * workers} of 256 replicas "
                              f"({n_rep} per process), {sweeps} sweeps"}
    out["value"] = out["all_cores"]["value"]
    out["cores"] = cores
    out["sample"] = out["all_cores"]["sample"] + "; one core: " + out["one_core"]["sample"]
    return out


def workload_config(world: int, sweeps: int) -> dict:
    """The "config" of the cubic bench line (both arms)."""
    return {"workload": WORKLOAD, "L": L, "d": D, "m": M, "replicas": R, "rho": list(RHOS),
            "sweeps_per_step": sweeps, "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (576 MiB of state per GPU)"}


def run_reference(args, rank: int) -> None:
    """The oracle on every host core, each step one sweep of a block of 4
    replicas per process (rank 0 only; other ranks exit without work)."""
    if rank != 0:
        return
    cores = args.ref_cores or host_cores()
    n_rep = 4
    blocks = OracleBlocks(cores, n_rep)
    for _ in range(args.warmup):
        blocks.step(1)
    dt = sum(blocks.step(1) for _ in range(args.steps))
    blocks.close()
    value = N_SITES * n_rep * cores * args.steps / dt
    sample = (f"oracle on {cores} processes ({cpu_model()}): L=128 d=3 m=3 rho=0.80, "
              f"{n_rep * cores} of 256 replicas ({n_rep} per process), 1 sweep per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": workload_config(args.gpus, args.sweeps),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def max_over_ranks(x: float, dist=None, device: str = "cpu") -> float:
    """The largest x over all ranks (x itself on one process): the job's time
    is its slowest rank's."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_seed(rank: int) -> int:
    """Dynamics seed of a rank: every rank simulates its own replicas (weak scaling)."""
    return SEED + 1000 * rank


def _apportion(region_ms: float, iso_ms: np.ndarray, dirs, launches: int) -> float:
    """Average chained launch time (ms) of the launches of directions `dirs`:
    the timed region split by the kernels' shares of the same launches timed
    one by one (events around each)."""
    share = float(iso_ms[list(dirs)].sum() / iso_ms.sum())
    return region_ms * share / launches


def run_rrg(dev: int, stream, sweeps: int) -> dict:
    """Random regular graph N=2^20, z=4, m=2, 64 replicas at each of
    rho = 0.55 .. 0.90, `sweeps` sweeps per density (initial states untimed),
    CUDA events around the sweeps: first one 64-replica context per density
    (and one density's launches timed one by one), then the eight densities
    as the eight words of one 512-replica context (the key's value)."""
    import torch

    import paper_1710_05155_gb300 as K

    t0 = time.perf_counter()
    sim = K.Simulation(topo=K.KA_RRG, N=RRG_N, z=RRG_Z, m=RRG_M, replicas=RRG_R,
                       graph_seed=RRG_GRAPH_SEED, device=dev, stream=stream)
    build_s = time.perf_counter() - t0
    nclass = sim.info["nclass"]
    total_ms = 0.0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rho in RRG_RHOS:
        sim.init(SEED, rho)
        K.ka_sweep(sim.ctx, 2)  # warm-up
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        K.ka_sweep(sim.ctx, sweeps)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        total_ms += ev0.elapsed_time(ev1)
    moves = RRG_N * RRG_R * sweeps * len(RRG_RHOS)
    value = moves / (total_ms / 1000.0)
    K.ka_profile_enable(sim.ctx, True)
    K.ka_sweep(sim.ctx, sweeps)
    iso_ms, iso_n = K.ka_profile_read_dirs(sim.ctx)
    K.ka_profile_enable(sim.ctx, False)
    # The same work with the densities packed: the eight densities' 64-replica
    # initial states (one seed each, drawn by the context above) loaded as the
    # eight words of one 512-replica context, so that a gathered 32-byte
    # sector carries four densities' words instead of one (four words per
    # site and plane).  Same sites, replicas per density and sweeps; each
    # density keeps its own random stream (its word index in the gates).
    words = []
    for k, rho in enumerate(RRG_RHOS):
        sim.init(SEED + k, rho)
        words.append(sim.get_state()[0][0])
    sim.close()
    n8 = np.ascontiguousarray(np.stack(words))
    packed = K.Simulation(topo=K.KA_RRG, N=RRG_N, z=RRG_Z, m=RRG_M, replicas=64 * len(RRG_RHOS),
                          graph_seed=RRG_GRAPH_SEED, device=dev, stream=stream)
    packed.set_state(n8, n8.copy(), np.full_like(n8, np.uint64(0xFFFFFFFFFFFFFFFF)), 0, SEED)
    K.ka_sweep(packed.ctx, 2)  # warm-up
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    K.ka_sweep(packed.ctx, sweeps)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    packed_ms = ev0.elapsed_time(ev1)
    packed_words = packed.info["plane_words"]
    packed.close()
    packed_value = RRG_N * 64 * len(RRG_RHOS) * sweeps / (packed_ms / 1000.0)
    launches = nclass * sweeps * len(RRG_RHOS)
    avg_ms = total_ms / launches  # the class launches are the whole timed region
    sweep_ms = total_ms / (sweeps * len(RRG_RHOS))
    bytes_per_sweep = RRG_BYTES_PER_SITE_WORD_SWEEP * RRG_N * (RRG_R // 64)
    achieved = bytes_per_sweep / (sweep_ms / 1000.0) / 1e9
    peak, peak_kind = _peaks()
    traffic = measured_traffic(PROFILE_GRAPH, SRC_GRAPH)
    # packed: one sweep moves all eight densities' words
    p_launches = nclass * sweeps
    p_achieved = bytes_per_sweep * len(RRG_RHOS) * sweeps / (packed_ms / 1000.0) / 1e9
    return {
        "metric": METRIC, "value": packed_value, "unit": UNIT,
        "workload": f"RRG N=2^20 z=4 m=2, graph seed 1, rho {RRG_RHOS[0]}..{RRG_RHOS[-1]} "
                    f"(8 densities, 64 replicas each, initial state of density k from seed "
                    f"1 + k), {sweeps} sweeps; the densities run as the eight replica words "
                    f"of one 512-replica context (four words per site and plane, dynamics "
                    f"seed 1)",
        "ms_per_sweep": packed_ms / sweeps, "classes_per_sweep": nclass,
        "graph_build_s": build_s,
        "roofline": {"bound": "hbm", "achieved": p_achieved, "peak": peak, "unit": "GB/s",
                     "frac": p_achieved / peak, "traffic": None, "kernel": "k_graph_class",
                     "peak_kind": peak_kind, "plane_words": packed_words,
                     "bytes_per_site_word_sweep": RRG_BYTES_PER_SITE_WORD_SWEEP,
                     "avg_launch_us": 1000.0 * packed_ms / p_launches},
        "separate_contexts": {
            "value": value, "unit": UNIT, "ms_per_sweep": sweep_ms,
            "workload": "one 64-replica context per density (one word per site), initial "
                        "states from seed 1",
            "roofline": {"achieved": achieved, "frac": achieved / peak, "traffic": traffic,
                         "avg_launch_us": 1000.0 * avg_ms,
                         "avg_launch_us_isolated":
                             1000.0 * float(iso_ms.sum() / max(iso_n.sum(), 1))}},
        "gpu_launches": launches + p_launches,
    }


def rrg_oracle_baseline(n_rep: int = 8, sweeps: int = 2) -> dict:
    """The oracle on every host core for the random regular graph workload
    (N=2^20, z=4, m=2, rho=0.55): n_rep replicas per process, `sweeps` sweeps."""
    cores = host_cores()
    blocks = OracleBlocks(min(cores, 8), n_rep, RRG_RHOS[0], ORACLE_RRG)  # 64 replicas at most
    dt = blocks.step(sweeps)
    blocks.close()
    nrep = n_rep * blocks.workers
    return {"value": RRG_N * nrep * sweeps / dt, "unit": UNIT, "kind": "oracle",
            "cores": blocks.workers, "cpu_model": cpu_model(),
            "sample": f"RRG N=2^20 z=4 m=2 rho=0.55, {nrep} of 64 replicas ({n_rep} per process), "
                      f"{sweeps} sweeps after an untimed initial state"}


def run_small(dev: int, stream, oracle: bool) -> dict:
    """The small configuration in full: d=3, L=16, m=3, rho=0.70, 64 replicas,
    1000 sweeps observed every 10 sweeps (101 observations), seed 1 -- on the
    GPU (counts into device memory, one context) and, when asked, the oracle
    on 8 host processes of 8 replicas each, the same sweeps and observations."""
    import torch

    import paper_1710_05155_gb300 as K

    Ls, sweeps, every, rho = 16, 1000, 10, 0.70
    sim = K.Simulation(topo=K.KA_CUBIC, d=3, L=Ls, m=3, replicas=64, device=dev, stream=stream)
    counts = torch.zeros((sweeps // every + 1, 64, 4), dtype=torch.int64, device=f"cuda:{dev}")
    runs = []
    for _ in range(3):  # the first run warms up
        sim.init(SEED, rho)
        torch.cuda.synchronize(dev)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        K.ka_observe_device(sim.ctx, counts[0].data_ptr())
        for k in range(1, sweeps // every + 1):
            K.ka_sweep(sim.ctx, every)
            K.ka_observe_device(sim.ctx, counts[k].data_ptr())
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        runs.append(ev0.elapsed_time(ev1))
    kernel = sim.info["kernel"]
    sim.close()
    ms = min(runs[1:])
    moves = Ls ** 3 * 64 * sweeps
    out = {"value": moves / (ms / 1000.0), "unit": UNIT, "ms": ms, "kernel": kernel,
           "workload": "cubic d=3 L=16 z=6 m=3, rho=0.70, 64 replicas, 1000 sweeps, "
                       "observed every 10 sweeps, seed 1"}
    if oracle:
        blocks = OracleBlocks(8, 8, rho, ORACLE_SMALL)
        dt = blocks.step(0, True)
        for _ in range(sweeps // every):
            dt += blocks.step(every, True)
        blocks.close()
        out["cpu_baseline"] = {"value": moves / dt, "unit": UNIT, "kind": "oracle", "cores": 8,
                               "cpu_model": cpu_model(), "seconds": dt,
                               "sample": "the whole run: 64 replicas in 8 processes of 8, "
                                         "1000 sweeps and 101 observations"}
    return out


def run_batched_sample(dev: int, jobs_n: int, scale: float) -> dict:
    """A bounded sample of the 512-instance mix, batched and per-job plain."""
    import paper_1710_05155_gb300 as K
    from paper_1710_05155_gb300 import workloads

    jobs = workloads.instance_mix(512, master=1)[:jobs_n]
    jobs = [workloads.Job(j.params, max(1, round(j.sweeps * scale)), j.every, j.seed, j.rho)
            for j in jobs]
    moves = float(sum(j.work for j in jobs))
    t0 = time.perf_counter()
    ms_b, rounds, k = _run_batch(jobs, K.KA_BATCH_GRAPH, dev, 0)
    own = _run_batch.own_tiles
    ms_p, _, _ = _run_batch(jobs, K.KA_BATCH_PLAIN, dev, k)
    return {"value": moves / (ms_b / 1000.0), "unit": UNIT, "own_launch_tiles": own,
            "workload": f"the first {jobs_n} of the 512-instance mix (cubic d=3 m=3 L in "
                        f"{{16..96}} or RRG z=4 m=2 N=2^12..2^18, R=64), sweeps x {scale}",
            "plain": moves / (ms_p / 1000.0), "ms": ms_b, "plain_ms": ms_p,
            "batched_over_plain": ms_p / ms_b, "round_sweeps": k, "rounds": rounds,
            "wall_s": time.perf_counter() - t0}


def native_line(*, world, steps, warmup, sweeps, ms, value, achieved, peak, peak_kind, traffic,
                pencil_ms, pencil_iso_ms, row_ms, row_iso_ms, bytes_per_launch, nq,
                path_achieved, cpu, e2e_value, h2d, d2h, gpu_launches, clocks,
                extra=None) -> dict:
    """The JSON line of the native cubic arm from its measured numbers (times
    in ms; rates in GB/s)."""
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(world, sweeps),
        "roofline": {
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
            "kernel": "k_pencils", "peak_kind": peak_kind,
            "bytes_per_launch": bytes_per_launch, "planes_per_launch": nq,
            "avg_launch_us": 1000.0 * pencil_ms,
            "avg_launch_us_isolated": 1000.0 * pencil_iso_ms,
            # the DRAM bytes the kernel moves per launch (the committed ncu
            # capture) over the same launch time
            "dram_achieved": traffic / (pencil_ms / 1000.0) / 1e9 if traffic else None,
            "dram_frac": traffic / (pencil_ms / 1000.0) / 1e9 / peak if traffic else None,
            "k_rows": {"avg_launch_us": 1000.0 * row_ms,
                       "avg_launch_us_isolated": 1000.0 * row_iso_ms,
                       "achieved": bytes_per_launch / (row_ms / 1000.0) / 1e9},
            # every group launch and observation of the timed region together
            "path_achieved": path_achieved, "path_frac": path_achieved / peak,
        },
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        # a sweep attempts each of the N z / 2 bonds once per replica: z / 2 = d
        # bond attempts per site-replica move
        "bond_attempts_per_s": value * D,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    line.update(extra or {})
    if "batched" in line:
        line["batched_over_plain"] = line["batched"]["batched_over_plain"]
    return line


def run_served_sample(jobs_n: int, scale: float, round_sweeps: int = 0) -> dict:
    """A bounded sample of the request trace through the serving loop: the
    first jobs_n requests at 200/s, then the same requests at 0.7 of the
    capacity (jobs/s) the first run measured."""
    import paper_1710_05155_gb300.serve as Sv
    from paper_1710_05155_gb300 import workloads

    budget = int(150 * (1 << 30))

    def serve(rate):
        jobs = workloads.scaled(workloads.request_trace(jobs_n, rate, 1), scale)
        be = Sv.DeviceBackend(0, budget, True, 4)
        try:
            rep = Sv.Server(be, round_sweeps=round_sweeps).run(jobs)
        finally:
            be.close()
        rep["rate_per_s"] = rate
        rep["mean_job_moves"] = float(np.mean([j.work for j in jobs]))
        return rep

    first = serve(200.0)
    capacity = first["moves_per_s"] / first["mean_job_moves"]
    second = serve(0.7 * capacity)
    keep = ("moves_per_s", "latency_p50_s", "latency_p99_s", "queue_p50_s", "service_p50_s",
            "makespan_s", "done", "max_running", "rate_per_s")
    return {"value": first["moves_per_s"], "unit": UNIT,
            "workload": f"the first {jobs_n} requests of the Poisson trace (200/s; cubic L in "
                        f"4*[8..32] or RRG z=4 N=2^14..2^20, m in {{2,3}}, R in {{64..256}}), "
                        f"sweeps x {scale}, 150 GB budget",
            "offered_200_per_s": {k: first[k] for k in keep},
            "at_0.7_capacity": {"capacity_jobs_per_s": capacity, **{k: second[k] for k in keep}}}


def run_native(args, rank: int, world: int) -> None:
    import torch

    import paper_1710_05155_gb300 as K

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", dev))
    stream = torch.cuda.current_stream(dev)
    S = args.sweeps

    # one context per density; weak scaling: every rank runs its own replicas
    sims = []
    for k, rho in enumerate(RHOS):
        sim = K.Simulation(topo=K.KA_CUBIC, d=D, L=L, m=M, replicas=R, device=dev, stream=stream)
        sim.init(rank_seed(rank), rho)
        sims.append(sim)
    counts_dev = [torch.zeros((R, 4), dtype=torch.int64, device=f"cuda:{dev}") for _ in sims]
    info = sims[0].info
    P, nq = info["planes"], info["planes_per_launch"]
    sets = -(-P // nq)  # launches per group and sweep
    sweep_launches_per_step = len(sims) * sets * S * GROUPS
    launches_per_step = sweep_launches_per_step + len(sims)  # + one observation each

    def step():
        for sim, cd in zip(sims, counts_dev):
            K.ka_sweep(sim.ctx, S)
            K.ka_observe_device(sim.ctx, cd.data_ptr())

    # Device warm-up, untimed: on a GPU that has just come out of idle the
    # first seconds of sweeps ran ~15 % slower than the same sweeps later in
    # the same process (measured: the first process on a fresh box, any
    # number of warm-up steps), so the contexts sweep for at least
    # args.settle seconds before the warm-up steps proper.
    t_settle = time.perf_counter()
    while time.perf_counter() - t_settle < args.settle:
        step()
        torch.cuda.synchronize(dev)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    local_ms = ms  # this GPU's timed region (the job's time is the max over ranks)
    clk = clocks.stop()
    if dist:
        ms = max_over_ranks(ms, dist, f"cuda:{dev}")
        dist.barrier()
    moves = N_SITES * R * S * len(sims) * args.steps * world
    value = moves / (ms / 1000.0)

    # Roofline.  The group launches are the timed region (one observation per
    # context and step aside).  The same launches of one step, timed one by
    # one with events around each (ka_profile_read_dirs, by direction), give
    # each kernel's share of the region: k_rows runs the groups along x,
    # k_pencils those along y and z (two thirds of the launches).  A launch
    # covers nq planes of one group: 32 bytes per site-word-sweep / 6 groups.
    iso_ms, iso_n = np.zeros(4), np.zeros(4, np.int64)
    for sim in sims:
        K.ka_profile_enable(sim.ctx, True)
        K.ka_sweep(sim.ctx, S)
        a_ms, a_n = K.ka_profile_read_dirs(sim.ctx)
        K.ka_profile_enable(sim.ctx, False)
        iso_ms += a_ms
        iso_n += a_n
    region_launches = sweep_launches_per_step * args.steps
    pencil_launches = region_launches * 2 // 3
    row_launches = region_launches - pencil_launches
    bytes_per_launch = BYTES_PER_SITE_WORD_SWEEP * N_SITES * nq / GROUPS
    pencil_ms = _apportion(local_ms, iso_ms, (1, 2), pencil_launches)
    row_ms = _apportion(local_ms, iso_ms, (0,), row_launches)
    achieved = bytes_per_launch / (pencil_ms / 1000.0) / 1e9
    path_achieved = BYTES_PER_SITE_WORD_SWEEP * N_SITES * WORDS * S * len(sims) * args.steps / (
        local_ms / 1000.0) / 1e9
    peak, peak_kind = _peaks()
    traffic = measured_traffic(PROFILE_STREAM, SRC_STREAM)

    # end to end through the C ABI: initial state from pinned host memory,
    # S sweeps, counts back to the host, for every context.  Each context runs
    # on its own stream: its state is uploaded (ka_set_state_async) while the
    # previous context sweeps, and its sweeps wait for the previous context's
    # to finish, so that one context at a time holds the L2.
    host_init = []
    for sim in sims:
        n, n0, p = sim.get_state()
        pinned = []
        for a in (n, n0, p):
            t = torch.empty(a.shape, dtype=torch.int64, pin_memory=True)
            t.numpy().view(np.uint64)[...] = a
            pinned.append(t.numpy().view(np.uint64))
        host_init.append(pinned)
    out = [np.zeros((R, 4), np.int64) for _ in sims]
    e2e_steps = max(2, min(args.steps, 5))

    e2e_streams = [torch.cuda.Stream(dev) for _ in sims]
    e2e_sims = [K.Simulation(topo=K.KA_CUBIC, d=D, L=L, m=M, replicas=R, device=dev, stream=st)
                for st in e2e_streams]

    def e2e_step():
        prev = None
        for sim, st, hs in zip(e2e_sims, e2e_streams, host_init):
            K.ka_set_state_async(sim.ctx, hs[0], hs[1], hs[2], 0, SEED)
            if prev is not None:
                st.wait_event(prev)
            K.ka_sweep(sim.ctx, S)
            prev = torch.cuda.Event()
            prev.record(st)
        for sim, o in zip(e2e_sims, out):
            K.ka_observe(sim.ctx, o)

    e2e_step()
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    if dist:
        e2e_s = max_over_ranks(e2e_s, dist, f"cuda:{dev}")
    e2e_value = N_SITES * R * S * len(sims) * e2e_steps * world / e2e_s
    h2d = len(sims) * 3 * WORDS * N_SITES * 8
    d2h = len(sims) * R * 4 * 8
    for sim in sims + e2e_sims:
        sim.close()

    if rank == 0:
        extra = {}
        if world == 1:
            if not args.no_rrg:
                extra["rrg"] = run_rrg(dev, stream, args.rrg_sweeps)
                if not args.no_cpu_baseline:
                    extra["rrg"]["cpu_baseline"] = rrg_oracle_baseline()
            if not args.no_small:
                extra["small"] = run_small(dev, stream, not args.no_cpu_baseline)
            if not args.no_batched:
                extra["batched"] = run_batched_sample(dev, args.batched_jobs, args.batched_scale)
            if not args.no_served:
                extra["served"] = run_served_sample(args.served_jobs, args.batched_scale)
            if not args.no_cpu_baseline:
                extra["cpu_baseline"] = cpu_baseline()
        line = native_line(
            world=world, steps=args.steps, warmup=args.warmup, sweeps=S, ms=ms, value=value,
            achieved=achieved, peak=peak, peak_kind=peak_kind, traffic=traffic,
            pencil_ms=pencil_ms, pencil_iso_ms=float(iso_ms[1:3].sum() / iso_n[1:3].sum()),
            row_ms=row_ms, row_iso_ms=float(iso_ms[0] / iso_n[0]),
            bytes_per_launch=bytes_per_launch, nq=nq, path_achieved=path_achieved,
            cpu=extra.pop("cpu_baseline", None), e2e_value=e2e_value, h2d=h2d, d2h=d2h,
            gpu_launches=launches_per_step * args.steps, clocks=clk, extra=extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _run_batch(jobs, flags, dev, k):
    """Run every job to its target in one batch; returns (device ms, rounds, round length)."""
    import torch

    import paper_1710_05155_gb300 as K

    stream = torch.cuda.Stream(device=dev)
    b = K.Batch(device=dev, stream=stream.cuda_stream, flags=flags)
    for j in jobs:
        b.add(j.sweeps, j.every, j.seed, j.rho, **j.params)
    torch.cuda.synchronize(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    rounds = 0
    if k == 0 and not (flags & K.KA_BATCH_PLAIN):
        k = b.autotune()  # times real rounds of this batch: part of the timed work
    own_tiles = b.tuning()[1]
    while b.info()["active"]:
        b.step(k or 16)
        rounds += 1
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms = ev0.elapsed_time(ev1)
    b.close()
    _run_batch.own_tiles = own_tiles
    return ms, rounds, k


def run_batched(args) -> None:
    """Instance mix: the same jobs batched (graph-captured rounds) and with
    per-job launches (one ka_sweep loop per instance on one stream)."""
    import torch

    import paper_1710_05155_gb300 as K
    from paper_1710_05155_gb300 import workloads

    dev = 0
    torch.cuda.set_device(dev)
    jobs = workloads.instance_mix(args.jobs, master=1)
    jobs = [workloads.Job(j.params, max(1, round(j.sweeps * args.sweep_scale)), j.every, j.seed,
                          j.rho) for j in jobs]
    moves = float(sum(j.work for j in jobs))
    clocks = ClockSampler(dev)
    clocks.start()
    ms_b, rounds, k = _run_batch(jobs, K.KA_BATCH_GRAPH, dev, args.round)
    own = _run_batch.own_tiles
    ms_p, _, _ = _run_batch(jobs, K.KA_BATCH_PLAIN, dev, k)
    _run_batch.own_tiles = own
    clk = clocks.stop()
    value = moves / (ms_b / 1000.0)
    line = {
        "metric": METRIC + ", batched vs plain", "value": value, "unit": UNIT, "n_gpus": 1,
        "steps": 1, "warmup": 0, "ms_per_step": ms_b, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": f"{args.jobs} instances: cubic d=3 m=3 L in {{16..96}} or RRG "
                               f"z=4 m=2 N=2^12..2^18, R=64, rho U[0.75,0.88], sweeps "
                               f"U[1000,20000] x {args.sweep_scale}, observe every 100",
                   "round_sweeps": k, "own_launch_tiles": _run_batch.own_tiles,
                   "rounds": rounds, "site_replica_moves": moves},
        "plain": {"value": moves / (ms_p / 1000.0), "unit": UNIT, "ms": ms_p},
        "batched_over_plain": ms_p / ms_b,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_served(args) -> None:
    """Request trace through the serving loop, then again at a fraction of the
    capacity the first run measured."""
    import paper_1710_05155_gb300.serve as S
    from paper_1710_05155_gb300 import workloads

    budget = int(150 * (1 << 30))

    def serve(rate):
        jobs = workloads.scaled(workloads.request_trace(args.jobs, rate, 1), args.sweep_scale)
        be = S.DeviceBackend(0, budget, True, 4)
        try:
            rep = S.Server(be, round_sweeps=args.round).run(jobs)
        finally:
            be.close()
        rep["rate_per_s"] = rate
        rep["mean_job_moves"] = float(np.mean([j.work for j in jobs]))
        return rep

    clocks = ClockSampler(0)
    clocks.start()
    first = serve(200.0)
    capacity = first["moves_per_s"] / first["mean_job_moves"]
    second = serve(0.7 * capacity)
    clk = clocks.stop()
    line = {
        "metric": METRIC + ", served", "value": first["moves_per_s"], "unit": UNIT, "n_gpus": 1,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic",
        "config": {"workload": f"{args.jobs} Poisson requests at 200/s: cubic L in 4*[8..32] or "
                               f"RRG z=4 N=2^14..2^20, m in {{2,3}}, R in {{64..256}}, "
                               f"sweeps log-U[1e3,1e5] x {args.sweep_scale}, 150 GB budget"},
        "offered_200_per_s": first,
        "at_0.7_capacity": {"capacity_jobs_per_s": capacity, **second},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--sweeps", type=int, default=100, help="sweeps per context per step")
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--settle", type=float, default=3.0,
                    help="seconds of untimed sweeps before the warm-up steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-cores", type=int, default=0,
                    help="reference arm: oracle processes (0: every host core)")
    ap.add_argument("--no-rrg", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-served", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--served-jobs", type=int, default=40,
                    help="served sample of the main line: requests of the trace")
    ap.add_argument("--rrg-sweeps", type=int, default=100, help="rrg: sweeps per density")
    ap.add_argument("--batched-jobs", type=int, default=512,
                    help="batched sample of the main line: instances of the mix")
    ap.add_argument("--batched-scale", type=float, default=0.05,
                    help="batched sample of the main line: fraction of each job's sweeps")
    ap.add_argument("--workload", choices=["cubic", "batched", "served"], default="cubic")
    ap.add_argument("--jobs", type=int, default=0, help="instances (batched: 512, served: 100)")
    ap.add_argument("--sweep-scale", type=float, default=0.05,
                    help="batched/served: fraction of each job's sweeps that is run")
    ap.add_argument("--round", type=int, default=0, help="batched/served: sweeps per round "
                                                         "(0: autotuned)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.workload != "cubic":
        if args.impl == "reference" or world > 1:
            if rank == 0:
                print(json.dumps({"impl": args.impl, "unavailable":
                                  "the batched and served workloads run on one GPU, natively"}))
            return
        args.jobs = args.jobs or (512 if args.workload == "batched" else 100)
        (run_batched if args.workload == "batched" else run_served)(args)
    elif args.impl == "reference":
        run_reference(args, rank)
    else:
        run_native(args, rank, world)


if __name__ == "__main__":
    main()
