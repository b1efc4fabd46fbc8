"""The benchmark's CPU legs (no GPU): the reference arm's JSON line, and how
the arms behave under several ranks or on the workloads that have no
reference arm.
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(env_extra, *args):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                          capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)


def test_reference_arm_line():
    import bench

    r = _bench({}, "--impl", "reference", "--steps", "1", "--warmup", "0", "--ref-cores", "2")
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    # the native arm's metric, unit, direction and config
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True
    assert d["config"] == bench.workload_config(1, 100)
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    cb = d["cpu_baseline"]
    # two oracle processes, each sweeping its own block of replicas
    assert cb["kind"] == "oracle" and cb["cores"] == 2 and cb["value"] == d["value"]
    assert "replicas" in cb["sample"] and "2 processes" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_without_work():
    r = _bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"},
               "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_batched_and_served_have_no_reference_arm():
    for workload in ("batched", "served"):
        r = _bench({}, "--impl", "reference", "--workload", workload)
        assert r.returncode == 0, r.stderr
        d = json.loads(r.stdout)
        assert d["impl"] == "reference" and d["unavailable"]


def test_native_line_contract():
    import bench

    clocks = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 20}
    cpu = {"value": 3.5e8, "unit": bench.UNIT, "cores": 16, "kind": "oracle", "sample": "s",
           "one_core": {"value": 3.3e7, "cores": 1}, "nproc": 16, "cpu_model": "x"}
    batched = {"value": 2e12, "plain": 6e11, "batched_over_plain": 3.3}
    kw = dict(world=1, steps=20, warmup=3, sweeps=100, ms=1900.0, value=1.69e12, achieved=2150.0,
              peak=6670.0, peak_kind="measured", traffic=1.2e7, pencil_ms=0.0155,
              pencil_iso_ms=0.0165, row_ms=0.0135, row_iso_ms=0.0145, bytes_per_launch=2.2e7,
              nq=2, path_achieved=2100.0, cpu=cpu, e2e_value=1.6e12,
              h2d=3 * 3 * 4 * 2097152 * 8, d2h=3 * 256 * 4 * 8, gpu_launches=36060,
              clocks=clocks, extra={"batched": batched, "rrg": {"value": 2.5e11}})
    line = bench.native_line(**kw)
    json.dumps(line)  # serialisable
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks", "rrg", "batched",
                "batched_over_plain"):
        assert key in line, key
    assert line["ms_per_step"] == 1900.0 / 20 and line["n_gpus"] == 1
    assert line["config"] == bench.workload_config(1, 100) and "workload" in line["config"]
    assert line["batched_over_plain"] == 3.3
    r = line["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["frac"] == 2150.0 / 6670.0
    assert r["kernel"] == "k_pencils" and r["traffic"] == 1.2e7
    assert abs(r["dram_achieved"] - 1.2e7 / 15.5e-6 / 1e9) < 1e-6
    assert abs(r["frac_of_nominal"] - 2150.0 / 7900.0) < 1e-12
    assert abs(r["k_rows"]["achieved"] - 2.2e7 / 13.5e-6 / 1e9) < 1e-6
    assert set(line["e2e"]) == {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert line["bond_attempts_per_s"] == 1.69e12 * 3
    # a kernel changed since the committed capture: no traffic, no DRAM rate
    kw["traffic"] = None
    r = bench.native_line(**kw)["roofline"]
    assert r["traffic"] is None and r["dram_achieved"] is None and r["dram_frac"] is None


def test_apportion_splits_the_region_by_isolated_shares():
    import numpy as np

    import bench

    iso = np.array([1.0, 1.5, 1.5, 0.0])
    # 8 pencil launches and 4 row launches in a 10 ms region: 3/4 of it to the pencils
    assert abs(bench._apportion(10.0, iso, (1, 2), 8) - 10.0 * 0.75 / 8) < 1e-12
    assert abs(bench._apportion(10.0, iso, (0,), 4) - 10.0 * 0.25 / 4) < 1e-12


def test_measured_traffic_needs_the_captured_source(tmp_path):
    import hashlib

    import bench

    src = tmp_path / "k.cu"
    src.write_bytes(b"kernel v1")
    prof = tmp_path / "p.md"
    digest = hashlib.sha256(b"kernel v1").hexdigest()[:16]
    prof.write_text(f"traffic_bytes_per_launch: 1234\nkernel_source_sha256_16: {digest}\n")
    assert bench.measured_traffic(str(prof), str(src)) == 1234.0
    src.write_bytes(b"kernel v2")
    assert bench.measured_traffic(str(prof), str(src)) is None


def test_oracle_blocks_time_cubic_and_graph_workloads():
    # the processes behind the CPU-baseline keys: each holds its own block of
    # replicas of a workload and sweeps (and observes) on request
    import bench

    for spec in (("cubic", (3, 8), 3), ("rrg", (512, 4, 1), 2)):
        blocks = bench.OracleBlocks(2, 4, 0.7, spec)
        try:
            assert blocks.step(2) > 0 and blocks.step(1, True) > 0
        finally:
            blocks.close()
        assert blocks.workers == 2 and blocks.n_rep == 4
