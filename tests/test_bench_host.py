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

    r = _bench({}, "--impl", "reference", "--steps", "1", "--warmup", "0")
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
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    assert "replicas" in cb["sample"]
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
    cpu = {"value": 3.5e7, "unit": bench.UNIT, "cores": 1, "kind": "oracle", "sample": "s"}
    kw = dict(world=1, steps=20, warmup=3, sweeps=100, ms=1900.0, value=1.69e12, achieved=845.0,
              peak=6670.0, peak_kind="measured copy", traffic=1.228e8, avg_launch_ms=0.053,
              isolated_launch_ms=0.057, bytes_per_launch=4.47e7, cpu=cpu, e2e_value=1.6e12,
              h2d=3 * 3 * 4 * 2097152 * 8, d2h=3 * 256 * 4 * 8, gpu_launches=36060, clocks=clocks)
    line = bench.native_line(**kw)
    json.dumps(line)  # serialisable
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert key in line, key
    assert line["ms_per_step"] == 1900.0 / 20 and line["n_gpus"] == 1
    assert line["config"] == bench.workload_config(1, 100) and "workload" in line["config"]
    r = line["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["frac"] == 845.0 / 6670.0
    assert r["traffic"] == 1.228e8
    assert abs(r["dram_achieved"] - 1.228e8 / 53e-6 / 1e9) < 1e-6
    assert abs(r["frac_of_nominal"] - 845.0 / 7900.0) < 1e-12
    assert set(line["e2e"]) == {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert line["bond_attempts_per_s"] == 1.69e12 * 3
    # a kernel changed since the committed capture: no traffic, no DRAM rate
    kw["traffic"] = None
    r = bench.native_line(**kw)["roofline"]
    assert r["traffic"] is None and r["dram_achieved"] is None and r["dram_frac"] is None
