"""The random-sequential schedule on the GPU (ka_sweep_sequential) against the oracle.

Every word of n, n0, p and every count must equal the oracle's after every sweep: cubic
lattices from coordinates (one-, two- and four-word planes; shared-memory and global-memory
chains, with exact and shared conflict stamps), the edge-gather tables, random regular and layered graphs, and sequential sweeps
after class sweeps (the sweep counter keys both streams).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_1710_05155_gb300 as K  # noqa: E402


def _same(sim, st, what):
    n, n0, p = sim.get_state()
    assert (n == O.pack_words(st.n)).all(), f"n differs {what}"
    assert (n0 == O.pack_words(st.n0)).all(), f"n0 differs {what}"
    assert (p == O.pack_words(st.p)).all(), f"p differs {what}"
    t, counts = sim.observe()
    assert t == st.t and (counts == O.observe(st)).all(), f"counts differ {what}"


def _topo(kw):
    if kw["topo"] == K.KA_CUBIC:
        return O.cubic(kw["d"], kw["L"])
    if kw["topo"] == K.KA_GRAPH:
        # the library keeps a caller's rows in ascending order; slots follow that order
        rows = np.sort(np.asarray(kw["nbr"], np.int32), axis=1)
        return O.graph(kw["N"], kw["z"], np.ascontiguousarray(rows).ravel())
    return O.rrg(kw["N"], kw["z"], kw.get("graph_seed", 1))


CASES = [
    dict(topo=K.KA_CUBIC, d=2, L=8, m=2, replicas=64),
    dict(topo=K.KA_CUBIC, d=3, L=8, m=3, replicas=128),
    dict(topo=K.KA_CUBIC, d=3, L=8, m=3, replicas=256),
    dict(topo=K.KA_CUBIC, d=1, L=32, m=0, replicas=192),
    dict(topo=K.KA_CUBIC, d=3, L=24, m=3, replicas=64),   # 13824 sites: global-memory chain
    dict(topo=K.KA_CUBIC, d=2, L=256, m=2, replicas=64),  # 65536 sites: sites share stamp words
    dict(topo=K.KA_CUBIC, d=4, L=8, m=5, replicas=64),    # z = 8
    dict(topo=K.KA_CUBIC, d=3, L=8, m=2, replicas=64, flags=K.KA_FLAG_GENERIC),
    dict(topo=K.KA_RRG, N=1000, z=3, m=1, replicas=128, graph_seed=4),
    dict(topo=K.KA_RRG, N=2048, z=4, m=2, replicas=256, graph_seed=5),
]


@pytest.mark.parametrize("kw", CASES, ids=lambda k: "-".join(f"{a}{b}" for a, b in k.items()
                                                             if a in ("d", "L", "N", "z", "m", "replicas", "flags")))
def test_sequential_matches_oracle(kw):
    topo = _topo(kw)
    sim = K.Simulation(**kw)
    sim.init(31, 0.66)
    st = O.init(topo.N, kw["replicas"], 31, 0.66)
    sweeps = 1 if topo.N > 10000 else 3
    for s in range(sweeps):
        sim.sweep_sequential(1)
        O.sequential_sweeps(topo, kw["m"], st, 31, 1)
        _same(sim, st, f"after sequential sweep {s + 1}")
    sim.close()


def test_layered_graph_sequential():
    nbr = O.layered_graph(3, 4, 4, 2)
    kw = dict(topo=K.KA_GRAPH, N=nbr.shape[0], z=6, m=3, replicas=64, nbr=nbr)
    topo = _topo(kw)
    sim = K.Simulation(**kw)
    sim.init(8, 0.7)
    st = O.init(topo.N, 64, 8, 0.7)
    sim.sweep_sequential(2)
    O.sequential_sweeps(topo, 3, st, 8, 2)
    _same(sim, st, "after two sweeps")
    sim.close()


def test_class_then_sequential_sweeps():
    kw = dict(topo=K.KA_CUBIC, d=3, L=8, m=3, replicas=64)
    topo = _topo(kw)
    sim = K.Simulation(**kw)
    sim.init(2, 0.75)
    st = O.init(topo.N, 64, 2, 0.75)
    sim.sweep(3)
    O.sweeps(topo, 3, st, 2, 3)
    sim.sweep_sequential(2)
    O.sequential_sweeps(topo, 3, st, 2, 2)
    _same(sim, st, "after 3 class sweeps and 2 sequential sweeps")
    sim.sweep(1)
    O.sweeps(topo, 3, st, 2, 1)
    _same(sim, st, "after one more class sweep")
    sim.close()


def test_sequential_before_init():
    sim = K.Simulation(topo=K.KA_CUBIC, d=2, L=8, m=2, replicas=64)
    with pytest.raises(K.KaError) as e:
        sim.sweep_sequential(1)
    assert e.value.status == K.KA_ESTATE
    sim.close()


def test_command_line_runner():
    # the runner prints one JSON line per observation and a timing line
    import json
    import subprocess
    import sys

    out = subprocess.run([sys.executable, "-m", "paper_1710_05155_gb300.cli", "--topo", "cubic",
                          "--d", "3", "--L", "16", "--m", "3", "--replicas", "64", "--rho", "0.7",
                          "--sweeps", "20", "--every", "10"],
                         capture_output=True, text=True, check=True).stdout.strip().splitlines()
    rows = [json.loads(x) for x in out]
    assert [r["sweep"] for r in rows[:-1]] == [0, 10, 20]
    assert rows[0]["C"] == pytest.approx(1.0) and rows[0]["phi"] == pytest.approx(1.0)
    assert rows[0]["chi4"] == pytest.approx(0.0, abs=1e-9)
    assert rows[-1]["sweeps"] == 20 and rows[-1]["site_replica_moves_per_s"] > 0
