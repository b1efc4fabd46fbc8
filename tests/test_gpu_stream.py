"""GPU parity of the group kernels of three-dimensional lattices (L % 4 == 0, L <= 128).

These kernels run every sweep of three-dimensional lattices of those sides
(32, 64 and 128 with the side fixed at compile time, every other side with the
geometry read at run time: partial warps of rows, blocks of fewer pencils and
several layers per warp, chunks of unequal length along the pencils);
planes hold one 64-replica word per site in split-row order (even x, then odd
x, in every row), which get_state / set_state translate.  Integer work, so
every compared word must equal the oracle's.  The cases cover one to five
planes (R = 64 .. 320), every activation number m = 0 .. 5, the degenerate
densities, both kernels (rows for mu = 0; pencils walked in chunks along mu
for mu > 0, including the periodic x neighbours of the first and last pencils
of a half-row and the chunk that wraps around), and the benchmark's own
configuration (L = 128, 256 replicas, the three densities, 20 sweeps) on
sampled replicas.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1710_05155_gb300 as K  # noqa: E402


def _assert_same(sim, st, what=""):
    n, n0, p = sim.get_state()
    assert (n == O.pack_words(st.n)).all(), f"n differs {what}"
    assert (n0 == O.pack_words(st.n0)).all(), f"n0 differs {what}"
    assert (p == O.pack_words(st.p)).all(), f"p differs {what}"


def _run(L, m, R, seed, rho, sweeps, per_call=1):
    topo = O.cubic(3, L)
    sim = K.Simulation(topo=K.KA_CUBIC, d=3, L=L, m=m, replicas=R)
    assert sim.info["kernel"] == 3 and sim.info["plane_words"] == 1 and sim.info["planes"] == R // 64
    sim.init(seed, rho)
    st = O.init(topo.N, R, seed, rho)
    _assert_same(sim, st, "after init")
    done = 0
    while done < sweeps:
        k = min(per_call, sweeps - done)
        sim.sweep(k)
        O.sweeps(topo, m, st, seed, k)
        done += k
        _assert_same(sim, st, f"after sweep {done}")
        t, counts = sim.observe()
        assert t == done and (counts == O.observe(st)).all()
    sim.close()


@pytest.mark.parametrize("m,R,rho", [(3, 64, 0.7), (0, 128, 0.5), (2, 192, 0.8), (5, 256, 0.88),
                                     (4, 320, 0.3), (1, 64, 0.95)])
def test_l32_every_sweep(m, R, rho):
    _run(32, m, R, seed=5 + m, rho=rho, sweeps=4)


@pytest.mark.parametrize("rho", [0.0, 1.0, 1.0 / 32768, 32767.0 / 32768])
def test_l32_degenerate_densities(rho):
    _run(32, 3, 64, seed=2, rho=rho, sweeps=2)


def test_l32_sweeps_in_one_call():
    # several sweeps per call: the launches of one call chain on the stream
    _run(32, 3, 128, seed=8, rho=0.75, sweeps=6, per_call=3)


def test_l64_every_sweep():
    _run(64, 3, 128, seed=11, rho=0.8, sweeps=2)


@pytest.mark.parametrize("L,m,R,sweeps", [
    (4, 3, 128, 4), (8, 2, 128, 4), (12, 3, 192, 4), (16, 3, 192, 4), (20, 1, 128, 4),
    (24, 4, 256, 3), (28, 3, 128, 3), (36, 3, 128, 2), (40, 5, 128, 2), (48, 3, 320, 2),
    (52, 0, 128, 2), (60, 3, 192, 2), (80, 2, 128, 1), (96, 3, 64, 1), (100, 3, 128, 1),
    (112, 4, 64, 1), (120, 3, 64, 1), (124, 3, 128, 1)])
def test_runtime_side_every_sweep(L, m, R, sweeps):
    # sides other than 32, 64, 128: the general form, geometry read at run time
    # (from two planes up, and one plane at the sides where they are faster)
    _run(L, m, R, seed=100 + L, rho=0.8, sweeps=sweeps)


def test_one_plane_kernel_choice():
    for L, kernel in ((72, 0), (100, 0), (80, 3), (96, 3)):
        sim = K.Simulation(topo=K.KA_CUBIC, d=3, L=L, m=3, replicas=64)
        assert sim.info["kernel"] == kernel
        sim.close()


def test_l128_one_plane():
    # one plane: the mu > 0 launches have fewer work items than SMs
    _run(128, 3, 64, seed=4, rho=0.85, sweeps=1)


def _oracle_bits(L, R0, Rs, seed, rho, sweeps):
    """Replicas R0 .. R0 + Rs - 1 after `sweeps` sweeps (run in a worker process)."""
    topo = O.cubic(3, L)
    st = O.init(topo.N, Rs, seed, rho, r0=R0)
    O.sweeps(topo, 3, st, seed, sweeps)
    return st.n, st.p, O.observe(st)


def _bits(words, b0, nb):
    # [N] uint64 -> [N, nb] bytes of bits b0 .. b0 + nb - 1
    shifts = np.arange(b0, b0 + nb, dtype=np.uint64)
    return ((words[:, None] >> shifts) & np.uint64(1)).astype(np.uint8)


def test_l128_bench_configuration_prefix():
    """The benchmark's workload: d=3, L=128, m=3, 256 replicas, seed 1, at each
    of rho = 0.80, 0.85, 0.88, 20 sweeps in one call (the launch sequence the
    benchmark times).  Sampled replicas -- 8 of word 0 and 8 of word 3 -- are
    compared bit for bit with the oracle run on those replicas alone, with
    their counts."""
    L, R, seed, sweeps, nb = 128, 256, 1, 20, 8
    rhos = (0.80, 0.85, 0.88)
    samples = [(0, 0), (3, 56)]  # (word, first bit)
    ctx = mp.get_context("spawn")
    with cf.ProcessPoolExecutor(max_workers=6, mp_context=ctx) as pool:
        futs = {(rho, w, b): pool.submit(_oracle_bits, L, 64 * w + b, nb, seed, rho, sweeps)
                for rho in rhos for (w, b) in samples}
        for rho in rhos:
            sim = K.Simulation(topo=K.KA_CUBIC, d=3, L=L, m=3, replicas=R)
            sim.init(seed, rho)
            sim.sweep(sweeps)
            n, _, p = sim.get_state()
            _, counts = sim.observe()
            sim.close()
            for (w, b) in samples:
                on, op, oc = futs[(rho, w, b)].result()
                assert (_bits(n[w], b, nb) == on).all(), f"n rho={rho} word {w}"
                assert (_bits(p[w], b, nb) == op).all(), f"p rho={rho} word {w}"
                assert (counts[64 * w + b:64 * w + b + nb] == oc).all()


def test_profile_by_direction():
    # one sweep of one plane set: two group launches per direction; a graph
    # context books every class launch under direction 0
    sim = K.Simulation(topo=K.KA_CUBIC, d=3, L=32, m=3, replicas=128)
    assert sim.info["planes_per_launch"] == 2
    sim.init(1, 0.8)
    K.ka_profile_enable(sim.ctx, True)
    sim.sweep(1)
    ms, n = K.ka_profile_read_dirs(sim.ctx)
    assert list(n) == [2, 2, 2, 0] and (ms[:3] > 0).all() and ms[3] == 0
    sim.sweep(2)
    tot, nl = K.ka_profile_read(sim.ctx)
    assert nl == 12 and tot > 0
    K.ka_profile_enable(sim.ctx, False)
    sim.sweep(1)
    assert K.ka_profile_read(sim.ctx)[1] == 0
    sim.close()
    g = K.Simulation(topo=K.KA_RRG, N=4096, z=4, m=2, replicas=64, graph_seed=3)
    g.init(1, 0.7)
    K.ka_profile_enable(g.ctx, True)
    g.sweep(1)
    ms, n = K.ka_profile_read_dirs(g.ctx)
    assert n[0] == g.info["nclass"] and (n[1:] == 0).all()
    g.close()
