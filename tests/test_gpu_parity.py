"""GPU parity: the CUDA path against the CPU oracle, bit-exact.

Every compared word of n (occupation), n0 (reference) and p (persistence)
must be identical after every compared sweep, and the per-replica counts must
be identical integers.  The cases span several warps and blocks with ragged
tails (pencil lengths L = 12, 20, 24 leave idle lanes and partly filled last
warps), every dimension, odd and even word counts (V = 1 and V = 2 plane
layouts), the edge-gather path on cubic lattices and random regular graphs,
and the degenerate densities rho = 0 and 1.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1710_05155_gb300 as K  # noqa: E402


def _oracle_topo(kw):
    if kw.get("topo", K.KA_CUBIC) == K.KA_CUBIC:
        return O.cubic(kw["d"], kw["L"])
    if kw["topo"] == K.KA_GRAPH:
        return O.graph(kw["N"], kw["z"], np.ascontiguousarray(kw["nbr"], np.int32).ravel())
    return O.rrg(kw["N"], kw["z"], kw.get("graph_seed", 1))


def _assert_same(sim, st, what=""):
    n, n0, p = sim.get_state()
    assert (n == O.pack_words(st.n)).all(), f"n differs {what}"
    assert (n0 == O.pack_words(st.n0)).all(), f"n0 differs {what}"
    assert (p == O.pack_words(st.p)).all(), f"p differs {what}"


def _run_case(kw, seed, rho, sweeps, check_every=1):
    topo = _oracle_topo(kw)
    sim = K.Simulation(**kw)
    R = kw["replicas"]
    sim.init(seed, rho)
    st = O.init(topo.N, R, seed, rho)
    _assert_same(sim, st, "after init")
    done = 0
    while done < sweeps:
        k = min(check_every, sweeps - done)
        sim.sweep(k)
        O.sweeps(topo, kw["m"], st, seed, k)
        done += k
        _assert_same(sim, st, f"after sweep {done}")
        t, counts = sim.observe()
        assert t == done
        assert (counts == O.observe(st)).all(), f"counts differ after sweep {done}"
    sim.close()


CUBIC = [
    dict(d=1, L=8, m=1, replicas=64),
    dict(d=1, L=32, m=0, replicas=128),
    dict(d=2, L=4, m=1, replicas=64),
    dict(d=2, L=8, m=2, replicas=128),
    dict(d=2, L=12, m=3, replicas=64),
    dict(d=2, L=20, m=1, replicas=192),
    dict(d=3, L=4, m=3, replicas=64),
    dict(d=3, L=8, m=3, replicas=192),
    dict(d=3, L=12, m=2, replicas=128),
    dict(d=3, L=16, m=3, replicas=256),
    dict(d=3, L=20, m=3, replicas=64),
    dict(d=3, L=24, m=4, replicas=128),
    dict(d=3, L=16, m=0, replicas=64),
    dict(d=3, L=16, m=5, replicas=64),
    dict(d=4, L=4, m=5, replicas=64),
    dict(d=4, L=8, m=4, replicas=128),
]


@pytest.mark.parametrize("kw", CUBIC, ids=lambda k: f"d{k['d']}L{k['L']}m{k['m']}R{k['replicas']}")
def test_cubic_pencil_kernel_every_sweep(kw):
    _run_case(dict(topo=K.KA_CUBIC, **kw), seed=1000 + kw["L"], rho=0.68, sweeps=5)


@pytest.mark.parametrize("kw", CUBIC[::3], ids=lambda k: f"d{k['d']}L{k['L']}m{k['m']}R{k['replicas']}")
def test_cubic_gather_kernel_every_sweep(kw):
    _run_case(dict(topo=K.KA_CUBIC, flags=K.KA_FLAG_GENERIC, **kw), seed=7, rho=0.6, sweeps=4)


def test_cubic_info_reports_kernel():
    # 3: group kernels of three-dimensional lattices; 0: general pencil
    # kernel; 1: edge gather
    a = K.Simulation(topo=K.KA_CUBIC, d=3, L=8, m=3, replicas=64)
    b = K.Simulation(topo=K.KA_CUBIC, d=3, L=8, m=3, replicas=64, flags=K.KA_FLAG_GENERIC)
    c = K.Simulation(topo=K.KA_CUBIC, d=2, L=8, m=2, replicas=64)
    d = K.Simulation(topo=K.KA_CUBIC, d=3, L=24, m=3, replicas=64)
    assert a.info["kernel"] == 3 and b.info["kernel"] == 1 and c.info["kernel"] == 0
    assert d.info["kernel"] == 0
    assert a.info["nclass"] == 24 and a.info["nbonds"] == 3 * 512


RRG = [
    dict(N=64, z=4, m=2, replicas=64),
    dict(N=4096, z=4, m=2, replicas=64),
    dict(N=1000, z=3, m=1, replicas=128),
    dict(N=500, z=6, m=3, replicas=192),
    dict(N=2000, z=4, m=3, replicas=256),
    dict(N=3000, z=4, m=2, replicas=512),   # four-word planes, two of them
    dict(N=1024, z=3, m=1, replicas=256),
]


@pytest.mark.parametrize("kw", RRG, ids=lambda k: f"N{k['N']}z{k['z']}m{k['m']}R{k['replicas']}")
def test_rrg_every_sweep(kw):
    _run_case(dict(topo=K.KA_RRG, graph_seed=3, **kw), seed=11, rho=0.7, sweeps=4)


@pytest.mark.parametrize("d,L,M,m,R", [(3, 4, 4, 3, 64), (3, 6, 2, 2, 128), (2, 8, 8, 1, 256)])
def test_layered_graph_every_sweep(d, L, M, m, R):
    # section 5.2 graph from the oracle's generator, run as a caller-supplied graph
    nbr = O.layered_graph(d, L, M, 3)
    _run_case(dict(topo=K.KA_GRAPH, N=M * L ** d, z=2 * d, m=m, replicas=R, nbr=nbr),
              seed=13, rho=0.7, sweeps=4)


def test_rrg_tables_match_oracle():
    sim = K.Simulation(topo=K.KA_RRG, N=4096, z=4, m=2, replicas=64, graph_seed=5)
    t = K.ka_graph_tables(sim.ctx)
    o = O.rrg(4096, 4, 5)
    assert (t["nbr"] == o.nbr).all() and (t["class_off"] == o.class_off).all()
    assert (t["bu"] == o.bu).all() and (t["bv"] == o.bv).all() and (t["bid"] == o.bid).all()


@pytest.mark.parametrize("rho", [0.0, 1.0, 1.0 / 512, 511.0 / 512])
def test_degenerate_densities(rho):
    _run_case(dict(topo=K.KA_CUBIC, d=3, L=8, m=3, replicas=128), seed=2, rho=rho, sweeps=3)


def test_config_small_cubic_full_run():
    """d=3, L=16, z=6, m=3, rho=0.70, 64 replicas, 1000 sweeps, Philox seed 1;
    counts every 10 sweeps and the full state at 500 and 1000 sweeps."""
    kw = dict(topo=K.KA_CUBIC, d=3, L=16, m=3, replicas=64)
    topo = O.cubic(3, 16)
    sim = K.Simulation(**kw)
    sim.init(1, 0.70)
    st = O.init(topo.N, 64, 1, 0.70)
    assert O.particles(0.70, topo.N) == 2867
    for k in range(101):
        if k:
            sim.sweep(10)
            O.sweeps(topo, 3, st, 1, 10)
        t, counts = sim.observe()
        assert t == 10 * k
        assert (counts == O.observe(st)).all(), f"counts differ at sweep {t}"
        if t in (500, 1000):
            _assert_same(sim, st, f"at sweep {t}")
    assert (counts[:, 0] == 2867).all()


def test_sweeps_compose_and_checkpoint():
    kw = dict(topo=K.KA_CUBIC, d=3, L=16, m=3, replicas=128)
    a = K.Simulation(**kw)
    a.init(5, 0.75)
    a.sweep(12)
    ref = a.get_state()
    b = K.Simulation(**kw)
    b.init(5, 0.75)
    for _ in range(5):
        b.sweep(1)
    snap = b.get_state()
    c = K.Simulation(**kw)
    c.set_state(*snap, sweep=5, seed=5)
    c.sweep(3)
    c.sweep(4)
    got = c.get_state()
    for x, y in zip(ref, got):
        assert (x == y).all()


@pytest.mark.parametrize("replicas", [64, 256])
def test_asynchronous_state_load(replicas):
    # ka_set_state_async from page-locked memory on a side stream, then sweeps
    # queued behind it: the same state as the synchronous load
    kw = dict(topo=K.KA_CUBIC, d=3, L=16, m=3, replicas=replicas)
    a = K.Simulation(**kw)
    a.init(5, 0.75)
    a.sweep(5)
    snap = a.get_state()
    a.sweep(7)
    ref = a.get_state()
    pinned = []
    for x in snap:
        t = torch.empty(x.shape, dtype=torch.int64, pin_memory=True)
        t.numpy().view(np.uint64)[...] = x
        pinned.append(t.numpy().view(np.uint64))
    st = torch.cuda.Stream()
    b = K.Simulation(stream=st, **kw)
    b.set_state_async(*pinned, sweep=5, seed=5)
    b.sweep(7)
    K.ka_sync(b.ctx)
    assert not b.ctx.inflight
    got = b.get_state()
    for x, y in zip(ref, got):
        assert (x == y).all()
    with pytest.raises(ValueError):
        b.set_state_async(snap[0][:, ::2], snap[1], snap[2], sweep=0, seed=5)
    a.close()
    b.close()


def test_errors_surface_as_status():
    sim = K.Simulation(topo=K.KA_CUBIC, d=2, L=8, m=1, replicas=64)
    with pytest.raises(K.KaError) as e:
        sim.sweep(1)
    assert e.value.status == K.KA_ESTATE
    with pytest.raises(K.KaError) as e:
        sim.init(1, 1.5)
    assert e.value.status == K.KA_EINVAL
    sim.init(1, 0.5)
    with pytest.raises(K.KaError) as e:
        sim.sweep(-1)
    assert e.value.status == K.KA_EINVAL
    sim.sweep(0)
    assert sim.observe()[0] == 0


def test_library_allocated_context():
    p, _ = K.make_params(topo=K.KA_CUBIC, d=3, L=8, m=3, replicas=64)
    ctx = K.ka_create(p)
    K.ka_init(ctx, 3, 0.6)
    K.ka_sweep(ctx, 4)
    st = O.init(512, 64, 3, 0.6)
    O.sweeps(O.cubic(3, 8), 3, st, 3, 4)
    n, n0, pp = K.ka_get_state(ctx)
    assert (n == O.pack_words(st.n)).all() and (pp == O.pack_words(st.p)).all()
    K.ka_destroy(ctx)


def test_large_cubic_prefix_sampled_words():
    """d=3, L=128 (2,097,152 sites), m=3, rho=0.80, 256 replicas: two sweeps in
    the launch configuration the benchmark uses; replica words 0 and 3 (both
    plane halves) compared with the oracle run on those 64 replicas only."""
    L, R, seed, rho = 128, 256, 1, 0.80
    topo = O.cubic(3, L)
    sim = K.Simulation(topo=K.KA_CUBIC, d=3, L=L, m=3, replicas=R)
    sim.init(seed, rho)
    sim.sweep(2)
    n, n0, p = sim.get_state()
    _, counts = sim.observe()
    K_ = O.particles(rho, topo.N)
    assert (counts[:, 0] == K_).all()
    for w in (0, 3):
        st = O.init(topo.N, 64, seed, rho, r0=64 * w)
        assert (n0[w] == O.pack_words(st.n0)[0]).all()
        O.sweeps(topo, 3, st, seed, 2)
        assert (n[w] == O.pack_words(st.n)[0]).all()
        assert (p[w] == O.pack_words(st.p)[0]).all()
        assert (counts[64 * w:64 * w + 64] == O.observe(st)).all()


def test_large_rrg_prefix():
    """Random regular graph N=2^20, z=4, m=2, 64 replicas, rho=0.75: graph,
    initial state and two sweeps against the oracle."""
    N, z, m, R, seed, rho = 1 << 20, 4, 2, 64, 1, 0.75
    sim = K.Simulation(topo=K.KA_RRG, N=N, z=z, m=m, replicas=R, graph_seed=1)
    topo = O.rrg(N, z, 1)
    t = K.ka_graph_tables(sim.ctx)
    assert (t["nbr"] == topo.nbr).all() and (t["class_off"] == topo.class_off).all()
    sim.init(seed, rho)
    st = O.init(N, R, seed, rho)
    sim.sweep(2)
    O.sweeps(topo, m, st, seed, 2)
    _assert_same(sim, st, "after 2 sweeps")


def _rrg_bits(N, z, m, graph_seed, R0, Rs, seed, rho, sweeps):
    """Replicas R0 .. R0 + Rs - 1 of a random regular graph run by the oracle
    (in a worker process): n, p as [N, Rs] bytes, and their counts."""
    topo = O.rrg(N, z, graph_seed)
    st = O.init(N, Rs, seed, rho, r0=R0)
    O.sweeps(topo, m, st, seed, sweeps)
    return st.n, st.p, O.observe(st)


def test_large_rrg_twenty_sweeps_sampled_replicas():
    """Random regular graph N=2^20, z=4, m=2, 64 replicas at rho = 0.55 and
    0.90 (the ends of the density range), 20 sweeps in one call: replicas
    0-7 and 56-63 bit for bit against the oracle run on those replicas
    alone, with their counts."""
    import concurrent.futures as cf
    import multiprocessing as mp

    N, z, m, R, seed, sweeps, nb = 1 << 20, 4, 2, 64, 1, 20, 8
    samples = (0, 56)
    rhos = (0.55, 0.90)
    with cf.ProcessPoolExecutor(max_workers=4, mp_context=mp.get_context("spawn")) as pool:
        futs = {(rho, b): pool.submit(_rrg_bits, N, z, m, 1, b, nb, seed, rho, sweeps)
                for rho in rhos for b in samples}
        for rho in rhos:
            sim = K.Simulation(topo=K.KA_RRG, N=N, z=z, m=m, replicas=R, graph_seed=1)
            sim.init(seed, rho)
            sim.sweep(sweeps)
            n, _, p = sim.get_state()
            _, counts = sim.observe()
            sim.close()
            for b in samples:
                on, op, oc = futs[(rho, b)].result()
                shifts = np.arange(b, b + nb, dtype=np.uint64)
                bits = lambda w: ((w[0][:, None] >> shifts) & np.uint64(1)).astype(np.uint8)
                assert (bits(n) == on).all(), f"n rho={rho} replicas {b}..{b + nb - 1}"
                assert (bits(p) == op).all(), f"p rho={rho} replicas {b}..{b + nb - 1}"
                assert (counts[b:b + nb] == oc).all()


def test_large_cubic_two_planes_sampled_words():
    """d=3, L=128, 512 replicas (eight one-word planes, four launches of two
    planes per group): words 3 and 7 against the oracle on their 64 replicas,
    after two sweeps."""
    L, R, seed, rho = 128, 512, 3, 0.85
    topo = O.cubic(3, L)
    sim = K.Simulation(topo=K.KA_CUBIC, d=3, L=L, m=3, replicas=R)
    assert sim.info["planes"] == 8 and sim.info["plane_words"] == 1
    sim.init(seed, rho)
    sim.sweep(2)
    n, _, p = sim.get_state()
    for w in (3, 7):
        st = O.init(topo.N, 64, seed, rho, r0=64 * w)
        O.sweeps(topo, 3, st, seed, 2)
        assert (n[w] == O.pack_words(st.n)[0]).all()
        assert (p[w] == O.pack_words(st.p)[0]).all()
    sim.close()


def test_large_rrg_four_word_planes_sampled_word():
    """Random regular graph N=2^20, z=4, m=2, 256 replicas (one plane of four
    words): the last word after two sweeps against the oracle on its 64 replicas."""
    N, z, m, R, seed, rho = 1 << 20, 4, 2, 256, 2, 0.8
    sim = K.Simulation(topo=K.KA_RRG, N=N, z=z, m=m, replicas=R, graph_seed=1)
    assert sim.info["plane_words"] == 4
    topo = O.rrg(N, z, 1)
    sim.init(seed, rho)
    sim.sweep(2)
    n, _, p = sim.get_state()
    st = O.init(N, 64, seed, rho, r0=192)
    O.sweeps(topo, m, st, seed, 2)
    assert (n[3] == O.pack_words(st.n)[0]).all()
    assert (p[3] == O.pack_words(st.p)[0]).all()
    sim.close()


@pytest.mark.parametrize("kw,rho", [
    (dict(topo=K.KA_CUBIC, d=3, L=48, m=3, replicas=128), 0.3),   # candidate lists, split rows
    (dict(topo=K.KA_CUBIC, d=3, L=48, m=3, replicas=128), 0.85),
    (dict(topo=K.KA_CUBIC, d=3, L=64, m=3, replicas=256), 0.5),   # four one-word planes
    (dict(topo=K.KA_CUBIC, d=3, L=48, m=3, replicas=64), 0.6),
    (dict(topo=K.KA_CUBIC, d=1, L=4096, m=1, replicas=256), 0.6),  # index order, four-word planes
    (dict(topo=K.KA_RRG, N=1 << 17, z=4, m=2, replicas=64, graph_seed=2), 0.7),  # full scans
])
def test_initial_state_of_larger_lattices(kw, rho):
    """The initial state (exactly K particles per replica, the K smallest
    Philox keys) of lattices large enough for the candidate-list passes."""
    sim = K.Simulation(**kw)
    sim.init(19, rho)
    n, n0, p = sim.get_state()
    N = kw["N"] if "N" in kw else kw["L"] ** kw["d"]
    st = O.init(N, kw["replicas"], 19, rho)
    assert (n == O.pack_words(st.n)).all() and (n0 == n).all()
    assert (p == np.uint64(0xFFFFFFFFFFFFFFFF)).all()
    sim.close()


@pytest.mark.parametrize("kw", [
    dict(topo=K.KA_CUBIC, d=2, L=132, m=2, replicas=64),    # above the pencil kernel's L <= 128
    dict(topo=K.KA_CUBIC, d=1, L=256, m=1, replicas=128),   # edge-gather path, two-word planes
    dict(topo=K.KA_CUBIC, d=4, L=16, m=5, replicas=256),    # d = 4 with four-word planes
    dict(topo=K.KA_CUBIC, d=2, L=128, m=3, replicas=256),   # the pencil kernel's longest pencils
    dict(topo=K.KA_RRG, N=4096, z=4, m=0, replicas=256, graph_seed=6),   # m = 0, four-word planes
    dict(topo=K.KA_RRG, N=4096, z=4, m=3, replicas=256, graph_seed=7),   # m = z - 1: no constraint
], ids=lambda k: "-".join(f"{a}{b}" for a, b in k.items() if a != "topo"))
def test_edge_shapes_every_sweep(kw):
    _run_case(dict(kw), seed=23, rho=0.64, sweeps=3)
