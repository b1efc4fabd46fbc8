"""Four-point correlations on the GPU (ka_four_point) against the oracle.

The state is taken from the device (its parity with the oracle is tested
elsewhere), handed to the oracle's brute-force pair sum, and both must agree on
every (replica, shell) count and every shell of psi, bit for bit.  At full size
(L=128, 256 replicas) the small shells are checked against numpy shifts of the
state for the first 64 replicas, and psi against per-site counts.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU-only hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_1710_05155_gb300 as K  # noqa: E402


def _oracle_state(sim):
    n, n0, p = sim.get_state()
    N = n.shape[1]
    st = O.State(N, 64 * n.shape[0])
    st.n[...] = O.unpack_words(n)
    st.n0[...] = O.unpack_words(n0)
    st.p[...] = O.unpack_words(p)
    return st


CASES = [
    dict(d=2, L=8, m=2, replicas=64, smax=32),      # every shell of the lattice
    dict(d=3, L=8, m=3, replicas=128, smax=48),     # two-word planes, every shell
    dict(d=3, L=12, m=3, replicas=192, smax=20),    # one-word planes, three of them
    dict(d=3, L=16, m=3, replicas=256, smax=12),    # four-word planes
    dict(d=1, L=32, m=1, replicas=64, smax=256),
    dict(d=4, L=4, m=4, replicas=64, smax=16),
    dict(d=3, L=8, m=3, replicas=64, smax=0),
]


@pytest.mark.parametrize("kw", CASES, ids=lambda k: f"d{k['d']}L{k['L']}R{k['replicas']}s{k['smax']}")
def test_four_point_matches_oracle(kw):
    kw = dict(kw)
    smax = kw.pop("smax")
    sim = K.Simulation(topo=K.KA_CUBIC, **kw)
    sim.init(21, 0.62)
    sim.sweep(3)
    phi, psi = sim.four_point(smax)
    st = _oracle_state(sim)
    want_phi, want_psi = O.four_point(kw["d"], kw["L"], st, smax)
    assert (phi == want_phi).all()
    assert (psi == want_psi).all()
    # shell 0 is each replica's overlap
    _, counts = sim.observe()
    assert (phi[:, 0] == counts[:, 1]).all()
    sim.close()


def test_g4_sums_to_chi4_on_device_counts():
    d, L, R = 3, 8, 256
    sim = K.Simulation(topo=K.KA_CUBIC, d=d, L=L, m=3, replicas=R)
    sim.init(5, 0.7)
    sim.sweep(20)
    phi, psi = sim.four_point(d * (L // 2) ** 2)
    _, counts = sim.observe()
    N = L ** d
    Kp = int(counts[0, 0])
    g4 = K.four_point_g4(phi, psi, N, Kp)
    assert g4.sum() == pytest.approx(K.susceptibility(counts, N, Kp), rel=1e-9, abs=1e-12)
    sim.close()


def test_four_point_edge_cases():
    sim = K.Simulation(topo=K.KA_CUBIC, d=3, L=8, m=3, replicas=64)
    with pytest.raises(K.KaError) as e:
        sim.four_point(2)
    assert e.value.status == K.KA_ESTATE
    sim.init(1, 0.0)  # empty lattice: nothing overlaps
    phi, psi = sim.four_point(48)
    assert not phi.any() and not psi.any()
    with pytest.raises(K.KaError) as e:
        sim.four_point(49)  # above d (L/2)^2
    assert e.value.status == K.KA_EINVAL
    sim.init(1, 1.0)  # full lattice: every pair overlaps
    phi, psi = sim.four_point(48)
    assert (phi.sum(axis=1) == 512 * 512).all() and psi.sum() == (512 * 64) ** 2
    sim.close()
    g = K.Simulation(topo=K.KA_RRG, N=1024, z=4, m=2, replicas=64)
    g.init(1, 0.5)
    with pytest.raises(K.KaError) as e:
        g.four_point(1)
    assert e.value.status == K.KA_EINVAL
    g.close()


def _popcount64(a):
    table = np.array([bin(i).count("1") for i in range(1 << 16)], np.uint8)
    v = a.view(np.uint16)
    return table[v].reshape(a.shape + (4,)).sum(axis=-1, dtype=np.int64)


def test_full_size_small_shells():
    d, L, R, smax = 3, 128, 256, 2
    sim = K.Simulation(topo=K.KA_CUBIC, d=d, L=L, m=3, replicas=R)
    sim.init(1, 0.8)
    sim.sweep(2)
    phi, psi = sim.four_point(smax)
    n, n0, _ = sim.get_state()
    q = n & n0  # [W, N] words
    # per-site counts M and psi by periodic shifts of the lattice
    M = _popcount64(q).sum(axis=0).reshape(L, L, L)  # axes (z, y, x)
    vecs = {0: [(0, 0, 0)], 1: [], 2: []}
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                s = dx * dx + dy * dy + dz * dz
                if 0 < s <= 2:
                    vecs[s].append((dx, dy, dz))
    for s in range(smax + 1):
        tot = 0
        for dx, dy, dz in vecs[s]:
            tot += int((M * np.roll(M, shift=(-dz, -dy, -dx), axis=(0, 1, 2))).sum())
        assert psi[s] == tot
    # phi of the first 64 replicas: bits of word 0
    bits = ((q[0][:, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)).astype(np.uint8)
    bits = bits.reshape(L, L, L, 64)
    for s in range(smax + 1):
        tot = np.zeros(64, np.int64)
        for dx, dy, dz in vecs[s]:
            tot += (bits & np.roll(bits, shift=(-dz, -dy, -dx), axis=(0, 1, 2))).sum(
                axis=(0, 1, 2), dtype=np.int64)
        assert (phi[:64, s] == tot).all()
    sim.close()
