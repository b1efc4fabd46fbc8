"""Pins for the oracle's dynamics and observables.

What the paper fixes and these tests check:
  * particle number is conserved (section 2.1);
  * every accepted move can be undone by the reverse move (the detailed
    balance remark of section 2.1), and blocked configurations never change;
  * the flat Gibbs measure of section 2.2: each bond class is a doubly
    stochastic map, so the uniform measure is stationary; the oracle's
    empirical law after t sweeps matches exact propagation of the chain on
    every configuration of a 4x4 torus (chi-square, alpha = 1e-6);
  * one bit per replica (section 3.1): a replica's trajectory is the same
    whatever other replicas share its word;
  * C(0) = 1 with the normalisation of section 3.3, and C -> 0 in the
    ergodic phase (section 2.2).
"""
import itertools

import numpy as np
import pytest
from scipy import sparse, stats

import oracle as O


def _verbal_allowed(nbr, z, state, i, j, m):
    """Rules (a)-(c) of section 2.1 for the bond (i, j) in one configuration."""
    ni, nj = state[i], state[j]
    if ni == nj:
        return False
    src, dst = (i, j) if ni == 1 else (j, i)
    s_src = sum(state[k] for k in nbr[src * z:(src + 1) * z])
    s_dst = sum(state[k] for k in nbr[dst * z:(dst + 1) * z])
    return s_src <= m and s_dst <= m + 1


def test_conservation_and_reversibility_per_class():
    topo = O.cubic(3, 8)
    m, seed = 3, 17
    st = O.init(topo.N, 64, seed, 0.62)
    K = O.particles(0.62, topo.N)
    for t in range(3):
        for c in range(topo.nclass):
            before = st.n.copy()
            O.class_step(topo, m, st, c, seed, t=t)
            assert (st.n.sum(axis=0) == K).all()
            changed = np.nonzero((before != st.n).any(axis=1))[0]
            lo, hi = topo.class_off[c], topo.class_off[c + 1]
            ends = set(topo.bu[lo:hi].tolist()) | set(topo.bv[lo:hi].tolist())
            assert set(changed.tolist()) <= ends
            for b in range(lo, hi):
                i, j = int(topo.bu[b]), int(topo.bv[b])
                for r in np.nonzero(before[i] != st.n[i])[0]:
                    # swapped: j changed too, and the reverse move is allowed now
                    assert before[j, r] != st.n[j, r]
                    assert _verbal_allowed(topo.nbr, topo.z, st.n[:, r], i, j, m)
                    assert _verbal_allowed(topo.nbr, topo.z, before[:, r], i, j, m)
                    assert st.p[i, r] == 0 and st.p[j, r] == 0


def _checkerboard(d, L):
    return np.array([sum((i // L ** k) % L for k in range(d)) % 2 for i in range(L ** d)], np.uint8)


@pytest.mark.parametrize("d,L,m", [(2, 4, 2), (2, 8, 1), (3, 8, 3), (3, 4, 4)])
def test_blocked_configurations_stay_frozen(d, L, m):
    topo = O.cubic(d, L)
    st = O.State(topo.N, 64)
    st.n[:] = _checkerboard(d, L)[:, None]
    st.n0[:] = st.n
    st.p[:] = 1
    O.sweeps(topo, m, st, 5, 20)
    assert (st.n == st.n0).all() and (st.p == 1).all()


@pytest.mark.parametrize("rho", [0.0, 1.0])
def test_empty_and_full_lattices_never_move(rho):
    topo = O.cubic(2, 8)
    st = O.init(topo.N, 64, 3, rho)
    O.sweeps(topo, 3, st, 3, 10)
    assert (st.n == st.n0).all() and (st.p == 1).all()


def test_order_inside_a_class_does_not_matter():
    topo = O.cubic(3, 8)
    rng = np.random.default_rng(0)
    perm_bu, perm_bv, perm_bid = topo.bu.copy(), topo.bv.copy(), topo.bid.copy()
    for c in range(topo.nclass):
        lo, hi = topo.class_off[c], topo.class_off[c + 1]
        p = lo + rng.permutation(hi - lo)
        perm_bu[lo:hi], perm_bv[lo:hi], perm_bid[lo:hi] = topo.bu[p], topo.bv[p], topo.bid[p]
    shuffled = O.Topology(topo.N, topo.z, topo.nbr, topo.class_off, perm_bu, perm_bv, perm_bid,
                          cubic_L=topo.cubic_L)
    a = O.init(topo.N, 64, 9, 0.7)
    b = a.copy()
    O.sweeps(topo, 3, a, 9, 6)
    O.sweeps(shuffled, 3, b, 9, 6)
    assert (a.n == b.n).all() and (a.p == b.p).all()


def test_replica_independent_of_its_word():
    topo = O.cubic(2, 8)
    full = O.init(topo.N, 128, 21, 0.55)
    O.sweeps(topo, 2, full, 21, 15)
    for r in (0, 63, 64, 100):
        one = O.init(topo.N, 1, 21, 0.55, r0=r)
        O.sweeps(topo, 2, one, 21, 15)
        assert (one.n[:, 0] == full.n[:, r]).all()
        assert (one.p[:, 0] == full.p[:, r]).all()


def test_graph_gate_bit_convention():
    # on a graph the gate of word w of edge e is half (w mod 2) of block (t, c, e, w // 2)
    topo = O.rrg(64, 4, 3)
    R, seed, t = 192, 5, 2
    for c in range(topo.nclass):
        lo, hi = topo.class_off[c], topo.class_off[c + 1]
        b = lo
        u = int(topo.bu[b])
        st = O.State(topo.N, R)
        st.n[u, :] = 1
        st.n0[:] = st.n
        st.p[:] = 1
        O.class_step(topo, 0, st, c, seed, t=t)
        for r in range(R):
            g = (O.gate_word(seed, t, c, int(topo.bid[b]), r // 64) >> (r % 64)) & 1
            # the lone particle sits on one end of this edge; other edges of the
            # class do not touch it (strong matching)
            assert st.n[u, r] == 1 - g


def test_sweeps_compose():
    topo = O.rrg(256, 4, 2)
    a = O.init(topo.N, 64, 4, 0.7)
    b = a.copy()
    O.sweeps(topo, 2, a, 4, 10)
    O.sweeps(topo, 2, b, 4, 4)
    O.sweeps(topo, 2, b, 4, 6)
    assert (a.n == b.n).all() and (a.p == b.p).all()


# ---------------------------------------------------------------------------
# exact enumeration on the 4x4 torus (N = 16, z = 4)
# ---------------------------------------------------------------------------

def _torus_classes(L):
    """Bond classes of the 2-d torus, written out from their definition."""
    def idx(x, y):
        return (x % L) + L * (y % L)
    classes = []
    for mu in range(2):
        for par in range(2):
            for a in range(4):
                bonds = []
                for y in range(L):
                    for x in range(L):
                        xm, perp = (x, y) if mu == 0 else (y, x)
                        if xm % 4 == a and perp % 2 == par:
                            bonds.append((idx(x, y), idx(x + 1, y) if mu == 0 else idx(x, y + 1)))
                classes.append(bonds)
    return classes


def _torus_nbr(L):
    nbr = []
    for i in range(L * L):
        x, y = i % L, i // L
        nbr.append([(x + 1) % L + L * y, (x - 1) % L + L * y, x + L * ((y + 1) % L), x + L * ((y - 1) % L)])
    return nbr


def _class_matrices(L, K, m):
    """Exact transition matrix of every bond class on all K-particle states:
    each bond that can exchange does so with probability 1/2, independently."""
    N = L * L
    nbr = _torus_nbr(L)
    states = [sum(1 << s for s in comb) for comb in itertools.combinations(range(N), K)]
    index = {s: k for k, s in enumerate(states)}
    mats = []
    for bonds in _torus_classes(L):
        rows, cols, vals = [], [], []
        for k, s in enumerate(states):
            occ = [(s >> i) & 1 for i in range(N)]
            active = []
            for i, j in bonds:
                if occ[i] == occ[j]:
                    continue
                src, dst = (i, j) if occ[i] else (j, i)
                if sum(occ[q] for q in nbr[src]) <= m and sum(occ[q] for q in nbr[dst]) <= m + 1:
                    active.append((1 << i) | (1 << j))
            w = 1.0 / (1 << len(active))
            for sub in itertools.product((0, 1), repeat=len(active)):
                t = s
                for bit, mask in zip(sub, active):
                    if bit:
                        t ^= mask
                rows.append(k)
                cols.append(index[t])
                vals.append(w)
        mats.append(sparse.csr_matrix((vals, (rows, cols)), shape=(len(states), len(states))))
    return states, index, mats


@pytest.mark.parametrize("K,m", [(3, 1), (5, 2), (1, 0)])
def test_class_maps_are_doubly_stochastic(K, m):
    _, _, mats = _class_matrices(4, K, m)
    for T in mats:
        assert np.allclose(T.sum(axis=1), 1.0)
        assert np.allclose(T.sum(axis=0), 1.0)  # uniform measure is stationary


@pytest.mark.parametrize("K,m,t,seed", [(3, 1, 2, 11), (3, 1, 25, 12), (5, 2, 1, 13),
                                        (1, 0, 3, 14), (8, 2, 2, 15)])
def test_exact_law_on_4x4_torus(K, m, t, seed):
    L, N, R = 4, 16, 64 * 160
    states, index, mats = _class_matrices(L, K, m)
    rng = np.random.default_rng(seed)
    start = sorted(rng.choice(N, K, replace=False).tolist())
    s0 = sum(1 << i for i in start)
    prob = np.zeros(len(states))
    prob[index[s0]] = 1.0
    for _ in range(t):
        for T in mats:
            prob = T.T @ prob
    # oracle: R replicas from the same start, t sweeps
    topo = O.cubic(2, L)
    st = O.State(N, R)
    st.n[start, :] = 1
    st.n0[:] = st.n
    st.p[:] = 1
    O.sweeps(topo, m, st, seed, t)
    weights = (1 << np.arange(N, dtype=np.int64))
    codes = (st.n.astype(np.int64) * weights[:, None]).sum(axis=0)
    counts = np.zeros(len(states))
    for c in codes:
        counts[index[int(c)]] += 1
    expected = prob * R
    assert abs(counts.sum() - R) < 1e-9
    # pool bins with small expectation, then chi-square
    big = expected >= 5
    obs = np.append(counts[big], counts[~big].sum())
    exp = np.append(expected[big], expected[~big].sum())
    keep = exp > 0
    obs, exp = obs[keep], exp[keep]
    assert counts[expected == 0].sum() == 0  # no impossible configuration reached
    chi2 = ((obs - exp) ** 2 / exp).sum()
    pval = stats.chi2.sf(chi2, max(len(obs) - 1, 1))
    assert pval > 1e-6, (chi2, len(obs), pval)


# ---------------------------------------------------------------------------
# observables
# ---------------------------------------------------------------------------

def _C(counts, N, K):
    rho = K / N
    return ((counts[:, 1] - N * rho * rho) / (N * rho * (1 - rho))).mean()


def test_observables_initial_values_and_monotone_persistence():
    topo = O.cubic(3, 8)
    N, K = topo.N, O.particles(0.7, topo.N)
    st = O.init(N, 64, 5, 0.7)
    c0 = O.observe(st)
    assert (c0[:, 0] == K).all() and (c0[:, 1] == K).all()
    assert (c0[:, 2] == K).all() and (c0[:, 3] == N).all()
    assert abs(_C(c0, N, K) - 1.0) < 1e-12
    prev = c0
    for _ in range(5):
        O.sweeps(topo, 3, st, 5, 3)
        c = O.observe(st)
        assert (c[:, 0] == K).all()
        assert (c[:, 2] <= c[:, 1]).all()
        assert (c[:, 3] <= prev[:, 3]).all() and (c[:, 2] <= prev[:, 2]).all()
        prev = c


def test_correlation_decays_in_free_gas():
    # no constraint (m = z - 1), low density: C(t) -> 0 (section 2.2)
    topo = O.cubic(2, 8)
    N = topo.N
    st = O.init(N, 128, 8, 0.3)
    K = O.particles(0.3, N)
    O.sweeps(topo, 3, st, 8, 300)
    assert abs(_C(O.observe(st), N, K)) < 0.1


def test_gate_bit_convention_in_class_step():
    # a lone particle has no constraint, so on a bond touching it it hops iff
    # the replica's gate bit is set: replica r reads bit r % 64 of gate word r // 64
    topo = O.cubic(2, 8)
    assert topo.cubic_L == 8
    R, seed, t = 192, 77, 5
    for c in range(topo.nclass):
        lo, hi = topo.class_off[c], topo.class_off[c + 1]
        for b in range(lo, hi):
            if topo.bu[b] != 9 and topo.bv[b] != 9:
                continue
            st = O.State(topo.N, R)
            st.n[9, :] = 1
            st.n0[:] = st.n
            st.p[:] = 1
            O.class_step(topo, 0, st, c, seed, t=t)
            for r in range(R):
                g = (O.cubic_gate_word(seed, t, c, int(topo.bid[b]), r // 64, 8) >> (r % 64)) & 1
                assert st.n[9, r] == 1 - g
