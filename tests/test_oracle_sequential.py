"""Pins of the oracle's random-sequential mode (section 3.2, time unit of section 2.1).

Each attempt draws one bond (a site and one of its neighbour slots, uniformly), shared by
the 64 replicas of a word, and exchanges wherever the rule allows it (no gate); N attempts
make a sweep.  Pins: particle conservation and persistence only cleared; a full lattice and
an empty one stay put; replicas of one word that start alike stay alike (the shared bond
sequence), replicas of different words do not; and the exact law on the 4x4 torus: the
one-attempt transition matrix averages the rule over the N z (site, slot) pairs, and after
t sweeps the empirical law of one replica per word matches P^(N t) (chi-square, alpha 1e-6).
"""
import itertools

import numpy as np
import pytest
from scipy import sparse, stats

import oracle as O


def _torus_nbr(L):
    out = []
    for i in range(L * L):
        x, y = i % L, i // L
        out.append([(x + 1) % L + L * y, (x - 1) % L + L * y, x + L * ((y + 1) % L),
                    x + L * ((y - 1) % L)])
    return out


def test_conservation_and_persistence():
    topo = O.cubic(3, 8)
    st = O.init(topo.N, 128, 3, 0.6)
    before = O.observe(st)[:, 0].copy()
    p0 = st.p.copy()
    O.sequential_sweeps(topo, 3, st, 3, 4)
    assert (O.observe(st)[:, 0] == before).all()
    assert (st.p <= p0).all()
    assert (st.p[st.n != st.n0] == 0).all()  # a site that changed has moved
    assert st.t == 4


@pytest.mark.parametrize("rho", [0.0, 1.0])
def test_empty_and_full_lattices_stay(rho):
    topo = O.cubic(2, 8)
    st = O.init(topo.N, 64, 1, rho)
    n = st.n.copy()
    O.sequential_sweeps(topo, 2, st, 1, 3)
    assert (st.n == n).all() and (st.p == 1).all()


def test_a_word_shares_its_bond_sequence():
    topo = O.cubic(2, 8)
    st = O.State(topo.N, 128)
    start = np.random.default_rng(0).choice(topo.N, 30, replace=False)
    st.n[start, :] = 1
    st.n0[:] = st.n
    st.p[:] = 1
    O.sequential_sweeps(topo, 3, st, 9, 5)  # m = 3 = z - 1: free gas
    assert (st.n[:, :64] == st.n[:, :1]).all() and (st.n[:, 64:] == st.n[:, 64:65]).all()
    assert not (st.n[:, 0] == st.n[:, 64]).all()


def _attempt_matrix(L, K, m):
    N, z = L * L, 4
    nbr = _torus_nbr(L)
    states = [sum(1 << s for s in c) for c in itertools.combinations(range(N), K)]
    index = {s: k for k, s in enumerate(states)}
    rows, cols, vals = [], [], []
    for k, s in enumerate(states):
        occ = [(s >> i) & 1 for i in range(N)]
        stay = 1.0
        for i in range(N):
            for slot in range(z):
                j = nbr[i][slot]
                if occ[i] == occ[j]:
                    continue
                src, dst = (i, j) if occ[i] else (j, i)
                if sum(occ[q] for q in nbr[src]) <= m and sum(occ[q] for q in nbr[dst]) <= m + 1:
                    s2 = s ^ (1 << i) ^ (1 << j)
                    rows.append(k)
                    cols.append(index[s2])
                    vals.append(1.0 / (N * z))
                    stay -= 1.0 / (N * z)
        rows.append(k)
        cols.append(k)
        vals.append(stay)
    P = sparse.csr_matrix((vals, (rows, cols)), shape=(len(states), len(states)))
    return states, index, P


@pytest.mark.parametrize("K,m,t,seed", [(3, 1, 2, 1), (5, 2, 1, 2), (4, 0, 3, 3)])
def test_exact_law_on_4x4_torus(K, m, t, seed):
    L, N, words = 4, 16, 3000
    states, index, P = _attempt_matrix(L, K, m)
    assert np.allclose(np.asarray(P.sum(axis=0)).ravel(), 1.0)  # doubly stochastic
    start = sorted(np.random.default_rng(seed).choice(N, K, replace=False).tolist())
    prob = np.zeros(len(states))
    prob[index[sum(1 << i for i in start)]] = 1.0
    for _ in range(N * t):
        prob = P.T @ prob
    topo = O.cubic(2, L)
    st = O.State(N, 64 * words)
    st.n[start, :] = 1
    st.n0[:] = st.n
    st.p[:] = 1
    O.sequential_sweeps(topo, m, st, seed, t)
    sample = st.n[:, ::64]  # one replica per word: the words are independent
    codes = (sample.astype(np.int64) * (1 << np.arange(N, dtype=np.int64))[:, None]).sum(axis=0)
    counts = np.zeros(len(states))
    for c in codes:
        counts[index[int(c)]] += 1
    expected = prob * words
    assert counts[expected < 1e-12].sum() == 0
    big = expected >= 5
    obs = np.append(counts[big], counts[~big].sum())
    exp = np.append(expected[big], expected[~big].sum())
    keep = exp > 0
    chi2 = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    assert stats.chi2.sf(chi2, max(keep.sum() - 1, 1)) > 1e-6
