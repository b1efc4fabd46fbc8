"""Pins of the oracle's layered random graph (section 5.2).

M copies of the periodic cubic lattice, the M links of every base bond rewired
by an independent uniform permutation of the copies.  Pins: M = 1 is the cubic
lattice itself; the graph is 2d-regular, simple and symmetric; every entry
projects onto the base lattice's neighbour in the same slot; the links of each
base bond form a perfect matching between the copies; the permutations are
uniform (chi-square over all M! permutations, alpha = 1e-6).
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O


@pytest.mark.parametrize("d,L", [(1, 8), (2, 4), (3, 4), (3, 8)])
def test_one_layer_is_the_cubic_lattice(d, L):
    g = O.layered_graph(d, L, 1, 5)
    base = O.cubic(d, L).nbr.reshape(L ** d, 2 * d)
    assert (g == base).all()


@pytest.mark.parametrize("d,L,M", [(3, 4, 2), (3, 6, 4), (2, 8, 8), (1, 16, 3), (4, 3, 2)])
def test_regular_simple_symmetric_and_projected(d, L, M):
    N = L ** d
    g = O.layered_graph(d, L, M, 9)
    assert g.shape == (M * N, 2 * d)
    assert ((g >= 0) & (g < M * N)).all()
    v = np.arange(M * N)[:, None]
    assert (g != v).all()  # no self-loops
    assert all(len(set(row)) == 2 * d for row in g)  # no repeated edges
    # symmetric, and the up link along mu of u is a down link along mu of its end
    for u in range(M * N):
        for mu in range(d):
            w = g[u, 2 * mu]
            assert g[w, 2 * mu + 1] == u
    # projection onto the base lattice (site index = sum x_k L^k: axis d-1-mu is x_mu)
    for mu in range(d):
        up = np.roll(np.arange(N).reshape((L,) * d), -1, axis=d - 1 - mu).ravel()
        dn = np.roll(np.arange(N).reshape((L,) * d), 1, axis=d - 1 - mu).ravel()
        assert (g[:, 2 * mu] % N == np.tile(up, M)).all()
        assert (g[:, 2 * mu + 1] % N == np.tile(dn, M)).all()
    # each base bond's links match the copies one to one
    for i in range(N):
        for mu in range(d):
            layers = sorted(g[a * N + i, 2 * mu] // N for a in range(M))
            assert layers == list(range(M))


@pytest.mark.parametrize("d,L,M", [(3, 8, 3), (3, 12, 4)])
def test_permutations_are_uniform(d, L, M):
    N = L ** d
    g = O.layered_graph(d, L, M, 17)
    index = {p: k for k, p in enumerate(itertools.permutations(range(M)))}
    counts = np.zeros(len(index))
    for i in range(N):
        for mu in range(d):
            perm = tuple(int(g[a * N + i, 2 * mu] // N) for a in range(M))
            counts[index[perm]] += 1
    expected = np.full(len(index), N * d / math.factorial(M))
    assert stats.chisquare(counts, expected).pvalue > 1e-6


def test_seeds():
    a = O.layered_graph(3, 4, 4, 1)
    assert (a == O.layered_graph(3, 4, 4, 1)).all()
    assert not (a == O.layered_graph(3, 4, 4, 2)).all()
