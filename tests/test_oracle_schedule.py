"""Pins for the oracle's bond-class schedules and random regular graphs.

Checked independently of the oracle's own checker, from coordinates on the
torus: every bond class is a strong matching (no two bonds share a site or
touch through an edge, so the order of bonds inside a class cannot matter),
and a sweep attempts every bond of the lattice exactly once.  Random regular
graphs (section 2.1, Bollobas' configuration model) are checked for
regularity and simplicity, and for uniformity over all labelled graphs of a
tiny size.
"""
import itertools
from collections import Counter

import numpy as np
import pytest
from scipy import stats

import oracle as O


def _coords(i, d, L):
    return [(i // L ** k) % L for k in range(d)]


def _torus_l1(a, b, L):
    return sum(min((x - y) % L, (y - x) % L) for x, y in zip(a, b))


@pytest.mark.parametrize("d,L", [(1, 4), (1, 12), (2, 4), (2, 8), (3, 4), (3, 8), (4, 4)])
def test_cubic_schedule_is_strong_matching(d, L):
    topo = O.cubic(d, L)
    N = L ** d
    assert topo.nclass == (4 if d == 1 else 8 * d)
    allbonds = Counter()
    for c in range(topo.nclass):
        lo, hi = topo.class_off[c], topo.class_off[c + 1]
        ends = []
        for b in range(lo, hi):
            u, v = int(topo.bu[b]), int(topo.bv[b])
            cu, cv = _coords(u, d, L), _coords(v, d, L)
            assert _torus_l1(cu, cv, L) == 1  # a lattice bond
            assert topo.bid[b] == u  # Philox bond id = base site
            allbonds[frozenset((u, v))] += 1
            ends.append((cu, cv))
        # distance >= 2 between any endpoints of two different bonds
        for (a1, a2), (b1, b2) in itertools.combinations(ends, 2):
            for x in (a1, a2):
                for y in (b1, b2):
                    assert _torus_l1(x, y, L) >= 2
    assert len(allbonds) == d * N and set(allbonds.values()) == {1}


def test_cubic_neighbour_table():
    d, L = 3, 8
    topo = O.cubic(d, L)
    z = 2 * d
    for i in range(L ** d):
        nb = sorted(int(x) for x in topo.nbr[i * z:(i + 1) * z])
        want = sorted(j for j in range(L ** d) if _torus_l1(_coords(i, d, L), _coords(j, d, L), L) == 1)
        assert nb == want


def _check_simple_regular(N, z, nbr):
    nbr = nbr.reshape(N, z)
    for v in range(N):
        row = list(nbr[v])
        assert row == sorted(row)
        assert v not in row
        assert len(set(row)) == z
        for u in row:
            assert v in nbr[u]


@pytest.mark.parametrize("N,z,seed", [(64, 4, 1), (1000, 4, 3), (4096, 4, 1), (200, 6, 2),
                                      (50, 3, 5), (31, 2, 4)])
def test_rrg_is_simple_and_regular(N, z, seed):
    nbr, att = O.rrg_neighbours(N, z, seed)
    assert att >= 1
    _check_simple_regular(N, z, nbr)


def test_rrg_uniform_over_labelled_graphs():
    # all 70 labelled 3-regular graphs on 6 vertices come out equally often
    N, z = 6, 3
    edges = list(itertools.combinations(range(N), 2))
    graphs = []
    for sub in itertools.combinations(edges, N * z // 2):
        deg = Counter(x for e in sub for x in e)
        if all(deg[v] == z for v in range(N)):
            graphs.append(frozenset(sub))
    assert len(graphs) == 70
    index = {g: k for k, g in enumerate(graphs)}
    counts = np.zeros(len(graphs))
    for seed in range(1, 3501):
        nbr, _ = O.rrg_neighbours(N, z, seed)
        nbr = nbr.reshape(N, z)
        g = frozenset((min(u, int(v)), max(u, int(v))) for u in range(N) for v in nbr[u])
        counts[index[g]] += 1
    p = stats.chisquare(counts).pvalue
    assert p > 1e-6, p


def test_rrg_deterministic_in_seed():
    a, _ = O.rrg_neighbours(500, 4, 11)
    b, _ = O.rrg_neighbours(500, 4, 11)
    c, _ = O.rrg_neighbours(500, 4, 12)
    assert (a == b).all() and not (a == c).all()


@pytest.mark.parametrize("N,z,seed", [(64, 4, 1), (4096, 4, 1), (300, 6, 2), (40, 3, 7)])
def test_graph_classes_strong_and_greedy(N, z, seed):
    nbr, _ = O.rrg_neighbours(N, z, seed)
    topo = O.graph(N, z, nbr)
    adj = nbr.reshape(N, z)
    eu, ev = O.graph_edges(N, z, nbr)
    E = len(eu)
    assert topo.class_off[-1] == E
    colour = np.full(E, -1)
    for c in range(topo.nclass):
        lo, hi = topo.class_off[c], topo.class_off[c + 1]
        ids = topo.bid[lo:hi]
        assert (np.diff(ids) > 0).all()  # edge-id order inside a class
        colour[ids] = c
        closed = []
        for b in range(lo, hi):
            u, v = int(topo.bu[b]), int(topo.bv[b])
            assert (eu[topo.bid[b]], ev[topo.bid[b]]) == (u, v)
            closed.append(({u, v}, {u, v} | set(adj[u].tolist()) | set(adj[v].tolist())))
        for (e1, n1), (e2, n2) in itertools.combinations(closed, 2):
            assert not (e1 & n2) and not (e2 & n1)
    assert (colour >= 0).all()
    # greedy: every smaller colour is taken by an earlier edge in conflict
    inc = [[] for _ in range(N)]
    for f in range(E):
        inc[int(eu[f])].append(f)
        inc[int(ev[f])].append(f)
    for e in range(E):
        u, v = int(eu[e]), int(ev[e])
        near = {u, v} | set(adj[u].tolist()) | set(adj[v].tolist())
        earlier = {int(colour[f]) for w in near for f in inc[w] if f < e}
        assert all(c in earlier for c in range(colour[e]))
        assert colour[e] not in earlier
