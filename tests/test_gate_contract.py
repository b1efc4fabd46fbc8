"""The random-gate contract written in include/ka.h, recomputed from its own words.

A lone particle can always hop (it has no occupied neighbour, and its target
has exactly one, itself), so over one sweep its path is decided by the gate
bits alone: at every class that holds a bond through its site it crosses that
bond iff its replica's gate bit is 1 (section 2.1 rules (a)-(c) with the
gate).  The tests below walk such particles with gate words computed from the
header's description of the Philox counters, and require the oracle (CPU) and
the library (GPU, through the C ABI) to produce the same positions and
persistence bits.
"""
import numpy as np
import pytest

import oracle as O

SEED = 0x0123_4567_89AB_CDEF


def _block(ctr, seed):
    return O.philox4x32_10(ctr, [seed & 0xFFFFFFFF, seed >> 32])


def _half(blk, h):
    lo, hi = (blk[0], blk[1]) if h == 0 else (blk[2], blk[3])
    return int(lo) | (int(hi) << 32)


def header_cubic_gate(seed, t, c, i, w, L):
    """ka.h, cubic lattices: half (c mod 2) of the block at counter
    (t, c - (c mod 2), i - (c mod 2) L^mu, w); i is the bond's base site."""
    mu = c // 8
    h = c % 2
    return _half(_block([t, c - h, i - h * L ** mu, w], seed), h)


def header_graph_gate(seed, t, c, e, w):
    """ka.h, graphs: half (w mod 2) of the block at counter (t, c, e, w / 2)."""
    return _half(_block([t, c, e, w // 2], seed), w % 2)


def _coords(i, d, L):
    return [(i // L ** k) % L for k in range(d)]


def _index(x, L):
    return sum(v * L ** k for k, v in enumerate(x))


def cubic_walk(d, L, start, R, t):
    """Positions and persistence after sweep t of one lone particle per replica."""
    N = L ** d
    nclass = 4 if d == 1 else 8 * d
    pos = list(start)
    moved = [set() for _ in range(R)]
    for c in range(nclass):
        mu, par, a = c // 8, (c // 4) % 2, c % 4
        for r in range(R):
            s = _coords(pos[r], d, L)
            for base_is_s in (True, False):
                x = list(s)
                if not base_is_s:
                    x[mu] = (x[mu] - 1) % L
                perp = sum(x[k] for k in range(d) if k != mu) % 2
                if x[mu] % 4 != a or perp != par:
                    continue
                i = _index(x, L)
                y = list(x)
                y[mu] = (y[mu] + 1) % L
                j = _index(y, L)
                g = header_cubic_gate(SEED, t, c, i, r // 64, L)
                if (g >> (r % 64)) & 1:
                    moved[r].update((i, j))
                    pos[r] = j if pos[r] == i else i
                break
    n = np.zeros((N, R), np.uint8)
    p = np.ones((N, R), np.uint8)
    for r in range(R):
        n[pos[r], r] = 1
        for k in moved[r]:
            p[k, r] = 0
    return n, p


def graph_walk(topo, start, R, t):
    N = topo.N
    pos = list(start)
    moved = [set() for _ in range(R)]
    for c in range(topo.nclass):
        lo, hi = int(topo.class_off[c]), int(topo.class_off[c + 1])
        for r in range(R):
            for b in range(lo, hi):
                u, v = int(topo.bu[b]), int(topo.bv[b])
                if pos[r] not in (u, v):
                    continue
                g = header_graph_gate(SEED, t, c, int(topo.bid[b]), r // 64)
                if (g >> (r % 64)) & 1:
                    moved[r].update((u, v))
                    pos[r] = v if pos[r] == u else u
                break
    n = np.zeros((N, R), np.uint8)
    p = np.ones((N, R), np.uint8)
    for r in range(R):
        n[pos[r], r] = 1
        for k in moved[r]:
            p[k, r] = 0
    return n, p


def _lone_state(N, R, start):
    st = O.State(N, R)
    for r in range(R):
        st.n[start[r], r] = 1
    st.n0[...] = st.n
    st.p[...] = 1
    return st


CUBIC_CASES = [(1, 16), (2, 8), (3, 8)]


@pytest.mark.parametrize("d,L", CUBIC_CASES)
def test_oracle_follows_header_cubic_gates(d, L):
    N, R, t = L ** d, 128, 3
    start = [(37 * r + 5) % N for r in range(R)]
    st = _lone_state(N, R, start)
    st.t = t
    O.sweeps(O.cubic(d, L), 0, st, SEED, 1)
    n, p = cubic_walk(d, L, start, R, t)
    assert (st.n == n).all()
    assert (st.p == p).all()


def test_oracle_follows_header_graph_gates():
    topo = O.rrg(64, 4, 5)
    R, t = 128, 2
    start = [(11 * r + 3) % 64 for r in range(R)]
    st = _lone_state(64, R, start)
    st.t = t
    O.sweeps(topo, 0, st, SEED, 1)
    n, p = graph_walk(topo, start, R, t)
    assert (st.n == n).all()
    assert (st.p == p).all()


def test_header_cubic_rule_differs_from_graph_rule():
    # the two layouts are not the same stream: a reader who applied the graph
    # rule to a cubic lattice would get other bits
    L, diff = 8, 0
    for c in range(1, 24, 2):
        mu, par, a = c // 8, (c // 4) % 2, c % 4
        x = [1, 2, 5]
        x[mu] = a
        other = [k for k in range(3) if k != mu][0]
        if sum(x[k] for k in range(3) if k != mu) % 2 != par:
            x[other] += 1
        i = _index(x, L)
        diff += header_cubic_gate(SEED, 0, c, i, 0, L) != header_graph_gate(SEED, 0, c, i, 0)
    assert diff == 12


def _library_walk(K, params, N, R, start, t):
    sim = K.Simulation(**params, replicas=R, device=0)
    try:
        n0 = np.zeros((N, R), np.uint8)
        for r in range(R):
            n0[start[r], r] = 1
        words = O.pack_words(n0)
        ones = O.pack_words(np.ones((N, R), np.uint8))
        K.ka_set_state(sim.ctx, words, words, ones, t, SEED)
        K.ka_sweep(sim.ctx, 1)
        n, _, p = K.ka_get_state(sim.ctx)
        return O.unpack_words(n), O.unpack_words(p)
    finally:
        sim.close()


@pytest.mark.gpu
@pytest.mark.parametrize("d,L", CUBIC_CASES + [(3, 32)])
def test_library_follows_header_cubic_gates(d, L):
    import paper_1710_05155_gb300 as K

    N, R, t = L ** d, 128, 7
    start = [(37 * r + 5) % N for r in range(R)]
    n, p = _library_walk(K, dict(topo=K.KA_CUBIC, d=d, L=L, m=0), N, R, start, t)
    en, ep = cubic_walk(d, L, start, R, t)
    assert (n == en).all()
    assert (p == ep).all()


@pytest.mark.gpu
def test_library_follows_header_graph_gates():
    import paper_1710_05155_gb300 as K

    R, t = 128, 4
    topo = O.rrg(64, 4, 5)
    start = [(11 * r + 3) % 64 for r in range(R)]
    n, p = _library_walk(K, dict(topo=K.KA_RRG, N=64, z=4, m=0, graph_seed=5), 64, R, start, t)
    en, ep = graph_walk(topo, start, R, t)
    assert (n == en).all()
    assert (p == ep).all()
