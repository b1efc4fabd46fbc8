"""Pins of the oracle's four-point correlations (section 2.2 g_4, section 3.3 Phi).

Every ordered site pair (i, j) falls in exactly one shell s = |delta|^2 of its
representative displacement (components in [-L/2, L/2)), so:
* summed over all shells, phi of replica b is (sum_i q_i)^2 = overlap_b^2 and psi is
  (sum_i M_i)^2; shell 0 holds the diagonal (overlap_b, sum M_i^2);
* a checkerboard (n = n0) pairs i with i + delta iff the components of delta sum to an even
  number: phi[s] = N/2 * #{representatives delta in shell s with even component sum};
* a lone particle has phi = 1 in shell 0 and 0 elsewhere; a periodic shift changes nothing;
* g_4 summed over all shells is chi_4 (section 2.2), with the normalisation read from that identity.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_1710_05155_gb300 import four_point_g4, susceptibility


def _reps(d, L):
    return list(itertools.product(range(-L // 2, L // 2), repeat=d))


def _evolved(d, L, R, seed, rho, sweeps, m):
    topo = O.cubic(d, L)
    st = O.init(topo.N, R, seed, rho)
    O.sweeps(topo, m, st, seed, sweeps)
    return topo, st


@pytest.mark.parametrize("d,L,R", [(2, 8, 16), (3, 4, 24), (1, 16, 8), (3, 8, 4)])
def test_shells_partition_the_pairs(d, L, R):
    topo, st = _evolved(d, L, R, 7, 0.6, 3, d)
    smax = d * (L // 2) ** 2
    phi, psi = O.four_point(d, L, st, smax)
    ov = O.observe(st)[:, 1]
    assert (phi.sum(axis=1) == ov ** 2).all()
    assert (phi[:, 0] == ov).all()
    M = (st.n & st.n0).sum(axis=1).astype(np.int64)
    assert psi.sum() == M.sum() ** 2
    assert psi[0] == (M * M).sum()
    # shells with no representative vector are empty
    norms = {sum(x * x for x in v) for v in _reps(d, L)}
    for s in range(smax + 1):
        if s not in norms:
            assert phi[:, s].sum() == 0 and psi[s] == 0


@pytest.mark.parametrize("d,L", [(2, 8), (3, 4), (3, 8)])
def test_checkerboard_closed_form(d, L):
    N = L ** d
    st = O.State(N, 2)
    for i in range(N):
        x, par = i, 0
        for _ in range(d):
            par += x % L
            x //= L
        st.n[i, :] = (par % 2 == 0)
    st.n0[...] = st.n
    smax = d * (L // 2) ** 2
    phi, _ = O.four_point(d, L, st, smax)
    want = np.zeros(smax + 1, np.int64)
    for v in _reps(d, L):
        if sum(v) % 2 == 0:
            want[sum(x * x for x in v)] += N // 2
    assert (phi[0] == want).all() and (phi[1] == want).all()


def test_lone_particle_and_shift_invariance():
    d, L = 3, 8
    N = L ** d
    st = O.State(N, 1)
    st.n[17, 0] = st.n0[17, 0] = 1
    phi, psi = O.four_point(d, L, st, 48)
    assert phi[0, 0] == 1 and phi[0, 1:].sum() == 0 and psi[0] == 1
    topo, ev = _evolved(d, L, 4, 3, 0.5, 2, 3)
    a, pa = O.four_point(d, L, ev, 20)
    sh = O.State(N, 4)
    idx = np.arange(N).reshape((L,) * d)
    perm = np.roll(idx, shift=(1, 2, 3), axis=(0, 1, 2)).ravel()
    sh.n[...] = ev.n[perm]
    sh.n0[...] = ev.n0[perm]
    b, pb = O.four_point(d, L, sh, 20)
    assert (a == b).all() and (pa == pb).all()


def test_g4_sums_to_chi4():
    d, L, R = 2, 8, 64
    topo, st = _evolved(d, L, R, 11, 0.7, 5, 2)
    N = topo.N
    K = int(O.observe(st)[0, 0])
    phi, psi = O.four_point(d, L, st, d * (L // 2) ** 2)
    g4 = four_point_g4(phi, psi, N, K)
    assert g4.sum() == pytest.approx(susceptibility(O.observe(st), N, K), rel=1e-9)
