"""Pins for the oracle's random streams and its initial state.

Philox4x32-10 is pinned to published known-answer vectors; the initial state is
pinned to the paper's requirement (section 3.1: draw configurations at fixed
density at random) by exact particle counts and a uniformity test over all
K-subsets of a tiny lattice.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle as O


def _kat_rows(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([int(x, 16) for x in line.split()])
    return rows


def test_philox_known_answers(golden_dir):
    rows = _kat_rows(golden_dir)
    assert len(rows) == 3
    for r in rows:
        out = O.philox4x32_10(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


def test_gate_word_layout():
    # word w of a bond takes half (w mod 2) of the Philox block with c3 = w // 2
    seed = 0x1234_5678_9ABC_DEF0
    for (t, c, b) in [(0, 0, 0), (7, 13, 4095), (99999, 23, 2097151)]:
        for w in range(4):
            blk = O.philox4x32_10([t, c, b, w // 2], [seed & 0xFFFFFFFF, seed >> 32])
            lo, hi = (blk[0], blk[1]) if w % 2 == 0 else (blk[2], blk[3])
            assert O.gate_word(seed, t, c, b, w) == int(lo) | (int(hi) << 32)


def test_cubic_gate_word_layout():
    # bonds at pencil positions 4k + 2b and 4k + 2b + 1 share the block with
    # counter (t, 4g + 2b, first base site, w): half 0 for the first, 1 for the second
    seed, L = 77, 8
    for mu, stride in ((0, 1), (1, 8), (2, 64)):
        for par in (0, 1):
            for a in range(4):
                cls = 4 * (2 * mu + par) + a
                for base in (3 * stride * 4 + 5 if mu else 36, 100):
                    for w in range(3):
                        first = base - (a % 2) * stride
                        blk = O.philox4x32_10([9, cls - cls % 2, first, w], [seed, 0])
                        lo, hi = (blk[0], blk[1]) if a % 2 == 0 else (blk[2], blk[3])
                        got = O.cubic_gate_word(seed, 9, cls, base, w, L)
                        assert got == int(lo) | (int(hi) << 32)


def test_gate_bits_are_fair():
    # Bernoulli(1/2) per replica: 64 * 4000 bits, mean within 5 sigma of 1/2
    words = [O.gate_word(1, t, 5, b, 0) for t in range(40) for b in range(50)]
    words += [O.cubic_gate_word(1, t, 5, b, 1, 16) for t in range(40) for b in range(50)]
    ones = sum(bin(w).count("1") for w in words)
    n = 64 * len(words)
    assert abs(ones - n / 2) < 5 * math.sqrt(n / 4)


@pytest.mark.parametrize("rho,N,K", [(0.70, 4096, 2867), (0.80, 128 ** 3, 1677722),
                                     (0.85, 128 ** 3, 1782579), (0.88, 128 ** 3, 1845494),
                                     (0.55, 1 << 20, 576717), (0.75, 1 << 20, 786432),
                                     (0.5, 7, 4), (0.0, 10, 0), (1.0, 10, 10)])
def test_particle_count_rounding(rho, N, K):
    # K = rho * N rounded half away from zero (values worked out by hand)
    assert O.particles(rho, N) == K


def test_init_exact_count_and_reference():
    st = O.init(512, 128, 7, 0.37)
    K = O.particles(0.37, 512)
    assert (st.n.sum(axis=0) == K).all()
    assert (st.n0 == st.n).all()
    assert (st.p == 1).all()


def test_init_selects_smallest_keys():
    # the occupied sites of replica r are the K smallest (key, site) pairs,
    # key = half (r mod 2) of the Philox block with counter (r // 2, TAG_INIT, site, 0)
    N, R, seed, rho = 50, 6, 99, 0.3
    st = O.init(N, R, seed, rho)
    K = O.particles(rho, N)
    for r in range(R):
        keys = []
        for i in range(N):
            blk = O.philox4x32_10([r // 2, O.TAG_INIT, i, 0], [seed & 0xFFFFFFFF, seed >> 32])
            lo, hi = (blk[0], blk[1]) if r % 2 == 0 else (blk[2], blk[3])
            keys.append((int(lo) | (int(hi) << 32), i))
        chosen = sorted(i for _, i in sorted(keys)[:K])
        assert chosen == sorted(np.nonzero(st.n[:, r])[0].tolist())


def test_init_uniform_over_subsets():
    # all C(6,2) = 15 placements equally likely (chi-square, alpha = 1e-6)
    N, K, R = 6, 2, 64 * 96
    st = O.init(N, R, 2024, K / N)
    assert (st.n.sum(axis=0) == K).all()
    subsets = {s: k for k, s in enumerate(itertools.combinations(range(N), K))}
    counts = np.zeros(len(subsets))
    for r in range(R):
        counts[subsets[tuple(np.nonzero(st.n[:, r])[0])]] += 1
    p = stats.chisquare(counts).pvalue
    assert p > 1e-6, p


def test_init_replicas_independent_of_block():
    # a replica's placement does not depend on which other replicas are computed
    full = O.init(300, 128, 5, 0.6)
    part = O.init(300, 3, 5, 0.6, r0=61)
    assert (full.n[:, 61:64] == part.n).all()
