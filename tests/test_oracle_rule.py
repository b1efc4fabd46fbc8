"""Pins for the oracle's exchange rule.

Three statements of "allowed move" from the paper are checked against the
oracle over every local configuration:
  * rules (a)-(c) of section 2.1, in words (full neighbourhood sums);
  * the Karnaugh-map form of section 3.2 (s_k4 / s_k5 as negated ORs of ANDs
    over 4- and 5-subsets of the neighbours), generalised to any m;
  * Table 1 of section 3.2 (the 16-row update truth table).
"""
import itertools
import os
import random

import pytest

import oracle as O


def _table1(golden_dir):
    tab = {}
    with open(os.path.join(golden_dir, "tabup.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            ni, nj, si, sj, a, b = (int(x) for x in line.split())
            tab[(ni, nj, si, sj)] = (a, b)
    assert len(tab) == 16
    return tab


def _karnaugh_at_most(values, T):
    """Negated OR over all (T+1)-subsets of the AND of the subset: 1 iff at most T ones."""
    if T + 1 > len(values):
        return 1
    anyall = 0
    for sub in itertools.combinations(values, T + 1):
        anyall |= int(all(sub))
    return 1 - anyall


def _verbal(z, m, ni, nj, oi, oj):
    """Section 2.1: a particle at the source hops to the empty target iff the
    source has at most m occupied neighbours and the target at most m + 1."""
    if ni == nj:
        return ni, nj
    full_i = list(oi) + [nj]  # all z neighbours of i
    full_j = list(oj) + [ni]  # all z neighbours of j
    src, dst = (full_i, full_j) if ni == 1 else (full_j, full_i)
    if sum(src) <= m and sum(dst) <= m + 1:
        return nj, ni
    return ni, nj


def test_table1_with_karnaugh_flags(golden_dir):
    tab = _table1(golden_dir)
    z, m = 6, 3
    for ni, nj in itertools.product((0, 1), repeat=2):
        for oi in itertools.product((0, 1), repeat=z - 1):
            for oj in itertools.product((0, 1), repeat=z - 1):
                nbi, nbj = list(oi) + [nj], list(oj) + [ni]
                s_i4, s_i5 = _karnaugh_at_most(nbi, 3), _karnaugh_at_most(nbi, 4)
                s_j4, s_j5 = _karnaugh_at_most(nbj, 3), _karnaugh_at_most(nbj, 4)
                s_i, s_j = s_i4 & s_j5, s_j4 & s_i5
                want = tab[(ni, nj, s_i, s_j)]
                assert O.local_move(z, m, ni, nj, oi, oj, 1) == want
                assert O.local_move(z, m, ni, nj, oi, oj, 0) == (ni, nj)


@pytest.mark.parametrize("z", [2, 3, 4, 5, 6, 7])
def test_rule_matches_words_exhaustive(z):
    for m in range(z):
        for ni, nj in itertools.product((0, 1), repeat=2):
            for oi in itertools.product((0, 1), repeat=z - 1):
                for oj in itertools.product((0, 1), repeat=z - 1):
                    assert O.local_move(z, m, ni, nj, oi, oj, 1) == _verbal(z, m, ni, nj, oi, oj)


def test_rule_matches_words_sampled_z8():
    rng = random.Random(8)
    z = 8
    for _ in range(20000):
        m = rng.randrange(z)
        ni, nj = rng.randrange(2), rng.randrange(2)
        oi = [rng.randrange(2) for _ in range(z - 1)]
        oj = [rng.randrange(2) for _ in range(z - 1)]
        assert O.local_move(z, m, ni, nj, oi, oj, 1) == _verbal(z, m, ni, nj, oi, oj)


@pytest.mark.parametrize("z", [4, 6])
def test_rule_matches_generalised_karnaugh(z):
    # move i -> j allowed iff s_i^(m) and s_j^(m+1), the section 3.2 form with m in place of 3
    for m in range(z):
        for ni, nj in ((1, 0), (0, 1)):
            for oi in itertools.product((0, 1), repeat=z - 1):
                for oj in itertools.product((0, 1), repeat=z - 1):
                    nbi, nbj = list(oi) + [nj], list(oj) + [ni]
                    if ni == 1:
                        ok = _karnaugh_at_most(nbi, m) & _karnaugh_at_most(nbj, m + 1)
                    else:
                        ok = _karnaugh_at_most(nbj, m) & _karnaugh_at_most(nbi, m + 1)
                    want = (nj, ni) if ok else (ni, nj)
                    assert O.local_move(z, m, ni, nj, oi, oj, 1) == want


def test_free_gas_limit():
    # m = z - 1 removes the constraint: every particle-hole bond exchanges
    for z in (4, 6):
        for oi in itertools.product((0, 1), repeat=z - 1):
            for oj in itertools.product((0, 1), repeat=z - 1):
                assert O.local_move(z, z - 1, 1, 0, oi, oj, 1) == (0, 1)
                assert O.local_move(z, z - 1, 0, 1, oi, oj, 1) == (1, 0)
