"""Host observables derived from the per-replica counts: C(t) and chi_4(t) (section 2.2).

chi_4(t) = N (<q^2> - <q>^2) with q the normalised overlap.  Pins:
* t = 0: every replica's overlap is K, so q = 1 for all and chi_4 = 0;
* the ergodic long-time limit (chi_4 -> 1 as N -> infinity, section 2.2): when the
  configurations are independent and uniform over the K-subsets, the overlap with a fixed
  K-subset is hypergeometric, of variance K^2 (N-K)^2 / (N^2 (N-1)), hence chi_4 = N/(N-1)
  exactly over the population of all C(N, K) configurations;
* the free gas (m >= z - 1: no constraint) mixes to that law: chi_4 of the oracle's replicas
  after many sweeps is N/(N-1) within sampling error, and C(t) -> 0.
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_1710_05155_gb300 import correlation, susceptibility


def _counts_from_overlaps(overlap, K):
    c = np.zeros((len(overlap), 4), np.int64)
    c[:, 0] = K
    c[:, 1] = overlap
    return c


def test_chi4_vanishes_at_time_zero():
    N, K = 4096, 2867
    c = _counts_from_overlaps(np.full(64, K), K)
    assert susceptibility(c, N, K) == pytest.approx(0.0, abs=1e-9)
    assert correlation(c, N, K) == pytest.approx(1.0)


@pytest.mark.parametrize("N,K", [(10, 4), (12, 6), (9, 2)])
def test_chi4_of_all_configurations_is_exact(N, K):
    ref = set(range(K))
    overlap = [len(ref.intersection(S)) for S in itertools.combinations(range(N), K)]
    c = _counts_from_overlaps(np.array(overlap), K)
    assert susceptibility(c, N, K) == pytest.approx(N / (N - 1), rel=1e-12)
    assert correlation(c, N, K) == pytest.approx(0.0, abs=1e-12)


def test_chi4_of_the_mixed_free_gas_tends_to_one():
    # d = 2, L = 8 torus, no constraint (m = z - 1 = 3), half filling, 1024 replicas
    topo = O.cubic(2, 8)
    N, R = topo.N, 1024
    st = O.init(N, R, 5, 0.5)
    K = int(st.n[:, 0].sum())
    O.sweeps(topo, 3, st, 5, 300)
    counts = O.observe(st)
    chi4 = susceptibility(counts, N, K)
    # sample variance of R draws: relative standard error ~ sqrt(2 / R) ~ 4.4 %
    assert chi4 == pytest.approx(N / (N - 1), rel=0.2)
    assert abs(correlation(counts, N, K)) < 4.0 / np.sqrt(R)
