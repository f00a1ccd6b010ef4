"""Pins of the oracle's hybrid selection (reading R9; section "A new hybrid
treecode-FMM with auto-tuning" and the N_crit discussion of the results).

The interaction type of a MAC-accepted pair is looked up in a table over the
count buckets of the two cells; particle-particle pairs may then sit above the
leaf level.  Pinned here by what the method fixes independently of the oracle:
* the bucket function against its closed form (floating-point log2);
* an all-M2L table is the plain FMM, pair for pair;
* an all-P2P table leaves no far field, so the result is the direct sum;
* any table keeps the stencil exclusive: every ordered particle pair is
  covered exactly once (brute force);
* replacing far pairs by exact ones does not lose accuracy."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_5815_gb300 import inputs
from tests.oracle_helpers import coverage_matrix

NB = O.SEL_NB


def _bucket_closed_form(n):
    if n < 4:
        return n - 1
    m, e = math.frexp(n)  # n = m * 2^e, m in [0.5, 1)
    e -= 1                # floor(log2 n)
    frac = n / 2.0 ** e - 1.0
    return 3 + 4 * (e - 2) + int(math.floor(4 * frac))


def test_count_bucket_closed_form():
    for n in list(range(1, 5000)) + [2 ** k + d for k in range(12, 31) for d in (-1, 0, 1)]:
        assert O.count_bucket(n) == _bucket_closed_form(n), n
    assert [O.count_bucket(n) for n in (1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 16)] == \
        [0, 1, 2, 3, 4, 5, 6, 7, 7, 8, 9, 11]
    assert O.count_bucket(2 ** 31 - 1) == 118 < NB


def _threshold_table(k):
    """P2P iff the product of the buckets' smallest counts is <= k."""
    lo = np.zeros(NB, dtype=np.int64)
    for n in range(1, 1 << 16):
        b = O.count_bucket(n)
        if lo[b] == 0:
            lo[b] = n
    lo[lo == 0] = 1 << 40
    return (lo[:, None] * lo[None, :] <= k).astype(np.uint8)


def test_all_m2l_table_is_plain_fmm():
    x, q = inputs.make("plummer", 3000, 5)
    a = O.Fmm(x, q, 4, 0.5, 8)
    b = O.Fmm(x, q, 4, 0.5, 8, sel=np.zeros((NB, NB), np.uint8))
    la, lb = a.lists(), b.lists()
    for k in la:
        assert np.array_equal(la[k], lb[k])


@pytest.mark.parametrize("dist", ["uniform", "plummer"])
def test_all_p2p_table_is_direct_sum(dist):
    x, q = inputs.make(dist, 2500, 8)
    f = O.Fmm(x, q, 3, 0.5, 8, sel=np.ones((NB, NB), np.uint8))
    assert f.nm2l == 0
    phi, grad = f.evaluate()
    dphi, dgrad = O.direct(x, q)
    assert np.abs(phi - dphi).max() <= 1e-11 * np.abs(dphi).max()
    assert np.abs(grad - dgrad).max() <= 1e-11 * np.abs(dgrad).max()


@pytest.mark.parametrize("dist,theta,ncrit,k", [("uniform", 0.5, 4, 64), ("plummer", 0.6, 2, 200),
                                               ("shell", 0.5, 4, 1000), ("uniform", 0.4, 8, 10 ** 9)])
def test_exclusive_coverage_with_selection(dist, theta, ncrit, k):
    x, q = inputs.make(dist, 1200, 33)
    f = O.Fmm(x, q, 2, theta, ncrit, sel=_threshold_table(k))
    c, L = f.cells(), f.lists()
    assert np.all(coverage_matrix(f.N, c, L) == 1)
    if k < 10 ** 9:
        # particle-particle pairs above the leaf level are exercised
        assert np.any(c["nchild"][L["p2p_t"]] > 0) or np.any(c["nchild"][L["p2p_s"]] > 0)


def test_random_tables_keep_coverage():
    rng = np.random.default_rng(4)
    x, q = inputs.make("plummer", 900, 12)
    for _ in range(3):
        sel = (rng.random((NB, NB)) < 0.5).astype(np.uint8)
        f = O.Fmm(x, q, 2, 0.5, 3, sel=sel)
        assert np.all(coverage_matrix(f.N, f.cells(), f.lists()) == 1)


def test_selection_does_not_lose_accuracy():
    x, q = inputs.make("uniform", 6000, 3)
    dphi, dgrad = O.direct(x, q)
    plain = O.Fmm(x, q, 4, 0.5, 8)
    hyb = O.Fmm(x, q, 4, 0.5, 8, sel=_threshold_table(256))
    assert hyb.nm2l < plain.nm2l
    e = []
    for f in (plain, hyb):
        phi, grad = f.evaluate()
        e.append((np.linalg.norm(phi - dphi) / np.linalg.norm(dphi),
                  np.linalg.norm(grad - dgrad) / np.linalg.norm(dgrad)))
    assert e[1][0] <= e[0][0] and e[1][1] <= e[0][1]
