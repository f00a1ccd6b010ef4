"""Pins of the oracle's cell-particle interaction (M2P, the treecode kernel) and
of selection-table value 2 (reading R9; the paper's treecode performs
cell-particle interactions for every accepted pair, Results section).

* the M2P gradient against central differences of the M2P potential;
* M2P of a cluster converges to the direct potential and field with p;
* a table of all 2 is the treecode: no cell-cell pairs, every ordered particle
  pair covered exactly once, error falling with p;
* mixed tables keep the coverage exact."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_5815_gb300 import inputs
from tests.oracle_helpers import coverage_matrix

NB = O.SEL_NB


def _cluster(seed=0, n=40, a=0.3):
    rng = np.random.default_rng(seed)
    y = rng.uniform(-a, a, (n, 3)) / np.sqrt(3)
    return y, rng.uniform(-1, 1, n)


def test_m2p_gradient_matches_central_differences():
    y, q = _cluster()
    c = np.array([0.02, -0.01, 0.03])
    x = np.array([1.3, 0.7, -0.9])
    for p in (1, 4, 9):
        M = O.p2m(c, y, q, p)
        phi, g = O.m2p_grad(c, p, M, x)
        assert abs(phi - O.m2p(c, p, M, x)) <= 1e-14 * abs(phi)
        h = 1e-5
        fd = np.array([(O.m2p(c, p, M, x + h * e) - O.m2p(c, p, M, x - h * e)) / (2 * h) for e in np.eye(3)])
        assert np.max(np.abs(fd - g)) <= 1e-8 * np.max(np.abs(g))


def test_m2p_converges_to_direct_field():
    y, q = _cluster(seed=2)
    c = np.zeros(3)
    x = np.array([1.1, -0.9, 0.6])
    d = x - y
    r = np.linalg.norm(d, axis=1)
    phi_ex = np.sum(q / r)
    g_ex = -np.sum(q[:, None] * d / r[:, None] ** 3, axis=0)
    errs = []
    for p in range(1, 15):
        phi, g = O.m2p_grad(c, p, O.p2m(c, y, q, p), x)
        errs.append(np.linalg.norm(g - g_ex) / np.linalg.norm(g_ex))
        assert abs(phi - phi_ex) / abs(phi_ex) < 0.5 * 0.4 ** p + 1e-14
    assert errs[-1] < 1e-5 * errs[0]


@pytest.mark.parametrize("dist,ncrit", [("uniform", 8), ("plummer", 4), ("shell", 6)])
def test_treecode_table_covers_every_pair_once(dist, ncrit):
    x, q = inputs.make(dist, 1200, 55)
    f = O.Fmm(x, q, 3, 0.5, ncrit, sel=np.full((NB, NB), 2, np.uint8))
    assert f.nm2l == 0
    L = f.lists()
    L["m2p_t"], L["m2p_s"] = f.m2p_list()
    assert len(L["m2p_t"]) > 0
    assert np.all(coverage_matrix(f.N, f.cells(), L) == 1)


def test_treecode_error_falls_with_p():
    x, q = inputs.make("uniform", 4000, 9)
    dphi, dgrad = O.direct(x, q)
    e = []
    for p in (2, 4, 6, 8):
        phi, grad = O.Fmm(x, q, p, 0.5, 16, sel=np.full((NB, NB), 2, np.uint8)).evaluate()
        e.append(np.linalg.norm(grad - dgrad) / np.linalg.norm(dgrad))
    assert all(b < 0.5 * a for a, b in zip(e, e[1:]))
    assert e[-1] < 1e-4


def test_mixed_tables_keep_coverage_and_accuracy():
    rng = np.random.default_rng(8)
    x, q = inputs.make("plummer", 1000, 13)
    for _ in range(3):
        sel = rng.integers(0, 3, (NB, NB)).astype(np.uint8)
        f = O.Fmm(x, q, 6, 0.5, 4, sel=sel)
        L = f.lists()
        L["m2p_t"], L["m2p_s"] = f.m2p_list()
        assert np.all(coverage_matrix(f.N, f.cells(), L) == 1)
        dphi, _ = O.direct(x, q)
        phi, _ = f.evaluate()
        assert np.linalg.norm(phi - dphi) / np.linalg.norm(dphi) < 1e-3


def test_p2l_converges_to_direct_field():
    # charges far from the expansion centre; evaluation points near it
    y, q = _cluster(seed=5, n=30, a=0.3)
    y = y + np.array([2.2, -1.1, 0.9])
    c = np.zeros(3)
    x = np.array([0.15, -0.1, 0.2])
    d = x - y
    r = np.linalg.norm(d, axis=1)
    phi_ex = np.sum(q / r)
    g_ex = -np.sum(q[:, None] * d / r[:, None] ** 3, axis=0)
    prev = None
    for p in range(2, 15, 2):
        phi, g = O.l2p(c, p, O.p2l(c, y, q, p), x)
        err = np.linalg.norm(g - g_ex) / np.linalg.norm(g_ex)
        assert abs(phi - phi_ex) / abs(phi_ex) < 0.2 ** p
        if prev is not None:
            assert err < 0.5 * prev
        prev = err
    assert prev < 1e-7


@pytest.mark.parametrize("dist,ncrit", [("uniform", 6), ("plummer", 3)])
def test_p2l_table_covers_every_pair_once_and_stays_accurate(dist, ncrit):
    x, q = inputs.make(dist, 1100, 71)
    rng = np.random.default_rng(3)
    for sel in (np.full((NB, NB), 3, np.uint8), rng.integers(0, 4, (NB, NB)).astype(np.uint8)):
        f = O.Fmm(x, q, 8, 0.5, ncrit, sel=sel)
        L = f.lists()
        L["m2p_t"], L["m2p_s"] = f.m2p_list()
        L["p2l_t"], L["p2l_s"] = f.p2l_list()
        assert len(L["p2l_t"]) > 0
        assert np.all(coverage_matrix(f.N, f.cells(), L) == 1)
        dphi, dgrad = O.direct(x, q)
        phi, grad = f.evaluate()
        assert np.linalg.norm(grad - dgrad) / np.linalg.norm(dgrad) < 1e-3
