"""Pins of the oracle's whole FMM against the exact direct sum.

* Error falls geometrically in p at fixed theta; p = 10 reaches about four
  significant digits or better (the paper: "p=10 giving an accuracy of 4
  significant digits in the potential for the Laplace kernel").
* A tiny theta sends every pair to the near field and reproduces the direct sum.
* The leaf-sampled evaluation (used at full size) agrees with the full one."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_5815_gb300 import inputs


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dist,theta", [("uniform", 0.5), ("plummer", 0.4)])
def test_error_falls_geometrically_in_p(dist, theta):
    x, q = inputs.make(dist, 3000, 31) if dist == "uniform" else inputs.plummer(3000, 31, equal_charges=False)
    pd, gd = O.direct(x, q)
    errs = []
    for p in range(1, 13):
        phi, g = O.Fmm(x, q, p, theta, 32).evaluate()
        errs.append((rel_l2(phi, pd), rel_l2(g, gd)))
    e = np.array(errs)
    # geometric decay: every 3 orders gain at least a factor 3
    assert np.all(e[3:, 0] < e[:-3, 0] / 3.0) and np.all(e[3:, 1] < e[:-3, 1] / 3.0)
    assert e[9, 0] < 1e-4 and e[9, 1] < 1e-4          # p = 10: four digits or better


def test_tiny_theta_is_direct_sum():
    x, q = inputs.uniform_cube(800, 8)
    phi, g = O.Fmm(x, q, 3, 1e-3, 8).evaluate()
    pd, gd = O.direct(x, q)
    assert rel_l2(phi, pd) < 1e-13 and rel_l2(g, gd) < 1e-13


def test_leaf_sampled_evaluation_matches_full():
    x, q = inputs.uniform_cube(5000, 12)
    f = O.Fmm(x, q, 6, 0.4, 32)
    phi, g = f.evaluate()
    c = f.cells()
    leaves = np.flatnonzero(c["nchild"] == 0)[::7]
    pos, ps, gs = f.evaluate_leaves(leaves)
    order = f.sorted()[1]
    assert np.allclose(ps, phi[order[pos]], rtol=1e-12, atol=1e-12)
    assert np.allclose(gs, g[order[pos]], rtol=1e-11, atol=1e-11)


def test_literal_leaf_first_variant_is_also_consistent():
    x, q = inputs.uniform_cube(2000, 13)
    pd, gd = O.direct(x, q)
    f1 = O.Fmm(x, q, 8, 0.5, 16)
    f2 = O.Fmm(x, q, 8, 0.5, 16, leaf_first=True)
    assert f2.np2p >= f1.np2p and f2.nm2l <= f1.nm2l
    assert rel_l2(f2.evaluate()[0], pd) <= rel_l2(f1.evaluate()[0], pd) * 1.5
