"""Pins of the oracle's exact direct sum against closed forms and invariants.

The direct sum is the definition of what the FMM approximates: the Laplace
potential and its gradient over all pairs (the O(N^2) all-pairs summation of
the paper's Introduction), with coincident pairs skipped."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_5815_gb300 import inputs


def test_two_charges_closed_form():
    x = np.array([[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]])
    q = np.array([1.0, 3.0])
    phi, g = O.direct(x, q)
    # phi_0 = 3/2, phi_1 = 1/2; grad_0 = -3*(0-2)/8 = +0.75 in x, grad_1 = -1*(2-0)/8 = -0.25
    assert phi == pytest.approx([1.5, 0.5], abs=1e-15)
    assert g[0] == pytest.approx([0.75, 0.0, 0.0], abs=1e-15)
    assert g[1] == pytest.approx([-0.25, 0.0, 0.0], abs=1e-15)


def test_cube_corners_closed_form():
    # unit charges on the 8 corners of the unit cube: each corner sees 3 edges,
    # 3 face diagonals and 1 body diagonal; by symmetry the potential gradient
    # at a corner points along the body diagonal towards the centre.
    corners = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], float)
    q = np.ones(8)
    phi, g = O.direct(corners, q)
    expect_phi = 3.0 + 3.0 / math.sqrt(2.0) + 1.0 / math.sqrt(3.0)
    assert np.allclose(phi, expect_phi, rtol=0, atol=1e-14)
    # x-component at the origin corner: -sum q (0 - xj)/r^3 over others
    # = sum xj / r^3 = 1 + 2/(2*sqrt2) + 1/(3*sqrt3)
    gx = 1.0 + 2.0 / (2.0 * math.sqrt(2.0)) + 1.0 / (3.0 * math.sqrt(3.0))
    assert g[0] == pytest.approx([gx, gx, gx], abs=1e-14)
    assert g[7] == pytest.approx([-gx, -gx, -gx], abs=1e-14)


def test_coincident_pairs_skipped():
    x = np.array([[0.5, 0.5, 0.5], [0.5, 0.5, 0.5], [1.5, 0.5, 0.5]])
    q = np.array([1.0, 2.0, 4.0])
    phi, g = O.direct(x, q)
    assert phi[0] == pytest.approx(4.0)      # the coincident charge contributes nothing
    assert phi[2] == pytest.approx(3.0)
    assert np.all(np.isfinite(g))


@pytest.mark.parametrize("dist", ["uniform", "plummer"])
def test_net_force_vanishes(dist):
    # Newton's third law: sum_i q_i grad_i = 0 for the exact pairwise sum.
    x, q = inputs.make(dist, 1500, 7) if dist != "plummer" else inputs.plummer(1500, 7, equal_charges=False)
    phi, g = O.direct(x, q)
    f = (q.astype(np.float64)[:, None] * g).sum(axis=0)
    scale = np.abs(q.astype(np.float64)[:, None] * g).sum()
    assert np.all(np.abs(f) <= 1e-12 * scale)


def test_targets_subset_and_scaling():
    x, q = inputs.uniform_cube(600, 3)
    t = np.array([0, 17, 599])
    phi_all, g_all = O.direct(x, q)
    phi_t, g_t = O.direct(x, q, targets=t)
    assert np.array_equal(phi_t, phi_all[t]) and np.array_equal(g_t, g_all[t])
    # homogeneity: scaling positions by 2 halves phi and quarters grad
    phi2, g2 = O.direct(2.0 * x.astype(np.float64), q)
    assert np.allclose(phi2, 0.5 * phi_all, rtol=1e-13, atol=0)
    assert np.allclose(g2, 0.25 * g_all, rtol=1e-12, atol=1e-12 * np.abs(g_all).max())
