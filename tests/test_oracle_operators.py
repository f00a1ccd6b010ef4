"""Pins of the oracle's spherical-harmonic expansions and translation operators.

Each check is fixed by mathematics independent of the oracle's code: closed
forms on the z axis, associated Legendre functions from scipy, harmonicity,
the addition theorem for 1/|x-y|, exactness of the multipole and local shifts,
the Greengard-Rokhlin truncation bound, and finite differences.  The
expansions are the spherical-harmonic ones the paper's kernels use (section
"Hybrid treecode/FMM algorithm")."""
import math

import numpy as np
import pytest
from scipy.special import lpmv

from oracle import oracle as O

H = O.hidx


def _sph(x):
    r = np.linalg.norm(x)
    return r, x[2] / r, math.atan2(x[1], x[0])


def test_z_axis_closed_forms():
    z = 0.7
    p = 12
    R = O.regular([0.0, 0.0, z], p)
    Ih = O.irregular([0.0, 0.0, z], p)
    for n in range(p + 1):
        assert R[H(n, 0)] == pytest.approx(z ** n / math.factorial(n), rel=1e-13)
        assert Ih[H(n, 0)] == pytest.approx(math.factorial(n) / z ** (n + 1), rel=1e-13)
        for m in range(1, n + 1):  # P_n^m(1) = 0 for m > 0
            assert abs(R[H(n, m)]) < 1e-15 and abs(Ih[H(n, -m)]) < 1e-9


@pytest.mark.parametrize("x", [[0.3, -0.4, 0.5], [-1.1, 0.2, -0.7], [0.05, 0.9, 0.01]])
def test_against_scipy_legendre(x):
    x = np.array(x)
    p = 10
    r, ct, ph = _sph(x)
    R = O.regular(x, p)
    Ih = O.irregular(x, p)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            P = lpmv(m, n, ct)  # includes the Condon-Shortley phase
            eR = r ** n * P * np.exp(1j * m * ph) / math.factorial(n + m)
            eI = math.factorial(n - m) * P * np.exp(1j * m * ph) / r ** (n + 1)
            assert abs(R[H(n, m)] - eR) <= 1e-12 * max(1.0, abs(eR))
            assert abs(Ih[H(n, m)] - eI) <= 1e-11 * max(1.0, abs(eI))


def test_harmonics_are_harmonic():
    # Both families solve Laplace's equation: the three second differences
    # cancel to O(h^2) relative to their own size.
    x = np.array([0.41, -0.33, 0.62])
    p, h = 6, 1e-3
    for fn in (O.regular, O.irregular):
        f0 = fn(x, p)
        terms = []
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            terms.append((fn(x + e, p) + fn(x - e, p) - 2.0 * f0) / (h * h))
        lap = terms[0] + terms[1] + terms[2]
        size = np.abs(terms[0]) + np.abs(terms[1]) + np.abs(terms[2])
        big = size > 1e-6 * size.max()
        assert np.all(np.abs(lap[big]) < 1e-4 * size[big])


def test_addition_theorem():
    # 1/|x - y| = sum_{n,m} conj(R_n^m(y)) I_n^m(x), |y| < |x|
    x = np.array([1.3, -0.7, 2.1])
    y = np.array([0.2, 0.1, -0.3])
    p = 40
    s = np.sum(np.conj(O.regular(y, p)) * O.irregular(x, p))
    assert s.real == pytest.approx(1.0 / np.linalg.norm(x - y), rel=1e-14)
    assert abs(s.imag) < 1e-15


def _cluster(n=25, seed=0, a=0.5):
    rng = np.random.default_rng(seed)
    y = rng.uniform(-a, a, (n, 3))
    q = rng.uniform(-1, 1, n)
    return y, q


def test_p2m_m2p_greengard_rokhlin_bound():
    y, q = _cluster()
    c = np.zeros(3)
    a = np.linalg.norm(y, axis=1).max()
    x = np.array([1.9, -0.8, 1.2])
    r = np.linalg.norm(x)
    exact = np.sum(q / np.linalg.norm(x - y, axis=1))
    errs = []
    for p in range(1, 13):
        M = O.p2m(c, y, q, p)
        err = abs(O.m2p(c, p, M, x) - exact)
        bound = np.abs(q).sum() / (r - a) * (a / r) ** (p + 1)
        assert err <= bound * (1 + 1e-9) + 1e-14
        errs.append(err)
    assert errs[-1] < 1e-3 * errs[0]


def test_m2m_is_exact():
    y, q = _cluster(seed=1, a=0.25)
    c = np.array([0.1, -0.05, 0.2])
    cp = np.array([0.35, 0.2, -0.05])
    for p in (3, 8, 12):
        shifted = O.m2m(c, cp, p, O.p2m(c, y, q, p))
        direct = O.p2m(cp, y, q, p)
        assert np.abs(shifted - direct).max() <= 1e-13 * np.abs(direct).max()


def _local_from_far_cluster(p, seed=2):
    y, q = _cluster(seed=seed, a=0.4)
    cs = np.zeros(3)
    ct = np.array([3.0, 1.0, -1.5])
    return y, q, cs, ct, O.m2l(cs, ct, p, O.p2m(cs, y, q, p))


def test_l2l_is_exact():
    p = 10
    y, q, cs, ct, L = _local_from_far_cluster(p)
    cc = ct + np.array([0.25, -0.25, 0.25])
    Lc = O.l2l(ct, cc, p, L)
    rng = np.random.default_rng(5)
    for _ in range(5):
        x = cc + rng.uniform(-0.2, 0.2, 3)
        a = O.l2p(ct, p, L, x)
        b = O.l2p(cc, p, Lc, x)
        assert b[0] == pytest.approx(a[0], rel=1e-12)
        assert np.allclose(b[1], a[1], rtol=1e-10, atol=1e-13)


def test_m2l_l2p_converges_to_m2p_and_direct():
    y, q = _cluster(seed=3, a=0.4)
    cs = np.zeros(3)
    ct = np.array([2.5, -1.0, 1.0])
    x = ct + np.array([0.3, -0.2, 0.25])
    exact = np.sum(q / np.linalg.norm(x - y, axis=1))
    gexact = -np.sum(q[:, None] * (x - y) / np.linalg.norm(x - y, axis=1)[:, None] ** 3, axis=0)
    prev = None
    for p in range(2, 15, 2):
        M = O.p2m(cs, y, q, p)
        L = O.m2l(cs, ct, p, M)
        phi, g = O.l2p(ct, p, L, x)
        err = abs(phi - exact) / abs(exact)
        gerr = np.linalg.norm(g - gexact) / np.linalg.norm(gexact)
        if prev is not None:
            assert err < 0.6 * prev[0] and gerr < 0.7 * prev[1]
        prev = (err, gerr)
    assert prev[0] < 1e-7 and prev[1] < 1e-6
    # M2L of a single charge at the source centre equals the exact local
    # expansion L_j^l = conj(I_j^l(c_s - c_t)) of 1/|x - c_s|.
    p = 6
    M = O.p2m(cs, cs[None, :], np.array([1.0]), p)
    L = O.m2l(cs, ct, p, M)
    expect = np.conj(O.irregular(cs - ct, p))
    assert np.abs(L - expect).max() <= 1e-14 * np.abs(expect).max()


def test_l2p_gradient_matches_finite_difference():
    p = 8
    _, _, _, ct, L = _local_from_far_cluster(p, seed=4)
    x = ct + np.array([0.1, 0.2, -0.15])
    h = 1e-5
    _, g = O.l2p(ct, p, L, x)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        fd = (O.l2p(ct, p, L, x + e)[0] - O.l2p(ct, p, L, x - e)[0]) / (2 * h)
        assert g[a] == pytest.approx(fd, rel=1e-6, abs=1e-9)
