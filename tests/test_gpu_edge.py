"""Edge cases and error behaviour of the C ABI on the GPU."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_5815_gb300 import inputs
from tests.gpu_helpers import gpu_solve, rel_l2, torch_cuda

pytestmark = pytest.mark.gpu


def test_single_particle():
    phi, grad = gpu_solve(np.array([[0.3, 0.2, 0.1]], np.float32), np.array([2.0], np.float32), 4, 0.5, 8)
    assert phi[0] == 0 and np.all(grad == 0)


def test_two_particles_closed_form():
    x = np.array([[0, 0, 0], [2, 0, 0]], np.float32)
    phi, grad = gpu_solve(x, np.array([1.0, 3.0], np.float32), 4, 0.5, 1)
    assert np.allclose(phi, [1.5, 0.5], rtol=1e-6)
    assert np.allclose(grad, [[0.75, 0, 0], [-0.25, 0, 0]], rtol=1e-6, atol=1e-7)


def test_identical_points_give_zero():
    x = np.tile(np.array([[0.4, 0.4, 0.4]], np.float32), (100, 1))
    phi, grad = gpu_solve(x, np.ones(100, np.float32), 5, 0.5, 4)
    assert np.all(phi == 0) and np.all(grad == 0)


def test_root_leaf_equals_direct():
    x, q = inputs.uniform_cube(60, 1)
    phi, grad = gpu_solve(x, q, 4, 0.5, 64)
    pd, gd = O.direct(x, q)
    assert rel_l2(phi, pd) < 1e-6 and rel_l2(grad, gd) < 1e-6


def test_depth_cap_and_box_faces():
    # lattice corners sit on the maximum faces; depth 2 forces crowded leaves
    g = np.stack(np.meshgrid(*[np.linspace(0, 1, 9)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = g.astype(np.float32)
    q = np.resize(np.array([1, -1, 0.5], np.float32), len(x))
    phi, grad = gpu_solve(x, q, 6, 0.5, 4, max_depth=2)
    f = O.Fmm(x, q, 6, 0.5, 4, max_depth=2)
    ophi, ograd = f.evaluate()
    assert rel_l2(phi, ophi) < 1e-5 and rel_l2(grad, ograd) < 1e-5


def test_pair_below_float_resolution_across_a_leaf_face_is_dropped():
    # box [-h, h)^3 with h = 2^-20: the face x = 0 puts two particles 2e-21 apart
    # in different leaves; their r^2 is below the smallest normal float, so the
    # P2P kernel drops the pair as it drops a coincident one (a pass that meets it
    # outside the target's own leaf is redone with the r = 0 guard on every pair)
    h = 2.0 ** -20
    x, q = inputs.uniform_cube(3000, 11)
    x = ((2.0 * x.astype(np.float64) - 1.0) * h).astype(np.float32)
    x[2], x[3] = -h, h                                      # box corners
    x[0] = np.array([-1e-21, 0.3 * h, -0.2 * h], np.float32)
    x[1] = np.array([1e-21, 0.3 * h, -0.2 * h], np.float32)
    p, theta, ncrit = 6, 0.5, 16
    phi, grad = gpu_solve(x, q, p, theta, ncrit)
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(grad))
    k = O.morton_keys(x)[2]
    assert (k[0] >> np.uint64(60)) != (k[1] >> np.uint64(60))  # different cells from level 1 on
    ophi, ograd = O.Fmm(x, q, p, theta, ncrit).evaluate()
    rest = np.arange(2, len(x))
    assert rel_l2(phi[rest], ophi[rest]) < 1e-5 and rel_l2(grad[rest], ograd[rest]) < 1e-5
    for i, j in ((0, 1), (1, 0)):  # each of the two sees everything but the other
        qj = q.copy()
        qj[j] = 0.0
        ephi, egrad = O.Fmm(x, qj, p, theta, ncrit).evaluate()
        assert abs(phi[i] - ephi[i]) <= 1e-4 * abs(ephi[i])
        assert np.linalg.norm(grad[i] - egrad[i]) <= 1e-4 * np.linalg.norm(egrad[i])


@pytest.mark.parametrize("n", [33, 65, 129, 257, 1025])
def test_ragged_small_sizes(n):
    x, q = inputs.plummer(n, n, equal_charges=False)
    phi, grad = gpu_solve(x, q, 5, 0.5, 4)
    ophi, ograd = O.Fmm(x, q, 5, 0.5, 4).evaluate()
    assert rel_l2(phi, ophi) < 1e-5 and rel_l2(grad, ograd) < 1e-5


def test_nonfinite_input_reported():
    from paper_1108_5815_gb300 import fmm
    x, q = inputs.uniform_cube(1000, 2)
    for bad in (np.nan, np.inf):
        xb = x.copy()
        xb[17, 1] = bad
        with pytest.raises(fmm.FmmError) as e:
            gpu_solve(xb, q, 4, 0.5, 16)
        assert e.value.status == fmm.FMM_ERR_NONFINITE
    # the context stays usable
    phi, _ = gpu_solve(x, q, 4, 0.5, 16)
    assert np.all(np.isfinite(phi))


@pytest.mark.parametrize("p,theta,ncrit", [(0, 0.5, 8), (21, 0.5, 8), (4, 0.0, 8), (4, 1.0, 8),
                                           (4, 0.5, 0)])
def test_bad_arguments(p, theta, ncrit):
    from paper_1108_5815_gb300 import fmm
    x, q = inputs.uniform_cube(100, 2)
    with pytest.raises(fmm.FmmError) as e:
        gpu_solve(x, q, p, theta, ncrit)
    assert e.value.status == fmm.FMM_ERR_ARG


def test_null_pointers_and_empty():
    from paper_1108_5815_gb300 import fmm
    L = fmm.load()
    assert L.fmm_laplace3d(None, None, 10, 4, 0.5, 8, None, None, None) == fmm.FMM_ERR_ARG
    assert "null" in fmm.last_error()
    import torch
    z = torch.zeros(3, device="cuda")
    assert L.fmm_laplace3d(z.data_ptr(), z.data_ptr(), 0, 4, 0.5, 8, z.data_ptr(), z.data_ptr(),
                           None) == fmm.FMM_ERR_ARG


def test_bounded_wait_reports_timeout_and_context_survives():
    """Failure detection without a GPU fault: a wait that nothing satisfies gives up
    after its poll limit, the host reads FMM_ERR_TIMEOUT from the device flag, and
    the next solve on the same context succeeds."""
    torch = torch_cuda()
    from paper_1108_5815_gb300 import fmm
    assert fmm.selftest_wait_timeout(1 << 14) == fmm.FMM_ERR_TIMEOUT
    assert "bounded" in fmm.last_error()
    x, q = inputs.uniform_cube(5000, 8)
    phi, grad = gpu_solve(x, q, 4, 0.5, 32)
    f = O.Fmm(x, q, 4, 0.5, 32)
    ophi, ograd = f.evaluate()
    assert rel_l2(phi, ophi) < 1e-5


def test_tree_read_back_once_when_sizes_repeat():
    # a solve of the same N, ncrit and depth limit as the previous one builds the
    # tree with the level ranges on the device (one read-back); the result equals
    # the level-by-level build of the first solve bit for bit
    from paper_1108_5815_gb300 import fmm
    torch = torch_cuda()
    x0, q0 = inputs.uniform_cube(1500, 90)
    gpu_solve(x0, q0, 5, 0.5, 16)  # another N first: the next solve builds level by level
    x, q = inputs.uniform_cube(40000, 91)
    xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    first = [t.cpu().numpy() for t in fmm.laplace3d(xt, qt, 6, 0.5, 32)]
    again = [t.cpu().numpy() for t in fmm.laplace3d(xt, qt, 6, 0.5, 32)]
    assert np.array_equal(first[0], again[0]) and np.array_equal(first[1], again[1])
    # same N, far deeper tree: the capacities of the previous solve do not hold, the
    # tree is rebuilt level by level, and the result still matches the oracle
    xp, qp = inputs.plummer(40000, 92, equal_charges=False)
    phi, grad = gpu_solve(xp, qp, 6, 0.5, 32)
    ophi, ograd = O.Fmm(xp, qp, 6, 0.5, 32).evaluate()
    assert rel_l2(phi, ophi) < 1e-5 and rel_l2(grad, ograd) < 1e-5


def test_fp32_ceilings_bound_the_p2p_kernel():
    # the interaction body on staged sources is an upper bound of the P2P kernel's
    # rate, and the FMA stream bounds the body (16 FP32-pipe lane operations per
    # interaction, 2 flop per FMA lane operation)
    from paper_1108_5815_gb300 import fmm
    torch_cuda()
    c = fmm.measure_fp32()
    assert c["ffma_tflops"] > 1 and c["body_interactions_per_s"] > 1e9
    assert c["body_interactions_per_s"] * 16 * 2 <= 1.05 * c["ffma_tflops"] * 1e12
    x, q = inputs.uniform_cube(1 << 18, 93)
    _, _, st = gpu_solve(x, q, 6, 0.5, 64, stats=True)
    rate = st["n_p2p_interactions"] / (st["ms_p2p"] * 1e-3)
    assert rate <= 1.05 * c["body_interactions_per_s"]


@pytest.mark.parametrize("dist", ["uniform", "plummer"])
def test_tree_from_previous_capacities_is_bit_exact(dist):
    # A second solve with the same N, ncrit and depth limit builds its tree with the
    # level ranges on the device (the first levels in one block, the rest level by
    # level): on new points its keys, order, cells and lists must still equal the
    # oracle's bit for bit, and its fields must match.
    from tests.test_gpu_parity import _compare_structure
    n = 50000
    x0, q0 = inputs.make(dist, n, 301)
    gpu_solve(x0, q0, 5, 0.5, 24)
    x, q = inputs.make(dist, n, 302)
    phi, grad = gpu_solve(x, q, 5, 0.5, 24)
    f = O.Fmm(x, q, 5, 0.5, 24)
    _compare_structure(f)
    ophi, ograd = f.evaluate()
    assert rel_l2(phi, ophi) < 1e-5 and rel_l2(grad, ograd) < 1e-5
