"""The uniform 1M workload (N = 1,048,576 uniform cube, p = 10, theta = 0.4,
ncrit = 64, depth <= 10) in the configuration the benchmark times: structure
bit-exact against the oracle at full size, fields on sampled leaves against the
oracle's leaf-restricted evaluation, and sampled targets against the FP64
direct sum (the 1e-4 accuracy target at p = 10)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_5815_gb300 import inputs
from tests.gpu_helpers import assert_pointwise, canonical_ids, gpu_cells, gpu_solve, pair_codes, rel_l2

pytestmark = pytest.mark.gpu

W = inputs.WORKLOADS["uniform1m"]


@pytest.fixture(scope="module")
def solved():
    x, q = inputs.uniform_cube(W["n"], W["seed"])
    phi, grad, st = gpu_solve(x, q, W["p"], W["theta"], W["ncrit"], max_depth=W["max_depth"],
                              stats=True)
    from paper_1108_5815_gb300 import fmm
    exports = {k: fmm.export(k) for k in ("keys", "order", "p2p", "m2l")}
    exports["cells"] = gpu_cells()
    f = O.Fmm(x, q, W["p"], W["theta"], W["ncrit"], max_depth=W["max_depth"])
    return x, q, phi, grad, st, exports, f


def test_structure_bit_exact(solved):
    x, q, phi, grad, st, ex, f = solved
    key, order = f.sorted()
    assert np.array_equal(ex["keys"], key)
    assert np.array_equal(ex["order"].astype(np.int64), order)
    oc, gc = f.cells(), ex["cells"]
    oid, oord = canonical_ids(oc["level"], oc["prefix"])
    gid, gord = canonical_ids(gc["level"], gc["prefix"])
    for k in ("level", "prefix", "begin", "end", "nchild"):
        assert np.array_equal(np.asarray(oc[k])[oord], np.asarray(gc[k])[gord])
    ol = f.lists()
    assert np.array_equal(pair_codes(ol["p2p_t"], ol["p2p_s"], oid, f.ncells),
                          pair_codes(ex["p2p"][:, 0], ex["p2p"][:, 1], gid, f.ncells))
    assert np.array_equal(pair_codes(ol["m2l_t"], ol["m2l_s"], oid, f.ncells),
                          pair_codes(ex["m2l"][:, 0], ex["m2l"][:, 1], gid, f.ncells))
    assert st["n_m2l_pairs"] == f.nm2l and st["n_p2p_pairs"] == f.np2p


def test_sampled_leaves_match_oracle(solved):
    x, q, phi, grad, st, ex, f = solved
    c = f.cells()
    leaves = np.flatnonzero(c["nchild"] == 0)
    pick = leaves[inputs.sample_indices(len(leaves), 48, 77)]
    pos, ophi, ograd = f.evaluate_leaves(pick)
    orig = f.sorted()[1][pos]
    assert rel_l2(phi[orig], ophi) < 1e-5
    assert rel_l2(grad[orig], ograd) < 1e-5
    assert_pointwise(phi[orig], ophi, grad[orig], ograd, 1e-4)


def test_sampled_targets_vs_direct(solved):
    x, q, phi, grad, st, ex, f = solved
    t = inputs.sample_indices(len(q), 2048, 1009)
    pd, gd = O.direct(x, q, targets=t)
    assert rel_l2(phi[t], pd) < 1e-4
    assert rel_l2(grad[t], gd) < 1e-4
    # the worst sampled target against the FP64 direct sum (the 1e-4 target at p = 10)
    assert_pointwise(phi[t], pd, grad[t], gd, 1e-4)


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_tensor_core_modes_at_full_size(solved, precision):
    """The tensor-core M2L modes on the same workload: the metric's 1e-4 against the
    FP64 direct sum, and the FP32 path's 1e-5 against the oracle (main and
    correction products accumulate separately and are summed with round-to-nearest)."""
    x, q, phi0, grad0, st, ex, f = solved
    phi, grad = gpu_solve(x, q, W["p"], W["theta"], W["ncrit"], max_depth=W["max_depth"],
                          precision=precision)
    t = inputs.sample_indices(len(q), 1024, 1013)
    pd, gd = O.direct(x, q, targets=t)
    assert rel_l2(phi[t], pd) < 1e-4 and rel_l2(grad[t], gd) < 1e-4
    c = f.cells()
    leaves = np.flatnonzero(c["nchild"] == 0)
    pick = leaves[inputs.sample_indices(len(leaves), 32, 79)]
    pos, ophi, ograd = f.evaluate_leaves(pick)
    orig = f.sorted()[1][pos]
    assert rel_l2(phi[orig], ophi) < 1e-5 and rel_l2(grad[orig], ograd) < 1e-5
    assert_pointwise(phi[orig], ophi, grad[orig], ograd, 1e-4)
