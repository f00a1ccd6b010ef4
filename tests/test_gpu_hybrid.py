"""Hybrid selection on the GPU vs the oracle (reading R9: the interaction type
of a MAC-accepted pair comes from a table over the count buckets of the two
cells; P2P may be taken above the leaf level).

Bit-exact: cells and both pair sets, with the oracle's P2P pairs expanded to
the target leaves below them.  Within 1e-5 relative L2 of the oracle: phi and
grad.  An all-P2P table leaves no far field: the result is the direct sum."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_5815_gb300 import inputs
from tests.gpu_helpers import (canonical_ids, expand_p2p_to_leaves, gpu_cells, gpu_solve,
                               pair_codes, rel_l2)

pytestmark = pytest.mark.gpu

NB = 128
TOL_ORACLE = 1e-5


def threshold_table(k):
    """P2P iff the product of the two buckets' smallest counts is <= k."""
    lo = np.zeros(NB, dtype=np.int64)
    for n in range(1, 1 << 16):
        b = O.count_bucket(n)
        if lo[b] == 0:
            lo[b] = n
    lo[lo == 0] = 1 << 40
    return (lo[:, None] * lo[None, :] <= k).astype(np.uint8)


def _compare(f, sel):
    from paper_1108_5815_gb300 import fmm
    assert np.array_equal(fmm.export("select"), sel)
    oc, gc = f.cells(), gpu_cells()
    assert len(gc["level"]) == f.ncells
    oid, oord = canonical_ids(oc["level"], oc["prefix"])
    gid, gord = canonical_ids(gc["level"], gc["prefix"])
    for k in ("level", "prefix", "begin", "end", "nchild"):
        assert np.array_equal(np.asarray(oc[k])[oord], np.asarray(gc[k])[gord]), k
    ol = f.lists()
    et, es = expand_p2p_to_leaves(oc, ol["p2p_t"], ol["p2p_s"])
    gp, gm = fmm.export("p2p"), fmm.export("m2l")
    assert np.array_equal(pair_codes(et, es, oid, f.ncells), pair_codes(gp[:, 0], gp[:, 1], gid, f.ncells))
    assert np.array_equal(pair_codes(ol["m2l_t"], ol["m2l_s"], oid, f.ncells),
                          pair_codes(gm[:, 0], gm[:, 1], gid, f.ncells))
    qt, qs = f.m2p_list()
    et, es = expand_p2p_to_leaves(oc, qt, qs)
    gq = fmm.export("m2p")
    assert np.array_equal(pair_codes(et, es, oid, f.ncells), pair_codes(gq[:, 0], gq[:, 1], gid, f.ncells))
    lt, ls = f.p2l_list()  # particle-cell pairs stay at their target cell
    gl = fmm.export("p2l")
    assert np.array_equal(pair_codes(lt, ls, oid, f.ncells), pair_codes(gl[:, 0], gl[:, 1], gid, f.ncells))
    return np.any(oc["nchild"][ol["p2p_t"]] > 0)


CASES = [
    ("uniform30k_k256", "uniform", 30000, 5, 0.5, 8, 256),
    ("plummer25k_k1024", "plummer", 25000, 6, 0.4, 4, 1024),
    ("shell15k_k64", "shell", 15000, 4, 0.5, 4, 64),
    ("uniform12k_k4096_ncrit32", "uniform", 12000, 8, 0.5, 32, 4096),
]


@pytest.mark.parametrize("name,dist,n,p,theta,ncrit,k", CASES, ids=[c[0] for c in CASES])
def test_threshold_table_matches_oracle(name, dist, n, p, theta, ncrit, k):
    x, q = inputs.make(dist, n, 900 + n)
    sel = threshold_table(k)
    phi, grad, st = gpu_solve(x, q, p, theta, ncrit, stats=True, select=sel)
    f = O.Fmm(x, q, p, theta, ncrit, sel=sel)
    above = _compare(f, sel)
    assert above  # P2P above the leaf level is exercised
    assert st["n_m2l_pairs"] == f.nm2l
    ophi, ograd = f.evaluate()
    assert rel_l2(phi, ophi) < TOL_ORACLE
    assert rel_l2(grad, ograd) < TOL_ORACLE


def test_random_table_matches_oracle():
    rng = np.random.default_rng(11)
    sel = (rng.random((NB, NB)) < 0.3).astype(np.uint8)
    x, q = inputs.make("plummer", 20000, 31)
    phi, grad = gpu_solve(x, q, 4, 0.5, 6, select=sel)
    f = O.Fmm(x, q, 4, 0.5, 6, sel=sel)
    _compare(f, sel)
    ophi, ograd = f.evaluate()
    assert rel_l2(phi, ophi) < TOL_ORACLE and rel_l2(grad, ograd) < TOL_ORACLE


def test_all_p2p_table_is_direct_sum():
    sel = np.ones((NB, NB), np.uint8)
    x, q = inputs.make("uniform", 16000, 5)
    phi, grad, st = gpu_solve(x, q, 4, 0.5, 8, stats=True, select=sel)
    assert st["n_m2l_pairs"] == 0
    assert st["n_p2p_interactions"] == 16000 * 16000
    dphi, dgrad = O.direct(x, q)
    assert rel_l2(phi, dphi) < 1e-5 and rel_l2(grad, dgrad) < 1e-5


def test_all_m2l_table_is_plain_and_tensor_modes_agree():
    x, q = inputs.make("uniform", 20000, 8)
    phi0, grad0 = gpu_solve(x, q, 6, 0.5, 16)
    phi1, grad1 = gpu_solve(x, q, 6, 0.5, 16, select=np.zeros((NB, NB), np.uint8))
    assert np.array_equal(phi0, phi1) and np.array_equal(grad0, grad1)
    sel = threshold_table(512)
    f = O.Fmm(x, q, 6, 0.5, 16, sel=sel)
    ophi, ograd = f.evaluate()
    for prec in ("tf32x3", "bf16x3"):
        phi, grad = gpu_solve(x, q, 6, 0.5, 16, precision=prec, select=sel)
        assert rel_l2(phi, ophi) < TOL_ORACLE and rel_l2(grad, ograd) < TOL_ORACLE


def test_batched_with_table_matches_separate_solves():
    torch = pytest.importorskip("torch")
    from paper_1108_5815_gb300 import fmm
    sel = threshold_table(256)
    x, q, off = inputs.batched_systems(6, 77, nmin=2000, nmax=9000)
    xt, qt = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    phi, grad = fmm.laplace3d_batched(xt, qt, off, 5, 0.5, 6, select=sel)
    phi, grad = phi.cpu().numpy(), grad.cpu().numpy()
    for s in range(6):
        a, b = int(off[s]), int(off[s + 1])
        f = O.Fmm(x[a:b], q[a:b], 5, 0.5, 6, sel=sel)
        ophi, ograd = f.evaluate()
        assert rel_l2(phi[a:b], ophi) < TOL_ORACLE and rel_l2(grad[a:b], ograd) < TOL_ORACLE


@pytest.mark.parametrize("dist,n,p,theta,ncrit", [("uniform", 20000, 5, 0.5, 8), ("plummer", 15000, 8, 0.4, 6),
                                                  ("shell", 12000, 4, 0.5, 12)])
def test_treecode_matches_oracle(dist, n, p, theta, ncrit):
    from paper_1108_5815_gb300 import fmm
    x, q = inputs.make(dist, n, 300 + n)
    phi, grad, st = gpu_solve(x, q, p, theta, ncrit, stats=True, select="treecode")
    sel = np.full((NB, NB), 2, np.uint8)
    f = O.Fmm(x, q, p, theta, ncrit, sel=sel)
    _compare(f, sel)
    assert st["n_m2l_pairs"] == 0 and st["n_m2p_pairs"] > 0
    ophi, ograd = f.evaluate()
    assert rel_l2(phi, ophi) < TOL_ORACLE and rel_l2(grad, ograd) < TOL_ORACLE


def test_three_way_random_table_matches_oracle():
    rng = np.random.default_rng(21)
    sel = rng.integers(0, 3, (NB, NB)).astype(np.uint8)
    x, q = inputs.make("plummer", 25000, 61)
    phi, grad = gpu_solve(x, q, 6, 0.45, 5, select=sel)
    f = O.Fmm(x, q, 6, 0.45, 5, sel=sel)
    _compare(f, sel)
    ophi, ograd = f.evaluate()
    assert rel_l2(phi, ophi) < TOL_ORACLE and rel_l2(grad, ograd) < TOL_ORACLE


@pytest.mark.parametrize("dist,n,p,theta,ncrit,seed", [("plummer", 20000, 8, 0.45, 5, 23),
                                                       ("uniform", 25000, 10, 0.4, 8, 24)])
def test_four_way_table_with_p2l_matches_oracle(dist, n, p, theta, ncrit, seed):
    rng = np.random.default_rng(seed)
    sel = rng.integers(0, 4, (NB, NB)).astype(np.uint8)
    x, q = inputs.make(dist, n, 700 + seed)
    phi, grad, st = gpu_solve(x, q, p, theta, ncrit, stats=True, select=sel)
    f = O.Fmm(x, q, p, theta, ncrit, sel=sel)
    _compare(f, sel)
    assert st["n_p2l_pairs"] > 0
    ophi, ograd = f.evaluate()
    assert rel_l2(phi, ophi) < TOL_ORACLE and rel_l2(grad, ograd) < TOL_ORACLE


def test_all_p2l_table_matches_oracle():
    sel = np.full((NB, NB), 3, np.uint8)
    x, q = inputs.make("uniform", 20000, 19)
    phi, grad, st = gpu_solve(x, q, 6, 0.5, 16, stats=True, select=sel)
    assert st["n_m2l_pairs"] == 0 and st["n_p2l_pairs"] > 0
    f = O.Fmm(x, q, 6, 0.5, 16, sel=sel)
    _compare(f, sel)
    ophi, ograd = f.evaluate()
    assert rel_l2(phi, ophi) < TOL_ORACLE and rel_l2(grad, ograd) < TOL_ORACLE
