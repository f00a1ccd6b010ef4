"""Captured plans (fmm_plan_*): the solve with every size on the device, captured
into one CUDA graph and replayed for new particle data.

* a replay of the plan's own first input gives exactly the plain solve's result,
  and that result matches the oracle at equal p and theta;
* replays on new positions and on new charges that fit the plan equal the plain
  solve of the same data bit for bit, with no synchronisation between replays;
* batched systems, the tensor-core M2L and hybrid tables (M2P and P2L lists)
  replay the same way;
* a replay that needs a deeper tree than the plan holds is reported as
  FMM_ERR_CAPACITY, the context stays usable, and the next fitting replay of the
  same plan is valid again;
* the graph holds the whole solve: its kernel nodes are every launch of a solve."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1108_5815_gb300 import inputs
from tests.gpu_helpers import rel_l2, torch_cuda

pytestmark = pytest.mark.gpu

CAPACITY = 3


def _dev(x, q):
    torch = torch_cuda()
    return (torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda())


def _plain(xt, qt, p, theta, ncrit, **kw):
    from paper_1108_5815_gb300 import fmm
    torch = torch_cuda()
    phi, grad = fmm.laplace3d(xt, qt, p, theta, ncrit, replay=False, **kw)
    torch.cuda.synchronize()
    return phi.cpu().numpy(), grad.cpu().numpy()


def _replay(plan, xt=None, qt=None):
    phi, grad = plan.execute(xt, qt)
    status = plan.check()
    return status, phi.cpu().numpy(), grad.cpu().numpy()


def test_replay_equals_plain_solve_and_oracle():
    from paper_1108_5815_gb300 import fmm
    x, q = inputs.uniform_cube(20000, 301)
    xt, qt = _dev(x, q)
    p, theta, ncrit = 6, 0.5, 32
    phi0, grad0 = _plain(xt, qt, p, theta, ncrit)
    plan = fmm.Plan(xt, qt, p, theta, ncrit)
    for _ in range(2):  # the plan's own input, twice: same result each time
        status, phi1, grad1 = _replay(plan)
        assert status == 0
        assert np.array_equal(phi1, phi0) and np.array_equal(grad1, grad0)
    ophi, ograd = O.Fmm(x, q, p, theta, ncrit).evaluate()
    assert rel_l2(phi1, ophi) < 1e-5 and rel_l2(grad1, ograd) < 1e-5
    info = plan.info()
    assert info["last_valid"] == 1 and info["graph_kernels"] > 50 and info["graph_nodes"] >= info["graph_kernels"]
    plan.close()


def test_replays_on_new_positions_and_charges():
    from paper_1108_5815_gb300 import fmm
    torch = torch_cuda()
    p, theta, ncrit = 6, 0.45, 24
    data = [inputs.uniform_cube(30000, s) for s in (401, 402, 403)]
    dev = [_dev(x, q) for x, q in data]
    plain = [_plain(xt, qt, p, theta, ncrit) for xt, qt in dev]  # also builds every class operator
    plan = fmm.Plan(dev[0][0], dev[0][1], p, theta, ncrit, headroom=1.5)
    # all replays queued back to back, checked afterwards
    outs = []
    for xt, qt in dev[1:] + dev[:1]:
        outs.append(plan.execute(xt, qt))
    assert plan.check() == 0
    for (phi, grad), (pphi, pgrad) in zip(outs, plain[1:] + plain[:1]):
        # results of earlier replays were copied out before the next one ran
        assert np.array_equal(phi.cpu().numpy(), pphi) and np.array_equal(grad.cpu().numpy(), pgrad)
    # new charges only
    q2 = np.random.default_rng(5).uniform(-1, 1, 30000).astype(np.float32)
    q2t = torch.from_numpy(q2).cuda()
    status, phi, grad = _replay(plan, dev[2][0], q2t)
    assert status == 0
    pphi, pgrad = _plain(dev[2][0], q2t, p, theta, ncrit)
    assert np.array_equal(phi, pphi) and np.array_equal(grad, pgrad)
    plan.close()


def test_batched_plan():
    from paper_1108_5815_gb300 import fmm
    torch = torch_cuda()
    rng = np.random.default_rng(17)
    sizes = np.exp(rng.uniform(np.log(200), np.log(3000), 40)).astype(np.int64)
    parts = [inputs.uniform_cube(int(n), 500 + i) if i % 2 == 0 else inputs.plummer(int(n), 500 + i, equal_charges=False)
             for i, n in enumerate(sizes)]
    x = np.concatenate([a for a, _ in parts])
    q = np.concatenate([b for _, b in parts])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    xt, qt = _dev(x, q)
    p, theta, ncrit = 5, 0.5, 16
    phi0, grad0 = fmm.laplace3d_batched(xt, qt, off, p, theta, ncrit, replay=False)
    torch.cuda.synchronize()
    plan = fmm.Plan(xt, qt, p, theta, ncrit, offsets=off)
    status, phi1, grad1 = _replay(plan)
    assert status == 0
    assert np.array_equal(phi1, phi0.cpu().numpy()) and np.array_equal(grad1, grad0.cpu().numpy())
    assert plan.info()["nsys"] == 40
    plan.close()


@pytest.mark.parametrize("precision", ["tf32x3", "bf16x3"])
def test_tensor_core_plan(precision):
    from paper_1108_5815_gb300 import fmm
    x, q = inputs.uniform_cube(40000, 611)
    xt, qt = _dev(x, q)
    p, theta, ncrit = 8, 0.45, 32
    phi0, grad0 = _plain(xt, qt, p, theta, ncrit, precision=precision)
    plan = fmm.Plan(xt, qt, p, theta, ncrit, precision=precision)
    status, phi1, grad1 = _replay(plan)
    assert status == 0
    assert np.array_equal(phi1, phi0) and np.array_equal(grad1, grad0)
    assert plan.info()["last_units"] > 0
    plan.close()


def test_hybrid_table_plan():
    from paper_1108_5815_gb300 import fmm
    x, q = inputs.plummer(20000, 77, equal_charges=False)
    xt, qt = _dev(x, q)
    sel = np.random.default_rng(9).integers(0, 4, (fmm.SELECT_NB, fmm.SELECT_NB)).astype(np.uint8)
    p, theta, ncrit = 5, 0.5, 8
    phi0, grad0 = _plain(xt, qt, p, theta, ncrit, select=sel)
    plan = fmm.Plan(xt, qt, p, theta, ncrit, select=sel)
    status, phi1, grad1 = _replay(plan)
    assert status == 0
    assert np.array_equal(phi1, phi0) and np.array_equal(grad1, grad0)
    plan.close()


def test_capacity_overflow_is_reported_and_plan_recovers():
    from paper_1108_5815_gb300 import fmm
    p, theta, ncrit = 5, 0.5, 32
    x, q = inputs.uniform_cube(20000, 701)
    xt, qt = _dev(x, q)
    plan = fmm.Plan(xt, qt, p, theta, ncrit, headroom=1.0)
    xp, qp = inputs.plummer(20000, 702, equal_charges=False)  # a far deeper tree
    xpt, qpt = _dev(xp, qp)
    phi, grad = plan.execute(xpt, qpt)
    assert plan.check() == CAPACITY
    assert plan.info()["last_valid"] == 0
    # the context is usable: a plain solve of the same data matches the oracle
    pphi, pgrad = _plain(xpt, qpt, p, theta, ncrit)
    ophi, ograd = O.Fmm(xp, qp, p, theta, ncrit).evaluate()
    assert rel_l2(pphi, ophi) < 1e-5 and rel_l2(pgrad, ograd) < 1e-5
    # and the plan is valid again on data that fits it
    status, phi1, grad1 = _replay(plan, xt, qt)
    assert status == 0
    phi0, grad0 = _plain(xt, qt, p, theta, ncrit)
    assert np.array_equal(phi1, phi0) and np.array_equal(grad1, grad0)
    plan.close()
