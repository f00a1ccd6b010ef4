"""Repeated solves through the public entry points (fmm_options.replay, the
default): from the third call of one key on, a call replays the plan the library
captured after the second, reading and writing each call's arrays in place.

* a replayed call gives exactly the plain solve's result (replay=False) of the
  same data, for new positions and charges too, also when they are written into
  the same arrays;
* calls that alternate between two sets of arrays replay on each set and stay right;
* data that outgrows the plan (a clustered set after a uniform one of the same
  N) is solved again plainly, with the plain result, and later calls stay right;
* batched systems and a selection table replay the same way;
* a non-finite coordinate is reported as FMM_ERR_NONFINITE by a replayed call as
  by a plain one, and the next call is valid again."""
import numpy as np
import pytest

from paper_1108_5815_gb300 import inputs
from tests.gpu_helpers import torch_cuda

pytestmark = pytest.mark.gpu


def _dev(x, q):
    torch = torch_cuda()
    return (torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(q, np.float32)).cuda())


def _solve(xt, qt, args, **kw):
    from paper_1108_5815_gb300 import fmm
    torch = torch_cuda()
    phi, grad = fmm.laplace3d(xt, qt, *args, **kw)
    torch.cuda.synchronize()
    return phi.cpu().numpy(), grad.cpu().numpy()


def _equal(a, b):
    return np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_replayed_calls_equal_the_plain_solve():
    x, q = inputs.uniform_cube(30000, 801)
    args = (6, 0.5, 32)
    xt, qt = _dev(x, q)
    plain = _solve(xt, qt, args, replay=False)
    runs = [_solve(xt, qt, args) for _ in range(4)]  # plain, plain + capture, replay, replay
    for r in runs:
        assert _equal(r, plain)
    # new charges and jittered positions: the replay equals the plain solve of that data
    rng = np.random.default_rng(802)
    x2 = np.clip(x + rng.normal(0.0, 1e-3, x.shape), 0.0, 1.0).astype(np.float32)
    q2 = rng.uniform(-1.0, 1.0, len(q)).astype(np.float32)
    xt2, qt2 = _dev(x2, q2)
    assert _equal(_solve(xt2, qt2, args), _solve(xt2, qt2, args, replay=False))


def test_data_that_outgrows_the_plan_is_solved_plainly():
    n = 20000
    xu, qu = inputs.uniform_cube(n, 803)
    xp, qp = inputs.plummer(n, 804, equal_charges=False)
    args = (5, 0.5, 16)
    xut, qut = _dev(xu, qu)
    xpt, qpt = _dev(xp, qp)
    for _ in range(3):
        _solve(xut, qut, args)  # the plan is captured from the uniform set
    clustered = _solve(xpt, qpt, args)  # a much deeper tree than the plan holds
    assert _equal(clustered, _solve(xpt, qpt, args, replay=False))
    assert _equal(_solve(xut, qut, args), _solve(xut, qut, args, replay=False))


def test_batched_and_selection_table_replays():
    from paper_1108_5815_gb300 import fmm
    torch = torch_cuda()
    sizes = [3000, 500, 7000]
    parts = [inputs.uniform_cube(s, 810 + i) for i, s in enumerate(sizes)]
    x = np.concatenate([a for a, _ in parts])
    q = np.concatenate([b for _, b in parts])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    xt, qt = _dev(x, q)

    def batched(**kw):
        phi, grad = fmm.laplace3d_batched(xt, qt, off, 5, 0.5, 16, **kw)
        torch.cuda.synchronize()
        return phi.cpu().numpy(), grad.cpu().numpy()

    plain = batched(replay=False)
    for _ in range(3):
        assert _equal(batched(), plain)

    x1, q1 = inputs.uniform_cube(20000, 815)
    xt1, qt1 = _dev(x1, q1)
    args = (6, 0.5, 8)
    plain = _solve(xt1, qt1, args, select="autotune", replay=False)
    for _ in range(3):
        assert _equal(_solve(xt1, qt1, args, select="autotune"), plain)


def test_nonfinite_input_in_a_replayed_call():
    from paper_1108_5815_gb300 import fmm
    x, q = inputs.uniform_cube(10000, 820)
    args = (4, 0.5, 16)
    xt, qt = _dev(x, q)
    plain = _solve(xt, qt, args, replay=False)
    for _ in range(3):
        _solve(xt, qt, args)
    bad = x.copy()
    bad[17, 1] = np.nan
    xbt, qbt = _dev(bad, q)
    with pytest.raises(fmm.FmmError) as e:
        _solve(xbt, qbt, args)
    assert e.value.status == fmm.FMM_ERR_NONFINITE
    assert _equal(_solve(xt, qt, args), plain)


def test_new_data_in_the_same_arrays_and_alternating_arrays():
    torch = torch_cuda()
    from paper_1108_5815_gb300 import fmm
    args = (6, 0.5, 32)
    xa, qa = inputs.uniform_cube(25000, 830)
    xb, qb = inputs.uniform_cube(25000, 831)
    xta, qta = _dev(xa, qa)
    xtb, qtb = _dev(xb, qb)
    pa = torch.empty(25000, device="cuda")
    ga = torch.empty(25000, 3, device="cuda")

    def run(xt, qt, **kw):
        fmm.laplace3d(xt, qt, *args, out=(pa, ga), **kw)
        torch.cuda.synchronize()
        return pa.cpu().numpy().copy(), ga.cpu().numpy().copy()

    for _ in range(3):
        run(xta, qta)  # the third call replays the plan on these very arrays
    # new data written into the same arrays: the replay reads it in place
    xta.copy_(xtb)
    qta.copy_(qtb)
    ref_b = run(xtb, qtb, replay=False)
    assert _equal(run(xta, qta), ref_b)
    # alternating arrays: the same plan replays on each set
    xta.copy_(torch.from_numpy(xa).cuda())
    qta.copy_(torch.from_numpy(qa).cuda())
    ref_a = run(xta, qta, replay=False)
    for _ in range(2):
        assert _equal(run(xtb, qtb), ref_b)
        assert _equal(run(xta, qta), ref_a)
