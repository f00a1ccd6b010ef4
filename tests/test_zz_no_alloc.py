"""The allocation-free entry point fmm_morton_sort_noalloc against the solve.

Callers that may not allocate device memory after start-up (code inside another
framework's memory pool, plugin hosts) use this entry point for the key/sort
stage; its fixed scratch array is shared by all calls and keeps the previous
call's contents, so two calls in a row on different inputs must both give the
same keys, order and box as a full solve on the same points.  The cases span
one point, ragged sizes and the largest size the scratch holds (where the
sort's look-back words fill it); a NaN coordinate is rejected; and once a
device has had its first call, a call takes no device memory."""
import numpy as np
import pytest

from paper_1108_5815_gb300 import inputs

pytestmark = pytest.mark.gpu

MAX_N = 1 << 20


def _solve_exports(torch, fmm, x, q):
    xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    fmm.laplace3d(xd, qd, 4, 0.5, 32)
    torch.cuda.synchronize()
    return fmm.export("keys"), fmm.export("order"), fmm.export("box").reshape(-1)


def _check_against_solve(torch, fmm, x, q):
    keys, order, box = fmm.morton_sort_noalloc(torch.from_numpy(x).cuda())
    torch.cuda.synchronize()
    k_ref, o_ref, b_ref = _solve_exports(torch, fmm, x, q)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), k_ref)
    assert np.array_equal(order.cpu().numpy(), o_ref)
    assert np.array_equal(box.cpu().numpy(), b_ref)


def test_noalloc_sort_matches_solve_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    from paper_1108_5815_gb300 import fmm
    cases = [inputs.uniform_cube(300000, 41), inputs.plummer(70001, 42, equal_charges=False)]
    for x, q in cases:
        _check_against_solve(torch, fmm, x, q)


def test_noalloc_sort_at_the_maximum_size_and_one_point():
    torch = pytest.importorskip("torch")
    from paper_1108_5815_gb300 import fmm
    # the largest N the scratch holds (256 sort tiles x 8 passes of look-back
    # words), then a single point, then the maximum again on other points
    for x, q in (inputs.uniform_cube(MAX_N, 43), inputs.uniform_cube(1, 44),
                 inputs.plummer(MAX_N, 45, equal_charges=False)):
        _check_against_solve(torch, fmm, x, q)


def test_noalloc_rejects_nan_then_recovers():
    torch = pytest.importorskip("torch")
    from paper_1108_5815_gb300 import fmm
    x, q = inputs.uniform_cube(5000, 46)
    bad = x.copy()
    bad[1234, 1] = np.nan
    with pytest.raises(fmm.FmmError) as e:
        fmm.morton_sort_noalloc(torch.from_numpy(bad).cuda())
    assert e.value.status == fmm.FMM_ERR_NONFINITE
    # the flag is cleared on the next call
    _check_against_solve(torch, fmm, x, q)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_1108_5815_gb300 import fmm
    L = fmm.load()
    x = torch.zeros(8, 3, device="cuda")
    k = torch.zeros(8, dtype=torch.int64, device="cuda")
    o = torch.zeros(8, dtype=torch.int32, device="cuda")
    b = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = L.fmm_morton_sort_noalloc(x.data_ptr(), MAX_N + 1, k.data_ptr(), o.data_ptr(),
                                   b.data_ptr(), None)
    assert st == fmm.FMM_ERR_ARG and "1048576" in fmm.last_error()


def test_noalloc_call_takes_no_device_memory():
    torch = pytest.importorskip("torch")
    from paper_1108_5815_gb300 import fmm
    L = fmm.load()
    x, _ = inputs.uniform_cube(200000, 47)
    xd = torch.from_numpy(x).cuda()
    k = torch.empty(len(x), dtype=torch.int64, device="cuda")
    o = torch.empty(len(x), dtype=torch.int32, device="cuda")
    b = torch.empty(4, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream

    def call():
        rc = L.fmm_morton_sort_noalloc(xd.data_ptr(), len(x), k.data_ptr(), o.data_ptr(),
                                       b.data_ptr(), st)
        assert rc == fmm.FMM_OK, fmm.last_error()

    call()  # the device's first call (module set-up) may take device memory
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    keys1 = k.clone()
    call()
    assert torch.equal(k, keys1)
