"""The allocation-free entry point fmm_morton_sort_noalloc against the solve.

Callers that may not allocate device memory after start-up (code inside another
framework's memory pool, plugin hosts) use this entry point for the key/sort
stage; its fixed scratch array is shared by all calls and keeps the previous
call's contents, so two calls in a row on different inputs must both give the
same keys, order and box as a full solve on the same points."""
import ctypes

import numpy as np
import pytest

from paper_1108_5815_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solve_exports(torch, fmm, x, q):
    xd, qd = torch.from_numpy(x).cuda(), torch.from_numpy(q).cuda()
    fmm.laplace3d(xd, qd, 4, 0.5, 32)
    torch.cuda.synchronize()
    return fmm.export("keys"), fmm.export("order"), fmm.export("box").reshape(-1)


def test_noalloc_sort_matches_solve_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    from paper_1108_5815_gb300 import fmm
    cases = [inputs.uniform_cube(300000, 41), inputs.plummer(70001, 42, equal_charges=False)]
    for x, q in cases:
        keys, order, box = fmm.morton_sort_noalloc(torch.from_numpy(x).cuda())
        torch.cuda.synchronize()
        k_ref, o_ref, b_ref = _solve_exports(torch, fmm, x, q)
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), k_ref)
        assert np.array_equal(order.cpu().numpy(), o_ref)
        assert np.array_equal(box.cpu().numpy(), b_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_1108_5815_gb300 import fmm
    L = fmm.load()
    x = torch.zeros(8, 3, device="cuda")
    k = torch.zeros(8, dtype=torch.int64, device="cuda")
    o = torch.zeros(8, dtype=torch.int32, device="cuda")
    b = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = L.fmm_morton_sort_noalloc(x.data_ptr(), (1 << 20) + 1, k.data_ptr(), o.data_ptr(),
                                   b.data_ptr(), None)
    assert st == fmm.FMM_ERR_ARG and "1048576" in fmm.last_error()
