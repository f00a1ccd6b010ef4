"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
bring its intermediate arrays into the oracle's vocabulary."""
import math

import numpy as np

from oracle import oracle as O


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


def gpu_solve(xyz, q, p, theta, ncrit, max_depth=0, precision="fp32", stats=False, select="plain"):
    torch = torch_cuda()
    from paper_1108_5815_gb300 import fmm
    x = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.float32)).cuda()
    qq = torch.from_numpy(np.ascontiguousarray(q, dtype=np.float32)).cuda()
    res = fmm.laplace3d(x, qq, p, theta, ncrit, max_depth=max_depth, precision=precision,
                        stats=stats, select=select)
    torch.cuda.synchronize()
    out = [res[0].cpu().numpy().astype(np.float64), res[1].cpu().numpy().astype(np.float64)]
    if stats:
        out.append(res[2])
    return tuple(out)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def assert_pointwise(phi, ophi, grad, ograd, tol=1e-4):
    """Worst particle, beside the relative L2 norm: max_i |phi_i - phi*_i| <=
    tol * max_j |phi*_j|, and the same for the gradient vectors (Euclidean
    length per particle), so that a few bad targets cannot hide under the norm."""
    phi, grad = np.asarray(phi, np.float64), np.asarray(grad, np.float64).reshape(-1, 3)
    ograd = np.asarray(ograd, np.float64).reshape(-1, 3)
    ep = np.abs(phi - ophi).max()
    eg = np.linalg.norm(grad - ograd, axis=1).max()
    sp = np.abs(ophi).max()
    sg = np.linalg.norm(ograd, axis=1).max()
    assert ep <= tol * sp, f"worst |dphi| {ep:.3e} > {tol} * {sp:.3e}"
    assert eg <= tol * sg, f"worst |dgrad| {eg:.3e} > {tol} * {sg:.3e}"


def canonical_ids(level, prefix):
    """Rank of each cell in (level, prefix) order -- identical for both sides
    when the cell sets agree."""
    order = np.lexsort((np.asarray(prefix, np.uint64), np.asarray(level, np.int64)))
    ids = np.empty(len(order), dtype=np.int64)
    ids[order] = np.arange(len(order))
    return ids, order


def gpu_cells():
    from paper_1108_5815_gb300 import fmm
    c = fmm.export("cells")
    return dict(level=c[:, 0], prefix=c[:, 1].astype(np.uint64), begin=c[:, 2], end=c[:, 3],
                parent=c[:, 4], nchild=c[:, 5])


def pair_codes(t, s, ids, ncells):
    return np.sort(ids[np.asarray(t, np.int64)] * ncells + ids[np.asarray(s, np.int64)])


def nu(n, m):
    return math.sqrt(math.factorial(n - m) * math.factorial(n + m))


def oracle_to_gpu_layout(E, p, side, which, P2pad):
    """Oracle complex coefficients (signed m, index n*n+n+m) of a cell with side
    ``side`` -> the GPU's real, unit-scaled, order-normalised row."""
    row = np.zeros(P2pad)
    for n in range(p + 1):
        for m in range(n + 1):
            c = E[n * n + n + m]
            if which == "M":
                c = c * side ** (-n) * nu(n, m)
            else:
                c = c * side ** (n + 1) / nu(n, m)
            if m == 0:
                row[n * n] = c.real
            else:
                row[n * n + 2 * m - 1] = c.real
                row[n * n + 2 * m] = c.imag
    return row


def expand_p2p_to_leaves(cells, t, s):
    """P2P pairs (T, S) with any target cell -> (leaf below T, S), the per-leaf
    form the GPU lists use."""
    b, e, nch = (np.asarray(cells[k], np.int64) for k in ("begin", "end", "nchild"))
    leaves = np.flatnonzero(nch == 0)
    lb = b[leaves]
    order = np.argsort(lb)
    leaves, lb = leaves[order], lb[order]
    out_t, out_s = [], []
    for tt, ss in zip(np.asarray(t, np.int64), np.asarray(s, np.int64)):
        if nch[tt] == 0:
            out_t.append(tt)
            out_s.append(ss)
            continue
        i0, i1 = np.searchsorted(lb, b[tt]), np.searchsorted(lb, e[tt])
        out_t.extend(leaves[i0:i1])
        out_s.extend([ss] * (i1 - i0))
    return np.asarray(out_t, np.int64), np.asarray(out_s, np.int64)
