"""Helpers for tests: geometry decoded from cell (level, key prefix) with numpy."""
import numpy as np


def compact3(v):
    v = np.asarray(v, dtype=np.uint64)
    out = np.zeros_like(v)
    for b in range(21):
        out |= ((v >> np.uint64(3 * b)) & np.uint64(1)) << np.uint64(b)
    return out


def cell_index(level, prefix):
    """Integer cell coordinates (k_x, k_y, k_z) at the cell's own level."""
    prefix = np.asarray(prefix, dtype=np.uint64)
    return np.stack([compact3(prefix >> np.uint64(a)).astype(np.int64) for a in range(3)], axis=-1)


def coverage_matrix(n, cells, lists):
    """How many times each ordered particle pair (i, j) (sorted positions) is
    covered by a P2P leaf pair or by an M2L pair of cells containing i and j."""
    cov = np.zeros((n, n), dtype=np.int32)
    b, e = cells["begin"], cells["end"]
    for t, s in zip(lists["p2p_t"], lists["p2p_s"]):
        cov[b[t]:e[t], b[s]:e[s]] += 1
    for t, s in zip(lists["m2l_t"], lists["m2l_s"]):
        cov[b[t]:e[t], b[s]:e[s]] += 1
    for t, s in zip(lists.get("m2p_t", ()), lists.get("m2p_s", ())):
        cov[b[t]:e[t], b[s]:e[s]] += 1
    for t, s in zip(lists.get("p2l_t", ()), lists.get("p2l_s", ())):
        cov[b[t]:e[t], b[s]:e[s]] += 1
    return cov
