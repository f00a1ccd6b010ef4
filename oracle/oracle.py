"""ctypes wrapper of the FP64 CPU oracle (``fmm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  It shares no code with the
CUDA library and never imports it.  The C source documents what each function
computes and which passage of Yokota & Barba it follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U64 = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_direct.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_int64, _I64, _D, _D]
            L.orc_fmm_create.restype = ctypes.c_void_p
            L.orc_fmm_create.argtypes = [ctypes.c_int64, _D, _D, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]
            L.orc_count_bucket.restype = ctypes.c_int
            L.orc_count_bucket.argtypes = [ctypes.c_int64]
            for name in ("orc_fmm_upward", "orc_fmm_evaluate", "orc_fmm_destroy"):
                getattr(L, name).argtypes = [ctypes.c_void_p]
            L.orc_fmm_evaluate_leaves.argtypes = [ctypes.c_void_p, ctypes.c_int64, _I64, _D, _D, _I64]
            L.orc_fmm_sizes.argtypes = [ctypes.c_void_p, _I64]
            L.orc_fmm_box.argtypes = [ctypes.c_void_p, _D]
            L.orc_fmm_sorted.argtypes = [ctypes.c_void_p, _U64, _I64]
            L.orc_fmm_cells.argtypes = [ctypes.c_void_p, _I64, _U64, _I64, _I64, _I64, _I64]
            L.orc_fmm_lists.argtypes = [ctypes.c_void_p, _I64, _I64, _I64, _I64]
            L.orc_fmm_results.argtypes = [ctypes.c_void_p, _D, _D]
            L.orc_fmm_expansion.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, _D, _D]
            L.orc_fmm_centre.argtypes = [ctypes.c_void_p, ctypes.c_int64, _D]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            L.orc_morton_keys.restype = ctypes.c_int
            L.orc_morton_keys.argtypes = [ctypes.c_int64, _D, _D, _D, _U64]
            L.orc_regular_ri.argtypes = [_D, ctypes.c_int, _D]
            L.orc_irregular_ri.argtypes = [_D, ctypes.c_int, _D]
            L.orc_p2m_ri.argtypes = [_D, _D, _D, ctypes.c_int64, ctypes.c_int, _D]
            L.orc_m2m_ri.argtypes = [_D, _D, ctypes.c_int, _D, _D]
            L.orc_m2l_ri.argtypes = [_D, _D, ctypes.c_int, _D, _D]
            L.orc_l2l_ri.argtypes = [_D, _D, ctypes.c_int, _D, _D]
            L.orc_l2p_ri.argtypes = [_D, ctypes.c_int, _D, _D, _D]
            L.orc_m2p_grad_ri.argtypes = [_D, ctypes.c_int, _D, _D, _D]
            L.orc_fmm_m2p_list.argtypes = [ctypes.c_void_p, _I64, _I64, _I64]
            L.orc_fmm_p2l_list.argtypes = [ctypes.c_void_p, _I64, _I64, _I64]
            L.orc_p2l_ri.argtypes = [_D, _D, _D, ctypes.c_int64, ctypes.c_int, _D]
            L.orc_m2p_ri.restype = ctypes.c_double
            L.orc_m2p_ri.argtypes = [_D, ctypes.c_int, _D, _D]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on."""
    lib().orc_set_num_threads(int(n))


def nterms(p: int) -> int:
    return (p + 1) * (p + 1)


def hidx(n: int, m: int) -> int:
    """Index of coefficient (n, m), signed m, in the oracle's layout."""
    return n * n + n + m


# ---------------------------------------------------------------- direct sum

def direct(xyz, q, targets=None):
    """Exact FP64 potential and gradient (float32 inputs promoted to float64).

    ``targets``: optional array of target indices; returns values for those only."""
    x = _f64(xyz, (-1, 3))
    qq = _f64(q, (-1,))
    n = x.shape[0]
    if targets is None:
        nt = n
        tp = None
    else:
        t = np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
        nt = t.shape[0]
        tp = t.ctypes.data_as(_I64)
    phi = np.zeros(nt)
    grad = np.zeros((nt, 3))
    lib().orc_direct(n, _d(x), _d(qq), nt, tp, _d(phi), _d(grad))
    return phi, grad


def morton_keys(xyz):
    """(lo[3], side, keys) of reading R1; raises ValueError on non-finite input."""
    x = _f64(xyz, (-1, 3))
    lo = np.zeros(3)
    side = np.zeros(1)
    keys = np.zeros(x.shape[0], dtype=np.uint64)
    rc = lib().orc_morton_keys(x.shape[0], _d(x), _d(lo), _d(side), keys.ctypes.data_as(_U64))
    if rc:
        raise ValueError("non-finite coordinate")
    return lo, float(side[0]), keys


# ---------------------------------------------------------------- operators

def _cbuf(p):
    return np.zeros(nterms(p), dtype=np.complex128)


def regular(x, p):
    out = _cbuf(p)
    lib().orc_regular_ri(_d(_f64(x, (3,))), p, _d(out.view(np.float64)))
    return out


def irregular(x, p):
    out = _cbuf(p)
    lib().orc_irregular_ri(_d(_f64(x, (3,))), p, _d(out.view(np.float64)))
    return out


def p2m(c, y, q, p):
    y = _f64(y, (-1, 3))
    out = _cbuf(p)
    lib().orc_p2m_ri(_d(_f64(c, (3,))), _d(y), _d(_f64(q, (-1,))), y.shape[0], p,
                     _d(out.view(np.float64)))
    return out


def m2m(c, cp, p, M):
    M = np.ascontiguousarray(M, dtype=np.complex128)
    out = _cbuf(p)
    lib().orc_m2m_ri(_d(_f64(c, (3,))), _d(_f64(cp, (3,))), p, _d(M.view(np.float64)),
                     _d(out.view(np.float64)))
    return out


def m2l(cs, ct, p, M):
    M = np.ascontiguousarray(M, dtype=np.complex128)
    out = _cbuf(p)
    lib().orc_m2l_ri(_d(_f64(cs, (3,))), _d(_f64(ct, (3,))), p, _d(M.view(np.float64)),
                     _d(out.view(np.float64)))
    return out


def l2l(c, cp, p, L):
    L = np.ascontiguousarray(L, dtype=np.complex128)
    out = _cbuf(p)
    lib().orc_l2l_ri(_d(_f64(c, (3,))), _d(_f64(cp, (3,))), p, _d(L.view(np.float64)),
                     _d(out.view(np.float64)))
    return out


def l2p(c, p, L, x):
    """(phi, grad[3]) at x from the local expansion L about c."""
    L = np.ascontiguousarray(L, dtype=np.complex128)
    out = np.zeros(4)
    lib().orc_l2p_ri(_d(_f64(c, (3,))), p, _d(L.view(np.float64)), _d(_f64(x, (3,))), _d(out))
    return out[0], out[1:4].copy()


def p2l(c, y, q, p):
    """Local expansion about c of charges q at y (complex, index n*n+n+m)."""
    y = _f64(y, (-1, 3))
    q = _f64(q, (-1,))
    L = np.zeros((p + 1) ** 2, dtype=np.complex128)
    lib().orc_p2l_ri(_d(_f64(c, (3,))), _d(y), _d(q), y.shape[0], p, _d(L.view(np.float64)))
    return L


def m2p_grad(c, p, M, x):
    """(phi, grad[3]) at x from the multipole M about c."""
    M = np.ascontiguousarray(M, dtype=np.complex128)
    out = np.zeros(4)
    lib().orc_m2p_grad_ri(_d(_f64(c, (3,))), p, _d(M.view(np.float64)), _d(_f64(x, (3,))), _d(out))
    return float(out[0]), out[1:].copy()


def m2p(c, p, M, x):
    M = np.ascontiguousarray(M, dtype=np.complex128)
    return lib().orc_m2p_ri(_d(_f64(c, (3,))), p, _d(M.view(np.float64)), _d(_f64(x, (3,))))


# ---------------------------------------------------------------- full FMM

SEL_NB = 128


def count_bucket(n):
    """Count bucket of the hybrid selection table (reading R9)."""
    return int(lib().orc_count_bucket(int(n)))


class Fmm:
    """Oracle FMM: keys, tree and interaction lists are built on construction;
    ``evaluate()`` runs the upward and downward passes."""

    SPLIT_RULES = {"paper": 0, "smaller": 2, "source_on_tie": 4}

    def __init__(self, xyz, q, p, theta, ncrit, max_depth=21, leaf_first=False, sel=None,
                 split_rule="paper"):
        """``sel``: optional hybrid selection table (reading R9), uint8 [128, 128]
        indexed by the count buckets of (target, source); 1 = P2P for a MAC-accepted pair.

        ``split_rule``: "paper" (split the larger cell, the target on a tie) is the
        traversal; "smaller" and "source_on_tie" are deliberately wrong rules that
        only the tests use, to show that the pair-set pins catch them."""
        self.xyz = _f64(xyz, (-1, 3))
        self.q = _f64(q, (-1,))
        self.p = p
        st = ctypes.c_int(0)
        selp = None
        if sel is not None:
            sel = np.ascontiguousarray(np.asarray(sel, dtype=np.uint8).reshape(SEL_NB, SEL_NB))
            selp = sel.ctypes.data
        self._h = lib().orc_fmm_create(self.xyz.shape[0], _d(self.xyz), _d(self.q), p, theta,
                                       ncrit, max_depth,
                                       int(leaf_first) | self.SPLIT_RULES[split_rule], selp,
                                       ctypes.byref(st))
        if st.value != 0 or not self._h:
            self._h = None
            raise ValueError("non-finite coordinate")
        s = np.zeros(6, dtype=np.int64)
        lib().orc_fmm_sizes(self._h, s.ctypes.data_as(_I64))
        self.N, self.ncells, self.nm2l, self.np2p, self.depth, self.nleaves = (int(v) for v in s)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_fmm_destroy(self._h)
            self._h = None

    def box(self):
        b = np.zeros(4)
        lib().orc_fmm_box(self._h, _d(b))
        return b[:3].copy(), float(b[3])

    def sorted(self):
        key = np.zeros(self.N, dtype=np.uint64)
        order = np.zeros(self.N, dtype=np.int64)
        lib().orc_fmm_sorted(self._h, key.ctypes.data_as(_U64), order.ctypes.data_as(_I64))
        return key, order

    def cells(self):
        n = self.ncells
        level, begin, end, parent, nchild = (np.zeros(n, dtype=np.int64) for _ in range(5))
        prefix = np.zeros(n, dtype=np.uint64)
        lib().orc_fmm_cells(self._h, level.ctypes.data_as(_I64), prefix.ctypes.data_as(_U64),
                            begin.ctypes.data_as(_I64), end.ctypes.data_as(_I64),
                            parent.ctypes.data_as(_I64), nchild.ctypes.data_as(_I64))
        return dict(level=level, prefix=prefix, begin=begin, end=end, parent=parent, nchild=nchild)

    def lists(self):
        mt, ms = np.zeros(self.nm2l, dtype=np.int64), np.zeros(self.nm2l, dtype=np.int64)
        pt, ps = np.zeros(self.np2p, dtype=np.int64), np.zeros(self.np2p, dtype=np.int64)
        lib().orc_fmm_lists(self._h, mt.ctypes.data_as(_I64), ms.ctypes.data_as(_I64),
                            pt.ctypes.data_as(_I64), ps.ctypes.data_as(_I64))
        return dict(m2l_t=mt, m2l_s=ms, p2p_t=pt, p2p_s=ps)

    def p2l_list(self):
        """Particle-cell pairs (target cell, source cell) chosen by the selection table."""
        n = ctypes.c_int64(0)
        lib().orc_fmm_p2l_list(self._h, ctypes.byref(n), None, None)
        t = np.zeros(n.value, dtype=np.int64)
        s = np.zeros(n.value, dtype=np.int64)
        lib().orc_fmm_p2l_list(self._h, ctypes.byref(n), t.ctypes.data_as(_I64), s.ctypes.data_as(_I64))
        return t, s

    def m2p_list(self):
        """Cell-particle pairs (target cell, source cell) chosen by the selection table."""
        n = ctypes.c_int64(0)
        lib().orc_fmm_m2p_list(self._h, ctypes.byref(n), None, None)
        t = np.zeros(n.value, dtype=np.int64)
        s = np.zeros(n.value, dtype=np.int64)
        lib().orc_fmm_m2p_list(self._h, ctypes.byref(n), t.ctypes.data_as(_I64), s.ctypes.data_as(_I64))
        return t, s

    def upward(self):
        lib().orc_fmm_upward(self._h)

    def evaluate(self):
        """(phi[N], grad[N,3]) in the caller's particle order."""
        lib().orc_fmm_evaluate(self._h)
        phi = np.zeros(self.N)
        grad = np.zeros((self.N, 3))
        lib().orc_fmm_results(self._h, _d(phi), _d(grad))
        return phi, grad

    def evaluate_leaves(self, leaves):
        """FMM values for the particles of the given leaves only.

        Returns (sorted_positions, phi, grad); sorted_positions index the sorted
        order (map to caller order with ``sorted()[1]``)."""
        lv = np.ascontiguousarray(np.asarray(leaves, dtype=np.int64))
        cells = self.cells()
        cnt = int(np.sum(cells["end"][lv] - cells["begin"][lv]))
        phi = np.zeros(cnt)
        grad = np.zeros((cnt, 3))
        pos = np.zeros(cnt, dtype=np.int64)
        lib().orc_fmm_evaluate_leaves(self._h, lv.shape[0], lv.ctypes.data_as(_I64), _d(phi),
                                      _d(grad), pos.ctypes.data_as(_I64))
        return pos, phi, grad

    def expansion(self, which: str, c: int):
        """Complex coefficients (signed m, index n*n+n+m) of cell c: which='M' or 'L'."""
        P2 = nterms(self.p)
        re, im = np.zeros(P2), np.zeros(P2)
        lib().orc_fmm_expansion(self._h, 0 if which == "M" else 1, c, _d(re), _d(im))
        return re + 1j * im

    def centre(self, c: int):
        out = np.zeros(3)
        lib().orc_fmm_centre(self._h, c, _d(out))
        return out
