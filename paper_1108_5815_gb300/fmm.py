"""Python binding of the C ABI in ``include/fmm.h`` (argument marshalling only).

Every step of the solve runs in the CUDA library ``libfmm.so``; this module
passes device pointers and the current torch stream.  There is no CPU
fallback: if the library is missing or the tensors are not CUDA float32, the
call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfmm.so")

FMM_OK, FMM_ERR_ARG, FMM_ERR_NONFINITE, FMM_ERR_CAPACITY, FMM_ERR_CUDA, FMM_ERR_TIMEOUT, \
    FMM_ERR_NOMEM = range(7)
PRECISION = {"fp32": 0, "tf32x3": 1, "bf16x3": 2}
SELECT = {"plain": 0, "autotune": 1, "learned": 2, "table": 3, "treecode": 4}
SELECT_NB = 128
EXPORT = {"box": 0, "keys": 1, "order": 2, "cells": 3, "p2p": 4, "m2l": 5, "multipole": 6,
          "local": 7, "select": 8, "m2p": 9, "p2l": 10}

# every symbol the header declares
ABI_SYMBOLS = ("fmm_default_options", "fmm_laplace3d", "fmm_laplace3d_ex", "fmm_laplace3d_host",
               "fmm_laplace3d_batched",
               "fmm_direct", "fmm_export", "fmm_last_error", "fmm_morton_sort_noalloc",
               "fmm_selection_table", "fmm_cost_model_train", "fmm_cost_model_get",
               "fmm_cost_model_set", "fmm_cost_model_grad", "fmm_cost_model_adam_step",
               "fmm_cost_model_predict", "fmm_cost_model_samples", "fmm_tune_ncrit",
               "fmm_tune_schedule", "fmm_selftest_wait_timeout", "fmm_plan_create", "fmm_plan_execute",
               "fmm_plan_check", "fmm_plan_buffers", "fmm_plan_info", "fmm_plan_destroy", "fmm_measure_fp32",
               "fmm_cost_model_pick_ncrit")
COST_MODEL_PARAMS = 4610


class FmmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fmm status {status}: {msg}")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("max_depth", ctypes.c_int), ("precision_mode", ctypes.c_int),
                ("select_mode", ctypes.c_int), ("deterministic", ctypes.c_int),
                ("select_table", ctypes.c_void_p), ("m2l_unit_blocks", ctypes.c_int),
                ("serialize_phases", ctypes.c_int), ("replay", ctypes.c_int)]


class CostModelInfo(ctypes.Structure):
    _fields_ = [("n_samples_p2p", ctypes.c_int64), ("n_samples_m2l", ctypes.c_int64),
                ("steps", ctypes.c_int), ("loss_initial", ctypes.c_float),
                ("loss_final", ctypes.c_float), ("agreement", ctypes.c_float),
                ("ms_pretime", ctypes.c_float), ("ms_train", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PlanInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("nsys", ctypes.c_int), ("levels", ctypes.c_int),
                ("cell_cap", ctypes.c_int64), ("tile_cap", ctypes.c_int64), ("class_cap", ctypes.c_int64),
                ("entry_cap", ctypes.c_int64), ("unit_cap", ctypes.c_int64), ("m2l_cap", ctypes.c_int64),
                ("p2p_cap", ctypes.c_int64), ("operators", ctypes.c_int64), ("graph_nodes", ctypes.c_int64),
                ("graph_kernels", ctypes.c_int64), ("last_cells", ctypes.c_int64), ("last_leaves", ctypes.c_int64),
                ("last_classes", ctypes.c_int64), ("last_entries", ctypes.c_int64), ("last_units", ctypes.c_int64),
                ("last_valid", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("ncells", "nleaves", "depth", "n_p2p_pairs",
                                              "n_p2p_interactions", "n_m2l_pairs",
                                              "n_offset_classes", "n_m2l_blocks",
                                              "n_launches")] + \
               [(n, ctypes.c_float) for n in ("ms_tree", "ms_upward", "ms_traverse", "ms_m2l",
                                              "ms_downward", "ms_p2p", "ms_total")] + \
               [("n_m2p_pairs", ctypes.c_int64), ("n_p2l_pairs", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libfmm.so (built in-tree by ``paper_1108_5815_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or LIB_PATH
        if not os.path.exists(path):
            raise FmmError(FMM_ERR_CUDA, f"CUDA library not built: {path} is missing "
                                         "(run paper_1108_5815_gb300.build.build())")
        L = ctypes.CDLL(path)
        vp, i64, f32p = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
        L.fmm_default_options.argtypes = [ctypes.POINTER(Options)]
        L.fmm_default_options.restype = None
        L.fmm_laplace3d.argtypes = [vp, vp, i64, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp, vp, vp]
        L.fmm_laplace3d_ex.argtypes = L.fmm_laplace3d.argtypes + [ctypes.POINTER(Options),
                                                                  ctypes.POINTER(Stats)]
        L.fmm_laplace3d_host.argtypes = L.fmm_laplace3d_ex.argtypes
        L.fmm_direct.argtypes = [vp, vp, i64, vp, vp, vp]
        L.fmm_laplace3d_batched.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            ctypes.c_int, vp, vp, vp, ctypes.POINTER(Options),
                                            ctypes.POINTER(Stats)]
        L.fmm_export.argtypes = [ctypes.c_int, vp, i64, ctypes.POINTER(i64)]
        L.fmm_last_error.restype = ctypes.c_char_p
        L.fmm_morton_sort_noalloc.argtypes = [vp, i64, vp, vp, vp, vp]
        L.fmm_morton_sort_noalloc.restype = ctypes.c_int
        L.fmm_selection_table.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, vp]
        L.fmm_cost_model_train.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_uint64, ctypes.POINTER(CostModelInfo)]
        L.fmm_cost_model_get.argtypes = [vp, i64, ctypes.c_int]
        L.fmm_cost_model_set.argtypes = [vp, i64]
        L.fmm_cost_model_grad.argtypes = [vp, vp, vp, i64, vp, vp]
        L.fmm_cost_model_adam_step.argtypes = [vp, vp, vp, i64, ctypes.c_float, vp]
        L.fmm_cost_model_predict.argtypes = [vp, i64, vp]
        L.fmm_cost_model_samples.argtypes = [vp, vp, vp, i64, ctypes.POINTER(i64)]
        L.fmm_tune_ncrit.argtypes = [vp, vp, i64, ctypes.c_int, ctypes.c_double, vp, ctypes.POINTER(Options),
                                     vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int)]
        L.fmm_selftest_wait_timeout.argtypes = [i64, vp]
        L.fmm_selftest_wait_timeout.restype = ctypes.c_int
        L.fmm_tune_schedule.argtypes = [vp, vp, i64, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, vp,
                                        ctypes.POINTER(Options), vp, ctypes.c_int, vp, ctypes.c_int, vp,
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        L.fmm_plan_create.argtypes = [ctypes.POINTER(vp), vp, vp, i64, vp, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, ctypes.POINTER(Options), ctypes.c_double, vp]
        L.fmm_plan_execute.argtypes = [vp, vp, vp, vp, vp, vp]
        L.fmm_plan_check.argtypes = [vp, vp]
        L.fmm_plan_buffers.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(vp)]
        L.fmm_plan_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
        L.fmm_measure_fp32.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double), vp]
        L.fmm_cost_model_pick_ncrit.argtypes = [vp, vp, i64, ctypes.c_int, ctypes.c_double, vp,
                                                ctypes.POINTER(Options), vp, ctypes.c_int, vp,
                                                ctypes.POINTER(ctypes.c_int)]
        L.fmm_cost_model_pick_ncrit.restype = ctypes.c_int
        L.fmm_measure_fp32.restype = ctypes.c_int
        L.fmm_plan_destroy.argtypes = [vp]
        L.fmm_plan_destroy.restype = None
        for name in ("fmm_plan_create", "fmm_plan_execute", "fmm_plan_check", "fmm_plan_buffers",
                     "fmm_plan_info"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("fmm_laplace3d", "fmm_laplace3d_ex", "fmm_laplace3d_host", "fmm_direct",
                     "fmm_export", "fmm_laplace3d_batched", "fmm_selection_table",
                     "fmm_cost_model_train", "fmm_cost_model_get", "fmm_cost_model_set",
                     "fmm_cost_model_grad", "fmm_cost_model_adam_step", "fmm_cost_model_predict",
                     "fmm_cost_model_samples", "fmm_tune_ncrit", "fmm_tune_schedule"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def last_error() -> str:
    return load().fmm_last_error().decode()


def _check(status: int):
    if status != FMM_OK:
        raise FmmError(status, last_error())


def _options(max_depth=0, precision="fp32", select="plain", m2l_unit_blocks=0, serialize_phases=False,
             replay=True):
    """fmm_options for the call.  ``select`` is "plain", "autotune", "learned" or a
    uint8 [128, 128] selection table; the returned options keep the table alive.
    ``serialize_phases``: the far-field chain waits for P2P (phase times of the
    statistics are then each phase alone).  ``replay``: repeated solves of one
    key replay a captured plan (fmm_options.replay)."""
    o = Options()
    load().fmm_default_options(ctypes.byref(o))
    o.max_depth = max_depth
    o.precision_mode = PRECISION[precision]
    o.m2l_unit_blocks = m2l_unit_blocks
    o.serialize_phases = int(bool(serialize_phases))
    o.replay = int(bool(replay))
    if isinstance(select, str):
        o.select_mode = SELECT[select]
        o._table = None
    else:
        t = np.ascontiguousarray(np.asarray(select, dtype=np.uint8))
        if t.shape != (SELECT_NB, SELECT_NB):
            raise FmmError(FMM_ERR_ARG, f"selection table must be uint8 [{SELECT_NB}, {SELECT_NB}]")
        o.select_mode = SELECT["table"]
        o.select_table = t.ctypes.data
        o._table = t
    return o


def _stream_ptr(torch, device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev_f32(t, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise FmmError(FMM_ERR_ARG, f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32:
        raise FmmError(FMM_ERR_ARG, f"{name} must be float32")
    if tuple(t.shape) != shape:
        raise FmmError(FMM_ERR_ARG, f"{name} must have shape {shape}, got {tuple(t.shape)}")
    return t.contiguous()


def laplace3d(xyz, q, p: int, theta: float, ncrit: int, *, max_depth: int = 0,
              precision: str = "fp32", select="plain", m2l_unit_blocks: int = 0, stats: bool = False,
              out=None, serialize_phases: bool = False, replay: bool = True):
    """FMM potential and gradient for CUDA float32 xyz[N,3], q[N].

    Returns (phi[N], grad[N,3]) as CUDA tensors (and a stats dict if ``stats``)."""
    import torch
    n = int(xyz.shape[0]) if hasattr(xyz, "shape") else 0
    xyz = _dev_f32(xyz, (n, 3), "xyz")
    q = _dev_f32(q, (n,), "q")
    with torch.cuda.device(xyz.device):
        if out is None:
            phi = torch.empty(n, device=xyz.device, dtype=torch.float32)
            grad = torch.empty(n, 3, device=xyz.device, dtype=torch.float32)
        else:
            phi, grad = out
        o = _options(max_depth, precision, select, m2l_unit_blocks, serialize_phases, replay)
        st = Stats()
        _check(load().fmm_laplace3d_ex(xyz.data_ptr(), q.data_ptr(), n, p, float(theta), ncrit,
                                       phi.data_ptr(), grad.data_ptr(), _stream_ptr(torch, xyz.device),
                                       ctypes.byref(o), ctypes.byref(st) if stats else None))
    return (phi, grad, st.as_dict()) if stats else (phi, grad)


def laplace3d_host(xyz: np.ndarray, q: np.ndarray, p: int, theta: float, ncrit: int, *,
                   max_depth: int = 0, precision: str = "fp32", select="plain", m2l_unit_blocks: int = 0,
                   stats: bool = False,
                   out=None,
                   stream=None, serialize_phases: bool = False, replay: bool = True):
    """Same solve with host (numpy) arrays: the library copies in and out."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float32)
    q = np.ascontiguousarray(q, dtype=np.float32)
    n = xyz.shape[0]
    if out is None:
        phi = np.empty(n, dtype=np.float32)
        grad = np.empty((n, 3), dtype=np.float32)
    else:
        phi, grad = out
    o = _options(max_depth, precision, select, m2l_unit_blocks, serialize_phases, replay)
    st = Stats()
    _check(load().fmm_laplace3d_host(xyz.ctypes.data, q.ctypes.data, n, p, float(theta), ncrit,
                                     phi.ctypes.data, grad.ctypes.data,
                                     ctypes.c_void_p(stream or 0), ctypes.byref(o),
                                     ctypes.byref(st) if stats else None))
    return (phi, grad, st.as_dict()) if stats else (phi, grad)


def laplace3d_batched(xyz, q, offsets, p: int, theta: float, ncrit: int, *, max_depth: int = 0,
                      precision: str = "fp32", select="plain", m2l_unit_blocks: int = 0, stats: bool = False,
                      out=None, serialize_phases: bool = False, replay: bool = True):
    """Independent systems in one solve: system s = rows offsets[s]:offsets[s+1] of
    the CUDA float32 xyz[N,3], q[N]; offsets is a host int sequence (len nsys + 1)."""
    import torch
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    n = int(xyz.shape[0])
    if off.ndim != 1 or len(off) < 2 or off[-1] != n:
        raise FmmError(FMM_ERR_ARG, "offsets must be 1-D with offsets[-1] == N")
    xyz = _dev_f32(xyz, (n, 3), "xyz")
    q = _dev_f32(q, (n,), "q")
    with torch.cuda.device(xyz.device):
        if out is None:
            phi = torch.empty(n, device=xyz.device, dtype=torch.float32)
            grad = torch.empty(n, 3, device=xyz.device, dtype=torch.float32)
        else:
            phi, grad = out
        o = _options(max_depth, precision, select, m2l_unit_blocks, serialize_phases, replay)
        st = Stats()
        _check(load().fmm_laplace3d_batched(xyz.data_ptr(), q.data_ptr(), off.ctypes.data,
                                            len(off) - 1, p, float(theta), ncrit, phi.data_ptr(),
                                            grad.data_ptr(), _stream_ptr(torch, xyz.device),
                                            ctypes.byref(o), ctypes.byref(st) if stats else None))
    return (phi, grad, st.as_dict()) if stats else (phi, grad)


def cost_model_pick_ncrit(xyz, q, p: int, theta: float, candidates=(16, 32, 64, 128, 256), *, max_depth: int = 0,
                          precision: str = "fp32", select="plain"):
    """N_crit from the learned cost model (fmm_cost_model_pick_ncrit): (best,
    {candidate: predicted ms}).  Builds each candidate's tree and lists, times
    nothing."""
    import torch
    n = int(xyz.shape[0])
    xyz = _dev_f32(xyz, (n, 3), "xyz")
    q = _dev_f32(q, (n,), "q")
    cand = np.ascontiguousarray(np.asarray(candidates, dtype=np.int32))
    pred = np.zeros(len(cand), dtype=np.float32)
    best = ctypes.c_int()
    o = _options(max_depth, precision, select)
    with torch.cuda.device(xyz.device):
        _check(load().fmm_cost_model_pick_ncrit(xyz.data_ptr(), q.data_ptr(), n, p, float(theta),
                                                _stream_ptr(torch, xyz.device), ctypes.byref(o), cand.ctypes.data,
                                                len(cand), pred.ctypes.data, ctypes.byref(best)))
    return best.value, {int(c): float(m) for c, m in zip(cand, pred)}


def measure_fp32() -> dict:
    """FP32-pipe ceilings on the current device (fmm_measure_fp32): the rate of an
    FP32x2 FMA stream in TFLOP/s and the interactions per second of the P2P
    interaction body on staged sources."""
    import torch
    f, b = ctypes.c_double(), ctypes.c_double()
    dev = torch.cuda.current_device()
    _check(load().fmm_measure_fp32(ctypes.byref(f), ctypes.byref(b), _stream_ptr(torch, dev)))
    return {"ffma_tflops": f.value, "body_interactions_per_s": b.value}


class Plan:
    """A solve captured into one CUDA graph (fmm_plan_create): fixed N, systems,
    p, theta, ncrit and options; replayed for new particle data with one graph
    launch and no synchronisation.  ``check()`` tells whether the last replay
    stayed within the plan's capacities (else its results are invalid)."""

    def __init__(self, xyz, q, p: int, theta: float, ncrit: int, *, offsets=None, max_depth: int = 0,
                 precision: str = "fp32", select="plain", m2l_unit_blocks: int = 0, headroom: float = 1.25):
        import torch
        n = int(xyz.shape[0])
        xyz = _dev_f32(xyz, (n, 3), "xyz")
        q = _dev_f32(q, (n,), "q")
        self.n = n
        self.device = xyz.device
        off = None
        nsys = 1
        if offsets is not None:
            off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
            nsys = len(off) - 1
        self._off = off
        o = _options(max_depth, precision, select, m2l_unit_blocks)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(load().fmm_plan_create(ctypes.byref(h), xyz.data_ptr(), q.data_ptr(), n,
                                          off.ctypes.data if off is not None else None, nsys, p, float(theta),
                                          ncrit, ctypes.byref(o), float(headroom), _stream_ptr(torch, self.device)))
        self._h = h

    def execute(self, xyz=None, q=None, out=None):
        """Replays the plan on the current stream; xyz/q (CUDA float32) replace the
        plan's inputs when given.  Returns (phi, grad) CUDA tensors (new tensors
        unless ``out``); nothing is synchronised."""
        import torch
        n = self.n
        xp = _dev_f32(xyz, (n, 3), "xyz").data_ptr() if xyz is not None else None
        qp = _dev_f32(q, (n,), "q").data_ptr() if q is not None else None
        with torch.cuda.device(self.device):
            if out is None:
                phi = torch.empty(n, device=self.device, dtype=torch.float32)
                grad = torch.empty(n, 3, device=self.device, dtype=torch.float32)
            else:
                phi, grad = out
            _check(load().fmm_plan_execute(self._h, xp, qp, phi.data_ptr(), grad.data_ptr(),
                                           _stream_ptr(torch, self.device)))
        return phi, grad

    def execute_in_place(self):
        """Replays the plan on its own buffers (see ``buffers``): no copies."""
        import torch
        with torch.cuda.device(self.device):
            _check(load().fmm_plan_execute(self._h, None, None, None, None, _stream_ptr(torch, self.device)))

    def buffers(self):
        """Device pointers (ints) of the plan's xyz, q, phi and grad buffers."""
        ptrs = [ctypes.c_void_p() for _ in range(4)]
        _check(load().fmm_plan_buffers(self._h, *[ctypes.byref(x) for x in ptrs]))
        return tuple(x.value for x in ptrs)

    def check(self) -> int:
        """Synchronises the current stream; returns the status of the last replay
        (0 = valid, FMM_ERR_CAPACITY = it exceeded the plan)."""
        import torch
        with torch.cuda.device(self.device):
            return load().fmm_plan_check(self._h, _stream_ptr(torch, self.device))

    def info(self) -> dict:
        inf = PlanInfo()
        _check(load().fmm_plan_info(self._h, ctypes.byref(inf)))
        return inf.as_dict()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().fmm_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def direct(xyz, q):
    """Exact all-pairs sum on the GPU (FP32)."""
    import torch
    n = int(xyz.shape[0])
    xyz = _dev_f32(xyz, (n, 3), "xyz")
    q = _dev_f32(q, (n,), "q")
    with torch.cuda.device(xyz.device):
        phi = torch.empty(n, device=xyz.device, dtype=torch.float32)
        grad = torch.empty(n, 3, device=xyz.device, dtype=torch.float32)
        _check(load().fmm_direct(xyz.data_ptr(), q.data_ptr(), n, phi.data_ptr(), grad.data_ptr(),
                                 _stream_ptr(torch, xyz.device)))
    return phi, grad


_EXPORT_DTYPE = {"box": (np.float64, 4), "keys": (np.uint64, None), "order": (np.int32, None),
                 "cells": (np.int64, 6), "p2p": (np.int32, 2), "m2l": (np.int32, 3),
                 "multipole": (np.float32, "P2pad"), "local": (np.float32, "P2pad"),
                 "select": (np.uint8, SELECT_NB), "m2p": (np.int32, 2), "p2l": (np.int32, 2)}


def export(what: str, p: int | None = None) -> np.ndarray:
    """An intermediate array of the last solve on the current device (see fmm.h)."""
    L = load()
    need = ctypes.c_int64(0)
    _check(L.fmm_export(EXPORT[what], None, 0, ctypes.byref(need)))
    dt, width = _EXPORT_DTYPE[what]
    buf = np.empty(need.value // np.dtype(dt).itemsize, dtype=dt)
    _check(L.fmm_export(EXPORT[what], buf.ctypes.data, need.value, ctypes.byref(need)))
    if width == "P2pad":
        if p is None:
            raise ValueError("p is needed to shape expansion exports")
        width = ((p + 1) ** 2 + 31) // 32 * 32
    return buf.reshape(-1, width) if width else buf


def morton_sort_noalloc(xyz, out=None):
    """Morton keys, sorted order and box of CUDA float32 xyz[N,3] through the
    entry point that allocates no device memory (N <= 1048576).

    ``out`` = (keys int64-viewed uint64 [N], order int32 [N], box float64 [4]) CUDA
    tensors to fill; allocated with torch when omitted."""
    import torch
    n = int(xyz.shape[0])
    xyz = _dev_f32(xyz, (n, 3), "xyz")
    with torch.cuda.device(xyz.device):
        if out is None:
            keys = torch.empty(n, dtype=torch.int64, device=xyz.device)
            order = torch.empty(n, dtype=torch.int32, device=xyz.device)
            box = torch.empty(4, dtype=torch.float64, device=xyz.device)
        else:
            keys, order, box = out
        _check(load().fmm_morton_sort_noalloc(xyz.data_ptr(), n, keys.data_ptr(), order.data_ptr(),
                                              box.data_ptr(), _stream_ptr(torch, xyz.device)))
    return keys, order, box


# ---------------------------------------------------------------- hybrid selection

def _f32(a, shape):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if shape is not None and a.shape != shape:
        raise FmmError(FMM_ERR_ARG, f"expected shape {shape}, got {a.shape}")
    return a


def selection_table(mode: str, p: int, theta: float, precision: str = "fp32") -> np.ndarray:
    """uint8 [128, 128] table the "autotune" or "learned" mode uses (see fmm.h)."""
    t = np.zeros((SELECT_NB, SELECT_NB), dtype=np.uint8)
    _check(load().fmm_selection_table(SELECT[mode], p, float(theta), PRECISION[precision], t.ctypes.data))
    return t


def cost_model_train(precision: str = "fp32", p_lo: int = 3, p_hi: int = 12, steps: int = 2000,
                     seed: int = 1) -> dict:
    """Time the kernels on artificial data and train the cost-model network on the GPU."""
    info = CostModelInfo()
    _check(load().fmm_cost_model_train(PRECISION[precision], p_lo, p_hi, steps, seed, ctypes.byref(info)))
    return info.as_dict()


def cost_model_get(master: bool = False) -> np.ndarray:
    w = np.zeros(COST_MODEL_PARAMS, dtype=np.float32)
    _check(load().fmm_cost_model_get(w.ctypes.data, w.size, int(master)))
    return w


def cost_model_set(params) -> None:
    w = _f32(params, (COST_MODEL_PARAMS,))
    _check(load().fmm_cost_model_set(w.ctypes.data, w.size))


def cost_model_grad(x, t, m):
    """(loss, gradient[4610]) of the current network over a host batch, on the GPU."""
    x = _f32(x, None).reshape(-1, 4)
    b = x.shape[0]
    t, m = _f32(t, (b, 2)), _f32(m, (b, 2))
    loss = np.zeros(1, dtype=np.float32)
    g = np.zeros(COST_MODEL_PARAMS, dtype=np.float32)
    _check(load().fmm_cost_model_grad(x.ctypes.data, t.ctypes.data, m.ctypes.data, b, loss.ctypes.data,
                                      g.ctypes.data))
    return float(loss[0]), g


def cost_model_adam_step(x, t, m, lr: float) -> float:
    x = _f32(x, None).reshape(-1, 4)
    b = x.shape[0]
    t, m = _f32(t, (b, 2)), _f32(m, (b, 2))
    loss = np.zeros(1, dtype=np.float32)
    _check(load().fmm_cost_model_adam_step(x.ctypes.data, t.ctypes.data, m.ctypes.data, b, float(lr),
                                           loss.ctypes.data))
    return float(loss[0])


def cost_model_predict(x) -> np.ndarray:
    x = _f32(x, None).reshape(-1, 4)
    y = np.zeros((x.shape[0], 2), dtype=np.float32)
    _check(load().fmm_cost_model_predict(x.ctypes.data, x.shape[0], y.ctypes.data))
    return y


def cost_model_samples():
    """(x [n,4], t [n,2], m [n,2]) of the last training."""
    n = ctypes.c_int64(0)
    _check(load().fmm_cost_model_samples(None, None, None, 0, ctypes.byref(n)))
    k = n.value
    x = np.zeros((k, 4), np.float32)
    t = np.zeros((k, 2), np.float32)
    m = np.zeros((k, 2), np.float32)
    if k:
        _check(load().fmm_cost_model_samples(x.ctypes.data, t.ctypes.data, m.ctypes.data, k, ctypes.byref(n)))
    return x, t, m


def tune_ncrit(xyz, q, p: int, theta: float, candidates=(16, 32, 64, 128, 256), *, max_depth: int = 0,
               precision: str = "fp32", select="plain"):
    """Measured autotuner for ncrit: (best, {ncrit: ms}) over the candidates."""
    import torch
    n = int(xyz.shape[0])
    xyz = _dev_f32(xyz, (n, 3), "xyz")
    q = _dev_f32(q, (n,), "q")
    c = np.ascontiguousarray(np.asarray(candidates, dtype=np.int32))
    ms = np.zeros(len(c), dtype=np.float32)
    best = ctypes.c_int(0)
    with torch.cuda.device(xyz.device):
        o = _options(max_depth, precision, select)
        _check(load().fmm_tune_ncrit(xyz.data_ptr(), q.data_ptr(), n, p, float(theta),
                                     _stream_ptr(torch, xyz.device), ctypes.byref(o), c.ctypes.data,
                                     len(c), ms.ctypes.data, ctypes.byref(best)))
    return best.value, {int(k): float(v) for k, v in zip(c, ms)}


def tune_schedule(xyz, q, p: int, theta: float, offsets=None, ncrit_candidates=(16, 32, 64, 128),
                  unit_candidates=(0, 8, 32, 128), *, max_depth: int = 0, precision: str = "fp32",
                  select="plain"):
    """Measured autotuner for (ncrit, M2L work-unit size) of a single or batched solve:
    (best_ncrit, best_unit, {(ncrit, unit): ms})."""
    import torch
    n = int(xyz.shape[0])
    xyz = _dev_f32(xyz, (n, 3), "xyz")
    q = _dev_f32(q, (n,), "q")
    nc = np.ascontiguousarray(np.asarray(ncrit_candidates, dtype=np.int32))
    uc = np.ascontiguousarray(np.asarray(unit_candidates, dtype=np.int32))
    ms = np.zeros(len(nc) * len(uc), dtype=np.float32)
    bn, bu = ctypes.c_int(0), ctypes.c_int(0)
    off = None if offsets is None else np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    with torch.cuda.device(xyz.device):
        o = _options(max_depth, precision, select)
        _check(load().fmm_tune_schedule(xyz.data_ptr(), q.data_ptr(), n, None if off is None else off.ctypes.data,
                                        0 if off is None else len(off) - 1, p, float(theta),
                                        _stream_ptr(torch, xyz.device), ctypes.byref(o), nc.ctypes.data, len(nc),
                                        uc.ctypes.data, len(uc), ms.ctypes.data, ctypes.byref(bn), ctypes.byref(bu)))
    table = {(int(a), int(b)): float(ms[i * len(uc) + j]) for i, a in enumerate(nc) for j, b in enumerate(uc)}
    return bn.value, bu.value, table


def selftest_wait_timeout(polls: int = 1 << 16) -> int:
    """Run the bounded-wait self-test; returns the library status (FMM_ERR_TIMEOUT expected)."""
    import torch
    with torch.cuda.device(torch.cuda.current_device()):
        return int(load().fmm_selftest_wait_timeout(int(polls), _stream_ptr(torch, torch.cuda.current_device())))
