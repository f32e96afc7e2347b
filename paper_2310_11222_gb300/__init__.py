"""GB300-native Generalized-Euclidean (GE) node-vector distance.

    d(x, y)^2 = (x - y)^T L^+ (x - y)            (Section 3.1 of the paper, GE equation)

computed without forming L^+: the CUDA library (``_build/libnvd.so``, C ABI in
``include/nvd.h``) solves L z = x - y with a Jacobi-preconditioned conjugate
gradient (Section 3.2, the "CG" Laplacian solver) whose SpMV/SpMM, fused
update/inner-product passes, preconditioner and per-component projection are
hand-written sm_103a kernels.

This module only marshals arguments to the C ABI (ctypes); every step of the
computation runs in the library's kernels.  There is no CPU fallback: if the
library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

__all__ = [
    "Graph", "SolveOpts", "SolveStats", "ge_distance", "effective_resistance", "resistance_matrix",
    "network_variance", "ge_distance_batched", "ge_grad",
    "laplacian_apply", "dot_f32", "GEDistance", "ge_distance_autograd", "profile_enable", "profile_read",
    "library_path", "load_library", "NvdError", "MODE_FP64", "MODE_FP32", "MODE_MIXED",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libnvd.so")

F32, F64 = 0, 1
MODE_FP64, MODE_FP32, MODE_MIXED = 0, 1, 2
SOLVE_SINGLE_RHS = 1
SOLVE_D2_DEVICE = 2
SOLVE_HOST_INPUTS = 4
SOLVE_PERSISTENT = 8
SOLVE_NO_SYNC = 16
SOLVE_FOLD_DIRECTION = 32
SOLVE_TEST_TIMEOUT = 64
SOLVE_D2_STOP = 128
SOLVE_ELIMINATE = 256
GRAPH_DEVICE_PTRS = 1
GRAPH_SKIP_SYM_CHECK = 2
GRAPH_REORDER_DEGREE = 4
TUNE_SINGLE_RHS = 1
GATHER_SLICES, GATHER_STREAM, GATHER_TMA, GATHER_ACOPY = 0, 1, 2, 3   # nvd_tune_result.gather

STATUS = {0: "NVD_OK", 1: "NVD_ERR_INVALID_ARG", 2: "NVD_ERR_NOT_SYMMETRIC", 3: "NVD_ERR_BAD_WEIGHT",
          4: "NVD_ERR_OOM", 5: "NVD_ERR_CUDA", 6: "NVD_ERR_NOT_CONVERGED", 7: "NVD_ERR_NUMERIC",
          8: "NVD_ERR_TIMEOUT", 9: "NVD_ERR_UNSUPPORTED"}


class NvdError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class SolveOpts(ctypes.Structure):
    """Mirror of ``nvd_solve_opts``."""
    _fields_ = [("mode", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("rtol", ctypes.c_double),
                ("d2_rtol", ctypes.c_double), ("max_refine", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("kt", ctypes.c_int32), ("flags", ctypes.c_uint32)]


class SolveStats(ctypes.Structure):
    """Mirror of ``nvd_solve_stats``."""
    _fields_ = [("iters", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("rel_resid", ctypes.c_double), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ElimInfo(ctypes.Structure):
    """Mirror of ``nvd_elim_info``."""
    _fields_ = [("n_kept", ctypes.c_int64), ("nnz_kept", ctypes.c_int64), ("n_eliminated", ctypes.c_int64),
                ("rounds", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    """Mirror of ``nvd_tune_result``."""
    _fields_ = [("kt", ctypes.c_int32), ("row_max_pct", ctypes.c_int32), ("blocks_pct", ctypes.c_int32),
                ("persistent", ctypes.c_int32), ("candidates", ctypes.c_int32), ("fold_direction", ctypes.c_int32),
                ("gather", ctypes.c_int32), ("l2_hot", ctypes.c_int32),
                ("ms_per_iter", ctypes.c_double), ("ms_per_pair_iter", ctypes.c_double)]


_lib = None
_lock = threading.Lock()

_SIGS = {
    "nvd_graph_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.c_uint32, ctypes.c_void_p]),
    "nvd_graph_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "nvd_graph_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int64)]),
    "nvd_graph_set_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32,
                                             ctypes.c_void_p]),
    "nvd_solve_opts_default": (None, [ctypes.POINTER(SolveOpts)]),
    "nvd_graph_tune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32,
                                      ctypes.POINTER(TuneResult), ctypes.c_void_p]),
    "nvd_graph_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(TuneResult)]),
    "nvd_ge_distance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int32, ctypes.POINTER(SolveOpts), ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "nvd_ge_distance_batched": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                               ctypes.POINTER(SolveOpts), ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p]),
    "nvd_ge_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "nvd_graph_eliminate": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ElimInfo), ctypes.c_void_p]),
    "nvd_eliminate_host": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "nvd_eliminate_host_program": (ctypes.c_int, [ctypes.c_int64] + [ctypes.c_void_p] * 18),
    "nvd_ge_distance_warm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int32, ctypes.c_void_p, ctypes.POINTER(SolveOpts),
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "nvd_effective_resistance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.POINTER(SolveOpts), ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "nvd_resistance_matrix": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                             ctypes.POINTER(SolveOpts), ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p]),
    "nvd_network_variance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.POINTER(SolveOpts), ctypes.c_void_p, ctypes.c_void_p]),
    "nvd_laplacian_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_int32, ctypes.c_void_p]),
    "nvd_dot_f32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p]),
    "nvd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "nvd_last_error": (ctypes.c_char_p, []),
    "nvd_profile_enable": (ctypes.c_int, [ctypes.c_int32]),
    "nvd_profile_read": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "nvd_version": (ctypes.c_char_p, []),
    "nvd_kernel_launches": (ctypes.c_int64, []),
}


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Load ``libnvd.so`` (built by ``build.build()``); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise RuntimeError(f"CUDA library not built: {_LIB_PATH} is missing "
                                   "(run __graft_entry__.build() or paper_2310_11222_gb300/build.py)")
            lib = ctypes.CDLL(_LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int, where: str, allow=(0,)):
    if rc not in allow:
        detail = load_library().nvd_last_error()
        raise NvdError(rc, where, detail.decode() if detail else "")
    return rc


def _torch():
    import torch
    return torch


def _stream_ptr(device=None):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def default_opts(mode: int = MODE_FP64, **kw) -> SolveOpts:
    o = SolveOpts()
    load_library().nvd_solve_opts_default(ctypes.byref(o))
    o.mode = mode
    if mode == MODE_MIXED:
        o.rtol = 1e-4
    elif mode == MODE_FP32:
        o.rtol = 1e-5
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _weight_key(w):
    """(address, version) of a torch weight tensor: a changed key means new values
    (an optimizer step bumps the version); None for numpy or no weights."""
    if w is None or isinstance(w, np.ndarray) or not hasattr(w, "_version"):
        return None
    return (w.data_ptr(), int(w._version))


class Graph:
    """Handle on a graph held in device memory (``nvd_graph_create``).

    ``rowptr`` int64 [n+1], ``colidx`` int32 [nnz], ``w`` float32/float64 [nnz] (or None
    for unit weights) describe a symmetric CSR adjacency.  numpy arrays are copied
    from the host; torch CUDA tensors are read on the device.
    """

    def __init__(self, rowptr, colidx, w=None, *, skip_sym_check: bool = False, reorder: bool = False,
                 device=None):
        torch = _torch()
        lib = load_library()
        self._lib = lib
        self.handle = ctypes.c_void_p(None)
        flags = (GRAPH_SKIP_SYM_CHECK if skip_sym_check else 0) | (GRAPH_REORDER_DEGREE if reorder else 0)
        keep = []
        if isinstance(rowptr, np.ndarray):
            rp = np.ascontiguousarray(rowptr, dtype=np.int64)
            ci = np.ascontiguousarray(colidx, dtype=np.int32)
            wv = None if w is None else np.ascontiguousarray(w)
            if wv is not None and wv.dtype not in (np.float32, np.float64):
                wv = wv.astype(np.float64)
            wdt = F64 if (wv is None or wv.dtype == np.float64) else F32
            keep = [rp, ci, wv]
            p_rp, p_ci = rp.ctypes.data, ci.ctypes.data
            p_w = None if wv is None else wv.ctypes.data
            n = rp.shape[0] - 1
            nnz = ci.shape[0]
            dev = device if device is not None else torch.cuda.current_device()
        else:
            rp = rowptr.contiguous()
            ci = colidx.contiguous()
            wv = None if w is None else w.contiguous()
            if rp.dtype != torch.int64 or ci.dtype != torch.int32:
                raise TypeError("rowptr must be int64 and colidx int32")
            wdt = F64 if wv is None else _dtype_code(wv)
            keep = [rp, ci, wv]
            if rp.is_cuda:
                flags |= GRAPH_DEVICE_PTRS
                dev = rp.device.index
            else:
                dev = device if device is not None else torch.cuda.current_device()
            p_rp, p_ci = rp.data_ptr(), ci.data_ptr()
            p_w = None if wv is None else wv.data_ptr()
            n = rp.shape[0] - 1
            nnz = ci.shape[0]
        self.device = torch.device("cuda", dev)
        self.wdtype = wdt
        self.n_user = int(n)
        self.nnz_user = int(nnz)
        # the torch weight tensor (address, version) the handle's weights came from
        self._w_key = _weight_key(w)
        with torch.cuda.device(self.device):
            rc = lib.nvd_graph_create(ctypes.byref(self.handle), int(n), int(nnz), p_rp, p_ci, p_w, wdt,
                                      flags, _stream_ptr(self.device))
        del keep
        _check(rc, "nvd_graph_create")

    @classmethod
    def from_csr(cls, g, **kw):
        """From an object with ``rowptr``, ``colidx``, ``w`` numpy attributes."""
        return cls(g.rowptr, g.colidx, g.w, **kw)

    def set_weights(self, w, *, skip_sym_check: bool = False):
        """New weights for the same sparsity pattern (``nvd_graph_set_weights``), in the
        entry order of the CSR the graph was built from: numpy (host) or torch (host
        or this graph's device).  Converted to the graph's weight type."""
        torch = _torch()
        flags = GRAPH_SKIP_SYM_CHECK if skip_sym_check else 0
        if isinstance(w, np.ndarray):
            wv = np.ascontiguousarray(w, dtype=np.float64 if self.wdtype == F64 else np.float32)
            ptr = wv.ctypes.data
            key = None
        else:
            key = _weight_key(w)
            wv = w.detach().to(torch.float64 if self.wdtype == F64 else torch.float32).contiguous()
            if wv.is_cuda:
                flags |= GRAPH_DEVICE_PTRS
            ptr = wv.data_ptr()
        if wv.shape[0] != self.nnz_user:
            raise ValueError(f"expected {self.nnz_user} weights, got {wv.shape[0]}")
        with torch.cuda.device(self.device):
            rc = self._lib.nvd_graph_set_weights(self.handle, ptr, self.wdtype, flags, _stream_ptr(self.device))
        _check(rc, "nvd_graph_set_weights")
        self._w_key = key

    def info(self):
        n, nnz, nc, nb = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        _check(self._lib.nvd_graph_info(self.handle, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(nc),
                                        ctypes.byref(nb)), "nvd_graph_info")
        return {"n": n.value, "nnz": nnz.value, "ncomp": nc.value, "device_bytes": nb.value}

    def eliminate(self) -> dict:
        """Eliminate degree-1/2 nodes exactly (nvd_graph_eliminate); later solves with
        ``eliminate=True`` run PCG on the reduced graph."""
        info = ElimInfo()
        torch = _torch()
        with torch.cuda.device(self.device):
            _check(self._lib.nvd_graph_eliminate(self.handle, ctypes.byref(info), _stream_ptr(self.device)),
                   "nvd_graph_eliminate")
        return {"n_kept": info.n_kept, "nnz_kept": info.nnz_kept, "n_eliminated": info.n_eliminated,
                "rounds": info.rounds}

    def tune(self, *, mode: int = 0, k: int = 1, single_rhs: bool = False) -> dict:
        """Time the solve's work decompositions on this graph (``nvd_graph_tune``) and keep
        the fastest for later calls of ``mode``; returns the chosen setting."""
        torch = _torch()
        r = TuneResult()
        with torch.cuda.device(self.device):
            rc = self._lib.nvd_graph_tune(self.handle, int(mode), int(k), TUNE_SINGLE_RHS if single_rhs else 0,
                                          ctypes.byref(r), _stream_ptr(self.device))
        _check(rc, "nvd_graph_tune")
        return {f: getattr(r, f) for f, _ in TuneResult._fields_}

    def set_tuning(self, *, mode: int = 0, kt: int = 0, row_max_pct: int = 100, blocks_pct: int = 100,
                   persistent: bool = False, fold_direction: bool = False, gather: int = GATHER_SLICES,
                   l2_hot: bool = False):
        """Apply a work-decomposition setting without timing (``nvd_graph_set_tuning``).
        ``gather``: GATHER_SLICES (default), GATHER_STREAM, GATHER_TMA or GATHER_ACOPY; ``l2_hot``: keep the
        highest-degree rows of a degree-ordered graph persisting in L2."""
        r = TuneResult(kt=int(kt), row_max_pct=int(row_max_pct), blocks_pct=int(blocks_pct),
                       persistent=int(bool(persistent)), fold_direction=int(bool(fold_direction)),
                       gather=int(gather), l2_hot=int(bool(l2_hot)))
        _check(self._lib.nvd_graph_set_tuning(self.handle, int(mode), ctypes.byref(r)), "nvd_graph_set_tuning")

    @property
    def n(self) -> int:
        return self.n_user

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.nvd_graph_destroy(self.handle)
            self.handle = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ge_distance(graph: Graph, x, y, *, mode: int = MODE_FP64, rtol: Optional[float] = None,
                d2_rtol: float = 1e-8, max_iter: int = 10000, max_refine: int = 8, kt: int = 0,
                check_every: int = 4, single_rhs: bool = False, persistent: bool = False,
                fold_direction: bool = False, test_timeout: bool = False, d2_stop: bool = False,
                z0=None, eliminate: bool = False, return_z: bool = False, return_stats: bool = False,
                allow_not_converged: bool = False):
    """Squared GE distances d^2 for the k pairs (rows) of x, y ([k, n] or [n]).

    CUDA tensors run on the device (d^2 returned as a CUDA float64 tensor); CPU
    tensors / numpy arrays go through the host-buffer path of the C ABI (copies
    inside the call) and d^2 comes back on the host.  ``z0`` (CUDA, the shape and
    dtype of x, FP64 mode) warm-starts every solve from a saved solution, e.g. the
    z returned by an earlier call (nvd_ge_distance_warm).  ``eliminate`` solves on
    the reduced graph of ``graph.eliminate()`` (CUDA inputs; z by back-substitution).
    """
    torch = _torch()
    lib = load_library()
    if isinstance(x, np.ndarray):
        x = torch.from_numpy(x)
    if isinstance(y, np.ndarray):
        y = torch.from_numpy(y)
    one = x.dim() == 1
    X = (x[None] if one else x).contiguous()
    Y = (y[None] if one else y).contiguous()
    if X.shape != Y.shape or X.dtype != Y.dtype or X.shape[1] != graph.n:
        raise ValueError("x and y must both be [k, n] of the same dtype")
    k = X.shape[0]
    o = default_opts(mode, d2_rtol=d2_rtol, max_iter=max_iter, max_refine=max_refine, kt=kt,
                     check_every=check_every)
    if rtol is not None:
        o.rtol = rtol
    if single_rhs:
        o.flags |= SOLVE_SINGLE_RHS
    if persistent:
        o.flags |= SOLVE_PERSISTENT
    if fold_direction:
        o.flags |= SOLVE_FOLD_DIRECTION
    if test_timeout:
        o.flags |= SOLVE_TEST_TIMEOUT
    if d2_stop:
        o.flags |= SOLVE_D2_STOP
    if eliminate:
        o.flags |= SOLVE_ELIMINATE
    xdt = _dtype_code(X)
    stats = (SolveStats * max(k, 1))()
    if z0 is not None:
        Z0 = (z0[None] if one else z0).contiguous()
        if not (X.is_cuda and Z0.is_cuda) or Z0.shape != X.shape or Z0.dtype != X.dtype:
            raise ValueError("z0 must be a CUDA tensor of the shape and dtype of x (and x on the device)")
        d2 = torch.empty(k, dtype=torch.float64, device=X.device)
        Z = torch.empty_like(X) if return_z else None
        o.flags |= SOLVE_D2_DEVICE
        with torch.cuda.device(X.device):
            rc = lib.nvd_ge_distance_warm(graph.handle, k, X.data_ptr(), Y.data_ptr(), xdt, Z0.data_ptr(),
                                          ctypes.byref(o), d2.data_ptr(), None if Z is None else Z.data_ptr(),
                                          stats, _stream_ptr(X.device))
    elif X.is_cuda:
        d2 = torch.empty(k, dtype=torch.float64, device=X.device)
        Z = torch.empty_like(X) if return_z else None
        o.flags |= SOLVE_D2_DEVICE
        with torch.cuda.device(X.device):
            rc = lib.nvd_ge_distance(graph.handle, k, X.data_ptr(), Y.data_ptr(), xdt, ctypes.byref(o),
                                     d2.data_ptr(), None if Z is None else Z.data_ptr(), stats,
                                     _stream_ptr(X.device))
    else:
        d2 = torch.empty(k, dtype=torch.float64)
        Z = torch.empty_like(X) if return_z else None
        o.flags |= SOLVE_HOST_INPUTS
        with torch.cuda.device(graph.device):
            rc = lib.nvd_ge_distance(graph.handle, k, X.data_ptr(), Y.data_ptr(), xdt, ctypes.byref(o),
                                     d2.data_ptr(), None if Z is None else Z.data_ptr(), stats,
                                     _stream_ptr(graph.device))
    _check(rc, "nvd_ge_distance", allow=(0, 6) if allow_not_converged else (0,))
    out = [d2[0] if one else d2]
    if return_z:
        out.append(Z[0] if one else Z)
    if return_stats:
        out.append([{"iters": s.iters, "refine_steps": s.refine_steps, "rel_resid": s.rel_resid,
                     "status": s.status} for s in stats[:k]])
    return out[0] if len(out) == 1 else tuple(out)


def effective_resistance(graph: Graph, u, v, *, mode: int = MODE_FP64, rtol: Optional[float] = None,
                         d2_rtol: float = 1e-8, max_iter: int = 10000, kt: int = 0, persistent: bool = False,
                         d2_stop: bool = False, eliminate: bool = False, return_stats: bool = False,
                         allow_not_converged: bool = False):
    """Effective resistances R(u_j, v_j) = (e_u - e_v)^T L^+ (e_u - e_v) for node-id
    sequences u, v of equal length: 0 where u = v, inf across components.
    Returns a float64 numpy array."""
    lib = load_library()
    U = np.ascontiguousarray(np.atleast_1d(np.asarray(u)), dtype=np.int32)
    V = np.ascontiguousarray(np.atleast_1d(np.asarray(v)), dtype=np.int32)
    if U.shape != V.shape or U.ndim != 1:
        raise ValueError("u and v must be 1-D sequences of equal length")
    k = U.shape[0]
    o = default_opts(mode, d2_rtol=d2_rtol, max_iter=max_iter, kt=kt)
    if rtol is not None:
        o.rtol = rtol
    if persistent:
        o.flags |= SOLVE_PERSISTENT
    if d2_stop:
        o.flags |= SOLVE_D2_STOP
    if eliminate:
        o.flags |= SOLVE_ELIMINATE
    r = np.empty(k, np.float64)
    stats = (SolveStats * max(k, 1))()
    torch = _torch()
    with torch.cuda.device(graph.device):
        rc = lib.nvd_effective_resistance(graph.handle, k, U.ctypes.data, V.ctypes.data, ctypes.byref(o),
                                          r.ctypes.data, stats, _stream_ptr(graph.device))
    _check(rc, "nvd_effective_resistance", allow=(0, 6) if allow_not_converged else (0,))
    if return_stats:
        return r, [{"iters": s.iters, "refine_steps": s.refine_steps, "rel_resid": s.rel_resid,
                    "status": s.status} for s in stats[:k]]
    return r


def resistance_matrix(graph: Graph, nodes, *, mode: int = MODE_FP64, rtol: Optional[float] = None,
                      d2_rtol: float = 1e-8, max_iter: int = 10000, kt: int = 0, persistent: bool = False,
                      return_stats: bool = False, allow_not_converged: bool = False):
    """Effective-resistance matrix [s, s] of the node subset ``nodes`` (one solve per
    node and component beyond the first); inf across components.  float64 numpy."""
    lib = load_library()
    N = np.ascontiguousarray(np.atleast_1d(np.asarray(nodes)), dtype=np.int32)
    if N.ndim != 1:
        raise ValueError("nodes must be a 1-D sequence")
    s_n = N.shape[0]
    o = default_opts(mode, d2_rtol=d2_rtol, max_iter=max_iter, kt=kt)
    if rtol is not None:
        o.rtol = rtol
    if persistent:
        o.flags |= SOLVE_PERSISTENT
    R = np.empty((s_n, s_n), np.float64)
    stats = (SolveStats * max(s_n, 1))()
    torch = _torch()
    with torch.cuda.device(graph.device):
        rc = lib.nvd_resistance_matrix(graph.handle, s_n, N.ctypes.data, ctypes.byref(o), R.ctypes.data, stats,
                                       _stream_ptr(graph.device))
    _check(rc, "nvd_resistance_matrix", allow=(0, 6) if allow_not_converged else (0,))
    if return_stats:
        return R, [{"iters": s.iters, "refine_steps": s.refine_steps, "rel_resid": s.rel_resid,
                    "status": s.status} for s in stats[:s_n]]
    return R


def network_variance(graph: Graph, nodes, p, *, mode: int = MODE_FP64, rtol: Optional[float] = None,
                     d2_rtol: float = 1e-8, max_iter: int = 10000, kt: int = 0,
                     allow_not_converged: bool = False) -> float:
    """Network variance (1/2) sum_ij p_i p_j R(nodes[i], nodes[j]) of non-negative
    node weights p (a distribution on the graph); inf across components."""
    lib = load_library()
    N = np.ascontiguousarray(np.atleast_1d(np.asarray(nodes)), dtype=np.int32)
    P = np.ascontiguousarray(np.atleast_1d(np.asarray(p)), dtype=np.float64)
    if N.ndim != 1 or N.shape != P.shape:
        raise ValueError("nodes and p must be 1-D sequences of equal length")
    o = default_opts(mode, d2_rtol=d2_rtol, max_iter=max_iter, kt=kt)
    if rtol is not None:
        o.rtol = rtol
    out = ctypes.c_double(0.0)
    torch = _torch()
    with torch.cuda.device(graph.device):
        rc = lib.nvd_network_variance(graph.handle, N.shape[0], N.ctypes.data, P.ctypes.data, ctypes.byref(o),
                                      ctypes.byref(out), _stream_ptr(graph.device))
    _check(rc, "nvd_network_variance", allow=(0, 6) if allow_not_converged else (0,))
    return out.value


def ge_distance_batched(graphs: Sequence[Graph], xs, ys, *, mode: int = MODE_FP32,
                        rtol: Optional[float] = None, max_iter: int = 10000, return_stats: bool = False,
                        fold_direction: bool = False, persistent: bool = False):
    """d^2 for many graphs in one solve; xs[g], ys[g] are CUDA [k_g, n_g].  One launch per
    phase over all graphs, or with ``persistent`` one persistent launch per tile."""
    torch = _torch()
    lib = load_library()
    G = len(graphs)
    hs = (ctypes.c_void_p * G)(*[g.handle.value for g in graphs])
    ks = (ctypes.c_int32 * G)(*[int(x.shape[0]) for x in xs])
    xs = [x.contiguous() for x in xs]
    ys = [y.contiguous() for y in ys]
    px = (ctypes.c_void_p * G)(*[x.data_ptr() for x in xs])
    py = (ctypes.c_void_p * G)(*[y.data_ptr() for y in ys])
    total = sum(int(x.shape[0]) for x in xs)
    o = default_opts(mode, max_iter=max_iter)
    if rtol is not None:
        o.rtol = rtol
    if fold_direction:
        o.flags |= SOLVE_FOLD_DIRECTION
    if persistent:
        o.flags |= SOLVE_PERSISTENT
    d2 = torch.empty(total, dtype=torch.float64)
    stats = (SolveStats * max(total, 1))()
    dev = xs[0].device
    with torch.cuda.device(dev):
        rc = lib.nvd_ge_distance_batched(hs, G, ks, px, py, _dtype_code(xs[0]), ctypes.byref(o),
                                         d2.data_ptr(), stats, _stream_ptr(dev))
    _check(rc, "nvd_ge_distance_batched")
    if return_stats:
        return d2, [{"iters": s.iters, "rel_resid": s.rel_resid, "status": s.status} for s in stats[:total]]
    return d2


def ge_grad(graph: Graph, z, gbar, *, want_w: bool = True, want_x: bool = True):
    """Adjoint of d^2: (grad_w [nnz], grad_x [k, n], grad_y [k, n]) from z and gbar = dL/d(d^2)."""
    torch = _torch()
    lib = load_library()
    Z = z.contiguous()
    gb = gbar.to(device=Z.device, dtype=torch.float64).contiguous()
    wdt = torch.float64 if graph.wdtype == F64 else torch.float32
    gw = torch.empty(graph.nnz_user, dtype=wdt, device=Z.device) if want_w else None
    gx = torch.empty_like(Z) if want_x else None
    gy = torch.empty_like(Z) if want_x else None
    with torch.cuda.device(Z.device):
        rc = lib.nvd_ge_grad(graph.handle, Z.shape[0], Z.data_ptr(), _dtype_code(Z), gb.data_ptr(),
                             None if gw is None else gw.data_ptr(), None if gx is None else gx.data_ptr(),
                             None if gy is None else gy.data_ptr(), _stream_ptr(Z.device))
    _check(rc, "nvd_ge_grad")
    return gw, gx, gy


def dot_f32(a, b) -> float:
    """sum a_i b_i of two FP32 CUDA vectors with the FP32-mode solver's inner-product
    reduction (``nvd_dot_f32``: exact products in double-float, FP64 sums)."""
    torch = _torch()
    lib = load_library()
    A = a.contiguous().reshape(-1)
    B = b.contiguous().reshape(-1)
    if A.dtype != torch.float32 or B.dtype != torch.float32 or A.numel() != B.numel():
        raise ValueError("dot_f32: two FP32 tensors of the same length")
    out = torch.empty(1, dtype=torch.float64, device=A.device)
    with torch.cuda.device(A.device):
        rc = lib.nvd_dot_f32(A.data_ptr(), B.data_ptr(), A.numel(), out.data_ptr(), _stream_ptr(A.device))
    _check(rc, "nvd_dot_f32")
    return float(out.item())


def laplacian_apply(graph: Graph, x):
    """y = L x for each row of x ([k, n] CUDA tensor)."""
    torch = _torch()
    lib = load_library()
    X = (x[None] if x.dim() == 1 else x).contiguous()
    Yt = torch.empty_like(X)
    with torch.cuda.device(X.device):
        rc = lib.nvd_laplacian_apply(graph.handle, X.shape[0], X.data_ptr(), Yt.data_ptr(), _dtype_code(X),
                                     _stream_ptr(X.device))
    _check(rc, "nvd_laplacian_apply")
    return Yt[0] if x.dim() == 1 else Yt


def kernel_launches() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load_library().nvd_kernel_launches())


def profile_enable(on=True, every: int = 1):
    """on: False/0 off, True/1 time the SpMV launches, 2 also the vector passes;
    every: time one SpMV launch in ``every`` (1..255)."""
    code = int(on)
    if code and every > 1:
        code |= (min(int(every), 255) & 0xff) << 8
    _check(load_library().nvd_profile_enable(code), "nvd_profile_enable")


def profile_read(kernel_class: int = 0):
    """(launches, total_ms, algorithmic_bytes) since the last read: class 0 = the SpMV/SpMM
    kernel, class 1 = the vector passes."""
    n, ms, b = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    _check(load_library().nvd_profile_read(kernel_class, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b)),
           "nvd_profile_read")
    return n.value, ms.value, b.value


def _make_autograd():
    torch = _torch()

    class GEDistance(torch.autograd.Function):
        """d^2 = (x - y)^T L^+ (x - y) with gradients for x, y and the CSR weights.

        forward(x, y, w, graph, opts) -> d^2 [k]; ``w`` holds the graph's weights in
        the entry order of its CSR.  When its values differ from the ones the graph
        holds (another tensor, or the same one after an in-place update such as an
        optimizer step) they are copied into the graph first
        (``nvd_graph_set_weights``), so the solve always uses the current ``w``.
        Backward reuses the forward z = L^+ delta (no new solve) through
        ``nvd_ge_grad``.
        """

        @staticmethod
        def forward(ctx, x, y, w, graph, opts):
            if w is not None and _weight_key(w) != graph._w_key:
                graph.set_weights(w)
            d2, z = ge_distance(graph, x, y, return_z=True, **(opts or {}))
            ctx.graph = graph
            ctx.save_for_backward(z)
            ctx.want_w = w is not None
            return d2

        @staticmethod
        def backward(ctx, gd2):
            (z,) = ctx.saved_tensors
            one = z.dim() == 1
            Z = z[None] if one else z
            g = gd2.reshape(-1)
            gw, gx, gy = ge_grad(ctx.graph, Z, g, want_w=ctx.want_w,
                                 want_x=ctx.needs_input_grad[0] or ctx.needs_input_grad[1])
            if gx is not None and one:
                gx, gy = gx[0], gy[0]
            return gx, gy, gw, None, None

    return GEDistance


class _Lazy:
    def __init__(self):
        self._cls = None

    def __getattr__(self, item):
        if self._cls is None:
            self._cls = _make_autograd()
        return getattr(self._cls, item)


GEDistance = _Lazy()


def ge_distance_autograd(graph: Graph, x, y, w=None, **opts):
    """Differentiable d^2 (see ``GEDistance``)."""
    return GEDistance.apply(x, y, w, graph, opts)
