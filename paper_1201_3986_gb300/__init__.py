"""Python binding of the qdvm C ABI (include/qdvm.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
kernels of ``libqdvm.so``.  PyTorch supplies device memory and the current
stream; nothing here computes any part of the operator.  Importing this
package loads the in-tree library and raises if it has not been built (there
is no fallback).

Names follow the C ABI: ``qdvm_plan_create``, ``qdvm_eval``,
``qdvm_eval_batched``, ``qdvm_jvp``, ``qdvm_vjp``, ``qdvm_moments``.  ``Plan``
wraps a plan handle, ``QdvmFunction`` exposes Q as a differentiable
``torch.autograd.Function`` (backward = ``qdvm_vjp``).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqdvm.so")

QDVM_KERNEL_UNIT, QDVM_KERNEL_HP = 0, 1
QDVM_F64, QDVM_F32, QDVM_F32_KAHAN = 0, 1, 2
QDVM_ENGINE_AUTO, QDVM_ENGINE_DIRECT, QDVM_ENGINE_SCAN = 0, 1, 2
QDVM_MAX_BATCH_PLANS = 16

KERNELS = {"unit": QDVM_KERNEL_UNIT, "hp": QDVM_KERNEL_HP}
PRECS = {"f64": QDVM_F64, "f32": QDVM_F32, "f32_kahan": QDVM_F32_KAHAN}
ENGINES = {"auto": QDVM_ENGINE_AUTO, "direct": QDVM_ENGINE_DIRECT, "scan": QDVM_ENGINE_SCAN}
QDVM_SCAN_J_DEFAULT = 0  # initial tuning scan_j of plans created with engine "auto" (qdvm.h)
_DTYPE = {QDVM_F64: torch.float64, QDVM_F32: torch.float32, QDVM_F32_KAHAN: torch.float32}


class QdvmError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        super().__init__(f"{where}: {detail}")


if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"qdvm CUDA library not built ({LIB_PATH} missing); run "
        "`python -c 'import __graft_entry__ as g; g.build()'` first")

_lib = ctypes.CDLL(LIB_PATH)
_vp = ctypes.c_void_p
_i = ctypes.c_int
_sz = ctypes.c_size_t
_P = ctypes.POINTER


def _sig(name, args):
    fn = getattr(_lib, name)
    fn.argtypes = args
    fn.restype = ctypes.c_int
    return fn


_sig("qdvm_plan_create", [_P(_vp), _i, _i, _i, ctypes.c_double, _i])
_sig("qdvm_plan_create_ex", [_P(_vp), _i, _i, _i, _i, ctypes.c_double, _i, _i])
_sig("qdvm_plan_destroy", [_vp])
_sig("qdvm_plan_info", [_vp, _P(_i), _P(_i), _P(_i), _P(_i), _P(_i), _P(ctypes.c_int64)])
_sig("qdvm_plan_lines", [_vp, _P(_i), _P(_i), _P(ctypes.c_double)])
_sig("qdvm_plan_row_info", [_vp, _P(_i), _P(_i)])
_sig("qdvm_eval_workspace", [_vp, _i, _P(_sz)])
_sig("qdvm_eval", [_vp, _vp, _vp, _i, _vp, _sz, _vp])
_sig("qdvm_eval_batched", [_P(_vp), _i, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp, _sz, _vp])
_sig("qdvm_jvp", [_vp, _vp, _vp, _vp, _i, _vp, _sz, _vp])
_sig("qdvm_vjp", [_vp, _vp, _vp, _vp, _i, _vp, _sz, _vp])
_sig("qdvm_batched_workspace", [_P(_vp), _i, _i, _i, _P(_sz)])
_sig("qdvm_jvp_batched", [_P(_vp), _i, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp, _sz, _vp])
_sig("qdvm_vjp_batched", [_P(_vp), _i, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp, _sz, _vp])
_sig("qdvm_moments", [_vp, _vp, _i, _vp, _vp])
class QdvmTuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("direct_j", ctypes.c_int), ("line_chunks", ctypes.c_int),
                ("loss_fft", ctypes.c_int), ("scan_j", ctypes.c_int)]


def _tuning_dict(t) -> dict:
    return {"threads": t.threads, "direct_j": t.direct_j, "line_chunks": t.line_chunks, "loss_fft": t.loss_fft,
            "scan_j": t.scan_j}


_sig("qdvm_plan_get_tuning", [_vp, _P(QdvmTuning)])
_sig("qdvm_plan_set_tuning", [_vp, _P(QdvmTuning)])
_sig("qdvm_tune_batched", [_P(_vp), _i, _i, _vp, _vp, _vp, _vp, _i, _vp, _sz, _vp, _P(QdvmTuning)])
_sig("qdvm_graph_capture_batched", [_P(_vp), _P(_vp), _i, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp, _sz])
_sig("qdvm_graph_launch", [_vp, _vp])
_sig("qdvm_graph_destroy", [_vp])
_sig("qdvm_eval_batched_noalloc", [_P(_vp), _i, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp])
_sig("qdvm_rk2_workspace", [_P(_vp), _i, _i, ctypes.c_int64, _i, _P(_sz)])
_sig("qdvm_rk2_batched", [_P(_vp), _i, _i, _vp, _vp, ctypes.c_int64, _vp, ctypes.c_double, _i, _vp, _i, _vp, _sz,
                          _vp])
_sig("qdvm_rk2_workspace_single", [_vp, _i, _P(_sz)])
_sig("qdvm_rk2", [_vp, _vp, ctypes.c_double, _i, _i, _vp, _sz, _vp])
_sig("qdvm_equilibrium_distance", [_P(_vp), _i, _i, _vp, _vp, _vp, _i, _vp, _vp])
_sig("qdvm_select_levels", [_i, _vp, _vp, _i, _i, _P(ctypes.c_double), _P(_i), _vp, _vp])
QDVM_MAX_LEVELS = 8
_sig("qdvm_eval_direct_batched", [_P(_vp), _i, _i, _vp, _vp, _vp, _vp, _vp, _i, _i, _vp])
_sig("qdvm_eval_direct_workspace", [_P(_sz)])
_sig("qdvm_eval_direct", [_vp, _vp, _vp, _i, _i, _vp, _sz, _vp])
_sig("qdvm_spectral_table_entries", [_vp, _P(_sz)])
_sig("qdvm_spectral_table", [_vp, _vp, _i, _vp])
_sig("qdvm_spectral_workspace", [_vp, _i, _i, _P(_sz)])
_sig("qdvm_eval_spectral", [_vp, _vp, _i, _vp, _vp, _i, _vp, _sz, _vp])
_BOUNDARY = {"periodic": 0, "box": 1}
_sig("qdvm_graph_capture_rk2", [_P(_vp), _P(_vp), _i, _i, _vp, _vp, ctypes.c_int64, _vp, ctypes.c_double, _i, _vp,
                                _i, _vp, _sz])
QDVM_NOALLOC_MAX_CELLS = 65536
_lib.qdvm_status_string.argtypes = [_i]
_lib.qdvm_status_string.restype = ctypes.c_char_p
_lib.qdvm_last_error.argtypes = []
_lib.qdvm_last_error.restype = ctypes.c_char_p
_lib.qdvm_version.argtypes = []
_lib.qdvm_version.restype = ctypes.c_char_p


def _check(status: int, where: str) -> None:
    if status != 0:
        s = _lib.qdvm_status_string(status).decode()
        detail = _lib.qdvm_last_error().decode()
        raise QdvmError(status, where, f"{s} ({detail})")


def version() -> str:
    return _lib.qdvm_version().decode()


def _ptr(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(device=None):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _prec(prec) -> int:
    return PRECS[prec] if isinstance(prec, str) else int(prec)


# ------------------------------------------------------------------- plans

def qdvm_plan_create(d: int, N: int, Nbar: int, L: float, kernel="unit", Ntilde: int | None = None,
                     engine="auto") -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
    e = ENGINES[engine] if isinstance(engine, str) else int(engine)
    _check(_lib.qdvm_plan_create_ex(ctypes.byref(h), d, N, Nbar, -1 if Ntilde is None else int(Ntilde),
                                    float(L), k, e), "qdvm_plan_create")
    return h


class Plan:
    """Owning wrapper of a qdvm plan (lines of A_m, windows, weights)."""

    def __init__(self, d: int, N: int, Nbar: int, L: float, kernel="unit", Ntilde: int | None = None,
                 engine="auto"):
        self.handle = None
        self.handle = qdvm_plan_create(d, N, Nbar, L, kernel, Ntilde, engine)
        vals = [ctypes.c_int() for _ in range(5)]
        nt = ctypes.c_int64()
        _check(_lib.qdvm_plan_info(self.handle, *[ctypes.byref(v) for v in vals], ctypes.byref(nt)), "qdvm_plan_info")
        self.d, self.N, self.Ntilde, self.m, self.n_lines = (v.value for v in vals)
        self.n_terms = nt.value
        self.L = float(L)
        self.h = 2.0 * self.L / self.N
        self.kernel = kernel

    def lines(self):
        """(dirs[n,3], J[n], c[n]) copied from the plan's tables."""
        n = self.n_lines
        dirs = np.zeros((n, 3), dtype=np.int32)
        J = np.zeros(n, dtype=np.int32)
        c = np.zeros(n, dtype=np.float64)
        _check(_lib.qdvm_plan_lines(self.handle, dirs.ctypes.data_as(_P(_i)), J.ctypes.data_as(_P(_i)),
                                    c.ctypes.data_as(_P(ctypes.c_double))), "qdvm_plan_lines")
        return dirs[:, :self.d], J, c

    def row_info(self):
        """(line classes, rows) of the 3D row decomposition; (0, 0) without."""
        nc, nr = ctypes.c_int(), ctypes.c_int()
        _check(_lib.qdvm_plan_row_info(self.handle, ctypes.byref(nc), ctypes.byref(nr)), "qdvm_plan_row_info")
        return nc.value, nr.value

    def eval_workspace(self, prec) -> int:
        b = ctypes.c_size_t()
        _check(_lib.qdvm_eval_workspace(self.handle, _prec(prec), ctypes.byref(b)), "qdvm_eval_workspace")
        return b.value

    def tuning(self) -> dict:
        t = QdvmTuning()
        _check(_lib.qdvm_plan_get_tuning(self.handle, ctypes.byref(t)), "qdvm_plan_get_tuning")
        return _tuning_dict(t)

    def set_tuning(self, threads=None, direct_j=None, line_chunks=None, loss_fft=None, scan_j=None) -> None:
        cur = self.tuning()
        t = QdvmTuning(cur["threads"] if threads is None else int(threads),
                       cur["direct_j"] if direct_j is None else int(direct_j),
                       cur["line_chunks"] if line_chunks is None else int(line_chunks),
                       cur["loss_fft"] if loss_fft is None else int(loss_fft),
                       cur["scan_j"] if scan_j is None else int(scan_j))
        _check(_lib.qdvm_plan_set_tuning(self.handle, ctypes.byref(t)), "qdvm_plan_set_tuning")

    @property
    def shape(self):
        return (self.N,) * self.d

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.qdvm_plan_destroy(self.handle)
            self.handle = None


def _workspace(nbytes: int, device) -> torch.Tensor | None:
    if nbytes == 0:
        return None
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def _check_batch(p: int, cell_plan: torch.Tensor, cell_offset: torch.Tensor, f: torch.Tensor,
                 Q: torch.Tensor | None = None, moments: torch.Tensor | None = None, n_mom: int = 4) -> None:
    """Argument checks of the batched calls, made before anything reaches
    the device: the cell layout (int32 plan indices, int64 offsets, one of
    each per cell), f and Q of the precision's dtype, and the moments array
    (float64, n_mom values per cell), all contiguous CUDA tensors on f's
    device.  A wrong array here would otherwise be read or written out of
    bounds by the kernels."""
    if cell_plan.dtype != torch.int32 or cell_offset.dtype != torch.int64:
        raise ValueError("cell_plan must be int32 and cell_offset int64")
    if f.dtype != _DTYPE[p] or not f.is_cuda or not f.is_contiguous():
        raise ValueError(f"f must be a contiguous CUDA {_DTYPE[p]} tensor")
    for name, t in (("cell_plan", cell_plan), ("cell_offset", cell_offset)):
        if not t.is_cuda or t.device != f.device or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CUDA tensor on {f.device}")
    if cell_plan.numel() != cell_offset.numel():
        raise ValueError("cell_plan and cell_offset must hold one entry per cell")
    if Q is not None:
        if Q.dtype != f.dtype or not Q.is_cuda or Q.device != f.device or not Q.is_contiguous() \
                or Q.numel() < f.numel():
            raise ValueError(f"Q must be a contiguous CUDA {f.dtype} tensor on {f.device} with f's size")
    if moments is not None:
        if moments.dtype != torch.float64 or not moments.is_cuda or moments.device != f.device \
                or not moments.is_contiguous() or moments.numel() < n_mom * cell_plan.numel():
            raise ValueError(f"moments must be a contiguous CUDA float64 tensor on {f.device} "
                             f"with at least {n_mom} values per cell")


# -------------------------------------------------------------- evaluation

def qdvm_eval(plan: Plan, f: torch.Tensor, prec="f64", out: torch.Tensor | None = None,
              workspace: torch.Tensor | None = None) -> torch.Tensor:
    p = _prec(prec)
    if f.dtype != _DTYPE[p] or not f.is_cuda or not f.is_contiguous() or tuple(f.shape) != plan.shape:
        raise ValueError(f"f must be a contiguous CUDA {_DTYPE[p]} tensor of shape {plan.shape}")
    Q = torch.empty_like(f) if out is None else out
    wsb = plan.eval_workspace(p)
    ws = workspace if workspace is not None else _workspace(wsb, f.device)
    _check(_lib.qdvm_eval(plan.handle, _ptr(f), _ptr(Q), p, _ptr(ws), 0 if ws is None else ws.numel(),
                          _stream(f.device)), "qdvm_eval")
    return Q


def qdvm_moments(plan: Plan, Q: torch.Tensor, prec="f64") -> torch.Tensor:
    p = _prec(prec)
    m = torch.empty(plan.d + 2, dtype=torch.float64, device=Q.device)
    _check(_lib.qdvm_moments(plan.handle, _ptr(Q), p, _ptr(m), _stream(Q.device)), "qdvm_moments")
    return m


def _plan_array(plans):
    arr = (ctypes.c_void_p * len(plans))(*[p.handle.value for p in plans])
    return arr


def batched_workspace_bytes(plans, n_cells: int, prec) -> int:
    b = ctypes.c_size_t()
    _check(_lib.qdvm_batched_workspace(_plan_array(plans), len(plans), int(n_cells), _prec(prec), ctypes.byref(b)),
           "qdvm_batched_workspace")
    return b.value


def qdvm_eval_batched(plans, cell_plan: torch.Tensor, cell_offset: torch.Tensor, f: torch.Tensor, prec="f32_kahan",
                      out: torch.Tensor | None = None, moments: torch.Tensor | bool | None = True,
                      workspace: torch.Tensor | None = None):
    """Evaluate Q on a ragged batch of cells in one persistent launch.

    Returns (Q, moments) where moments is an (n_cells, d+2) float64 tensor
    (or None when ``moments`` is False)."""
    p = _prec(prec)
    n_cells = int(cell_plan.numel())
    _check_batch(p, cell_plan, cell_offset, f)
    Q = torch.empty_like(f) if out is None else out
    d = plans[0].d
    mom = None
    if isinstance(moments, torch.Tensor):
        mom = moments
    elif moments:
        mom = torch.empty((n_cells, d + 2), dtype=torch.float64, device=f.device)
    _check_batch(p, cell_plan, cell_offset, f, Q, mom, d + 2)
    ws = workspace if workspace is not None else _workspace(batched_workspace_bytes(plans, n_cells, p), f.device)
    arr = _plan_array(plans)
    _check(_lib.qdvm_eval_batched(arr, len(plans), n_cells, _ptr(cell_plan), _ptr(cell_offset), _ptr(f), _ptr(Q),
                                  _ptr(mom), p, _ptr(ws), 0 if ws is None else ws.numel(), _stream(f.device)),
           "qdvm_eval_batched")
    return Q, mom


class BatchedGraph:
    """qdvm_eval_batched captured once into a CUDA graph (fixed tensors);
    ``launch()`` replays it on the current stream."""

    def __init__(self, plans, cell_plan, cell_offset, f, Q, moments, prec="f32_kahan", workspace=None):
        p = _prec(prec)
        n_cells = int(cell_plan.numel())
        _check_batch(p, cell_plan, cell_offset, f, Q, moments, plans[0].d + 2)
        self._keep = (plans, cell_plan, cell_offset, f, Q, moments)
        self.workspace = workspace if workspace is not None else _workspace(
            batched_workspace_bytes(plans, n_cells, p), f.device)
        self.handle = None
        h = ctypes.c_void_p()
        _check(_lib.qdvm_graph_capture_batched(ctypes.byref(h), _plan_array(plans), len(plans), n_cells,
                                               _ptr(cell_plan), _ptr(cell_offset), _ptr(f), _ptr(Q), _ptr(moments), p,
                                               _ptr(self.workspace),
                                               0 if self.workspace is None else self.workspace.numel()),
               "qdvm_graph_capture_batched")
        self.handle = h
        self.device = f.device

    def launch(self):
        _check(_lib.qdvm_graph_launch(self.handle, _stream(self.device)), "qdvm_graph_launch")

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.qdvm_graph_destroy(self.handle)
            self.handle = None


def rk2_workspace_bytes(plans, n_cells: int, n_elems: int, prec) -> int:
    b = ctypes.c_size_t()
    _check(_lib.qdvm_rk2_workspace(_plan_array(plans), len(plans), n_cells, int(n_elems), _prec(prec), ctypes.byref(b)),
           "qdvm_rk2_workspace")
    return b.value


def _rk2_args(plans, cell_plan, cell_offset, f, prec, moments, workspace):
    p = _prec(prec)
    n_cells = int(cell_plan.numel())
    if cell_plan.dtype != torch.int32 or cell_offset.dtype != torch.int64:
        raise ValueError("cell_plan must be int32 and cell_offset int64")
    if f.dtype != _DTYPE[p] or not f.is_cuda or not f.is_contiguous():
        raise ValueError(f"f must be a contiguous CUDA {_DTYPE[p]} tensor")
    mom = None
    if isinstance(moments, torch.Tensor):
        mom = moments
    elif moments:
        mom = torch.empty((n_cells, plans[0].d + 2), dtype=torch.float64, device=f.device)
    ws = workspace if workspace is not None else _workspace(rk2_workspace_bytes(plans, n_cells, f.numel(), p),
                                                            f.device)
    return p, n_cells, mom, ws


def qdvm_rk2_batched(plans, cell_plan: torch.Tensor, cell_offset: torch.Tensor, f: torch.Tensor, dt: float,
                     n_steps: int, prec="f32_kahan", moments: torch.Tensor | bool | None = False,
                     workspace: torch.Tensor | None = None):
    """Advance every cell of a ragged batch by n_steps second-order TVD
    Runge-Kutta steps of df/dt = Q(f), in place on f.  Returns (f, moments
    of the final f or None)."""
    p, n_cells, mom, ws = _rk2_args(plans, cell_plan, cell_offset, f, prec, moments, workspace)
    _check(_lib.qdvm_rk2_batched(_plan_array(plans), len(plans), n_cells, _ptr(cell_plan), _ptr(cell_offset), f.numel(),
                                 _ptr(f), float(dt), int(n_steps), _ptr(mom), p, _ptr(ws),
                                 0 if ws is None else ws.numel(), _stream(f.device)), "qdvm_rk2_batched")
    return f, mom


def rk2_workspace_single_bytes(plan: Plan, prec) -> int:
    b = ctypes.c_size_t()
    _check(_lib.qdvm_rk2_workspace_single(plan.handle, _prec(prec), ctypes.byref(b)), "qdvm_rk2_workspace_single")
    return b.value


def qdvm_rk2(plan: Plan, f: torch.Tensor, dt: float, n_steps: int, prec="f64",
             workspace: torch.Tensor | None = None) -> torch.Tensor:
    """Advance one cell by n_steps second-order TVD Runge-Kutta steps of
    df/dt = Q(f), in place on f."""
    p = _prec(prec)
    if f.dtype != _DTYPE[p] or not f.is_cuda or not f.is_contiguous():
        raise ValueError(f"f must be a contiguous CUDA {_DTYPE[p]} tensor")
    if workspace is None:
        workspace = _workspace(rk2_workspace_single_bytes(plan, p), f.device)
    _check(_lib.qdvm_rk2(plan.handle, _ptr(f), float(dt), int(n_steps), p, _ptr(workspace),
                         0 if workspace is None else workspace.numel(), _stream(f.device)), "qdvm_rk2")
    return f


def qdvm_eval_direct(plan: Plan, f: torch.Tensor, prec="f64", boundary="box",
                     out: torch.Tensor | None = None) -> torch.Tensor:
    """Term-by-term evaluation of one cell: boundary "box" gives the exactly
    conservative D^tr, "periodic" the periodised Q without the fast
    decomposition."""
    p = _prec(prec)
    if f.dtype != _DTYPE[p] or not f.is_cuda or not f.is_contiguous():
        raise ValueError(f"f must be a contiguous CUDA {_DTYPE[p]} tensor")
    Q = torch.empty_like(f) if out is None else out
    ws = torch.empty(256, dtype=torch.uint8, device=f.device)
    _check(_lib.qdvm_eval_direct(plan.handle, _ptr(f), _ptr(Q), p, _BOUNDARY[boundary], _ptr(ws), ws.numel(),
                                 _stream(f.device)), "qdvm_eval_direct")
    return Q


def spectral_table(plan: Plan, prec="f64", device=None) -> torch.Tensor:
    """The table beta~(K, L) of the pseudo-spectral route (N^d x N^d, row K,
    column L), built on the device."""
    p = _prec(prec)
    n = ctypes.c_size_t()
    _check(_lib.qdvm_spectral_table_entries(plan.handle, ctypes.byref(n)), "qdvm_spectral_table_entries")
    M = plan.N ** plan.d
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    table = torch.empty((M, M), dtype=_DTYPE[p], device=dev)
    assert table.numel() == n.value
    _check(_lib.qdvm_spectral_table(plan.handle, _ptr(table), p, _stream(dev)), "qdvm_spectral_table")
    return table


def spectral_workspace_bytes(plan: Plan, n_cells: int, prec) -> int:
    b = ctypes.c_size_t()
    _check(_lib.qdvm_spectral_workspace(plan.handle, int(n_cells), _prec(prec), ctypes.byref(b)),
           "qdvm_spectral_workspace")
    return b.value


def qdvm_eval_spectral(plan: Plan, table: torch.Tensor, f: torch.Tensor, prec="f64", out: torch.Tensor | None = None,
                       workspace: torch.Tensor | None = None) -> torch.Tensor:
    """Q of a batch of cells (f of shape (n_cells,) + plan.shape, or one cell
    of plan.shape) through the Fourier modes, eq. (sysDiff)."""
    p = _prec(prec)
    if f.dtype != _DTYPE[p] or not f.is_cuda or not f.is_contiguous():
        raise ValueError(f"f must be a contiguous CUDA {_DTYPE[p]} tensor")
    if table.dtype != _DTYPE[p] or not table.is_cuda or not table.is_contiguous():
        raise ValueError("table must come from spectral_table in the same precision")
    M = plan.N ** plan.d
    if f.numel() % M:
        raise ValueError("f must hold whole cells of N^d points")
    n_cells = f.numel() // M
    Q = torch.empty_like(f) if out is None else out
    ws = workspace if workspace is not None else _workspace(spectral_workspace_bytes(plan, n_cells, p), f.device)
    _check(_lib.qdvm_eval_spectral(plan.handle, _ptr(table), n_cells, _ptr(f), _ptr(Q), p, _ptr(ws),
                                   0 if ws is None else ws.numel(), _stream(f.device)), "qdvm_eval_spectral")
    return Q


def qdvm_eval_direct_batched(plans, cell_plan: torch.Tensor, cell_offset: torch.Tensor, f: torch.Tensor,
                             prec="f32_kahan", boundary="box", out: torch.Tensor | None = None,
                             moments: torch.Tensor | bool | None = True):
    """Term-by-term evaluation of a ragged batch; returns (Q, moments)."""
    p = _prec(prec)
    n_cells = int(cell_plan.numel())
    if cell_plan.dtype != torch.int32 or cell_offset.dtype != torch.int64:
        raise ValueError("cell_plan must be int32 and cell_offset int64")
    if f.dtype != _DTYPE[p] or not f.is_cuda or not f.is_contiguous():
        raise ValueError(f"f must be a contiguous CUDA {_DTYPE[p]} tensor")
    Q = torch.empty_like(f) if out is None else out
    mom = moments if isinstance(moments, torch.Tensor) else (
        torch.empty((n_cells, plans[0].d + 2), dtype=torch.float64, device=f.device) if moments else None)
    _check(_lib.qdvm_eval_direct_batched(_plan_array(plans), len(plans), n_cells, _ptr(cell_plan), _ptr(cell_offset),
                                         _ptr(f), _ptr(Q), _ptr(mom), p, _BOUNDARY[boundary], _stream(f.device)),
           "qdvm_eval_direct_batched")
    return Q, mom


def equilibrium_distance(plans, cell_plan: torch.Tensor, cell_offset: torch.Tensor, f: torch.Tensor,
                         prec="f32_kahan", out: torch.Tensor | None = None) -> torch.Tensor:
    """Per-cell FP64 distance sum|f - M[f]| / sum|f| to the Maxwellian with
    the cell's own discrete moments (+inf where undefined)."""
    p = _prec(prec)
    n_cells = int(cell_plan.numel())
    if f.dtype != _DTYPE[p] or not f.is_cuda or not f.is_contiguous():
        raise ValueError(f"f must be a contiguous CUDA {_DTYPE[p]} tensor")
    eps = torch.empty(n_cells, dtype=torch.float64, device=f.device) if out is None else out
    _check(_lib.qdvm_equilibrium_distance(_plan_array(plans), len(plans), n_cells, _ptr(cell_plan), _ptr(cell_offset),
                                          _ptr(f), p, _ptr(eps), _stream(f.device)), "qdvm_equilibrium_distance")
    return eps


def select_levels(eps: torch.Tensor, cell_base: torch.Tensor, thresholds, level_plan,
                  out: torch.Tensor | None = None) -> torch.Tensor:
    """cell_plan[c] = level_plan[cell_base[c]][level], level = number of the
    (strictly increasing) thresholds that eps[c] reaches."""
    lp = np.ascontiguousarray(np.asarray(level_plan, dtype=np.int32))
    if lp.ndim != 2:
        raise ValueError("level_plan must be a 2-D table (base, level)")
    thr = np.ascontiguousarray(np.asarray(thresholds, dtype=np.float64).reshape(-1))
    if thr.size != lp.shape[1] - 1:
        raise ValueError("need one threshold fewer than levels")
    n_cells = int(eps.numel())
    res = torch.empty(n_cells, dtype=torch.int32, device=eps.device) if out is None else out
    _check(_lib.qdvm_select_levels(n_cells, _ptr(eps), _ptr(cell_base), lp.shape[0], lp.shape[1],
                                   thr.ctypes.data_as(_P(ctypes.c_double)) if thr.size else None,
                                   lp.ctypes.data_as(_P(_i)), _ptr(res), _stream(eps.device)), "qdvm_select_levels")
    return res


class RK2Graph:
    """n_steps of qdvm_rk2_batched (fixed tensors, f updated in place)
    captured into one CUDA graph; ``launch()`` replays the whole loop."""

    def __init__(self, plans, cell_plan, cell_offset, f, dt, n_steps, prec="f32_kahan", moments=None,
                 workspace=None):
        p, n_cells, mom, ws = _rk2_args(plans, cell_plan, cell_offset, f, prec, moments, workspace)
        self._keep = (plans, cell_plan, cell_offset, f, mom)
        self.workspace = ws
        self.moments = mom
        self.handle = None
        h = ctypes.c_void_p()
        _check(_lib.qdvm_graph_capture_rk2(ctypes.byref(h), _plan_array(plans), len(plans), n_cells, _ptr(cell_plan),
                                           _ptr(cell_offset), f.numel(), _ptr(f), float(dt), int(n_steps), _ptr(mom),
                                           p, _ptr(ws), 0 if ws is None else ws.numel()), "qdvm_graph_capture_rk2")
        self.handle = h
        self.device = f.device

    def launch(self):
        _check(_lib.qdvm_graph_launch(self.handle, _stream(self.device)), "qdvm_graph_launch")

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.qdvm_graph_destroy(self.handle)
            self.handle = None


def qdvm_tune_batched(plans, cell_plan: torch.Tensor, cell_offset: torch.Tensor, f: torch.Tensor, prec="f32_kahan",
                      workspace: torch.Tensor | None = None) -> dict:
    """Time the candidate launch configurations on this batch, keep the
    fastest in every plan and return it."""
    p = _prec(prec)
    n_cells = int(cell_plan.numel())
    Q = torch.empty_like(f)
    ws = workspace if workspace is not None else _workspace(batched_workspace_bytes(plans, n_cells, p), f.device)
    t = QdvmTuning()
    _check(_lib.qdvm_tune_batched(_plan_array(plans), len(plans), n_cells, _ptr(cell_plan), _ptr(cell_offset), _ptr(f),
                                  _ptr(Q), p, _ptr(ws), 0 if ws is None else ws.numel(), _stream(f.device),
                                  ctypes.byref(t)), "qdvm_tune_batched")
    return _tuning_dict(t)


def qdvm_eval_batched_noalloc(plans, cell_plan: torch.Tensor, cell_offset: torch.Tensor, f: torch.Tensor, Q: torch.Tensor,
                              moments: torch.Tensor | None, prec="f32_kahan") -> None:
    """Batched 2D evaluation through the allocation-free entry point: the
    caller passes every array (f, Q, moments or None); the library uses its
    own static scratch and allocates nothing."""
    p = _prec(prec)
    _check_batch(p, cell_plan, cell_offset, f, Q, moments, 4)
    _check(_lib.qdvm_eval_batched_noalloc(_plan_array(plans), len(plans), int(cell_plan.numel()), _ptr(cell_plan),
                                          _ptr(cell_offset), _ptr(f), _ptr(Q), _ptr(moments), p, _stream(f.device)),
           "qdvm_eval_batched_noalloc")


def qdvm_jvp(plan: Plan, f: torch.Tensor, df: torch.Tensor, prec="f64", out=None, workspace=None) -> torch.Tensor:
    p = _prec(prec)
    dQ = torch.empty_like(f) if out is None else out
    wsb = plan.eval_workspace(p)
    ws = workspace if workspace is not None else _workspace(wsb, f.device)
    _check(_lib.qdvm_jvp(plan.handle, _ptr(f), _ptr(df), _ptr(dQ), p, _ptr(ws), 0 if ws is None else ws.numel(),
                         _stream(f.device)), "qdvm_jvp")
    return dQ


def qdvm_vjp(plan: Plan, f: torch.Tensor, g: torch.Tensor, prec="f64", out=None, workspace=None) -> torch.Tensor:
    p = _prec(prec)
    gr = torch.empty_like(f) if out is None else out
    wsb = plan.eval_workspace(p)
    ws = workspace if workspace is not None else _workspace(wsb, f.device)
    _check(_lib.qdvm_vjp(plan.handle, _ptr(f), _ptr(g), _ptr(gr), p, _ptr(ws), 0 if ws is None else ws.numel(),
                         _stream(f.device)), "qdvm_vjp")
    return gr


def _derivative_batched(fn, name, plans, cell_plan, cell_offset, f, a, prec, out, workspace):
    p = _prec(prec)
    n_cells = int(cell_plan.numel())
    if cell_plan.dtype != torch.int32 or cell_offset.dtype != torch.int64:
        raise ValueError("cell_plan must be int32 and cell_offset int64")
    for t in (f, a):
        if t.dtype != _DTYPE[p] or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"inputs must be contiguous CUDA {_DTYPE[p]} tensors")
    res = torch.empty_like(f) if out is None else out
    ws = workspace if workspace is not None else _workspace(batched_workspace_bytes(plans, n_cells, p), f.device)
    _check(fn(_plan_array(plans), len(plans), n_cells, _ptr(cell_plan), _ptr(cell_offset), _ptr(f), _ptr(a),
              _ptr(res), p, _ptr(ws), 0 if ws is None else ws.numel(), _stream(f.device)), name)
    return res


def qdvm_jvp_batched(plans, cell_plan, cell_offset, f, df, prec="f32", out=None, workspace=None):
    """dQ = Q'(f) df for every cell of a ragged batch."""
    return _derivative_batched(_lib.qdvm_jvp_batched, "qdvm_jvp_batched", plans, cell_plan, cell_offset, f, df,
                               prec, out, workspace)


def qdvm_vjp_batched(plans, cell_plan, cell_offset, f, g, prec="f32", out=None, workspace=None):
    """grad = Q'(f)^T g for every cell of a ragged batch."""
    return _derivative_batched(_lib.qdvm_vjp_batched, "qdvm_vjp_batched", plans, cell_plan, cell_offset, f, g,
                               prec, out, workspace)


class QdvmFunction(torch.autograd.Function):
    """Q(f) with a hand-written adjoint: backward calls qdvm_vjp."""

    @staticmethod
    def forward(ctx, f, plan, prec):
        ctx.plan = plan
        ctx.prec = prec
        ctx.save_for_backward(f)
        return qdvm_eval(plan, f.contiguous(), prec)

    @staticmethod
    def backward(ctx, g):
        (f,) = ctx.saved_tensors
        return qdvm_vjp(ctx.plan, f, g.contiguous(), ctx.prec), None, None


def collision(f: torch.Tensor, plan: Plan, prec="f64") -> torch.Tensor:
    """Differentiable Q(f)."""
    return QdvmFunction.apply(f, plan, prec)
