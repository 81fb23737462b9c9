"""GB300-native SCSF: sorting Chebyshev subspace filter for eigenvalue datasets.

Python binding of the C ABI in ``include/scsf.h`` (``libscsf.so``, built in-tree
for sm_103a by ``paper_2510_23215_gb300.build``). This module only marshals
arguments: every step of the sort and of the solver runs in the library's CUDA
kernels. PyTorch provides device memory and the CUDA stream. There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.

Paper: "Accelerating Eigenvalue Dataset Generation via Chebyshev Subspace
Filter" - truncated-FFT greedy sort (Alg. 2) and warm-started Chebyshev
filtered subspace iteration (Alg. 1, Alg. 3) over a sorted sequence of
discretised symmetric operators (Sec. 2.1, Eq. (eq:eq_basic)).
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

__all__ = [
    "ScsfError", "Operator", "Params", "Context", "Chain", "library", "lib_path",
    "sort", "solve", "cheb_filter", "assemble_bounds", "small_eigh", "block_width",
    "FP64", "MIXED", "DIV_A_GRAD", "LAP_PLUS_V", "EXPORTED_SYMBOLS", "launch_count",
    "PRODUCT_TENSOR", "PRODUCT_FP64", "block_gram", "block_rotate", "BOUND_GERSHGORIN",
    "BOUND_LANCZOS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
lib_path = os.path.join(_HERE, "libscsf.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_TIMEOUT, ERR_NO_MEMORY = range(7)
DIV_A_GRAD, LAP_PLUS_V, CSR, PLATE = 0, 1, 2, 3
FP64, MIXED = 0, 1
PRODUCT_TENSOR, PRODUCT_FP64 = 0, 1
BOUND_GERSHGORIN, BOUND_LANCZOS = 0, 1

EXPORTED_SYMBOLS = [
    "scsf_create", "scsf_destroy", "scsf_last_error", "scsf_version",
    "scsf_sort_workspace_size", "scsf_sort", "scsf_max_block_width",
    "scsf_solve_workspace_size", "scsf_chain_create", "scsf_chain_seed", "scsf_chain_step",
    "scsf_solve_workspace_size_rows", "scsf_chain_create_rows", "scsf_cholqr2_scratch",
    "scsf_cholqr2",
    "scsf_chain_destroy", "scsf_solve", "scsf_cheb_filter", "scsf_assemble_bounds",
    "scsf_small_eigh_scratch", "scsf_small_eigh", "scsf_set_timing", "scsf_launch_count",
    "scsf_sort_noalloc_capacity", "scsf_sort_noalloc", "scsf_cheb_filter_f32",
    "scsf_batch_workspace_size", "scsf_solve_batched",
    "scsf_proposal_param_count", "scsf_proposal_workspace_size", "scsf_proposal_init",
    "scsf_proposal_forward", "scsf_proposal_train_step", "scsf_proposal_target_scratch",
    "scsf_proposal_targets", "scsf_proposal_prolong",
    "scsf_cheb_filter_dc_scratch", "scsf_cheb_filter_dc", "scsf_sort_dist", "scsf_block_rotate",
    "scsf_block_product_scratch", "scsf_block_gram", "scsf_block_rotate_ex",
    "scsf_chain_restart", "scsf_far_steps", "scsf_block_gram_kernel_time",
    "scsf_cheb_filter_dc_grouped",
]


class ScsfError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"scsf status {status}: {message}")
        self.status = status


class _COperator(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_int), ("ax", ctypes.c_void_p),
                ("ay", ctypes.c_void_p), ("v", ctypes.c_void_p), ("rows", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p),
                ("plate_d", ctypes.c_void_p), ("plate_rho", ctypes.c_void_p),
                ("field", ctypes.c_void_p)]


class _CParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("nex", ctypes.c_int), ("degree", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("degree_fp32", ctypes.c_int),
                ("switch_tol", ctypes.c_double), ("products", ctypes.c_int),
                ("use_proposal", ctypes.c_int), ("proposal", ctypes.c_void_p),
                ("bound", ctypes.c_int), ("column_degree", ctypes.c_int)]


class _CStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int),
                ("filter_steps", ctypes.c_int), ("locked", ctypes.c_int),
                ("flops_fp64", ctypes.c_double), ("filter_bytes", ctypes.c_double),
                ("filter_elems", ctypes.c_double), ("rot_flops", ctypes.c_double),
                ("rot_launches", ctypes.c_int), ("launches", ctypes.c_int),
                ("t_filter_ms", ctypes.c_double), ("t_orth_ms", ctypes.c_double),
                ("t_rr_ms", ctypes.c_double), ("t_eig_ms", ctypes.c_double),
                ("t_rot_ms", ctypes.c_double), ("t_resid_ms", ctypes.c_double),
                ("iters_fp32", ctypes.c_int), ("filter32_steps", ctypes.c_int),
                ("filter32_elems", ctypes.c_double), ("t_filter32_ms", ctypes.c_double),
                ("filter_dc_steps", ctypes.c_int), ("filter_dc_elems", ctypes.c_double),
                ("t_filter_dc_ms", ctypes.c_double),
                ("history", ctypes.POINTER(ctypes.c_double)),
                ("beta", ctypes.c_double), ("beta_gershgorin", ctypes.c_double),
                ("chol_shifts", ctypes.c_int), ("chol_shifts_fp32", ctypes.c_int)]


class _CBatchChain(ctypes.Structure):
    _fields_ = [("ops", ctypes.POINTER(_COperator)), ("n_ops", ctypes.c_int64),
                ("params", _CParams), ("evals", ctypes.c_void_p), ("resid", ctypes.c_void_p),
                ("evecs", ctypes.c_void_p), ("stats", ctypes.POINTER(_CStats)),
                ("status", ctypes.c_int)]


_lib = None


def library() -> ctypes.CDLL:
    """Loads libscsf.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(lib_path):
        raise ImportError(f"{lib_path} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(lib_path)
    vp, i32, i64, dbl, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    L.scsf_create.argtypes = [ctypes.POINTER(vp), i32, vp]
    L.scsf_destroy.argtypes = [vp]
    L.scsf_destroy.restype = None
    L.scsf_last_error.argtypes = [vp]
    L.scsf_last_error.restype = ctypes.c_char_p
    L.scsf_sort_workspace_size.argtypes = [i64, i32]
    L.scsf_sort_workspace_size.restype = sz
    L.scsf_sort.argtypes = [vp, vp, i64, i32, i32, i32, vp, sz, vp]
    L.scsf_sort_dist.argtypes = [vp, vp, i64, i32, i32, i32, vp, sz, vp, vp]
    L.scsf_block_rotate.argtypes = [vp, vp, i32, i32, i32, vp, i32, i32, vp, i32]
    L.scsf_block_rotate.restype = ctypes.c_int
    L.scsf_sort_dist.restype = ctypes.c_int
    L.scsf_max_block_width.restype = i32
    L.scsf_solve_workspace_size.argtypes = [ctypes.POINTER(_CParams), i32]
    L.scsf_solve_workspace_size.restype = sz
    L.scsf_cholqr2_scratch.argtypes = [i32, i32]
    L.scsf_cholqr2_scratch.restype = sz
    L.scsf_cholqr2.argtypes = [vp, vp, i32, i32, i32, vp, i32, ctypes.POINTER(i32), vp, sz]
    L.scsf_cholqr2.restype = ctypes.c_int
    L.scsf_solve_workspace_size_rows.argtypes = [ctypes.POINTER(_CParams), i64]
    L.scsf_solve_workspace_size_rows.restype = sz
    L.scsf_chain_create_rows.argtypes = [vp, ctypes.POINTER(_CParams), i64, vp, sz,
                                         ctypes.POINTER(vp)]
    L.scsf_chain_create.argtypes = [vp, ctypes.POINTER(_CParams), i32, vp, sz, ctypes.POINTER(vp)]
    L.scsf_chain_seed.argtypes = [vp, vp, ctypes.POINTER(dbl)]
    L.scsf_chain_step.argtypes = [vp, ctypes.POINTER(_COperator), vp, vp, vp, ctypes.POINTER(_CStats)]
    L.scsf_chain_destroy.argtypes = [vp]
    L.scsf_chain_destroy.restype = None
    L.scsf_solve.argtypes = [vp, ctypes.POINTER(_COperator), i64, ctypes.POINTER(_CParams), vp, sz,
                             vp, vp, vp, ctypes.POINTER(_CStats)]
    L.scsf_cheb_filter.argtypes = [vp, ctypes.POINTER(_COperator), vp, i32, i32, i32, dbl, dbl, dbl,
                                   vp, i32, vp, sz]
    L.scsf_assemble_bounds.argtypes = [vp, ctypes.POINTER(_COperator), ctypes.POINTER(dbl), vp, sz]
    L.scsf_small_eigh_scratch.argtypes = [i32]
    L.scsf_small_eigh_scratch.restype = sz
    L.scsf_small_eigh.argtypes = [vp, vp, i32, vp, vp, vp, sz]
    L.scsf_set_timing.argtypes = [vp, i32]
    L.scsf_set_timing.restype = ctypes.c_int
    L.scsf_launch_count.argtypes = []
    L.scsf_launch_count.restype = ctypes.c_longlong
    L.scsf_batch_workspace_size.argtypes = [ctypes.POINTER(_CBatchChain), i32, i32]
    L.scsf_batch_workspace_size.restype = sz
    L.scsf_solve_batched.argtypes = [vp, ctypes.POINTER(_CBatchChain), i32, i32, vp, sz]
    L.scsf_solve_batched.restype = ctypes.c_int
    L.scsf_cheb_filter_f32.argtypes = [vp, ctypes.POINTER(_COperator), vp, i32, i32, i32, dbl, dbl,
                                       dbl, vp, i32, vp, sz]
    L.scsf_cheb_filter_f32.restype = ctypes.c_int
    L.scsf_proposal_param_count.restype = sz
    L.scsf_proposal_workspace_size.argtypes = [i32]
    L.scsf_proposal_workspace_size.restype = sz
    L.scsf_proposal_init.argtypes = [vp, vp, ctypes.c_uint64]
    L.scsf_proposal_init.restype = ctypes.c_int
    L.scsf_proposal_forward.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, sz]
    L.scsf_proposal_forward.restype = ctypes.c_int
    L.scsf_proposal_train_step.argtypes = [vp, vp, vp, vp, i32, ctypes.c_float, vp, i32, i32, vp, vp,
                                           ctypes.POINTER(dbl), vp, vp, sz]
    L.scsf_proposal_train_step.restype = ctypes.c_int
    L.scsf_proposal_target_scratch.restype = sz
    L.scsf_proposal_targets.argtypes = [vp, vp, i32, i32, i32, vp, vp, sz]
    L.scsf_proposal_targets.restype = ctypes.c_int
    L.scsf_proposal_prolong.argtypes = [vp, vp, i32, i32, vp, i32]
    L.scsf_proposal_prolong.restype = ctypes.c_int
    L.scsf_cheb_filter_dc_scratch.argtypes = [i32, i32, i32]
    L.scsf_cheb_filter_dc_scratch.restype = sz
    L.scsf_cheb_filter_dc.argtypes = [vp, ctypes.POINTER(_COperator), vp, i32, vp, i32, i32, dbl,
                                      dbl, dbl, vp, i32, vp, sz]
    L.scsf_cheb_filter_dc.restype = ctypes.c_int
    L.scsf_cheb_filter_dc_grouped.argtypes = [vp, ctypes.POINTER(_COperator), vp, i32, vp, i32, i32,
                                              ctypes.POINTER(ctypes.c_int), dbl, dbl, dbl, vp, i32,
                                              vp, sz]
    L.scsf_cheb_filter_dc_grouped.restype = ctypes.c_int
    L.scsf_sort_noalloc_capacity.argtypes = []
    L.scsf_sort_noalloc_capacity.restype = sz
    L.scsf_sort_noalloc.argtypes = [vp, vp, i64, i32, i32, i32, vp]
    L.scsf_sort_noalloc.restype = ctypes.c_int
    L.scsf_block_product_scratch.argtypes = [i64, i32, i32]
    L.scsf_block_product_scratch.restype = sz
    L.scsf_block_gram.argtypes = [vp, vp, i32, vp, i32, i32, i32, i32, i32, i32, i32, vp, i32, vp, sz]
    L.scsf_block_gram.restype = ctypes.c_int
    L.scsf_block_rotate_ex.argtypes = [vp, vp, i32, i32, i32, vp, i32, i32, dbl, dbl, i32, i32, vp,
                                       i32, vp, sz]
    L.scsf_block_rotate_ex.restype = ctypes.c_int
    L.scsf_block_gram_kernel_time.argtypes = [vp, vp, i32, i32, i32, i32, vp, sz,
                                              ctypes.POINTER(ctypes.c_float)]
    L.scsf_block_gram_kernel_time.restype = ctypes.c_int
    L.scsf_chain_restart.argtypes = [vp]
    L.scsf_chain_restart.restype = ctypes.c_int
    L.scsf_far_steps.argtypes = [ctypes.POINTER(dbl), i64, dbl, ctypes.POINTER(i32)]
    L.scsf_far_steps.restype = ctypes.c_int
    for name in EXPORTED_SYMBOLS:
        fn = getattr(L, name)
        if fn.restype is ctypes.c_int or name in (
                "scsf_create", "scsf_sort", "scsf_chain_create", "scsf_chain_seed", "scsf_chain_step",
                "scsf_solve", "scsf_cheb_filter", "scsf_assemble_bounds", "scsf_small_eigh"):
            fn.restype = ctypes.c_int
    L.scsf_version.restype = ctypes.c_int
    _lib = L
    return L


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _check(t: torch.Tensor, name: str, dtype=torch.float64, device=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name} must live on a CUDA device (the library has no CPU path)")
    if device is not None and t.device != device:
        raise ValueError(f"{name} is on {t.device}, expected {device}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def block_width(k: int, nex: int = -1) -> int:
    """k_b = k + nex, nex = ceil(0.2 k) by default (App. D.4)."""
    return k + (nex if nex >= 0 else int(math.ceil(0.2 * k)))


@dataclass
class Operator:
    """One discretised operator on the n x n interior grid (device FP64 tensors), or a
    general symmetric matrix in CSR form (kind CSR; n = 0, N = rows). Kind PLATE is the
    thin-plate problem div(grad(D lap u)) = lambda rho u (D, rho [n, n] at the nodes)."""
    kind: int
    n: int
    ax: Optional[torch.Tensor] = None   # [n+1, n]
    ay: Optional[torch.Tensor] = None   # [n, n+1]
    v: Optional[torch.Tensor] = None    # [n, n]
    rows: int = 0
    row_ptr: Optional[torch.Tensor] = None  # [rows + 1] int32
    col: Optional[torch.Tensor] = None      # [nnz] int32
    val: Optional[torch.Tensor] = None      # [nnz] FP64
    D: Optional[torch.Tensor] = None        # [n, n] (PLATE)
    rho: Optional[torch.Tensor] = None      # [n, n] (PLATE)
    field: Optional[torch.Tensor] = None    # [n, n] parameter field (learned-proposal heads)

    @staticmethod
    def csr(row_ptr, col, val, device="cuda") -> "Operator":
        """A symmetric matrix from CSR arrays (host or device; copied to the device)."""
        rp = torch.as_tensor(row_ptr, dtype=torch.int32, device=device).contiguous()
        return Operator(CSR, 0, rows=int(rp.numel()) - 1, row_ptr=rp,
                        col=torch.as_tensor(col, dtype=torch.int32, device=device).contiguous(),
                        val=torch.as_tensor(val, dtype=torch.float64, device=device).contiguous())

    @property
    def N(self) -> int:
        return self.rows if self.kind == CSR else self.n * self.n

    @staticmethod
    def from_workload(op, device="cuda") -> "Operator":
        """Uploads an ``scsf_inputs`` operator (numpy) to the device."""
        if hasattr(op, "row_ptr"):
            return Operator.csr(op.row_ptr, op.col, op.val, device)
        if hasattr(op, "rho"):
            return Operator(PLATE, op.n,
                            D=torch.as_tensor(op.D, dtype=torch.float64, device=device).contiguous(),
                            rho=torch.as_tensor(op.rho, dtype=torch.float64, device=device).contiguous())
        if hasattr(op, "ax"):
            return Operator(DIV_A_GRAD, op.n,
                            ax=torch.as_tensor(op.ax, dtype=torch.float64, device=device).contiguous(),
                            ay=torch.as_tensor(op.ay, dtype=torch.float64, device=device).contiguous(),
                            field=torch.as_tensor(op.P, dtype=torch.float64, device=device).contiguous())
        v = torch.as_tensor(op.V, dtype=torch.float64, device=device).contiguous()
        return Operator(LAP_PLUS_V, op.n, v=v, field=v)

    def _c(self) -> _COperator:
        if self.kind == DIV_A_GRAD:
            _check(self.ax, "ax")
            _check(self.ay, "ay", device=self.ax.device)
            if tuple(self.ax.shape) != (self.n + 1, self.n) or tuple(self.ay.shape) != (self.n, self.n + 1):
                raise ValueError("ax must be [n+1, n] and ay [n, n+1]")
        elif self.kind == LAP_PLUS_V:
            _check(self.v, "v")
            if tuple(self.v.shape) != (self.n, self.n):
                raise ValueError("v must be [n, n]")
        elif self.kind == PLATE:
            _check(self.D, "D")
            _check(self.rho, "rho", device=self.D.device)
            if tuple(self.D.shape) != (self.n, self.n) or tuple(self.rho.shape) != (self.n, self.n):
                raise ValueError("D and rho must be [n, n]")
        elif self.kind == CSR:
            _check(self.val, "val")
            _check(self.row_ptr, "row_ptr", dtype=torch.int32, device=self.val.device)
            _check(self.col, "col", dtype=torch.int32, device=self.val.device)
            if self.row_ptr.numel() != self.rows + 1 or self.col.numel() != self.val.numel():
                raise ValueError("row_ptr must have rows + 1 entries and col / val nnz each")
        else:
            raise ValueError(f"unknown operator kind {self.kind}")
        if self.field is not None:
            _check(self.field, "field")
            if tuple(self.field.shape) != (self.n, self.n):
                raise ValueError("field must be [n, n]")
        return _COperator(self.kind, self.n, _ptr(self.ax), _ptr(self.ay), _ptr(self.v),
                          self.rows, _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val),
                          _ptr(self.D), _ptr(self.rho), _ptr(self.field))

    @property
    def device(self):
        return {DIV_A_GRAD: self.ax, LAP_PLUS_V: self.v, CSR: self.val, PLATE: self.D}[self.kind].device


@dataclass
class Params:
    k: int
    degree: int = 20
    tol: float = 1e-8
    max_iter: int = 100
    nex: int = -1
    precision: int = FP64
    seed: int = 0
    degree_fp32: int = 0   # MIXED: degree of the FP32 phase (0: same as degree)
    switch_tol: float = 0.0  # MIXED: leave the FP32 phase at this wanted residual (0: off)
    products: int = PRODUCT_TENSOR  # block products on the tensor cores (or PRODUCT_FP64)
    proposal: Optional["Proposal"] = None  # chain heads start from this learned proposal
    bound: int = BOUND_GERSHGORIN  # upper end of the filter interval (or BOUND_LANCZOS)
    column_degree: bool = False  # MIXED: per-column-group degrees in the FP64 phase

    def _c(self) -> _CParams:
        use = self.proposal is not None
        return _CParams(self.k, self.nex, self.degree, self.tol, self.max_iter, self.precision,
                        self.seed & 0xFFFFFFFFFFFFFFFF, self.degree_fp32, self.switch_tol,
                        self.products, 1 if use else 0,
                        self.proposal.params.data_ptr() if use else None, self.bound,
                        1 if self.column_degree else 0)

    @property
    def kb(self) -> int:
        return block_width(self.k, self.nex)


class Context:
    """An scsf_ctx bound to one device and a CUDA stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        L = library()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the SCSF library has no CPU path")
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        st = L.scsf_create(ctypes.byref(h), device, ctypes.c_void_p(self.stream.cuda_stream))
        if st != OK:
            raise ScsfError(st, "scsf_create failed")
        self._h = h

    @property
    def handle(self):
        return self._h

    def set_timing(self, enable: bool = True):
        """Per-phase CUDA-event timing in the returned stats (adds event records, no syncs)."""
        self.check(library().scsf_set_timing(self._h, 1 if enable else 0))

    def check(self, status: int):
        if status != OK:
            msg = library().scsf_last_error(self._h).decode(errors="replace")
            raise ScsfError(status, msg)

    def close(self):
        if getattr(self, "_h", None):
            library().scsf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx: dict = {}


def _ctx(ctx: Optional[Context], device) -> Context:
    if ctx is not None:
        return ctx
    idx = torch.device(device).index or 0
    stream = torch.cuda.current_stream(idx)
    key = (idx, stream.cuda_stream)
    if key not in _default_ctx:
        _default_ctx[key] = Context(idx, stream)
    return _default_ctx[key]


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def sort(fields: torch.Tensor, p0: int, start: int = 0, ctx: Optional[Context] = None,
         return_distances: bool = False):
    """Alg. 2: visiting order of the problems (int32 [n_ops]) from fields [n_ops, p, p] FP64;
    with return_distances also the squared feature distance of each step (FP64 [n_ops])."""
    _check(fields, "fields")
    if fields.dim() != 3 or fields.shape[1] != fields.shape[2]:
        raise ValueError("fields must be [n_ops, p, p]")
    c = _ctx(ctx, fields.device)
    L = library()
    n_ops, p = int(fields.shape[0]), int(fields.shape[1])
    ws = _workspace(L.scsf_sort_workspace_size(n_ops, p0), fields.device)
    perm = torch.empty(n_ops, dtype=torch.int32, device=fields.device)
    if not return_distances:
        c.check(L.scsf_sort(c.handle, fields.data_ptr(), n_ops, p, p0, start, ws.data_ptr(),
                            ws.numel(), perm.data_ptr()))
        return perm
    dist = torch.empty(n_ops, dtype=torch.float64, device=fields.device)
    c.check(L.scsf_sort_dist(c.handle, fields.data_ptr(), n_ops, p, p0, start, ws.data_ptr(),
                             ws.numel(), perm.data_ptr(), dist.data_ptr()))
    return perm, dist


def sort_noalloc(fields: torch.Tensor, p0: int, start: int = 0,
                 ctx: Optional[Context] = None) -> torch.Tensor:
    """Alg. 2 through the allocation-free entry point: same result as sort(), with the
    library's static device scratch instead of a workspace (only perm_out is allocated,
    here by torch, because Python callers need a tensor to hold it)."""
    _check(fields, "fields")
    if fields.dim() != 3 or fields.shape[1] != fields.shape[2]:
        raise ValueError("fields must be [n_ops, p, p]")
    c = _ctx(ctx, fields.device)
    n_ops, p = int(fields.shape[0]), int(fields.shape[1])
    perm = torch.empty(n_ops, dtype=torch.int32, device=fields.device)
    c.check(library().scsf_sort_noalloc(c.handle, fields.data_ptr(), n_ops, p, p0, start,
                                        perm.data_ptr()))
    return perm


def _stats_dict(s: _CStats) -> dict:
    out = {name: getattr(s, name) for name, _ in _CStats._fields_ if name != "history"}
    out["converged"] = bool(s.converged)
    return out


def launch_count() -> int:
    """Kernels launched by libscsf.so in this process so far."""
    return int(library().scsf_launch_count())


class Chain:
    """A warm-started sequence of solves on one grid size (Alg. 3 along a sorted chain)."""

    def __init__(self, params: Params, n: int, device="cuda", ctx: Optional[Context] = None,
                 rows: Optional[int] = None):
        """A chain of n x n stencil operators, or (n = 0, rows given) of CSR operators."""
        self.ctx = _ctx(ctx, device)
        self.params = params
        self.n = n
        self.N = rows if rows is not None else n * n
        L = library()
        cp = params._c()
        if rows is not None:
            nbytes = L.scsf_solve_workspace_size_rows(ctypes.byref(cp), rows)
        else:
            nbytes = L.scsf_solve_workspace_size(ctypes.byref(cp), n)
        if nbytes == 0:
            raise ValueError("unsupported parameters (block width, size or precision)")
        self.workspace = _workspace(nbytes, self.ctx.device)
        h = ctypes.c_void_p()
        ws = (self.workspace.data_ptr(), self.workspace.numel(), ctypes.byref(h))
        if rows is not None:
            self.ctx.check(L.scsf_chain_create_rows(self.ctx.handle, ctypes.byref(cp), rows, *ws))
        else:
            self.ctx.check(L.scsf_chain_create(self.ctx.handle, ctypes.byref(cp), n, *ws))
        self._h = h

    def seed(self, block: torch.Tensor, ritz: Sequence[float]):
        _check(block, "block", device=self.ctx.device)
        kb = self.params.kb
        if tuple(block.shape) != (self.N, kb) or len(ritz) != kb:
            raise ValueError("block must be [N, k_b] with k_b Ritz values")
        arr = (ctypes.c_double * kb)(*[float(x) for x in ritz])
        self.ctx.check(library().scsf_chain_seed(self._h, block.data_ptr(), arr))

    def restart(self):
        """The next step starts as a chain head (the learned proposal when the params have one)."""
        self.ctx.check(library().scsf_chain_restart(self._h))

    def step(self, op: Operator, want_vectors: bool = True, raise_on_nonconvergence: bool = True,
             history: bool = False):
        """Solves the next problem. With history=True, stats["history"] lists per outer
        iteration (max residual, median residual of the wanted unlocked pairs, locked)."""
        k, N = self.params.k, self.N
        dev = self.ctx.device
        evals = torch.empty(k, dtype=torch.float64, device=dev)
        resid = torch.empty(k, dtype=torch.float64, device=dev)
        evecs = torch.empty((N, k), dtype=torch.float64, device=dev) if want_vectors else None
        stats = _CStats()
        hist = None
        if history:
            hist = (ctypes.c_double * (3 * self.params.max_iter))()
            stats.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
        cop = op._c()
        st = library().scsf_chain_step(self._h, ctypes.byref(cop), evals.data_ptr(), resid.data_ptr(),
                                       _ptr(evecs), ctypes.byref(stats))
        if st != OK and not (st == ERR_NOT_CONVERGED and not raise_on_nonconvergence):
            self.ctx.check(st)
        out = _stats_dict(stats)
        if hist is not None:
            out["history"] = [tuple(hist[3 * i: 3 * i + 3]) for i in range(stats.iters)]
        return evals, resid, evecs, out

    def close(self):
        if getattr(self, "_h", None):
            library().scsf_chain_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def far_steps(dist, quantile: float = 0.9) -> List[bool]:
    """scsf_far_steps: the head and every step whose squared feature distance to its sorted
    predecessor is above the given quantile of the chain's step distances."""
    d = [float(x) for x in (dist.tolist() if hasattr(dist, "tolist") else dist)]
    n = len(d)
    arr = (ctypes.c_double * n)(*d)
    out = (ctypes.c_int32 * n)()
    st = library().scsf_far_steps(arr, n, float(quantile), out)
    if st != OK:
        raise ScsfError(st, "scsf_far_steps: bad arguments")
    return [bool(x) for x in out]


def _product_scratch(rows: int, kmax: int, slices: int, device) -> torch.Tensor:
    nbytes = library().scsf_block_product_scratch(rows, kmax, slices)
    if nbytes == 0:
        raise ValueError("unsupported product sizes")
    return _workspace(nbytes, device)


def block_gram(A: torch.Tensor, B: Optional[torch.Tensor] = None, symmetric: bool = False,
               method: int = PRODUCT_TENSOR, slices: int = 8,
               ctx: Optional[Context] = None) -> torch.Tensor:
    """C = A^T B (FP64 [rows, m] and [rows, n] device tensors; B = A when omitted) by
    scsf_block_gram: on the tensor cores (digit split, `slices` digits) or the FP64 pipe."""
    B = A if B is None else B
    _check(A, "A")
    _check(B, "B", device=A.device)
    if A.dim() != 2 or B.dim() != 2 or A.shape[0] != B.shape[0]:
        raise ValueError("A and B must be [rows, m] and [rows, n]")
    c = _ctx(ctx, A.device)
    rows, m, n = int(A.shape[0]), int(A.shape[1]), int(B.shape[1])
    C = torch.empty((m, n), dtype=torch.float64, device=A.device)
    ws = _product_scratch(rows, max(m, n), slices, A.device)
    c.check(library().scsf_block_gram(c.handle, A.data_ptr(), m, B.data_ptr(), n, rows, m, n,
                                      1 if symmetric else 0, method, slices, C.data_ptr(), n,
                                      ws.data_ptr(), ws.numel()))
    return C


def block_gram_kernel_time(X: torch.Tensor, reps: int = 20, ctx: Optional[Context] = None) -> float:
    """Average device time (ms) of the tensor-core Gram kernel (8 digits) for X^T X alone."""
    _check(X, "X")
    c = _ctx(ctx, X.device)
    rows, m = int(X.shape[0]), int(X.shape[1])
    ws = _product_scratch(rows, m, 8, X.device)
    out = ctypes.c_float()
    c.check(library().scsf_block_gram_kernel_time(c.handle, X.data_ptr(), m, rows, m, reps,
                                                  ws.data_ptr(), ws.numel(), ctypes.byref(out)))
    return float(out.value)


def block_rotate(X: torch.Tensor, M: torch.Tensor, Y: Optional[torch.Tensor] = None,
                 alpha: float = 1.0, beta: float = 0.0, method: int = PRODUCT_TENSOR,
                 slices: int = 8, ctx: Optional[Context] = None) -> torch.Tensor:
    """Y = alpha X M + beta Y (FP64 [rows, k], [k, n], [rows, n]) by scsf_block_rotate_ex."""
    _check(X, "X")
    _check(M, "M", device=X.device)
    if X.dim() != 2 or M.dim() != 2 or X.shape[1] != M.shape[0]:
        raise ValueError("X must be [rows, k] and M [k, n]")
    rows, k, n = int(X.shape[0]), int(X.shape[1]), int(M.shape[1])
    if Y is None:
        if beta != 0.0:
            raise ValueError("beta != 0 needs Y")
        Y = torch.empty((rows, n), dtype=torch.float64, device=X.device)
    _check(Y, "Y", device=X.device)
    if tuple(Y.shape) != (rows, n):
        raise ValueError("Y must be [rows, n]")
    c = _ctx(ctx, X.device)
    ws = _product_scratch(rows, max(k, n), slices, X.device)
    c.check(library().scsf_block_rotate_ex(c.handle, X.data_ptr(), k, rows, k, M.data_ptr(), n, n,
                                           alpha, beta, method, slices, Y.data_ptr(), n,
                                           ws.data_ptr(), ws.numel()))
    return Y


def solve(ops: List[Operator], params: Params, want_vectors: bool = False,
          ctx: Optional[Context] = None):
    """scsf_solve over ops (already in solve order). Returns (evals, resid, evecs|None, stats)."""
    if not ops:
        raise ValueError("no operators")
    c = _ctx(ctx, ops[0].device)
    L = library()
    cp = params._c()
    if ops[0].kind == CSR:
        nbytes = L.scsf_solve_workspace_size_rows(ctypes.byref(cp), ops[0].rows)
    else:
        nbytes = L.scsf_solve_workspace_size(ctypes.byref(cp), ops[0].n)
    if nbytes == 0:
        raise ValueError("unsupported parameters (block width, size or precision)")
    ws = _workspace(nbytes, c.device)
    n_ops, k, N = len(ops), params.k, ops[0].N
    evals = torch.empty((n_ops, k), dtype=torch.float64, device=c.device)
    resid = torch.empty((n_ops, k), dtype=torch.float64, device=c.device)
    evecs = torch.empty((n_ops, N, k), dtype=torch.float64, device=c.device) if want_vectors else None
    cops = (_COperator * n_ops)(*[o._c() for o in ops])
    stats = (_CStats * n_ops)()
    c.check(L.scsf_solve(c.handle, cops, n_ops, ctypes.byref(cp), ws.data_ptr(), ws.numel(),
                         evals.data_ptr(), resid.data_ptr(), _ptr(evecs), stats))
    return evals, resid, evecs, [_stats_dict(s) for s in stats]


def solve_batched(chains, concurrency: int = 8, want_vectors: bool = False,
                  ctx: Optional[Context] = None, raise_on_error: bool = True):
    """scsf_solve_batched over chains = [(ops, Params), ...] (each ops list in solve order).

    Returns a list of (evals, resid, evecs|None, stats, status) per chain."""
    if not chains:
        raise ValueError("no chains")
    dev = chains[0][0][0].device
    c = _ctx(ctx, dev)
    keep, cchains, outs = [], [], []
    for ops, params in chains:
        if not ops:
            raise ValueError("empty chain")
        n_ops, k, N = len(ops), params.k, ops[0].N
        evals = torch.empty((n_ops, k), dtype=torch.float64, device=c.device)
        resid = torch.empty((n_ops, k), dtype=torch.float64, device=c.device)
        evecs = torch.empty((n_ops, N, k), dtype=torch.float64, device=c.device) if want_vectors else None
        cops = (_COperator * n_ops)(*[o._c() for o in ops])
        stats = (_CStats * n_ops)()
        keep.append((cops, stats))
        cchains.append(_CBatchChain(ctypes.cast(cops, ctypes.POINTER(_COperator)), n_ops, params._c(),
                                    evals.data_ptr(), resid.data_ptr(), _ptr(evecs),
                                    ctypes.cast(stats, ctypes.POINTER(_CStats)), 0))
        outs.append((evals, resid, evecs, stats))
    arr = (_CBatchChain * len(cchains))(*cchains)
    L = library()
    nbytes = L.scsf_batch_workspace_size(arr, len(cchains), concurrency)
    if nbytes == 0:
        raise ValueError("unsupported chain parameters")
    ws = _workspace(nbytes, c.device)
    st = L.scsf_solve_batched(c.handle, arr, len(cchains), concurrency, ws.data_ptr(), ws.numel())
    if st != OK and raise_on_error:
        c.check(st)
    return [(e, r, v, [_stats_dict(s) for s in stt], int(arr[i].status))
            for i, (e, r, v, stt) in enumerate(outs)]


def _plate_scratch(op: Operator) -> int:
    """Extra building-block scratch for the thin-plate operator's 13-slot CSR form."""
    return 4 * (14 * op.N + 1) + 104 * op.N + 1024 if op.kind == PLATE else 0


def cheb_filter(op: Operator, X: torch.Tensor, degree: int, lam: float, c: float, e: float,
                ctx: Optional[Context] = None) -> torch.Tensor:
    """Alg. 1: C_m(Abar) X / C_m(t_lambda) for X [N, ncols] FP64."""
    _check(X, "X")
    cx = _ctx(ctx, X.device)
    N, ncols = int(X.shape[0]), int(X.shape[1])
    if N != op.N:
        raise ValueError("X must have N rows")
    Y = torch.empty_like(X)
    ws = _workspace(8 * (2 * N * ncols + 3 * N + 2 * 2048) + 8192 + _plate_scratch(op), X.device)
    cop = op._c()
    cx.check(library().scsf_cheb_filter(cx.handle, ctypes.byref(cop), X.data_ptr(), ncols, ncols,
                                        degree, lam, c, e, Y.data_ptr(), ncols, ws.data_ptr(),
                                        ws.numel()))
    return Y


def cheb_filter_f32(op: Operator, X: torch.Tensor, degree: int, lam: float, c: float, e: float,
                    ctx: Optional[Context] = None) -> torch.Tensor:
    """Alg. 1 on an FP32 block (the mixed form's filter); ncols must be a multiple of 4."""
    _check(X, "X", dtype=torch.float32)
    cx = _ctx(ctx, X.device)
    N, ncols = int(X.shape[0]), int(X.shape[1])
    if N != op.N:
        raise ValueError("X must have N rows")
    Y = torch.empty_like(X)
    ws = _workspace(4 * 2 * N * ncols + 8 * 6 * N + (64 << 10), X.device)
    cop = op._c()
    cx.check(library().scsf_cheb_filter_f32(cx.handle, ctypes.byref(cop), X.data_ptr(), ncols,
                                            ncols, degree, lam, c, e, Y.data_ptr(), ncols,
                                            ws.data_ptr(), ws.numel()))
    return Y


def cheb_filter_dc(op: Operator, X: torch.Tensor, theta: torch.Tensor, degree: int, lam: float,
                   c: float, e: float, ctx: Optional[Context] = None,
                   group_degrees: Optional[Sequence[int]] = None) -> torch.Tensor:
    """Alg. 1 on an FP64 block through the defect-corrected form (FP32 remainder
    recurrence driven by the residual block of (X, theta)). With group_degrees (one int in
    [1, degree] per group of 4 columns), columns [4g, 4g+4) are filtered to degree
    group_degrees[g] (scsf_cheb_filter_dc_grouped)."""
    _check(X, "X")
    _check(theta, "theta")
    cx = _ctx(ctx, X.device)
    N, ncols = int(X.shape[0]), int(X.shape[1])
    if N != op.n * op.n or int(theta.numel()) != ncols:
        raise ValueError("X must have n*n rows and theta one entry per column")
    Y = torch.empty_like(X)
    L = library()
    nbytes = L.scsf_cheb_filter_dc_scratch(op.n, ncols, degree)
    if nbytes == 0:
        raise ValueError("unsupported filter shape")
    ws = _workspace(nbytes, X.device)
    cop = op._c()
    if group_degrees is None:
        cx.check(L.scsf_cheb_filter_dc(cx.handle, ctypes.byref(cop), X.data_ptr(), ncols,
                                       theta.data_ptr(), ncols, degree, lam, c, e, Y.data_ptr(),
                                       ncols, ws.data_ptr(), ws.numel()))
        return Y
    g = list(int(x) for x in group_degrees)
    if len(g) != (ncols + 3) // 4:
        raise ValueError("group_degrees needs one entry per group of 4 columns")
    garr = (ctypes.c_int * len(g))(*g)
    cx.check(L.scsf_cheb_filter_dc_grouped(cx.handle, ctypes.byref(cop), X.data_ptr(), ncols,
                                           theta.data_ptr(), ncols, degree, garr, lam, c, e,
                                           Y.data_ptr(), ncols, ws.data_ptr(), ws.numel()))
    return Y


def block_rotate_fp64(X: torch.Tensor, M: torch.Tensor, ctx: Optional[Context] = None) -> torch.Tensor:
    """Y = X M on the FP64 pipe (scsf_block_rotate): the rotation of Alg. 3 as a building block."""
    _check(X, "X")
    _check(M, "M")
    if X.dim() != 2 or M.dim() != 2 or X.shape[1] != M.shape[0]:
        raise ValueError("need X [rows, k] and M [k, n]")
    cx = _ctx(ctx, X.device)
    rows, k, n = int(X.shape[0]), int(X.shape[1]), int(M.shape[1])
    Y = torch.empty((rows, n), dtype=torch.float64, device=X.device)
    cx.check(library().scsf_block_rotate(cx.handle, X.data_ptr(), k, rows, k, M.data_ptr(), n, n,
                                         Y.data_ptr(), n))
    return Y


def assemble_bounds(op: Operator, ctx: Optional[Context] = None):
    """Gershgorin bounds (lo, hi) of the assembled operator."""
    cx = _ctx(ctx, op.device)
    N = op.N
    ws = _workspace(8 * (3 * N + 2 * 2048) + 8192 + _plate_scratch(op), op.device)
    out = (ctypes.c_double * 2)()
    cop = op._c()
    cx.check(library().scsf_assemble_bounds(cx.handle, ctypes.byref(cop), out, ws.data_ptr(),
                                            ws.numel()))
    return float(out[0]), float(out[1])


def cholqr2(X: torch.Tensor, ctx: Optional[Context] = None):
    """Cholesky QR2 of X [rows, ncols] FP64 (FP32 first factor, FP64 second). Returns
    (Q, (shifted restarts of pass 1, of pass 2))."""
    _check(X, "X")
    if X.dim() != 2:
        raise ValueError("X must be [rows, ncols]")
    rows, ncols = int(X.shape[0]), int(X.shape[1])
    cx = _ctx(ctx, X.device)
    L = library()
    nbytes = L.scsf_cholqr2_scratch(rows, ncols)
    if nbytes == 0:
        raise ValueError("need 1 <= ncols <= min(rows, 512)")
    ws = _workspace(nbytes, X.device)
    Q = torch.empty_like(X)
    shifts = (ctypes.c_int * 2)()
    cx.check(L.scsf_cholqr2(cx.handle, X.data_ptr(), ncols, rows, ncols, Q.data_ptr(), ncols,
                            shifts, ws.data_ptr(), ws.numel()))
    return Q, (int(shifts[0]), int(shifts[1]))


def small_eigh(S: torch.Tensor, ctx: Optional[Context] = None):
    """All eigenpairs of a small symmetric FP64 matrix (ascending), via the reduced eigensolver."""
    _check(S, "S")
    k = int(S.shape[0])
    cx = _ctx(ctx, S.device)
    L = library()
    ws = _workspace(L.scsf_small_eigh_scratch(k), S.device)
    evals = torch.empty(k, dtype=torch.float64, device=S.device)
    Z = torch.empty((k, k), dtype=torch.float64, device=S.device)
    cx.check(L.scsf_small_eigh(cx.handle, S.data_ptr(), k, evals.data_ptr(), Z.data_ptr(),
                               ws.data_ptr(), ws.numel()))
    return evals, Z


class Proposal:
    """The learned head proposal (a Fourier neural operator; all compute in libscsf).

    forward(fields) -> (bounds [B, 2] log(lambda_1), log(lambda_64); block [B, 1024, 64])
    train_step(fields, t_bounds, t_Q, lr) -> (subspace, orthonormality, bounds) loss terms
    Params(..., proposal=this) makes every chain head start from the proposal; the library
    composes the head block (scsf_params.use_proposal).
    """

    COARSE, KY = 32, 64

    def __init__(self, seed: int = 0, device="cuda", ctx: Optional[Context] = None):
        self.ctx = _ctx(ctx, device)
        L = library()
        self.count = int(L.scsf_proposal_param_count())
        dev = self.ctx.device
        self.params = torch.empty(self.count, dtype=torch.float32, device=dev)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.steps = 0
        self._ws = {}
        self.ctx.check(L.scsf_proposal_init(self.ctx.handle, self.params.data_ptr(), seed))

    def _workspace(self, batch: int) -> torch.Tensor:
        if batch not in self._ws:
            self._ws[batch] = _workspace(library().scsf_proposal_workspace_size(batch), self.ctx.device)
        return self._ws[batch]

    def forward(self, fields: torch.Tensor):
        _check(fields, "fields")
        B, s = int(fields.shape[0]), int(fields.shape[1])
        dev = self.ctx.device
        bounds = torch.empty((B, 2), dtype=torch.float32, device=dev)
        block = torch.empty((B, self.COARSE * self.COARSE, self.KY), dtype=torch.float32, device=dev)
        ws = self._workspace(B)
        self.ctx.check(library().scsf_proposal_forward(self.ctx.handle, self.params.data_ptr(),
                                                       fields.data_ptr(), B, s, bounds.data_ptr(),
                                                       block.data_ptr(), ws.data_ptr(), ws.numel()))
        return bounds, block

    def _train(self, fields, t_bounds, t_Q, lr, update: bool, want_grad: bool):
        _check(fields, "fields")
        _check(t_bounds, "t_bounds", dtype=torch.float32)
        _check(t_Q, "t_Q", dtype=torch.float32)
        B, s = int(fields.shape[0]), int(fields.shape[1])
        ws = self._workspace(B)
        loss = (ctypes.c_double * 3)()
        grad = torch.empty_like(self.params) if want_grad else None
        if update:
            self.steps += 1
        self.ctx.check(library().scsf_proposal_train_step(
            self.ctx.handle, self.params.data_ptr(), self.m.data_ptr() if update else None,
            self.v.data_ptr() if update else None, self.steps if update else 0, float(lr),
            fields.data_ptr(), B, s, t_bounds.data_ptr(), t_Q.data_ptr(), loss, _ptr(grad),
            ws.data_ptr(), ws.numel()))
        return (loss[0], loss[1], loss[2]), grad

    def train_step(self, fields, t_bounds, t_Q, lr: float = 1e-3):
        return self._train(fields, t_bounds, t_Q, lr, True, False)[0]

    def gradient(self, fields, t_bounds, t_Q):
        """Loss terms and the gradient w.r.t. the parameters (no update)."""
        return self._train(fields, t_bounds, t_Q, 0.0, False, True)

    def targets(self, evecs: torch.Tensor, n: int) -> torch.Tensor:
        """Coarse orthonormal targets from fine eigenvectors [B, n*n, >= 64] (FP64)."""
        _check(evecs, "evecs")
        B, lde = int(evecs.shape[0]), int(evecs.shape[2])
        Q = torch.empty((B, self.COARSE * self.COARSE, self.KY), dtype=torch.float32, device=evecs.device)
        L = library()
        scratch = _workspace(L.scsf_proposal_target_scratch(), evecs.device)
        self.ctx.check(L.scsf_proposal_targets(self.ctx.handle, evecs.data_ptr(), B, n, lde,
                                               Q.data_ptr(), scratch.data_ptr(), scratch.numel()))
        return Q
