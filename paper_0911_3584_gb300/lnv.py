"""ctypes binding of liblnv (include/lnv.h): argument marshalling only.

Every step of the computation runs in the CUDA library; this module checks
tensors (device, dtype, size, contiguity), passes raw pointers and raises
LnvError on a non-zero status.  PyTorch supplies device memory and the stream.
The library must have been built (``paper_0911_3584_gb300.build.build()``);
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from . import build as _build

_lib = None
_lock = threading.Lock()

FP64, FP32 = 0, 1
PREC = {"fp64": FP64, "fp32": FP32, FP64: FP64, FP32: FP32}
DTYPE = {FP64: torch.float64, FP32: torch.float32}
TRANS_A, TRANS_B, SYM_C = 1, 2, 4


class LnvError(RuntimeError):
    def __init__(self, what: str, status: int, msg: str):
        super().__init__(f"{what} failed with status {status}: {msg}")
        self.status = status


def lib():
    """Load liblnv.so; fail loudly if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(
                    f"liblnv is not built ({path} missing); run __graft_entry__.build() "
                    "or python -m paper_0911_3584_gb300.build")
            L = ctypes.CDLL(path)
            P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            PP = ctypes.POINTER(ctypes.c_void_p)
            sig = {
                "lnv_ctx_create": [i32, P, PP],
                "lnv_ctx_set_stream": [P, P],
                "lnv_ctx_destroy": [P],
                "lnv_ctx_device_status": [P],
                "lnv_ctx_set_wait_limit": [P, ctypes.c_uint64],
                "lnv_debug_expire_wait": [P],
                "lnv_probe_fma_rate": [P, i32, P],
                "lnv_pattern_build": [P, P, i64, P, dbl, PP],
                "lnv_pattern_build_batched": [P, P, i32, P, P, dbl, PP],
                "lnv_pattern_from_csr": [P, i64, P, P, PP],
                "lnv_pattern_info": [P, P, P, P, P, P, P],
                "lnv_pattern_destroy": [P],
                "lnv_plan_product": [P, P, P, P, i32, PP],
                "lnv_plan_info": [P, P, P],
                "lnv_plan_set_kernel": [P, P, i32],
                "lnv_plan_destroy": [P],
                "lnv_bsr_multiply": [P, P, i32, i32, P, P, P, dbl, dbl],
                "lnv_trace_product": [P, P, i32, i32, P, P, P, P],
                "lnv_system_create": [P, i32, i32, P, i64, i32, P, P, dbl, dbl, PP],
                "lnv_system_create_truncated": [P, i32, i32, P, i64, i32, P, P, dbl, dbl, dbl, dbl, PP],
                "lnv_system_patterns": [P, PP, PP],
                "lnv_system_workspace_size": [P, i32, P],
                "lnv_system_triples": [P, i32, P],
                "lnv_system_destroy": [P],
                "lnv_energy_grad": [P, P, P, P, P, P, P, P, P, ctypes.c_size_t],
                "lnv_energy_grad_host": [P, P, P, P, P, P, P],
                "lnv_system_profile": [P, i32],
                "lnv_system_stage_ms": [P, P],
                "lnv_system_stage_triples": [P, P],
                "lnv_system_stage_kernels": [P, P],
                "lnv_system_autotune": [P, P, P, P, P, i32, P],
                "lnv_system_set_stage_kernel": [P, P, i32, i32],
                "lnv_system_set_mirror": [P, P, i32],
                "lnv_system_mirror": [P, P],
                "lnv_system_info": [P, P, P, P],
                "lnv_pattern_remap": [P, P, P, i32, i32, P, P],
                "lnv_vec_axpby": [P, i32, i64, dbl, P, dbl, P, P],
                "lnv_vec_dot": [P, i32, i64, P, P, P],
                "lnv_minimize": [P, P, P, P, P, dbl, i32, dbl, P, P],
            }
            for name, args in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            L.lnv_last_error.restype = ctypes.c_char_p
            L.lnv_last_error.argtypes = []
            L.lnv_version.restype = ctypes.c_char_p
            L.lnv_version.argtypes = []
            L.lnv_launch_count.restype = ctypes.c_int64
            L.lnv_launch_count.argtypes = []
            _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        raise LnvError(what, status, lib().lnv_last_error().decode(errors="replace"))


def _ptr(t: torch.Tensor | None):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(None)


class _DevView:
    """Zero-copy __cuda_array_interface__ view of a library-owned device array."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {
            "shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 3,
            "strides": None}


def _view(ptr, n, typestr, device):
    if n == 0 or not ptr:
        return torch.empty(0, dtype={"<i8": torch.int64, "<i4": torch.int32}[typestr], device=device)
    return torch.as_tensor(_DevView(ptr, n, typestr), device=device)


def version() -> str:
    return lib().lnv_version().decode()


def launch_count() -> int:
    """Kernels liblnv has launched in this process."""
    return int(lib().lnv_launch_count())


class Context:
    """A device plus the stream the library enqueues on (torch's current one)."""

    def __init__(self, device=None, stream: torch.cuda.Stream | None = None):
        device = torch.device("cuda") if device is None else torch.device(device)
        if device.type != "cuda":
            raise ValueError("liblnv runs on CUDA devices only")
        if device.index is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        _check(lib().lnv_ctx_create(self.device.index, ctypes.c_void_p(self.stream.cuda_stream),
                                    ctypes.byref(h)), "lnv_ctx_create")
        self.h = h

    def set_stream(self, stream: torch.cuda.Stream):
        self.stream = stream
        _check(lib().lnv_ctx_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)), "lnv_ctx_set_stream")

    def device_status(self) -> int:
        """Synchronise the stream; 0, or LNV_ERR_TIMEOUT (-6) if a bounded
        device-side wait ran out since the last call (the word is cleared)."""
        return int(lib().lnv_ctx_device_status(self.h))

    def check_device(self):
        """Raise LnvError if a device-side wait ran out since the last check."""
        _check(lib().lnv_ctx_device_status(self.h), "device status")

    def set_wait_limit(self, ns: int):
        _check(lib().lnv_ctx_set_wait_limit(self.h, int(ns)), "lnv_ctx_set_wait_limit")

    def fma_rate(self, prec: str) -> float:
        """Measured FMA-pipe rate of this GPU in TFLOP/s ("fp32" or "fp64")."""
        v = ctypes.c_double()
        _check(lib().lnv_probe_fma_rate(self.h, 0 if prec == "fp64" else 1, ctypes.byref(v)),
               "lnv_probe_fma_rate")
        return float(v.value)

    def debug_expire_wait(self):
        """Launch one CTA whose bounded wait runs out (raises the status word)."""
        _check(lib().lnv_debug_expire_wait(self.h), "lnv_debug_expire_wait")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lnv_ctx_destroy(self.h)
            self.h = None


def _pos_tensor(pos, device):
    pos = torch.as_tensor(pos, dtype=torch.float64)
    if pos.device != device:
        pos = pos.to(device)
    pos = pos.contiguous()
    if pos.dim() != 2 or pos.shape[1] != 3:
        raise ValueError("positions must be [n, 3]")
    return pos


class Pattern:
    """A library-owned block-CSR range pattern."""

    def __init__(self, ctx: Context, handle, owner=None):
        self.ctx, self.h, self._owner = ctx, handle, owner
        n, nnzb, sym = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        rp, col, tr = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().lnv_pattern_info(self.h, ctypes.byref(n), ctypes.byref(nnzb), ctypes.byref(rp),
                                      ctypes.byref(col), ctypes.byref(tr), ctypes.byref(sym)),
               "lnv_pattern_info")
        self.n, self.nnzb, self.symmetric = n.value, nnzb.value, bool(sym.value)
        self._rp, self._col, self._tr = rp.value, col.value, tr.value

    @classmethod
    def build(cls, ctx: Context, pos, cell, cutoff: float) -> "Pattern":
        pos = _pos_tensor(pos, ctx.device)
        cellv = (ctypes.c_double * 3)(*[float(c) for c in cell])
        h = ctypes.c_void_p()
        _check(lib().lnv_pattern_build(ctx.h, _ptr(pos), pos.shape[0], cellv, float(cutoff),
                                       ctypes.byref(h)), "lnv_pattern_build")
        return cls(ctx, h)

    @classmethod
    def build_batched(cls, ctx: Context, pos, seg_off, cells, cutoff: float) -> "Pattern":
        pos = _pos_tensor(pos, ctx.device)
        off = (ctypes.c_int64 * len(seg_off))(*[int(x) for x in seg_off])
        flat = [float(c) for cell in cells for c in cell]
        cv = (ctypes.c_double * len(flat))(*flat)
        h = ctypes.c_void_p()
        _check(lib().lnv_pattern_build_batched(ctx.h, _ptr(pos), len(seg_off) - 1, off, cv,
                                               float(cutoff), ctypes.byref(h)),
               "lnv_pattern_build_batched")
        return cls(ctx, h)

    @classmethod
    def from_csr(cls, ctx: Context, row_ptr, col) -> "Pattern":
        rp = torch.as_tensor(row_ptr, dtype=torch.int64).to(ctx.device).contiguous()
        cl = torch.as_tensor(col, dtype=torch.int32).to(ctx.device).contiguous()
        h = ctypes.c_void_p()
        _check(lib().lnv_pattern_from_csr(ctx.h, rp.numel() - 1, _ptr(rp), _ptr(cl), ctypes.byref(h)),
               "lnv_pattern_from_csr")
        torch.cuda.current_stream(ctx.device).synchronize()
        return cls(ctx, h)

    @property
    def row_ptr(self) -> torch.Tensor:
        return _view(self._rp, self.n + 1, "<i8", self.ctx.device).clone()

    @property
    def col(self) -> torch.Tensor:
        return _view(self._col, self.nnzb, "<i4", self.ctx.device).clone()

    @property
    def tr(self) -> torch.Tensor:
        return _view(self._tr, self.nnzb, "<i8", self.ctx.device).clone()

    def values(self, nsf: int, dtype=torch.float64) -> torch.Tensor:
        return torch.zeros((self.nnzb, nsf, nsf), dtype=dtype, device=self.ctx.device)

    def remap(self, vals: torch.Tensor, to: "Pattern", out=None) -> torch.Tensor:
        """Block values on this pattern carried onto `to` (zeros where this
        pattern has no block), e.g. L of the previous geometry as the start of
        the next minimisation."""
        nsf = vals.shape[-1]
        prec = FP64 if vals.dtype == torch.float64 else FP32
        v = _vals(vals, self, nsf, prec, "vals")
        if out is None:
            out = torch.empty((to.nnzb, nsf, nsf), dtype=vals.dtype, device=self.ctx.device)
        o = _vals(out, to, nsf, prec, "out")
        _check(lib().lnv_pattern_remap(self.ctx.h, self.h, to.h, nsf, prec, v, o), "lnv_pattern_remap")
        return out

    def __del__(self):
        if getattr(self, "h", None) and self._owner is None and _lib is not None:
            _lib.lnv_pattern_destroy(self.h)
            self.h = None


def _vals(t: torch.Tensor, pattern: Pattern, nsf: int, prec: int, name: str):
    if not isinstance(t, torch.Tensor) or t.device != pattern.ctx.device:
        raise ValueError(f"{name} must be a tensor on {pattern.ctx.device}")
    if t.dtype != DTYPE[prec]:
        raise ValueError(f"{name} must be {DTYPE[prec]}, got {t.dtype}")
    if t.numel() != pattern.nnzb * nsf * nsf:
        raise ValueError(f"{name} holds {t.numel()} values; its pattern needs "
                         f"{pattern.nnzb} blocks of {nsf}x{nsf}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return _ptr(t)


class Plan:
    """C = mask_C(op(A) op(B)) on fixed patterns."""

    def __init__(self, ctx: Context, A: Pattern, B: Pattern, C: Pattern, trans_a=False, trans_b=False,
                 sym_c=False):
        """sym_c: the product is symmetric; only its upper triangle is formed and
        the lower one mirrored (C's pattern must be symmetric)."""
        self.ctx, self.A, self.B, self.C = ctx, A, B, C
        flags = (TRANS_A if trans_a else 0) | (TRANS_B if trans_b else 0) | (SYM_C if sym_c else 0)
        h = ctypes.c_void_p()
        _check(lib().lnv_plan_product(ctx.h, A.h, B.h, C.h, flags, ctypes.byref(h)), "lnv_plan_product")
        self.h = h
        t, m = ctypes.c_int64(), ctypes.c_int()
        _check(lib().lnv_plan_info(self.h, ctypes.byref(t), ctypes.byref(m)), "lnv_plan_info")
        self.triples, self.mode = t.value, self.KERNELS[m.value]

    KERNELS = ("push", "pull", "pull-merge", "group", "group-sparse", "group-pipe", "group-mma", "triples",
               "group-pipe-half", "tensor", "tensor9", "tensor-tile", "tensor-1pass", "tensor-tile-1pass")

    def set_kernel(self, kernel):
        k = self.KERNELS.index(kernel) if isinstance(kernel, str) else int(kernel)
        _check(lib().lnv_plan_set_kernel(self.ctx.h, self.h, k), "lnv_plan_set_kernel")
        self.mode = self.KERNELS[k]

    def multiply(self, A_vals, B_vals, C_vals=None, nsf=None, prec=None, alpha=1.0, beta=0.0):
        """C = alpha mask_C(op(A) op(B)) + beta C (C is overwritten when beta = 0)."""
        nsf = nsf or A_vals.shape[-1]
        prec = PREC[prec] if prec is not None else (FP64 if A_vals.dtype == torch.float64 else FP32)
        if C_vals is None:
            if beta != 0.0:
                raise ValueError("beta != 0 needs C_vals")
            C_vals = torch.empty((self.C.nnzb, nsf, nsf), dtype=DTYPE[prec], device=self.ctx.device)
        a = _vals(A_vals, self.A, nsf, prec, "A")
        b = _vals(B_vals, self.B, nsf, prec, "B")
        c = _vals(C_vals, self.C, nsf, prec, "C")
        _check(lib().lnv_bsr_multiply(self.ctx.h, self.h, nsf, prec, a, b, c, float(alpha), float(beta)),
               "lnv_bsr_multiply")
        return C_vals

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lnv_plan_destroy(self.h)
            self.h = None


def trace_product(ctx: Context, P: Pattern, A_vals, B_vals, out=None, scratch=None) -> torch.Tensor:
    """Tr[A B] (FP64) for A, B on the symmetric pattern P, as a 1-element device tensor."""
    nsf = A_vals.shape[-1]
    prec = FP64 if A_vals.dtype == torch.float64 else FP32
    a = _vals(A_vals, P, nsf, prec, "A")
    b = _vals(B_vals, P, nsf, prec, "B")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=ctx.device)
    if scratch is None:
        scratch = torch.empty(max(P.n, 1), dtype=torch.float64, device=ctx.device)
    _check(lib().lnv_trace_product(ctx.h, P.h, nsf, prec, a, b, _ptr(scratch), _ptr(out)),
           "lnv_trace_product")
    return out


def vec_axpby(ctx: Context, a: float, x: torch.Tensor, b: float, y: torch.Tensor, out=None) -> torch.Tensor:
    """out = a x + b y on the device (x, y, out contiguous, same dtype and size)."""
    prec = FP64 if x.dtype == torch.float64 else FP32
    if y.dtype != x.dtype or y.numel() != x.numel() or not (x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x and y must be contiguous tensors of one dtype and size")
    if out is None:
        out = torch.empty_like(x)
    _check(lib().lnv_vec_axpby(ctx.h, prec, x.numel(), float(a), _ptr(x), float(b), _ptr(y), _ptr(out)),
           "lnv_vec_axpby")
    return out


def vec_dot(ctx: Context, x: torch.Tensor, y: torch.Tensor, out=None) -> torch.Tensor:
    """x . y summed in FP64 in a fixed order, as a 1-element device tensor."""
    prec = FP64 if x.dtype == torch.float64 else FP32
    if y.dtype != x.dtype or y.numel() != x.numel() or not (x.is_contiguous() and y.is_contiguous()):
        raise ValueError("x and y must be contiguous tensors of one dtype and size")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=ctx.device)
    _check(lib().lnv_vec_dot(ctx.h, prec, x.numel(), _ptr(x), _ptr(y), _ptr(out)), "lnv_vec_dot")
    return out


def trace_product_noalloc(ctx: Context, P: Pattern, A_vals, B_vals, out=None) -> torch.Tensor:
    """Tr[A B] through lnv_trace_product_noalloc: no device allocation inside
    the library (its per-row sums use a built-in 2 MiB array, at most 262144
    rows).  Calls on one device must not overlap on the GPU."""
    nsf = A_vals.shape[-1]
    prec = FP64 if A_vals.dtype == torch.float64 else FP32
    a = _vals(A_vals, P, nsf, prec, "A")
    b = _vals(B_vals, P, nsf, prec, "B")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=ctx.device)
    f = lib().lnv_trace_product_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    _check(f(ctx.h, P.h, nsf, prec, a, b, _ptr(out)), "lnv_trace_product_noalloc")
    return out


class System:
    """One LNV system (or a batch of independent ones): patterns, plans, workspace."""

    def __init__(self, ctx: Context, nsf: int, prec, pos, cells, r_sh: float, r_l: float,
                 seg_off=None, r_x: float | None = None, r_t: float | None = None):
        """r_x, r_t: truncate X, Y, Z to r_x and T, U to r_t (None: the exact
        ranges r_l + r_sh and r_l + 2 r_sh)."""
        self.ctx, self.nsf, self.prec = ctx, int(nsf), PREC[prec]
        pos = _pos_tensor(pos, ctx.device)
        self.n = pos.shape[0]
        if seg_off is None:
            seg_off = [0, self.n]
            cells = [cells]
        self.n_seg = len(seg_off) - 1
        self.seg_off = [int(x) for x in seg_off]
        flat = [float(c) for cell in cells for c in cell]
        if len(flat) != 3 * self.n_seg:
            raise ValueError("one 3-vector cell per system is required")
        off = (ctypes.c_int64 * len(seg_off))(*self.seg_off)
        cv = (ctypes.c_double * len(flat))(*flat)
        h = ctypes.c_void_p()
        _check(lib().lnv_system_create_truncated(ctx.h, self.nsf, self.prec, _ptr(pos), self.n, self.n_seg,
                                                 off, cv, float(r_sh), float(r_l), float(r_x or 0.0),
                                                 float(r_t or 0.0), ctypes.byref(h)),
               "lnv_system_create_truncated")
        self.h = h
        self.r_sh, self.r_l = float(r_sh), float(r_l)
        sh, l = ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().lnv_system_patterns(self.h, ctypes.byref(sh), ctypes.byref(l)), "lnv_system_patterns")
        self.P_sh = Pattern(ctx, sh, owner=self)
        self.P_l = Pattern(ctx, l, owner=self)
        self.dtype = DTYPE[self.prec]

    def workspace_size(self, grad: bool = True) -> int:
        v = ctypes.c_size_t()
        _check(lib().lnv_system_workspace_size(self.h, int(grad), ctypes.byref(v)),
               "lnv_system_workspace_size")
        return v.value

    def triples(self, grad: bool = True) -> int:
        v = ctypes.c_int64()
        _check(lib().lnv_system_triples(self.h, int(grad), ctypes.byref(v)), "lnv_system_triples")
        return v.value

    def flops(self, grad: bool = True) -> int:
        """Algorithmic flops of one evaluation: 2 NSF^3 per contributing block triple."""
        return 2 * self.nsf ** 3 * self.triples(grad)

    def energy_grad(self, S, H, L, grad: bool = True, out=None, G=None, workspace=None,
                    grad_ne: bool = False, GN=None):
        """One evaluation; returns (out [n_seg, 6] FP64 device tensor, G or None),
        or (out, G or None, GN) with grad_ne.

        out[s] = (E, N_e, Tr[LSLH], Tr[LSLSLH], Tr[LSLS], Tr[LSLSLS]); G = dE/dL
        and GN = dN_e/dL on L's pattern.
        """
        s = _vals(S, self.P_sh, self.nsf, self.prec, "S")
        h = _vals(H, self.P_sh, self.nsf, self.prec, "H")
        l_ = _vals(L, self.P_l, self.nsf, self.prec, "L")
        if out is None:
            out = torch.empty((self.n_seg, 6), dtype=torch.float64, device=self.ctx.device)
        if grad and G is None:
            G = torch.empty_like(L)
        g = _vals(G, self.P_l, self.nsf, self.prec, "G") if grad else ctypes.c_void_p(None)
        if grad_ne and GN is None:
            GN = torch.empty_like(L)
        gn = _vals(GN, self.P_l, self.nsf, self.prec, "GN") if grad_ne else ctypes.c_void_p(None)
        ws, wsb = ctypes.c_void_p(None), 0
        if workspace is not None:
            ws, wsb = _ptr(workspace), workspace.numel() * workspace.element_size()
        _check(lib().lnv_energy_grad(self.ctx.h, self.h, s, h, l_, _ptr(out), g, gn, ws, wsb),
               "lnv_energy_grad")
        if grad_ne:
            return out, (G if grad else None), GN
        return out, (G if grad else None)

    def energy_grad_host(self, S, H, L, grad: bool = True, out=None, G=None):
        """One evaluation from host memory (lnv_energy_grad_host: the library
        copies S, H, L in and the results out, and synchronises).  S, H, L are
        contiguous CPU tensors in the system's precision (pinned ones copy
        fastest); returns (out [n_seg, 6] FP64 CPU tensor, G CPU tensor or None)."""
        def host(t, pattern, name):
            if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
                raise ValueError(f"{name} must be a CPU tensor")
            if t.dtype != DTYPE[self.prec] or t.numel() != pattern.nnzb * self.nsf * self.nsf \
                    or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous {DTYPE[self.prec]} tensor of "
                                 f"{pattern.nnzb} blocks of {self.nsf}x{self.nsf}")
            return ctypes.c_void_p(t.data_ptr())
        s, h, l_ = host(S, self.P_sh, "S"), host(H, self.P_sh, "H"), host(L, self.P_l, "L")
        if out is None:
            out = torch.empty((self.n_seg, 6), dtype=torch.float64)
        if grad and G is None:
            G = torch.empty(L.shape, dtype=L.dtype)
        g = host(G, self.P_l, "G") if grad else ctypes.c_void_p(None)
        _check(lib().lnv_energy_grad_host(self.ctx.h, self.h, s, h, l_, ctypes.c_void_p(out.data_ptr()), g),
               "lnv_energy_grad_host")
        return out, (G if grad else None)

    STAGES = ("XY", "TU", "Z", "traces", "Q", "W", "G")

    def minimize(self, S, H, L, mu: float, max_iter: int = 200, tol: float = 1e-8):
        """Minimise Omega = E - mu N_e over L (updated in place) by conjugate
        gradients with exact cubic line searches.  Returns (iterations, history
        [iterations + 1, 5] of (Omega, E, N_e, rms of dOmega/dL, previous step))."""
        if self.n_seg != 1:
            raise ValueError("minimize takes one system at a time")
        s = _vals(S, self.P_sh, self.nsf, self.prec, "S")
        h = _vals(H, self.P_sh, self.nsf, self.prec, "H")
        l_ = _vals(L, self.P_l, self.nsf, self.prec, "L")
        hist = np.zeros((int(max_iter) + 1, 5), dtype=np.float64)
        it = ctypes.c_int(0)
        _check(lib().lnv_minimize(self.ctx.h, self.h, s, h, l_, float(mu), int(max_iter), float(tol),
                                  hist.ctypes.data_as(ctypes.c_void_p), ctypes.byref(it)), "lnv_minimize")
        return it.value, hist[: it.value + 1]

    def capture(self, S, H, L, grad: bool = True, out=None, G=None, workspace=None):
        """Capture one evaluation in a CUDA graph; returns (graph, out, G).

        graph.replay() re-runs every kernel of the evaluation on the current
        contents of S, H, L (same device buffers) into out and G.  One warm-up
        evaluation runs first (outside the capture) so that no allocation or
        attribute change happens while capturing.
        """
        dev = self.ctx.device
        if out is None:
            out = torch.empty((self.n_seg, 6), dtype=torch.float64, device=dev)
        if grad and G is None:
            G = torch.empty_like(L)
        if workspace is None:
            workspace = torch.empty(self.workspace_size(grad), dtype=torch.uint8, device=dev)
        self.profile(False)
        self.energy_grad(S, H, L, grad=grad, out=out, G=G, workspace=workspace)
        torch.cuda.synchronize(dev)
        graph = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream(dev)
        old = self.ctx.stream
        with torch.cuda.graph(graph, stream=side):
            self.ctx.set_stream(side)
            try:
                self.energy_grad(S, H, L, grad=grad, out=out, G=G, workspace=workspace)
            finally:
                self.ctx.set_stream(old)
        self._graph_refs = (out, G, workspace)
        return graph, out, G

    def profile(self, enable: bool = True):
        _check(lib().lnv_system_profile(self.h, int(enable)), "lnv_system_profile")

    def stage_kernels(self) -> dict:
        """Kernel chosen for each product stage."""
        k = (ctypes.c_int * 7)()
        _check(lib().lnv_system_stage_kernels(self.h, k), "lnv_system_stage_kernels")
        return {s_: Plan.KERNELS[v] for s_, v in zip(self.STAGES, list(k)) if v >= 0}

    def set_stage_kernel(self, stage: str, kernel):
        """Pin the kernel of one product stage ("XY", "TU", "Z", "Q", "W")."""
        k = Plan.KERNELS.index(kernel) if isinstance(kernel, str) else int(kernel)
        _check(lib().lnv_system_set_stage_kernel(self.ctx.h, self.h, self.STAGES.index(stage), k),
               "lnv_system_set_stage_kernel")

    @property
    def mirror(self) -> bool:
        """True when T = SLS is formed on its upper triangle and mirrored."""
        v = ctypes.c_int()
        _check(lib().lnv_system_mirror(self.h, ctypes.byref(v)), "lnv_system_mirror")
        return bool(v.value)

    def set_mirror(self, on: bool):
        """Form T on its upper triangle and mirror it (True), or whole (False)."""
        _check(lib().lnv_system_set_mirror(self.ctx.h, self.h, int(on)), "lnv_system_set_mirror")

    def autotune(self, S, H, L, reps: int = 3) -> dict:
        """Time every applicable kernel per product stage on these inputs and
        keep the fastest; returns {stage: (kernel, ms)}."""
        s = _vals(S, self.P_sh, self.nsf, self.prec, "S")
        h = _vals(H, self.P_sh, self.nsf, self.prec, "H")
        l_ = _vals(L, self.P_l, self.nsf, self.prec, "L")
        nk = len(Plan.KERNELS)
        ms = (ctypes.c_double * (5 * nk))()
        _check(lib().lnv_system_autotune(self.ctx.h, self.h, s, h, l_, int(reps), ms), "lnv_system_autotune")
        ks = self.stage_kernels()
        self.tune_table = {st: {Plan.KERNELS[k]: ms[i * nk + k] for k in range(nk) if ms[i * nk + k] >= 0}
                           for i, st in enumerate(("XY", "TU", "Z", "Q", "W"))}
        return {st: (ks[st], self.tune_table[st][ks[st]]) for st in self.tune_table}

    def stage_triples(self) -> dict:
        """Contributing block triples of each stage."""
        t = (ctypes.c_int64 * 7)()
        _check(lib().lnv_system_stage_triples(self.h, t), "lnv_system_stage_triples")
        return dict(zip(self.STAGES, list(t)))

    def stage_ms(self) -> dict:
        """Per-stage milliseconds of the last profiled evaluation."""
        ms = (ctypes.c_double * 7)()
        _check(lib().lnv_system_stage_ms(self.h, ms), "lnv_system_stage_ms")
        return dict(zip(self.STAGES, list(ms)))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.lnv_system_destroy(self.h)
            self.h = None
