"""lnv_trace_product_noalloc, the trace entry point that allocates nothing.

It exists for callers that cannot allocate device memory or hand the library a
scratch buffer (a fixed device-memory budget owned by their own pool, or an
interface with no room for scratch).  Its per-row sums live in a built-in
device array, shared by every call on a device.  This file is collected last,
so a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from paper_0911_3584_gb300 import Context, Pattern, lib, trace_product

pytestmark = pytest.mark.gpu


def _noalloc(ctx, P, nsf, prec, A, B, out):
    f = lib().lnv_trace_product_noalloc
    f.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] * 2 + [ctypes.c_void_p] * 3
    f.restype = ctypes.c_int
    return f(ctx.h, P.h, nsf, prec, ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
             ctypes.c_void_p(out.data_ptr()))


@pytest.mark.parametrize("dtype,prec", [(torch.float64, 0), (torch.float32, 1)])
def test_noalloc_trace_matches_allocating_entry_point(cuda_device, dtype, prec):
    ctx = Context(cuda_device)
    rng = np.random.default_rng(17)
    pos, cell = synth.si_diamond_positions(4, rng)
    P = Pattern.build(ctx, pos, cell, 8.0)
    nsf = 4
    for call in range(2):  # two calls in a row share the built-in array
        A = torch.from_numpy(rng.standard_normal((P.nnzb, nsf, nsf))).to(cuda_device, dtype)
        B = torch.from_numpy(rng.standard_normal((P.nnzb, nsf, nsf))).to(cuda_device, dtype)
        out = torch.full((1,), np.nan, dtype=torch.float64, device=cuda_device)
        assert _noalloc(ctx, P, nsf, prec, A, B, out) == 0, lib().lnv_last_error()
        ref = trace_product(ctx, P, A, B)
        torch.cuda.synchronize()
        tol = 1e-12 * np.sqrt(P.nnzb) * nsf * nsf
        assert abs(out.item() - ref.item()) <= tol, (call, out.item(), ref.item())


def test_noalloc_trace_rejects_patterns_beyond_its_array(cuda_device):
    ctx = Context(cuda_device)
    n = (1 << 18) + 1
    rng = np.random.default_rng(2)
    pos = rng.uniform(0.0, 1000.0, size=(n, 3))
    P = Pattern.build(ctx, pos, [1000.0, 1000.0, 1000.0], 0.05)  # essentially diagonal rows
    A = torch.ones((P.nnzb, 1, 1), dtype=torch.float64, device=cuda_device)
    out = torch.zeros(1, dtype=torch.float64, device=cuda_device)
    assert _noalloc(ctx, P, 1, 0, A, A, out) == -5
    lib().lnv_last_error.restype = ctypes.c_char_p
    assert b"262144" in lib().lnv_last_error()


@pytest.mark.parametrize("dtype,prec", [(torch.float64, 0), (torch.float32, 1)])
def test_noalloc_trace_at_exactly_the_array_size(cuda_device, dtype, prec):
    """A diagonal NSF = 1 pattern of exactly 262144 rows: the last element of
    the built-in array is used; the result equals the allocating entry point."""
    ctx = Context(cuda_device)
    n = 1 << 18
    rp = torch.arange(n + 1, dtype=torch.int64, device=cuda_device)
    col = torch.arange(n, dtype=torch.int32, device=cuda_device)
    P = Pattern.from_csr(ctx, rp, col)
    rng = np.random.default_rng(5)
    for call in range(2):
        A = torch.from_numpy(rng.standard_normal((n, 1, 1))).to(cuda_device, dtype)
        B = torch.from_numpy(rng.standard_normal((n, 1, 1))).to(cuda_device, dtype)
        out = torch.full((1,), np.nan, dtype=torch.float64, device=cuda_device)
        assert _noalloc(ctx, P, 1, prec, A, B, out) == 0, lib().lnv_last_error()
        ref = trace_product(ctx, P, A, B)
        torch.cuda.synchronize()
        assert abs(out.item() - ref.item()) <= 1e-12 * np.sqrt(n), (call, out.item(), ref.item())


@pytest.mark.parametrize("dtype,prec", [(torch.float64, 0), (torch.float32, 1)])
def test_noalloc_trace_nsf9(cuda_device, dtype, prec):
    """9 x 9 blocks (s, p, d) on a 64-atom pattern: equal to the allocating entry point."""
    ctx = Context(cuda_device)
    rng = np.random.default_rng(9)
    pos, cell = synth.si_diamond_positions(2, rng)
    P = Pattern.build(ctx, pos, cell, 6.6)
    for call in range(2):
        A = torch.from_numpy(rng.standard_normal((P.nnzb, 9, 9))).to(cuda_device, dtype)
        B = torch.from_numpy(rng.standard_normal((P.nnzb, 9, 9))).to(cuda_device, dtype)
        out = torch.full((1,), np.nan, dtype=torch.float64, device=cuda_device)
        assert _noalloc(ctx, P, 9, prec, A, B, out) == 0, lib().lnv_last_error()
        ref = trace_product(ctx, P, A, B)
        torch.cuda.synchronize()
        assert abs(out.item() - ref.item()) <= 1e-12 * np.sqrt(P.nnzb) * 81, (call, out.item(), ref.item())
