"""FP64 CPU oracle for the LNV energy / electron count / gradient path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_0911_3584_gb300``) and never imports it.

The arithmetic lives in ``lnv_oracle.c`` (plain nested loops, FP64, compiled
with -ffp-contract=off, optional OpenMP over rows); this module marshals numpy
arrays and composes the steps in the order the equations give them.

What is computed (Bowler & Miyazaki, Sec. 2):

* K = 3 LSL - 2 LSLSL                        (Eq. 3, the LNV / ADM form)
* N_e = 2 Tr[K S]                            (Sec. 2, condition 2)
* E = 2 Tr[K H]                              (band energy of the fixed-H,
  non-self-consistent tight-binding level, Sec. 2; spin factor 2.  The paper
  does not print this formula; it is the energy whose minimisation over L the
  paper describes.)
* G = dE/dL = 6 (SLH + HLS) - 4 (SLSLH + SLHLS + HLSLS), kept on L's range
  pattern (L_ij = 0 beyond R_L, Sec. 2).  Derivative with respect to each
  stored entry L_ab taken as independent; S, H and L symmetric.

Matrices are block-CSR dicts {"rp": int64[n+1], "col": int32[nnzb],
"val": float64[nnzb, nsf, nsf]} (columns sorted inside each row).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lnv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblnv_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build (gcc, -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = _SO + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            lib.oracle_pattern_count.restype = i64
            lib.oracle_pattern_count.argtypes = [P, i64, P, ctypes.c_double, P]
            lib.oracle_pattern_fill.restype = None
            lib.oracle_pattern_fill.argtypes = [P, i64, P, ctypes.c_double, P, P]
            lib.oracle_mprod.restype = None
            lib.oracle_mprod.argtypes = [ctypes.c_int, i64] + [P] * 9 + [P, i64]
            lib.oracle_trace.restype = ctypes.c_double
            lib.oracle_trace.argtypes = [ctypes.c_int, i64] + [P] * 7 + [P, i64]
            lib.oracle_restrict.restype = None
            lib.oracle_restrict.argtypes = [ctypes.c_int, i64] + [P] * 6
            lib.oracle_transpose.restype = None
            lib.oracle_transpose.argtypes = [ctypes.c_int, i64] + [P] * 4
            lib.oracle_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def pattern(pos: np.ndarray, cell: np.ndarray, cutoff: float):
    """Block pattern {(i, j): d_ij^2 < cutoff^2}, minimum image, brute force.

    Returns (row_ptr int64[n+1], col int32[nnzb]), columns ascending.
    """
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    n = pos.shape[0]
    rp = np.zeros(n + 1, dtype=np.int64)
    nnz = lib.oracle_pattern_count(_p(pos), n, _p(cell), float(cutoff), _p(rp))
    col = np.zeros(max(nnz, 1), dtype=np.int32)
    lib.oracle_pattern_fill(_p(pos), n, _p(cell), float(cutoff), _p(rp), _p(col))
    return rp, col[:nnz]


def csr(rp, col, val=None, nsf=None):
    d = {"rp": np.ascontiguousarray(rp, dtype=np.int64),
         "col": np.ascontiguousarray(col, dtype=np.int32)}
    if val is None:
        d["val"] = np.zeros((d["col"].size, nsf, nsf))
    else:
        d["val"] = np.ascontiguousarray(val, dtype=np.float64)
    return d


def _rows(rows):
    if rows is None:
        return None, 0
    r = np.ascontiguousarray(rows, dtype=np.int64)
    return r, r.size


def mprod(A: dict, B: dict, C_pat: tuple, rows=None) -> dict:
    """mask(A B) on the block pattern C_pat = (row_ptr, col).

    With ``rows``, only those rows of C are formed (the rest stay zero).
    """
    lib = _load()
    nsf = A["val"].shape[-1]
    n = A["rp"].size - 1
    C = csr(C_pat[0], C_pat[1], nsf=nsf)
    r, nr = _rows(rows)
    lib.oracle_mprod(nsf, n, _p(A["rp"]), _p(A["col"]), _p(A["val"]),
                     _p(B["rp"]), _p(B["col"]), _p(B["val"]),
                     _p(C["rp"]), _p(C["col"]), _p(C["val"]),
                     _p(r) if r is not None else None, nr)
    return C


def trace(A: dict, B: dict, row_part: bool = False, rows=None):
    """Tr[A B] in FP64; optionally also the per-row partial sums.

    With ``rows``, the partial trace over those rows only.
    """
    lib = _load()
    nsf = A["val"].shape[-1]
    n = A["rp"].size - 1
    part = np.zeros(n) if row_part else None
    r, nr = _rows(rows)
    t = lib.oracle_trace(nsf, n, _p(A["rp"]), _p(A["col"]), _p(A["val"]),
                         _p(B["rp"]), _p(B["col"]), _p(B["val"]),
                         _p(part) if part is not None else None,
                         _p(r) if r is not None else None, nr)
    return (t, part) if row_part else t


def restrict(M: dict, C_pat: tuple) -> dict:
    lib = _load()
    nsf = M["val"].shape[-1]
    n = M["rp"].size - 1
    C = csr(C_pat[0], C_pat[1], nsf=nsf)
    lib.oracle_restrict(nsf, n, _p(M["rp"]), _p(M["col"]), _p(M["val"]),
                        _p(C["rp"]), _p(C["col"]), _p(C["val"]))
    return C


def transpose(M: dict) -> dict:
    """(M^T)_ij = (M_ji)^T on M's (symmetric) pattern."""
    lib = _load()
    nsf = M["val"].shape[-1]
    n = M["rp"].size - 1
    out = csr(M["rp"], M["col"], nsf=nsf)
    lib.oracle_transpose(nsf, n, _p(M["rp"]), _p(M["col"]), _p(M["val"]), _p(out["val"]))
    return out


def lnv_energy_grad(pos, cell, r_sh, r_l, S: dict, H: dict, L: dict, grad: bool = True,
                    keep: bool = False, grad_ne: bool = False) -> dict:
    """E, N_e and dE/dL of the LNV functional on range-truncated matrices.

    S and H share the block pattern of range r_sh, L has range r_l (Sec. 2).
    Each matrix product below is formed exactly on a pattern wide enough that
    nothing it is later used for is cut off: by the triangle inequality of the
    minimum-image distance, A B vanishes beyond R_A + R_B.

      X = L S, Y = L H                on range r_l + r_sh   (exact)
      T = S X = SLS, U = S Y = SLH    on range r_l + 2 r_sh (exact)
      Z = L T = LSLS                  on range r_l + r_sh   (every later use
                                       reads Z only inside that range)

    Eq. 3 with the linearity and cyclicity of the trace gives
      Tr[KH] = 3 Tr[LSLH] - 2 Tr[LSLSLH] = 3 Tr[XY] - 2 Tr[ZY]
      Tr[KS] = 3 Tr[LSLS] - 2 Tr[LSLSLS] = 3 Tr[XX] - 2 Tr[ZX]
    and each gradient term is one masked product onto L's pattern:
      SLH = S Y, HLS = H X, SLSLH = T Y, SLHLS = U X, HLSLS = H Z.
    With grad_ne, the electron count's gradient (the condition N_e = 2 Tr[KS]
    of Sec. 2 held during the minimisation needs it):
      dN_e/dL = 2 (3 * 2 SLS - 2 * 3 SLSLS) = 12 (SLS - SLSLS),
    with SLS = S X and SLSLS = T X, each masked onto L's pattern.
    """
    r_x = r_l + r_sh
    r_t = r_l + 2.0 * r_sh
    pat_x = pattern(pos, cell, r_x)
    pat_t = pattern(pos, cell, r_t)
    pat_l = (L["rp"], L["col"])
    X = mprod(L, S, pat_x)
    Y = mprod(L, H, pat_x)
    T = mprod(S, X, pat_t)
    Z = mprod(L, T, pat_x)
    t1 = trace(X, Y)
    t2 = trace(Z, Y)
    n1 = trace(X, X)
    n2 = trace(Z, X)
    out = {
        "E": 2.0 * (3.0 * t1 - 2.0 * t2),
        "Ne": 2.0 * (3.0 * n1 - 2.0 * n2),
        "traces": (t1, t2, n1, n2),
    }
    if grad:
        U = mprod(S, Y, pat_t)
        slh = mprod(S, Y, pat_l)
        hls = mprod(H, X, pat_l)
        slslh = mprod(T, Y, pat_l)
        slhls = mprod(U, X, pat_l)
        hlsls = mprod(H, Z, pat_l)
        G = 6.0 * (slh["val"] + hls["val"]) - 4.0 * (slslh["val"] + slhls["val"] + hlsls["val"])
        out["G"] = G
        if keep:
            out.update(U=U, slh=slh, hls=hls, slslh=slslh, slhls=slhls, hlsls=hlsls)
    if grad_ne:
        sls = mprod(S, X, pat_l)
        slsls = mprod(T, X, pat_l)
        out["GN"] = 12.0 * (sls["val"] - slsls["val"])
    if keep:
        out.update(X=X, Y=Y, T=T, Z=Z, pat_x=pat_x, pat_t=pat_t)
        if not grad:
            out["U"] = mprod(S, Y, pat_t)
    return out


def lnv_energy_grad_truncated(pos, cell, r_sh, r_l, r_x, r_t, S: dict, H: dict, L: dict,
                              grad: bool = True) -> dict:
    """E, N_e and G with the intermediates truncated below their exact ranges.

    The paper keeps every matrix sparse by range (Sec. 2) and leaves the
    ranges of products to "carefully constructed sparse matrix methods".  Here
    X = LS and Y = LH are kept within r_x, T = SX and U = SY within r_t, and
    Z = L T^T within r_x; then, as in the exact case,
      E = 2 (3 Tr[XY] - 2 Tr[ZY]),  N_e = 2 (3 Tr[XX] - 2 Tr[ZX]),
      G = 6 (U + U^T) - 4 (Q^T + W + Q) on L's pattern, Q = H Z,
      W = X^T U^T formed for j >= i and mirrored (W_ji = W_ij^T).
    With r_x = r_l + r_sh and r_t = r_l + 2 r_sh every product is exact and
    this equals lnv_energy_grad; below them, the association above defines
    the approximation (T is then not exactly symmetric, so Z uses T^T and W
    is taken from one triangle, as the exact plan's symmetric forms do).
    """
    pat_x = pattern(pos, cell, r_x)
    pat_t = pattern(pos, cell, r_t)
    pat_l = (L["rp"], L["col"])
    X = mprod(L, S, pat_x)
    Y = mprod(L, H, pat_x)
    T = mprod(S, X, pat_t)
    Z = mprod(L, transpose(T), pat_x)
    t1, t2, n1, n2 = trace(X, Y), trace(Z, Y), trace(X, X), trace(Z, X)
    out = {"E": 2.0 * (3.0 * t1 - 2.0 * t2), "Ne": 2.0 * (3.0 * n1 - 2.0 * n2), "traces": (t1, t2, n1, n2)}
    if grad:
        U = mprod(S, Y, pat_t)
        Ul = restrict(U, pat_l)
        Q = mprod(H, Z, pat_l)
        W = mprod(transpose(X), transpose(U), pat_l)
        rp, col = pat_l
        n = rp.size - 1
        rows = np.repeat(np.arange(n), np.diff(rp))
        low = col < rows
        Wv = W["val"].copy()
        Wt = transpose(W)["val"]
        Wv[low] = Wt[low]                       # W_ij = W_ji^T below the diagonal
        G = 6.0 * (Ul["val"] + transpose(Ul)["val"]) - 4.0 * (transpose(Q)["val"] + Wv + Q["val"])
        out["G"] = G
    return out


def lnv_rows(S: dict, H: dict, L: dict, full: dict, rows) -> float:
    """Every product and trace of one evaluation, restricted to output rows
    ``rows``, with the operands taken from ``full`` (a ``keep=True`` result of
    lnv_energy_grad).  Used to time bounded samples of the oracle; returns the
    partial sum 2 (3 Tr[XY] - 2 Tr[ZY]) over those rows."""
    px, pt, pl = full["pat_x"], full["pat_t"], (L["rp"], L["col"])
    mprod(L, S, px, rows)
    mprod(L, H, px, rows)
    mprod(S, full["X"], pt, rows)
    mprod(S, full["Y"], pt, rows)
    mprod(L, full["T"], px, rows)
    t1 = trace(full["X"], full["Y"], rows=rows)
    t2 = trace(full["Z"], full["Y"], rows=rows)
    trace(full["X"], full["X"], rows=rows)
    trace(full["Z"], full["X"], rows=rows)
    mprod(S, full["Y"], pl, rows)
    mprod(H, full["X"], pl, rows)
    mprod(full["T"], full["Y"], pl, rows)
    mprod(full["U"], full["X"], pl, rows)
    mprod(H, full["Z"], pl, rows)
    return 2.0 * (3.0 * t1 - 2.0 * t2)
