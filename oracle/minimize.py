"""FP64 CPU restatement of the LNV minimisation loop (test infrastructure only).

The paper (Sec. 2) asks for the energy to be minimised over the density
matrix with K = 3LSL - 2LSLSL (Eq. 3), the electron count being "relatively
easy to impose", and prints no algorithm.  This module takes the same reading
as the library's loop, written plainly with numpy on L's stored entries:

* the electron count is set by a chemical potential mu: the function
  minimised is the grand potential Omega = E - mu N_e = 2 Tr[K (H - mu S)],
  i.e. the band energy of H' = H - mu S, whose gradient is dE/dL with H';
* Polak-Ribiere conjugate gradients, d = -g + beta d_prev with beta =
  max(0, <g, g - g_prev> / <g_prev, g_prev>), reset to -g when not a descent;
* exact cubic line search: Omega(L + t d) = Omega + s t + c2 t^2 + c3 t^3
  (K is cubic in L) with s = <g, d>; c2, c3 from Omega at t1 and 2 t1; t =
  the positive root of the derivative where the curvature is positive.  The
  trial step t1 is the previous step, or 0.1 / |d| when that is smaller
  than 1e-3 of it.
* L and every gradient are kept exactly symmetric ((M + M^T) / 2 on L's
  pattern), the space the gradient formula is derived in.

With mu between the m-th and (m+1)-th generalised eigenvalues of (H, S) and
no truncation, the minimum is the projector on the m lowest states
(N_e = 2m, E = 2 sum eps_1..m).  Iteration stops when the root-mean-square
of g is at most tol, or when the line search finds no step (t below 1e-8 of
0.1 / |d|: the Omega differences have reached rounding).
"""
from __future__ import annotations

import numpy as np

from . import csr, lnv_energy_grad, transpose


def _fit_cubic(f0, f1, t1, fa, fb):
    """f(t1), f(2 t1) of f = f0 + f1 t + c2 t^2 + c3 t^3 -> (c2, c3)."""
    r1 = fa - f0 - f1 * t1
    r2 = fb - f0 - 2.0 * f1 * t1
    c3 = (r2 - 4.0 * r1) / (4.0 * t1 ** 3)
    c2 = (r1 - c3 * t1 ** 3) / t1 ** 2
    return c2, c3


def _cubic_min(slope, c2, c3, t_fallback):
    """Smallest positive t with slope + 2 c2 t + 3 c3 t^2 = 0 and 2 c2 + 6 c3 t > 0."""
    if c3 != 0.0:
        roots = np.roots([3.0 * c3, 2.0 * c2, slope])
    elif c2 != 0.0:
        roots = np.array([-slope / (2.0 * c2)])
    else:
        roots = np.array([])
    good = [r.real for r in np.atleast_1d(roots)
            if abs(r.imag) <= 1e-12 * max(1.0, abs(r.real)) and r.real > 0 and 2 * c2 + 6 * c3 * r.real > 0]
    return min(good) if good else t_fallback


def lnv_minimize(pos, cell, r_sh, r_l, S, H, L, mu, max_iter=200, tol=1e-8):
    """Minimise Omega = E - mu N_e over L's stored entries.  Returns the final
    L and history rows (Omega, E, N_e, |g|_rms, previous step)."""
    rp, col = L["rp"], L["col"]
    Hp = csr(H["rp"], H["col"], H["val"] - mu * S["val"])

    def sym(vals):
        return 0.5 * (vals + transpose(csr(rp, col, vals))["val"])

    lv = sym(L["val"])

    def ev(vals, grad):
        return lnv_energy_grad(pos, cell, r_sh, r_l, S, Hp, csr(rp, col, vals), grad=grad)

    hist = []
    d = g_old = None
    gg_old = t_prev = 0.0
    for it in range(max_iter + 1):
        o = ev(lv, True)
        g = sym(o["G"])
        gg = float((g * g).sum())
        rms = np.sqrt(gg / g.size)
        hist.append((o["E"], o["E"] + mu * o["Ne"], o["Ne"], rms, t_prev))
        if rms <= tol or it == max_iter:
            break
        beta = max(0.0, (gg - float((g * g_old).sum())) / gg_old) if it > 0 and gg_old > 0 else 0.0
        d = -g + beta * d if beta > 0.0 else -g
        slope = float((g * d).sum())
        if not slope < 0.0:
            d, slope = -g, -gg
        t_ref = 0.1 / np.sqrt(max(float((d * d).sum()), 1e-300))
        t1 = t_prev if t_prev > 1e-3 * t_ref else t_ref
        fa = ev(lv + t1 * d, False)["E"]
        fb = ev(lv + 2.0 * t1 * d, False)["E"]
        c2, c3 = _fit_cubic(o["E"], slope, t1, fa, fb)
        t = _cubic_min(slope, c2, c3, 2.0 * t1)
        if t < 1e-8 * t_ref:
            break
        lv = lv + t * d
        t_prev = t
        g_old, gg_old = g, gg
    return csr(rp, col, lv), np.array(hist)
