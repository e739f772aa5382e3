"""Shared helpers of the GPU parity tests (tests only)."""
import numpy as np
import torch

import oracle
import synth


def rel_fro(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (d if d > 0 else 1.0)


def workload(ncell, nsf, r_sh, r_l, seed=0):
    """Seeded Si workload plus its oracle matrices (patterns from the oracle)."""
    w = synth.si_workload(ncell, nsf, r_sh, r_l, seed, oracle.pattern)
    S = oracle.csr(w["sh_row_ptr"], w["sh_col"], w["S"])
    H = oracle.csr(w["sh_row_ptr"], w["sh_col"], w["H"])
    L = oracle.csr(w["l_row_ptr"], w["l_col"], w["L"])
    return w, S, H, L


def to_dev(a, dtype, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev, dtype)


def oracle_lnv(w, S, H, L, grad=True):
    return oracle.lnv_energy_grad(w["pos"], w["cell"], w["r_sh"], w["r_l"], S, H, L, grad=grad,
                                  grad_ne=grad)


def rounded(M, dtype):
    """Oracle matrix whose values are those of the GPU inputs in `dtype`."""
    if dtype == torch.float64:
        return M
    return oracle.csr(M["rp"], M["col"], M["val"].astype(np.float32).astype(np.float64))
