"""Dense numpy helpers used to pin the oracle on small inputs (tests only)."""
import numpy as np


def to_dense(rp, col, val):
    """Block-CSR -> dense (n*nsf) x (n*nsf) matrix."""
    rp = np.asarray(rp)
    n = rp.size - 1
    nsf = val.shape[-1]
    D = np.zeros((n * nsf, n * nsf))
    rows = np.repeat(np.arange(n), np.diff(rp))
    for p, (i, j) in enumerate(zip(rows, np.asarray(col))):
        D[i * nsf:(i + 1) * nsf, j * nsf:(j + 1) * nsf] = val[p]
    return D


def from_dense(D, rp, col, nsf):
    """Dense -> blocks on the given pattern."""
    rp = np.asarray(rp)
    n = rp.size - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    out = np.empty((len(col), nsf, nsf))
    for p, (i, j) in enumerate(zip(rows, np.asarray(col))):
        out[p] = D[i * nsf:(i + 1) * nsf, j * nsf:(j + 1) * nsf]
    return out


def mask_dense(rp, col, nsf):
    rp = np.asarray(rp)
    n = rp.size - 1
    return to_dense(rp, col, np.ones((len(col), nsf, nsf)))


def lnv_dense(S, H, L):
    """Eq. 3 and the energy / electron count / gradient, densely."""
    LS = L @ S
    K = 3 * LS @ L - 2 * LS @ LS @ L
    E = 2 * np.trace(K @ H)
    Ne = 2 * np.trace(K @ S)
    G = 6 * (S @ L @ H + H @ L @ S) - 4 * (S @ L @ S @ L @ H + S @ L @ H @ L @ S + H @ L @ S @ L @ S)
    return E, Ne, G, K


def ne_grad_dense(S, L):
    """dN_e/dL = 12 (SLS - SLSLS) for N_e = 2 Tr[KS], densely."""
    SLS = S @ L @ S
    return 12 * (SLS - SLS @ L @ S)


def random_blocks(rng, nnz, nsf):
    return rng.standard_normal((nnz, nsf, nsf))
