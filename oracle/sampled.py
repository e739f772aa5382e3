"""Gradient rows of the LNV energy from the dense definition, for a few atoms.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For systems too large for a full oracle evaluation, this forms the rows of
chosen atoms of

    G = dE/dL = 6 (SLH + HLS) - 4 (SLSLH + SLHLS + HLSLS)        (Sec. 2, Eq. 3)
    GN = dN_e/dL = 12 (SLS - SLSLS)

straight from their definition as matrix products: each row block is carried
left to right through the chain (rows of S L, then S L S, ...), every step a
sparse product of those rows with a whole input matrix (scipy.sparse, FP64),
with no mask and no range.  The result is then read on L's pattern.  The
scalar matrices are the block matrices over atoms (one block per ordered atom
pair, as the block-CSR input gives them).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _scalar(M: dict):
    """Block-CSR dict -> scalar CSR matrix of size (n nsf) x (n nsf)."""
    n = M["rp"].size - 1
    nsf = M["val"].shape[-1]
    return sp.bsr_matrix((M["val"], M["col"], M["rp"]), shape=(n * nsf, n * nsf)).tocsr()


def lnv_grad_rows(S: dict, H: dict, L: dict, atoms) -> dict:
    """Rows ``atoms`` of G and GN on L's pattern.

    Returns {"atoms": int64[m], "pos": int64[p] (positions of those rows'
    blocks in L's block arrays, row by row), "G": float64[p, nsf, nsf],
    "GN": float64[p, nsf, nsf]}.
    """
    atoms = np.asarray(atoms, dtype=np.int64)
    nsf = L["val"].shape[-1]
    Ss, Hs, Ls = _scalar(S), _scalar(H), _scalar(L)
    idx = (atoms[:, None] * nsf + np.arange(nsf)[None, :]).ravel()
    s0, h0 = Ss[idx], Hs[idx]
    SL, HL = s0 @ Ls, h0 @ Ls
    SLH, SLS, HLS = SL @ Hs, SL @ Ss, HL @ Ss
    SLSL = SLS @ Ls
    SLSLH = SLSL @ Hs
    SLSLS = SLSL @ Ss
    SLHLS = (SLH @ Ls) @ Ss
    HLSLS = (HLS @ Ls) @ Ss
    G = (6.0 * (SLH + HLS) - 4.0 * (SLSLH + SLHLS + HLSLS)).toarray()
    GN = (12.0 * (SLS - SLSLS)).toarray()
    pos, gb, nb = [], [], []
    for r, a in enumerate(atoms):
        rows = slice(r * nsf, (r + 1) * nsf)
        for q in range(int(L["rp"][a]), int(L["rp"][a + 1])):
            j = int(L["col"][q])
            cols = slice(j * nsf, (j + 1) * nsf)
            pos.append(q)
            gb.append(G[rows, cols])
            nb.append(GN[rows, cols])
    return {"atoms": atoms, "pos": np.asarray(pos, dtype=np.int64),
            "G": np.asarray(gb).reshape(-1, nsf, nsf), "GN": np.asarray(nb).reshape(-1, nsf, nsf)}
