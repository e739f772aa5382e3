"""Synthetic bulk-Si inputs for the LNV energy/gradient path.

The paper measures bulk silicon (Sec. 3, Fig. 2 and Fig. 3 / Table 1), with
real NSC-AITB Hamiltonians that are not reproducible here.  These generators
stand in for them: a jittered diamond lattice and random, range-limited,
symmetric block matrices S (overlap), H (Hamiltonian) and L (auxiliary density
matrix) with the envelopes below.

Recipe (seeded, all FP64):

* positions: conventional diamond cells of side a = 5.43 A, n x n x n of them,
  atom index = ((cx*n + cy)*n + cz)*8 + b for basis atom b; Gaussian jitter of
  sigma = 0.05 A per Cartesian component, then wrapped into [0, n*a).
* a symmetric matrix M on a symmetric block pattern (CSR over atoms, columns
  sorted, diagonal present): the diagonal block is a fixed matrix; every
  unordered pair i < j of the pattern, in lexicographic order, draws one
  NSF x NSF block of standard normals (row-major), scaled by amp*exp(-d/decay)
  with d the minimum-image distance; block (j, i) is its transpose.
* draw order from one numpy ``default_rng(seed)`` stream: jitter, then S pairs,
  then H pairs, then L pairs.

The block pattern is an input here: the caller builds it (with the oracle or
with the CUDA library, whose patterns are checked to be identical) and passes
it in, so this module does no neighbour search of its own.  The distance used
for the envelope is input-generation arithmetic only.
"""
from __future__ import annotations

import numpy as np

SI_A = 5.43  # conventional cubic lattice constant of Si, Angstrom

_DIAMOND_BASIS = np.array(
    [
        [0.0, 0.0, 0.0],
        [0.0, 0.5, 0.5],
        [0.5, 0.0, 0.5],
        [0.5, 0.5, 0.0],
        [0.25, 0.25, 0.25],
        [0.25, 0.75, 0.75],
        [0.75, 0.25, 0.75],
        [0.75, 0.75, 0.25],
    ]
)


def si_diamond_positions(n: int, rng: np.random.Generator | None, a: float = SI_A,
                         sigma: float = 0.05):
    """Jittered diamond lattice of n^3 conventional cells.

    Returns (pos [N,3] float64, cell [3] float64).  ``rng=None`` gives the
    perfect lattice (no draws).
    """
    c = np.stack(np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"), -1)
    c = c.reshape(-1, 1, 3).astype(np.float64)
    pos = ((c + _DIAMOND_BASIS[None]) * a).reshape(-1, 3)
    if rng is not None and sigma > 0:
        pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    box = n * a
    pos = np.mod(pos, box)
    pos[pos >= box] -= box  # np.mod of a tiny negative can round up to box
    cell = np.array([box, box, box], dtype=np.float64)
    return np.ascontiguousarray(pos), cell


def _min_image_dist(dvec: np.ndarray, cell: np.ndarray) -> np.ndarray:
    d = dvec - cell * np.rint(dvec / cell)
    return np.sqrt((d * d).sum(axis=-1))


def diag_block(kind: str, nsf: int) -> np.ndarray:
    """Fixed on-site blocks: S = I, L = 0.5 I, H = diag(-0.5, 0.2 x3, 0.6 x5)."""
    if kind == "S":
        return np.eye(nsf)
    if kind == "L":
        return 0.5 * np.eye(nsf)
    if kind == "H":
        d = [-0.5] + [0.2] * 3 + [0.6] * 5
        if nsf > len(d):
            d = d + [0.6] * (nsf - len(d))
        return np.diag(np.array(d[:nsf]))
    raise ValueError(kind)


ENVELOPE = {  # kind -> (amplitude, decay length in Angstrom)
    "S": (0.08, 1.5),
    "H": (0.3, 1.2),
    "L": (0.02, 2.0),
}


def sym_block_values(row_ptr: np.ndarray, col: np.ndarray, pos: np.ndarray,
                     cell: np.ndarray, nsf: int, kind: str,
                     rng: np.random.Generator) -> np.ndarray:
    """Random symmetric block matrix on a given symmetric block pattern.

    Returns values [nnzb, nsf, nsf] float64 in the pattern's block order.
    """
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = row_ptr.size - 1
    nnz = int(row_ptr[-1])
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    amp, decay = ENVELOPE[kind]
    vals = np.zeros((nnz, nsf, nsf), dtype=np.float64)
    upper = np.nonzero(col > rows)[0]
    iu, ju = rows[upper], col[upper]
    d = _min_image_dist(pos[ju] - pos[iu], cell)
    blocks = rng.standard_normal((upper.size, nsf, nsf))
    blocks *= (amp * np.exp(-d / decay))[:, None, None]
    vals[upper] = blocks
    key = rows * n + col  # sorted: rows ascending, columns ascending per row
    lower = np.searchsorted(key, ju * n + iu)
    if lower.size and not np.array_equal(key[np.minimum(lower, nnz - 1)], ju * n + iu):
        raise ValueError("block pattern is not symmetric")
    vals[lower] = blocks.transpose(0, 2, 1)
    dpos = np.nonzero(col == rows)[0]
    if dpos.size != n:
        raise ValueError("block pattern must hold every diagonal block")
    vals[dpos] = diag_block(kind, nsf)
    return vals


def si_workload(ncell: int, nsf: int, r_sh: float, r_l: float, seed: int, pattern_fn,
                sigma: float = 0.05, displace=None):
    """Positions plus S, H (range r_sh) and L (range r_l) for one Si supercell.

    ``pattern_fn(pos, cell, cutoff) -> (row_ptr, col)`` builds the block
    pattern {(i, j): d_ij^2 < cutoff^2}; it is supplied by the caller.
    ``displace`` (N x 3, Angstrom) moves the atoms after the jitter is drawn
    and before the values are: with the same seed, values then follow the
    new distances smoothly wherever the patterns do not change (a step of a
    geometry optimisation or of molecular dynamics).
    Returns a dict with pos, cell, the two patterns and S, H, L values.
    """
    rng = np.random.default_rng(seed)
    pos, cell = si_diamond_positions(ncell, rng, sigma=sigma)
    if displace is not None:
        pos = np.mod(pos + np.asarray(displace, np.float64), cell)
        pos[pos >= cell] -= cell[np.nonzero(pos >= cell)[1]]
    rp_sh, col_sh = pattern_fn(pos, cell, r_sh)
    rp_l, col_l = pattern_fn(pos, cell, r_l)
    S = sym_block_values(rp_sh, col_sh, pos, cell, nsf, "S", rng)
    H = sym_block_values(rp_sh, col_sh, pos, cell, nsf, "H", rng)
    L = sym_block_values(rp_l, col_l, pos, cell, nsf, "L", rng)
    return {
        "pos": pos, "cell": cell, "nsf": nsf, "r_sh": r_sh, "r_l": r_l,
        "sh_row_ptr": np.asarray(rp_sh, np.int64), "sh_col": np.asarray(col_sh, np.int32),
        "l_row_ptr": np.asarray(rp_l, np.int64), "l_col": np.asarray(col_l, np.int32),
        "S": S, "H": H, "L": L,
    }


def batch_cell_counts(n_sys: int = 64, lo: int = 2, hi: int = 10, seed: int = 0):
    """Cell counts n_s (cubic n_s^3 supercells) for the many-system batch."""
    rng = np.random.default_rng(seed)
    return [int(x) for x in rng.integers(lo, hi + 1, size=n_sys)]
