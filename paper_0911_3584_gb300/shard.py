"""Work distribution of the LNV evaluation over ranks (one GPU each).

The paper distributes atoms over cores in spatially compact partitions and
exchanges the matrix rows each product needs between them (Sec. 2,
partitions and bundles; Sec. 3, scaling studies).  Two forms are provided:

* Independent systems (the batched workload): whole systems per rank,
  assigned by their work (longest processing time first).  No data moves
  between ranks; the per-system scalars are gathered at the end.

* One large system: the atoms (block rows) are split into spatially compact
  parts, one per rank.  A masked product C = mask_C(A B) restricted to a
  rank's rows I reads A's rows I (local) and the rows of B indexed by the
  columns of those rows of A: the rows outside I among them are the halo,
  fetched from their owners before the product (point-to-point, one message
  per peer, only values: every rank holds every pattern).  A trace Tr[A B]
  over rows I reads the blocks B_ji for the columns j of A's rows: the halo
  of A's pattern again.  The traces then need one all-reduce of four
  scalars; the gradient is row-local.

The distribution logic here is independent of where the local products run:
``lnv_partitioned`` takes the local product and trace as callables on
block-CSR dicts ({"rp", "col", "val"}, full-size, valid on the rows the rank
holds), so the same code runs on CPU ranks (the tests) or around a GPU
product.
"""
from __future__ import annotations

from typing import Callable, Sequence

import numpy as np

# ---------------------------------------------------------------- independent systems


def assign_lpt(work: Sequence[float], n_ranks: int) -> list[list[int]]:
    """Whole systems to ranks, longest processing time first: systems in order
    of decreasing work (ties: lower index first), each to the currently least
    loaded rank (ties: lower rank).  Deterministic, so every rank computes the
    same assignment.  Returns each rank's system indices, ascending."""
    if n_ranks < 1:
        raise ValueError("n_ranks must be >= 1")
    load = [0.0] * n_ranks
    out: list[list[int]] = [[] for _ in range(n_ranks)]
    for s in sorted(range(len(work)), key=lambda i: (-float(work[i]), i)):
        r = min(range(n_ranks), key=lambda q: (load[q], q))
        out[r].append(s)
        load[r] += float(work[s])
    return [sorted(x) for x in out]


def lpt_loads(work: Sequence[float], assignment: list[list[int]]) -> list[float]:
    return [float(sum(work[i] for i in a)) for a in assignment]


# ---------------------------------------------------------------- one system, row parts


def row_parts(order: np.ndarray, n_ranks: int) -> list[np.ndarray]:
    """Split atoms, taken in `order` (a spatial order: consecutive atoms are
    neighbours, e.g. the cell order of the lattice or a space-filling curve),
    into n_ranks contiguous runs of near-equal size; each part sorted."""
    order = np.asarray(order, dtype=np.int64)
    bounds = np.linspace(0, order.size, n_ranks + 1).round().astype(np.int64)
    return [np.sort(order[bounds[r]:bounds[r + 1]]) for r in range(n_ranks)]


def owner_of(parts: list[np.ndarray], n: int) -> np.ndarray:
    own = np.full(n, -1, dtype=np.int64)
    for r, p in enumerate(parts):
        own[p] = r
    if (own < 0).any():
        raise ValueError("the parts do not cover every row")
    return own


def halo_rows(rp: np.ndarray, col: np.ndarray, owned: np.ndarray) -> np.ndarray:
    """Columns of the pattern's owned rows that are not owned: the rows of the
    right operand a rank must fetch before a product (or a trace) over its
    rows.  Sorted, unique."""
    rp = np.asarray(rp)
    owned = np.asarray(owned, dtype=np.int64)
    if owned.size == 0:
        return np.zeros(0, dtype=np.int64)
    cols = np.concatenate([np.asarray(col[rp[i]:rp[i + 1]], dtype=np.int64) for i in owned])
    return np.setdiff1d(np.unique(cols), owned)


class RowExchange:
    """Point-to-point exchange of block rows of a matrix whose pattern every
    rank knows (torch.distributed: gloo on CPU, NCCL on GPUs): each rank sends
    its peers the values of the owned rows they asked for.  Counts the values
    it receives (``received``)."""

    def __init__(self, dist, parts: list[np.ndarray], n: int):
        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()
        self.parts = parts
        self.owner = owner_of(parts, n)
        self.received = 0

    def fetch(self, M: dict, need: np.ndarray) -> None:
        """Fill M["val"] on the rows `need` (not owned here) from their owners."""
        import torch

        dist = self.dist
        needs: list = [None] * self.world
        dist.all_gather_object(needs, np.asarray(need, dtype=np.int64).tolist())
        rp, val = M["rp"], M["val"]
        blk = val.shape[1:]
        reqs, recv = [], []
        for q in range(self.world):
            if q == self.rank:
                continue
            give = [i for i in needs[q] if self.owner[i] == self.rank]
            take = [i for i in needs[self.rank] if self.owner[i] == q]
            if give:
                buf = np.concatenate([val[rp[i]:rp[i + 1]] for i in give]).reshape(-1)
                t = torch.from_numpy(np.ascontiguousarray(buf))
                reqs.append((dist.isend(t, dst=q), t))
            if take:
                cnt = int(sum(rp[i + 1] - rp[i] for i in take))
                t = torch.empty(cnt * int(np.prod(blk)), dtype=torch.from_numpy(val[:0]).dtype)
                reqs.append((dist.irecv(t, src=q), t))
                recv.append((take, t))
        for req, _ in reqs:
            req.wait()
        for take, t in recv:
            a = t.numpy().reshape((-1,) + blk)
            off = 0
            for i in take:
                nb = int(rp[i + 1] - rp[i])
                val[rp[i]:rp[i + 1]] = a[off:off + nb]
                off += nb
            self.received += a.size


def local_rows(M: dict, owned: np.ndarray) -> dict:
    """Copy of M holding only the owned rows' values (zeros elsewhere): what a
    rank starts from."""
    out = {"rp": M["rp"], "col": M["col"], "val": np.zeros_like(M["val"])}
    for i in owned:
        out["val"][M["rp"][i]:M["rp"][i + 1]] = M["val"][M["rp"][i]:M["rp"][i + 1]]
    return out


def lnv_partitioned(dist, parts: list[np.ndarray], pattern: Callable, pos, cell, r_sh: float, r_l: float,
                    S: dict, H: dict, L: dict, product: Callable, trace: Callable) -> dict:
    """E, N_e and this rank's rows of dE/dL, with the atoms split into `parts`.

    S, H (range r_sh) and L (range r_l) hold valid values on this rank's rows.
    Each masked product below is formed on the rank's rows after fetching its
    halo; the association is the plain one (every term of the gradient its own
    masked product onto L's pattern, as in Eq. 3's expansion):
      X = L S, Y = L H (range r_l + r_sh), T = S X, U = S Y (r_l + 2 r_sh),
      Z = L T (r_l + r_sh), E = 2 (3 Tr[XY] - 2 Tr[ZY]),
      N_e = 2 (3 Tr[XX] - 2 Tr[ZX]),
      G = 6 (S Y + H X) - 4 (T Y + U X + H Z) on L's pattern.
    `product(A, B, C_pat, rows)` forms rows `rows` of mask_{C_pat}(A B);
    `trace(A, B, rows)` is the partial trace over `rows`; `pattern(pos, cell,
    R)` the range pattern.  Returns {"E", "Ne", "G" (full-size array, this
    rank's rows valid), "halo_rows" (rows fetched per product)}.
    """
    import torch

    rank = dist.get_rank()
    mine = np.asarray(parts[rank], dtype=np.int64)
    n = L["rp"].size - 1
    ex = RowExchange(dist, parts, n)
    pat_x = pattern(pos, cell, r_l + r_sh)
    pat_t = pattern(pos, cell, r_l + 2.0 * r_sh)
    pat_l = (L["rp"], L["col"])
    fetched: dict = {}

    def prod(name, A, B, pat):
        need = halo_rows(A["rp"], A["col"], mine)
        ex.fetch(B, need)
        fetched[name] = need.size
        return product(A, B, pat, mine)

    def tr(A, B):
        ex.fetch(B, halo_rows(A["rp"], A["col"], mine))
        return trace(A, B, mine)

    X = prod("X", L, S, pat_x)
    Y = prod("Y", L, H, pat_x)
    T = prod("T", S, X, pat_t)
    Z = prod("Z", L, T, pat_x)
    part = torch.tensor([tr(X, Y), tr(Z, Y), tr(X, X), tr(Z, X)], dtype=torch.float64)
    dist.all_reduce(part)
    t1, t2, n1, n2 = (float(v) for v in part)
    U = prod("U", S, Y, pat_t)
    slh = prod("SLH", S, Y, pat_l)
    hls = prod("HLS", H, X, pat_l)
    slslh = prod("SLSLH", T, Y, pat_l)
    slhls = prod("SLHLS", U, X, pat_l)
    hlsls = prod("HLSLS", H, Z, pat_l)
    G = 6.0 * (slh["val"] + hls["val"]) - 4.0 * (slslh["val"] + slhls["val"] + hlsls["val"])
    return {"E": 2.0 * (3.0 * t1 - 2.0 * t2), "Ne": 2.0 * (3.0 * n1 - 2.0 * n2), "G": G,
            "halo_rows": fetched, "values_received": ex.received}
