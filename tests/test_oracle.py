"""Pins of the FP64 CPU oracle against things other than itself.

Each check targets a plausible mistake: a dropped or mis-signed term, a wrong
index, a transposed operand, a wrong range rule.  References are the dense
definition (numpy on small systems), closed forms, crystallographic counts,
a library neighbour search, exact finite differences of a cubic, and the
paper's constant energy per atom.
"""
import os

import numpy as np
import pytest

import oracle
import synth
from tests.dense_ref import from_dense, lnv_dense, mask_dense, ne_grad_dense, to_dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _si(ncell, nsf, r_sh, r_l, seed=0, sigma=0.05):
    w = synth.si_workload(ncell, nsf, r_sh, r_l, seed, oracle.pattern, sigma=sigma)
    S = oracle.csr(w["sh_row_ptr"], w["sh_col"], w["S"])
    H = oracle.csr(w["sh_row_ptr"], w["sh_col"], w["H"])
    L = oracle.csr(w["l_row_ptr"], w["l_col"], w["L"])
    return w, S, H, L


# ---------------------------------------------------------------- patterns

def _golden_shells():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "diamond_shells.txt"))
            if ln.strip() and not ln.startswith("#")]
    return [(int(a), int(b)) for a, b in rows]


@pytest.mark.parametrize("cutoff", [2.5, 4.0, 6.6, 8.0])
def test_pattern_ideal_lattice_shell_counts(cutoff):
    """Ideal diamond lattice: every row holds exactly the shells inside R."""
    pos, cell = synth.si_diamond_positions(4, None)  # 21.72 A box: no image folding at R <= 8
    rp, col = oracle.pattern(pos, cell, cutoff)
    unit2 = (synth.SI_A / 4.0) ** 2
    expect = sum(c for r2, c in _golden_shells() if r2 * unit2 < cutoff * cutoff)
    counts = np.diff(rp)
    assert np.all(counts == expect), (cutoff, expect, np.unique(counts))


def test_pattern_matches_kdtree_periodic():
    """Jittered lattice vs scipy's periodic k-d tree (an unrelated algorithm)."""
    spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(3)
    pos, cell = synth.si_diamond_positions(3, rng)
    for R in (3.0, 6.6, 7.9):
        rp, col = oracle.pattern(pos, cell, R)
        tree = spatial.cKDTree(pos, boxsize=cell)
        pairs = tree.query_pairs(R, output_type="ndarray")
        n = pos.shape[0]
        ref = np.zeros((n, n), bool)
        ref[pairs[:, 0], pairs[:, 1]] = True
        ref[pairs[:, 1], pairs[:, 0]] = True
        ref[np.arange(n), np.arange(n)] = True
        got = np.zeros((n, n), bool)
        got[np.repeat(np.arange(n), np.diff(rp)), col] = True
        assert np.array_equal(got, ref)


def test_pattern_sorted_symmetric_with_diagonal():
    w, S, H, L = _si(2, 1, 6.6, 8.0)
    for rp, col in ((S["rp"], S["col"]), (L["rp"], L["col"])):
        n = rp.size - 1
        for i in range(n):
            c = col[rp[i]:rp[i + 1]]
            assert np.all(np.diff(c) > 0)
            assert i in c
        d = mask_dense(rp, col, 1)
        assert np.array_equal(d, d.T)


def test_pattern_small_cell_is_dense():
    """Ranges beyond half the box: minimum image keeps one block per pair."""
    pos, cell = synth.si_diamond_positions(2, np.random.default_rng(1))
    rp, col = oracle.pattern(pos, cell, 21.2)
    assert np.all(np.diff(rp) == pos.shape[0])


# ---------------------------------------------------------------- products

@pytest.mark.parametrize("nsf", [1, 2, 4, 9])
@pytest.mark.parametrize("ranges", [(4.0, 6.6, 8.0), (6.6, 8.0, 3.0), (8.0, 6.6, 30.0)])
def test_mprod_equals_masked_dense_product(nsf, ranges):
    """mask(A B) against dense A @ B then masking; non-symmetric values so a
    transposed operand or a swapped index cannot pass."""
    ra, rb, rc = ranges
    rng = np.random.default_rng(nsf)
    pos, cell = synth.si_diamond_positions(2 if nsf < 9 else 1, rng)
    pa, pb, pc = (oracle.pattern(pos, cell, r) for r in (ra, rb, rc))
    A = oracle.csr(*pa, rng.standard_normal((pa[1].size, nsf, nsf)))
    B = oracle.csr(*pb, rng.standard_normal((pb[1].size, nsf, nsf)))
    C = oracle.mprod(A, B, pc)
    dense = to_dense(A["rp"], A["col"], A["val"]) @ to_dense(B["rp"], B["col"], B["val"])
    ref = from_dense(dense, pc[0], pc[1], nsf)
    np.testing.assert_allclose(C["val"], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_mprod_empty_rows_and_missing_blocks():
    """Rows of A without entries give zero rows of C."""
    rng = np.random.default_rng(5)
    n, nsf = 5, 2
    a_rp = np.array([0, 1, 1, 3, 3, 4])
    a_col = np.array([2, 0, 4, 1], np.int32)
    b_rp = np.array([0, 2, 3, 3, 4, 5])
    b_col = np.array([0, 3, 1, 2, 4], np.int32)
    c_rp = np.array([0, 5, 10, 15, 20, 25])
    c_col = np.tile(np.arange(5, dtype=np.int32), 5)
    A = oracle.csr(a_rp, a_col, rng.standard_normal((4, nsf, nsf)))
    B = oracle.csr(b_rp, b_col, rng.standard_normal((5, nsf, nsf)))
    C = oracle.mprod(A, B, (c_rp, c_col))
    ref = to_dense(a_rp, a_col, A["val"]) @ to_dense(b_rp, b_col, B["val"])
    np.testing.assert_allclose(to_dense(c_rp, c_col, C["val"]), ref, atol=1e-14)
    assert np.all(C["val"][5:10] == 0)


def test_trace_equals_dense_and_is_cyclic():
    rng = np.random.default_rng(7)
    pos, cell = synth.si_diamond_positions(2, rng)
    p = oracle.pattern(pos, cell, 6.0)
    for nsf in (1, 3, 4):
        A = oracle.csr(*p, rng.standard_normal((p[1].size, nsf, nsf)))
        B = oracle.csr(*p, rng.standard_normal((p[1].size, nsf, nsf)))
        Ad, Bd = to_dense(p[0], p[1], A["val"]), to_dense(p[0], p[1], B["val"])
        t = oracle.trace(A, B)
        assert t == pytest.approx(np.trace(Ad @ Bd), rel=1e-13)
        assert t == pytest.approx(oracle.trace(B, A), rel=1e-13)


def test_transpose_and_restrict():
    rng = np.random.default_rng(8)
    pos, cell = synth.si_diamond_positions(2, rng)
    p8, p4 = oracle.pattern(pos, cell, 8.0), oracle.pattern(pos, cell, 4.0)
    M = oracle.csr(*p8, rng.standard_normal((p8[1].size, 3, 3)))
    Md = to_dense(p8[0], p8[1], M["val"])
    Mt = oracle.transpose(M)
    np.testing.assert_array_equal(to_dense(p8[0], p8[1], Mt["val"]), Md.T)
    R = oracle.restrict(M, p4)
    np.testing.assert_array_equal(to_dense(p4[0], p4[1], R["val"]), Md * mask_dense(p4[0], p4[1], 3))


# ---------------------------------------------------------------- LNV energy / gradient

def _check_against_dense(w, S, H, L, rtol=1e-12):
    nsf = w["nsf"]
    out = oracle.lnv_energy_grad(w["pos"], w["cell"], w["r_sh"], w["r_l"], S, H, L, grad_ne=True)
    Sd = to_dense(S["rp"], S["col"], S["val"])
    Hd = to_dense(H["rp"], H["col"], H["val"])
    Ld = to_dense(L["rp"], L["col"], L["val"])
    E, Ne, G, _ = lnv_dense(Sd, Hd, Ld)
    assert out["E"] == pytest.approx(E, rel=rtol, abs=1e-12)
    assert out["Ne"] == pytest.approx(Ne, rel=rtol)
    Gref = from_dense(G, L["rp"], L["col"], nsf)
    err = np.linalg.norm(out["G"] - Gref) / np.linalg.norm(Gref)
    assert err < rtol
    GNref = from_dense(ne_grad_dense(Sd, Ld), L["rp"], L["col"], nsf)
    err = np.linalg.norm(out["GN"] - GNref) / np.linalg.norm(GNref)
    assert err < rtol
    return out


@pytest.mark.parametrize("ncell,nsf,r_sh,r_l", [(1, 1, 4.0, 5.0), (2, 2, 4.0, 5.0),
                                                (2, 4, 6.6, 8.0), (2, 9, 3.0, 4.0),
                                                (3, 4, 3.0, 4.5)])
def test_lnv_matches_dense_definition_small(ncell, nsf, r_sh, r_l):
    w, S, H, L = _si(ncell, nsf, r_sh, r_l, seed=ncell * 10 + nsf)
    _check_against_dense(w, S, H, L)


def test_lnv_matches_dense_definition_512_atoms():
    """The whole 4x4x4-cell workload (512 atoms, NSF=4, R_L = 8 A) densely."""
    w, S, H, L = _si(4, 4, 6.6, 8.0, seed=0)
    out = _check_against_dense(w, S, H, L)
    assert 0.0 < out["Ne"]


def test_overlap_is_positive_definite():
    w, S, H, L = _si(4, 4, 6.6, 8.0, seed=0)
    Sd = to_dense(S["rp"], S["col"], S["val"])
    np.linalg.cholesky(Sd)
    assert np.allclose(Sd, Sd.T)


@pytest.mark.parametrize("ncell,nsf", [(8, 4), (4, 9)])
def test_overlap_is_positive_definite_at_benchmark_sizes(ncell, nsf):
    """S of the 4096-atom benchmark workload (and of an NSF = 9 system) is
    symmetric and positive definite: its smallest eigenvalue, from Lanczos on
    the sparse matrix, is bounded away from zero.  Diagonal dominance alone
    does not guarantee it for every row."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla

    w, S, H, L = _si(ncell, nsf, 6.6, 8.0, seed=0)
    n = (len(S["rp"]) - 1) * nsf
    M = sp.bsr_matrix((S["val"], S["col"], S["rp"]), shape=(n, n)).tocsr()
    assert abs(M - M.T).max() == 0.0
    lam = sla.eigsh(M, k=1, which="SA", return_eigenvectors=False, tol=1e-8)[0]
    assert lam > 0.5, lam


# ---------------------------------------------------------------- sampled gradient rows

@pytest.mark.parametrize("ncell,nsf,r_sh,r_l", [(2, 4, 6.6, 8.0), (2, 9, 4.0, 5.0), (1, 4, 5.0, 5.0)])
def test_sampled_gradient_rows_match_dense_definition(ncell, nsf, r_sh, r_l):
    """The row-chain gradient (oracle/sampled.py) equals the dense definition
    of G and dN_e/dL, read on L's pattern, for chosen atoms."""
    from oracle.sampled import lnv_grad_rows

    w, S, H, L = _si(ncell, nsf, r_sh, r_l, seed=4)
    Sd, Hd, Ld = (to_dense(M["rp"], M["col"], M["val"]) for M in (S, H, L))
    _, _, Gd, _ = lnv_dense(Sd, Hd, Ld)
    G = from_dense(Gd, L["rp"], L["col"], nsf)
    GN = from_dense(ne_grad_dense(Sd, Ld), L["rp"], L["col"], nsf)
    n = L["rp"].size - 1
    r = lnv_grad_rows(S, H, L, [0, n // 2, n - 1])
    assert np.array_equal(r["pos"], np.concatenate([np.arange(L["rp"][a], L["rp"][a + 1]) for a in (0, n // 2, n - 1)]))
    assert np.linalg.norm(r["G"] - G[r["pos"]]) <= 1e-12 * np.linalg.norm(G[r["pos"]])
    assert np.linalg.norm(r["GN"] - GN[r["pos"]]) <= 1e-12 * np.linalg.norm(GN[r["pos"]])


def test_sampled_gradient_rows_match_full_oracle_512_atoms():
    """On the 512-atom workload (too large to form densely here), the row
    chain and the masked-product plan agree on sampled rows."""
    from oracle.sampled import lnv_grad_rows

    w, S, H, L = _si(4, 4, 6.6, 8.0, seed=0)
    ref = oracle.lnv_energy_grad(w["pos"], w["cell"], 6.6, 8.0, S, H, L, grad=True, grad_ne=True)
    r = lnv_grad_rows(S, H, L, [3, 200, 511])
    g, gn = ref["G"][r["pos"]], ref["GN"][r["pos"]]
    assert np.linalg.norm(r["G"] - g) <= 1e-12 * np.linalg.norm(g)
    assert np.linalg.norm(r["GN"] - gn) <= 1e-12 * np.linalg.norm(gn)


def _dense_system(nsf=4, seed=11):
    """One 8-atom cell with every range past the box: all matrices dense."""
    w, S, H, L = _si(1, nsf, 5.0, 5.0, seed=seed)
    assert np.all(np.diff(L["rp"]) == 8)
    return w, S, H, L


@pytest.mark.parametrize("c", [1.0, 0.5, 0.8])
def test_closed_form_scaled_inverse_overlap(c):
    """L = c S^-1 gives K = (3c^2 - 2c^3) S^-1, N_e = 2 (3c^2 - 2c^3) N NSF,
    E = 2 (3c^2 - 2c^3) Tr[S^-1 H], G = 12 (c - c^2) H and dN_e/dL =
    12 (c - c^2) S."""
    w, S, H, L = _dense_system()
    Sd = to_dense(S["rp"], S["col"], S["val"])
    Hd = to_dense(H["rp"], H["col"], H["val"])
    Linv = c * np.linalg.inv(Sd)
    L = oracle.csr(L["rp"], L["col"], from_dense(Linv, L["rp"], L["col"], 4))
    out = oracle.lnv_energy_grad(w["pos"], w["cell"], 5.0, 5.0, S, H, L, grad_ne=True)
    f = 3 * c * c - 2 * c ** 3
    assert out["Ne"] == pytest.approx(2 * f * Sd.shape[0], rel=1e-12)
    assert out["E"] == pytest.approx(2 * f * np.trace(np.linalg.solve(Sd, Hd)), rel=1e-12)
    Gref = from_dense(12 * (c - c * c) * Hd, L["rp"], L["col"], 4)
    assert np.abs(out["G"] - Gref).max() < 1e-12 * max(1.0, np.abs(Hd).max())
    GNref = from_dense(12 * (c - c * c) * Sd, L["rp"], L["col"], 4)
    assert np.abs(out["GN"] - GNref).max() < 1e-12 * max(1.0, np.abs(Sd).max())


@pytest.mark.parametrize("m", [5, 16])
def test_closed_form_ground_state_projector(m):
    """L = C C^T from the m lowest generalised eigenvectors of (H, S): K = L,
    N_e = 2m, E = 2 sum(eps_1..m), and both gradients vanish."""
    linalg = pytest.importorskip("scipy.linalg")
    w, S, H, L = _dense_system(seed=12)
    Sd = to_dense(S["rp"], S["col"], S["val"])
    Hd = to_dense(H["rp"], H["col"], H["val"])
    eps, C = linalg.eigh(Hd, Sd)
    Cm = C[:, :m]
    Ld = Cm @ Cm.T
    L = oracle.csr(L["rp"], L["col"], from_dense(Ld, L["rp"], L["col"], 4))
    out = oracle.lnv_energy_grad(w["pos"], w["cell"], 5.0, 5.0, S, H, L, grad_ne=True)
    assert out["Ne"] == pytest.approx(2 * m, rel=1e-11)
    assert out["E"] == pytest.approx(2 * eps[:m].sum(), rel=1e-11, abs=1e-11)
    assert np.abs(out["G"]).max() < 1e-11
    assert np.abs(out["GN"]).max() < 1e-11


def test_single_atom_scalar_polynomial():
    """NSF = 1, one atom: E = 2h(3 l^2 s - 2 l^3 s^2), N_e = 2(3 l^2 s^2 - 2 l^3 s^3),
    dE/dl = 2h(6 l s - 6 l^2 s^2), dN_e/dl = 2(6 l s^2 - 6 l^2 s^3)."""
    s, h, l = 1.3, -0.7, 0.45
    rp, col = np.array([0, 1]), np.array([0], np.int32)
    S = oracle.csr(rp, col, np.array([[[s]]]))
    H = oracle.csr(rp, col, np.array([[[h]]]))
    L = oracle.csr(rp, col, np.array([[[l]]]))
    out = oracle.lnv_energy_grad(np.zeros((1, 3)), np.array([10.0, 10.0, 10.0]), 3.0, 3.0, S, H, L,
                                 grad_ne=True)
    assert out["E"] == pytest.approx(2 * h * (3 * l * l * s - 2 * l ** 3 * s * s), rel=1e-14)
    assert out["Ne"] == pytest.approx(2 * (3 * l * l * s * s - 2 * l ** 3 * s ** 3), rel=1e-14)
    assert out["G"][0, 0, 0] == pytest.approx(2 * h * (6 * l * s - 6 * l * l * s * s), rel=1e-14)
    assert out["GN"][0, 0, 0] == pytest.approx(2 * (6 * l * s * s - 6 * l * l * s ** 3), rel=1e-14)


def test_gradient_against_exact_cubic_differences():
    """E(L + tD) is a cubic in t, so the 4-point Richardson difference
    [8(E(h)-E(-h)) - (E(2h)-E(-2h))] / 12h is exact up to rounding; it must equal
    <G, D> for symmetric D on L's pattern, and the same for N_e and dN_e/dL.
    Checked on 20 random blocks."""
    w, S, H, L = _si(2, 4, 6.6, 8.0, seed=21)
    rng = np.random.default_rng(99)
    base = oracle.lnv_energy_grad(w["pos"], w["cell"], 6.6, 8.0, S, H, L, grad_ne=True)
    G, GN = base["G"], base["GN"]
    rp, col = L["rp"], L["col"]
    n = rp.size - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    key = rows * n + col
    h = 1e-3
    picks = rng.choice(col.size, size=20, replace=False)
    for p in picks:
        i, j = rows[p], col[p]
        D = np.zeros_like(L["val"])
        blk = rng.standard_normal((4, 4))
        if i == j:
            blk = 0.5 * (blk + blk.T)
        D[p] = blk
        q = np.searchsorted(key, j * n + i)
        D[q] = blk.T

        def en_at(t):
            Lt = oracle.csr(rp, col, L["val"] + t * D)
            o = oracle.lnv_energy_grad(w["pos"], w["cell"], 6.6, 8.0, S, H, Lt, grad=False)
            return o["E"], o["Ne"]

        en = {t: en_at(t * h) for t in (-2, -1, 1, 2)}
        e = {t: v[0] for t, v in en.items()}
        ne = {t: v[1] for t, v in en.items()}
        fd = (8 * (e[1] - e[-1]) - (e[2] - e[-2])) / (12 * h)
        an = float((G * D).sum())
        assert fd == pytest.approx(an, rel=1e-8, abs=1e-10)
        fdn = (8 * (ne[1] - ne[-1]) - (ne[2] - ne[-2])) / (12 * h)
        # rounding of the four N_e values bounds the difference by about
        # 18 eps |N_e| / 12h = 3.3e-13 |N_e| at h = 1e-3
        assert fdn == pytest.approx(float((GN * D).sum()), rel=1e-8, abs=1e-12 * abs(base["Ne"]))
        # five points fix more than a cubic: the cubic through t=-2..2 must
        # also pass through E(0)
        t = np.array([-2.0, -1.0, 1.0, 2.0]) * h
        coef = np.polyfit(t, [e[-2], e[-1], e[1], e[2]], 3)
        assert np.polyval(coef, 0.0) == pytest.approx(base["E"], rel=1e-12, abs=1e-12)


def test_energy_per_atom_constant_under_tiling():
    """Sec. 3 / Table 1: the energy per atom is independent of cell size.
    Tiling a 4x4x4 system 2x2x2 times (all ranges below half the small box)
    must multiply E and N_e by exactly 8 and repeat G."""
    r_sh, r_l = 2.5, 3.0  # R_T = 8.0 < 10.86 = half the 21.72 A box
    w, S, H, L = _si(4, 4, r_sh, r_l, seed=5)
    small = oracle.lnv_energy_grad(w["pos"], w["cell"], r_sh, r_l, S, H, L)
    n = w["pos"].shape[0]
    box = w["cell"][0]
    shifts = np.array([[a, b, c] for a in (0, 1) for b in (0, 1) for c in (0, 1)], float) * box
    pos_big = np.concatenate([w["pos"] + s for s in shifts])
    cell_big = 2 * w["cell"]

    def tile(M, R):
        rp, col = oracle.pattern(pos_big, cell_big, R)
        rows = np.repeat(np.arange(8 * n), np.diff(rp))
        skey = np.repeat(np.arange(n), np.diff(M["rp"])) * n + M["col"]
        q = np.searchsorted(skey, (rows % n) * n + (col % n))
        assert np.array_equal(skey[q], (rows % n) * n + (col % n))
        return oracle.csr(rp, col, M["val"][q])

    Sb, Hb, Lb = tile(S, r_sh), tile(H, r_sh), tile(L, r_l)
    big = oracle.lnv_energy_grad(pos_big, cell_big, r_sh, r_l, Sb, Hb, Lb)
    assert big["E"] == pytest.approx(8 * small["E"], rel=1e-12)
    assert big["Ne"] == pytest.approx(8 * small["Ne"], rel=1e-12)
    Gs = tile(oracle.csr(L["rp"], L["col"], small["G"]), r_l)["val"]
    np.testing.assert_allclose(big["G"], Gs, rtol=0, atol=1e-12)


def test_row_subset_products_and_traces_equal_full_ones():
    """The row-restricted oracle entry points (used to time bounded samples)
    give exactly the full result's rows."""
    w, S, H, L = _si(3, 4, 6.6, 8.0, seed=2)
    pat = oracle.pattern(w["pos"], w["cell"], 14.6)
    full = oracle.mprod(L, S, pat)
    rows = np.array([0, 5, 17, 100, 215])
    part = oracle.mprod(L, S, pat, rows=rows)
    for i in rows:
        sl = slice(pat[0][i], pat[0][i + 1])
        np.testing.assert_array_equal(part["val"][sl], full["val"][sl])
    t_full, per_row = oracle.trace(full, full, row_part=True)
    assert oracle.trace(full, full, rows=rows) == pytest.approx(per_row[rows].sum(), rel=1e-14)


# ---------------------------------------------------------------- minimisation

def _fill_mu(Sd, Hd, m):
    linalg = pytest.importorskip("scipy.linalg")
    eps = linalg.eigh(Hd, Sd, eigvals_only=True)
    return eps, 0.5 * (eps[m - 1] + eps[m])


@pytest.mark.parametrize("m", [5, 16, 24])
def test_minimisation_reaches_ground_state_projector(m):
    """Untruncated system, mu in the gap above the m-th state: minimising
    Omega = E - mu N_e from L = S^-1 / 2 reaches the projector on the m lowest
    generalised eigenvectors of (H, S): E = 2 sum eps_1..m, N_e = 2m, LSL = L,
    with Omega never rising along the way."""
    from oracle.minimize import lnv_minimize
    w, S, H, L = _dense_system(seed=12)
    Sd = to_dense(S["rp"], S["col"], S["val"])
    Hd = to_dense(H["rp"], H["col"], H["val"])
    eps, mu = _fill_mu(Sd, Hd, m)
    L0 = oracle.csr(L["rp"], L["col"], from_dense(0.5 * np.linalg.inv(Sd), L["rp"], L["col"], 4))
    Lf, hist = lnv_minimize(w["pos"], w["cell"], 5.0, 5.0, S, H, L0, mu, max_iter=400, tol=1e-9)
    omega, E, Ne = hist[-1, 0], hist[-1, 1], hist[-1, 2]
    assert E == pytest.approx(2 * eps[:m].sum(), rel=1e-10, abs=1e-10)
    assert Ne == pytest.approx(2 * m, rel=1e-10)
    assert omega == pytest.approx(2 * (eps[:m] - mu).sum(), rel=1e-10)
    assert np.all(np.diff(hist[:, 0]) <= 1e-12 * abs(omega))
    Ld = to_dense(Lf["rp"], Lf["col"], Lf["val"])
    assert np.linalg.norm(Ld @ Sd @ Ld - Ld) <= 1e-6 * np.linalg.norm(Ld)


def test_minimisation_single_atom_closed_form():
    """NSF = 1, one atom: Omega(l) = 2(h - mu s)(3 l^2 s - 2 l^3 s^2) has its
    minimum at l = 1/s (the occupied state) when h < mu s."""
    from oracle.minimize import lnv_minimize
    s, h, mu = 1.3, -0.7, 0.0
    rp, col = np.array([0, 1]), np.array([0], np.int32)
    S = oracle.csr(rp, col, np.array([[[s]]]))
    H = oracle.csr(rp, col, np.array([[[h]]]))
    L = oracle.csr(rp, col, np.array([[[0.5 / s]]]))
    Lf, hist = lnv_minimize(np.zeros((1, 3)), np.array([10.0, 10.0, 10.0]), 3.0, 3.0, S, H, L, mu,
                            max_iter=50, tol=1e-12)
    assert Lf["val"][0, 0, 0] == pytest.approx(1.0 / s, rel=1e-9)
    assert hist[-1, 1] == pytest.approx(2 * h / s, rel=1e-12)
    assert hist[-1, 2] == pytest.approx(2.0, rel=1e-12)


# ---------------------------------------------------------------- truncated intermediates

def test_truncated_plan_at_exact_ranges_is_the_exact_evaluation():
    w, S, H, L = _si(2, 4, 6.6, 8.0, seed=4)
    ex = oracle.lnv_energy_grad(w["pos"], w["cell"], 6.6, 8.0, S, H, L)
    tr = oracle.lnv_energy_grad_truncated(w["pos"], w["cell"], 6.6, 8.0, 14.6, 21.2, S, H, L)
    assert tr["E"] == pytest.approx(ex["E"], rel=1e-13)
    assert tr["Ne"] == pytest.approx(ex["Ne"], rel=1e-13)
    assert np.linalg.norm(tr["G"] - ex["G"]) <= 1e-12 * np.linalg.norm(ex["G"])


def test_truncation_error_shrinks_with_the_ranges():
    """512 atoms, R_SH = 3, R_L = 4.5 (exact R_X = 7.5, R_T = 10.5 inside the
    21.7 A box): the errors of E, N_e and G against the exact evaluation fall
    as the intermediates' ranges grow, and vanish at the exact ranges."""
    w, S, H, L = _si(4, 4, 3.0, 4.5, seed=6)
    ex = oracle.lnv_energy_grad(w["pos"], w["cell"], 3.0, 4.5, S, H, L)
    errs = []
    for r_x, r_t in [(4.5, 4.5), (5.0, 6.0), (6.0, 8.0), (7.5, 10.5)]:
        tr = oracle.lnv_energy_grad_truncated(w["pos"], w["cell"], 3.0, 4.5, r_x, r_t, S, H, L)
        errs.append((abs(tr["E"] - ex["E"]) / abs(ex["E"]), abs(tr["Ne"] - ex["Ne"]) / abs(ex["Ne"]),
                     np.linalg.norm(tr["G"] - ex["G"]) / np.linalg.norm(ex["G"])))
    errs = np.array(errs)
    assert np.all(errs[:-1, 2] > errs[-1, 2])
    assert np.all(np.diff(errs[:-1, 2]) < 0)
    assert np.all(errs[-1] < 1e-12)
    assert errs[0, 2] > 1e-6  # the truncation is really felt


@pytest.mark.parametrize("nsf", [2, 4])
@pytest.mark.parametrize("r_x,r_t", [(5.0, 6.0), (6.0, 8.0)])
def test_truncated_oracle_against_dense_masked_definition(nsf, r_x, r_t):
    """The truncated evaluation written out densely with 0/1 block masks on a
    64-atom system, at ranges below the exact ones (R_X = 7.5, R_T = 10.5)
    where T = SX is not symmetric, so the association matters:
      X = M_rx o (L S), Y = M_rx o (L H), T = M_rt o (S X), U = M_rt o (S Y),
      Z = M_rx o (L T^T), Q = M_L o (H Z), W = M_L o (X^T U^T) taken on the
      block upper triangle (j >= i) and mirrored below it,
      E = 2 (3 Tr[XY] - 2 Tr[ZY]), N_e = 2 (3 Tr[XX] - 2 Tr[ZX]),
      G = M_L o (6 (U + U^T) - 4 (Q^T + W + Q)).
    Z from T instead of T^T, or W mirrored from the other triangle, fails."""
    w, S, H, L = _si(2, nsf, 3.0, 4.5, seed=11)
    pos, cell = w["pos"], w["cell"]
    n = pos.shape[0]
    Sd, Hd, Ld = (to_dense(M["rp"], M["col"], M["val"]) for M in (S, H, L))
    Mx = mask_dense(*oracle.pattern(pos, cell, r_x), nsf)
    Mt = mask_dense(*oracle.pattern(pos, cell, r_t), nsf)
    Ml = mask_dense(L["rp"], L["col"], nsf)
    X, Y = Mx * (Ld @ Sd), Mx * (Ld @ Hd)
    T, U = Mt * (Sd @ X), Mt * (Sd @ Y)
    assert np.linalg.norm(T - T.T) > 1e-5 * np.linalg.norm(T)  # the association is felt
    Z = Mx * (Ld @ T.T)
    E = 2 * (3 * np.trace(X @ Y) - 2 * np.trace(Z @ Y))
    Ne = 2 * (3 * np.trace(X @ X) - 2 * np.trace(Z @ X))
    Q = Ml * (Hd @ Z)
    W = Ml * (X.T @ U.T)
    blk = np.kron(np.arange(n)[:, None] <= np.arange(n)[None, :], np.ones((nsf, nsf)))    # j >= i
    strict = np.kron(np.arange(n)[:, None] < np.arange(n)[None, :], np.ones((nsf, nsf)))  # j > i
    Wm = blk * W + (strict * W).T
    Gd = Ml * (6 * (U + U.T) - 4 * (Q.T + Wm + Q))
    tr = oracle.lnv_energy_grad_truncated(pos, cell, 3.0, 4.5, r_x, r_t, S, H, L)
    assert tr["E"] == pytest.approx(E, rel=1e-12)
    assert tr["Ne"] == pytest.approx(Ne, rel=1e-12)
    G = from_dense(Gd, L["rp"], L["col"], nsf)
    assert np.linalg.norm(tr["G"] - G) <= 1e-12 * np.linalg.norm(G)
    # the plausible slips the pin guards against are far off
    Z_bad = Mx * (Ld @ T)
    E_bad = 2 * (3 * np.trace(X @ Y) - 2 * np.trace(Z_bad @ Y))
    assert abs(E_bad - E) > 1e-9 * abs(E)
    W_bad = blk.T * W + (strict.T * W).T
    G_bad = from_dense(Ml * (6 * (U + U.T) - 4 * (Q.T + W_bad + Q)), L["rp"], L["col"], nsf)
    assert np.linalg.norm(G_bad - G) > 1e-6 * np.linalg.norm(G)


# ---------------------------------------------------------------- precision reading

def _tf32(x):
    """x rounded to the nearest TF32 value (10 explicit significand bits, ties
    away from zero), held in FP32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    return ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def _lnv_emulated(S, H, L, mm):
    """Eq. 3's E, N_e and dE/dL with every matrix product formed by mm (FP32
    intermediates) and the traces and combinations in FP64."""
    f = lambda M: np.asarray(M, dtype=np.float32)
    S, H, L = f(S), f(H), f(L)
    LS, LH = mm(L, S), mm(L, H)
    SLS, SLH = mm(S, LS), mm(S, LH)
    LSLS = mm(L, SLS)
    K = 3.0 * mm(LS, L).astype(np.float64) - 2.0 * mm(LSLS, L).astype(np.float64)
    E = 2.0 * np.sum(K * H.T.astype(np.float64))
    Ne = 2.0 * np.sum(K * S.T.astype(np.float64))
    HLS, HLSLS, SLSLH, SLHLS = mm(H, LS), mm(H, LSLS), mm(SLS, LH), mm(SLH, LS)
    G = 6.0 * (SLH.astype(np.float64) + HLS) - 4.0 * (SLSLH.astype(np.float64) + SLHLS + HLSLS)
    return E, Ne, G


def test_single_pass_tf32_misses_the_fp32_bound():
    """The reading behind the tensor-core kernels' split operands: with every
    product's operands rounded once to TF32 (FP32 accumulation, emulated on the
    CPU) the gradient of a 64-atom NSF = 4 system misses the FP32 path's bound
    of 2e-5 relative, while the hi*hi + hi*lo + lo*hi split (3xTF32) meets it."""
    w = synth.si_workload(2, 4, 6.6, 8.0, 5, oracle.pattern)
    S = to_dense(w["sh_row_ptr"], w["sh_col"], w["S"])
    H = to_dense(w["sh_row_ptr"], w["sh_col"], w["H"])
    L = to_dense(w["l_row_ptr"], w["l_col"], w["L"])
    S32, H32, L32 = (M.astype(np.float32).astype(np.float64) for M in (S, H, L))
    E0, N0, G0, _ = lnv_dense(S32, H32, L32)

    def one_pass(A, B):
        return _tf32(A) @ _tf32(B)

    def three_pass(A, B):
        Ah, Bh = _tf32(A), _tf32(B)
        Al, Bl = _tf32(A - Ah), _tf32(B - Bh)
        return (Ah @ Bh + Ah @ Bl) + Al @ Bh

    errs = {}
    for name, mm in (("1xTF32", one_pass), ("3xTF32", three_pass)):
        E, Ne, G = _lnv_emulated(S32, H32, L32, mm)
        errs[name] = (abs(E - E0) / abs(E0), abs(Ne - N0) / abs(N0), np.linalg.norm(G - G0) / np.linalg.norm(G0))
    assert errs["1xTF32"][2] > 2e-5, errs
    assert max(errs["3xTF32"]) < 2e-5, errs
