"""GPU path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 path, relative Frobenius error <= 1e-12 for matrices and
relative error <= 1e-10 for E and N_e; FP32 path (FP32 products, FP64 traces
and gradient combination), <= 2e-5 for both, measured against the oracle run
on the FP64 inputs.  Integer work (patterns, transpose maps) is bit-exact.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_0911_3584_gb300 import Context, LnvError, Pattern, Plan, System, trace_product
from tests.gpu_util import oracle_lnv, rel_fro, rounded, to_dev, workload

pytestmark = pytest.mark.gpu

TOL = {torch.float64: (1e-12, 1e-10), torch.float32: (2e-5, 2e-5)}
PREC = {torch.float64: "fp64", torch.float32: "fp32"}


@pytest.fixture(scope="module")
def ctx(cuda_device):
    return Context(cuda_device)


def _pattern_np(P):
    return P.row_ptr.cpu().numpy(), P.col.cpu().numpy()


# ------------------------------------------------------------------ a0 patterns

@pytest.mark.parametrize("ncell,cutoffs", [(4, (2.5, 6.6, 8.0, 14.6, 21.2)), (2, (6.6, 21.2)),
                                           (1, (3.0, 30.0))])
def test_pattern_identical_to_oracle(ctx, ncell, cutoffs):
    rng = np.random.default_rng(ncell)
    pos, cell = synth.si_diamond_positions(ncell, rng)
    for R in cutoffs:
        P = Pattern.build(ctx, pos, cell, R)
        rp, col = _pattern_np(P)
        orp, ocol = oracle.pattern(pos, cell, R)
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol), R
        assert P.symmetric
        tr = P.tr.cpu().numpy()
        rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        assert np.array_equal(col[tr], rows) and np.array_equal(rows[tr], col)


def test_pattern_random_orthorhombic_box_and_unwrapped_positions(ctx):
    """Non-cubic box, positions partly outside [0, box): same set as the oracle."""
    rng = np.random.default_rng(11)
    cell = np.array([17.3, 23.9, 31.1])
    pos = rng.uniform(-0.3, 1.3, size=(700, 3)) * cell
    for R in (2.0, 5.5, 9.0, 12.0):
        P = Pattern.build(ctx, pos, cell, R)
        rp, col = _pattern_np(P)
        orp, ocol = oracle.pattern(pos, cell, R)
        assert np.array_equal(rp, orp) and np.array_equal(col, ocol)


def test_pattern_isolated_atoms_and_single_atom(ctx):
    pos = np.array([[0.0, 0.0, 0.0], [10.0, 10.0, 10.0], [20.0, 0.0, 5.0]])
    P = Pattern.build(ctx, pos, [40.0, 40.0, 40.0], 3.0)
    rp, col = _pattern_np(P)
    assert rp.tolist() == [0, 1, 2, 3] and col.tolist() == [0, 1, 2]
    P1 = Pattern.build(ctx, pos[:1], [5.0, 5.0, 5.0], 3.0)
    assert _pattern_np(P1)[1].tolist() == [0]


def test_pattern_batched_is_block_diagonal_union(ctx):
    sizes = [2, 3, 1, 2]
    pos_all, cells, off = [], [], [0]
    for k, n in enumerate(sizes):
        p, c = synth.si_diamond_positions(n, np.random.default_rng(100 + k))
        pos_all.append(p)
        cells.append(c)
        off.append(off[-1] + p.shape[0])
    P = Pattern.build_batched(ctx, np.concatenate(pos_all), off, cells, 8.0)
    rp, col = _pattern_np(P)
    exp_rp, exp_col = [0], []
    for k in range(len(sizes)):
        orp, ocol = oracle.pattern(pos_all[k], cells[k], 8.0)
        exp_col.append(ocol + off[k])
        exp_rp.extend((orp[1:] + exp_rp[-1]).tolist())
    assert np.array_equal(rp, np.array(exp_rp)) and np.array_equal(col, np.concatenate(exp_col))


def test_pattern_from_csr_rejects_unsorted_rows(ctx):
    with pytest.raises(LnvError) as e:
        Pattern.from_csr(ctx, [0, 2, 3], [1, 0, 1])
    assert e.value.status == -4
    P = Pattern.from_csr(ctx, [0, 2, 3], [0, 1, 1])
    assert not P.symmetric


# ------------------------------------------------------------------ a1-a3, a5, a6 products

PRODUCT_CASES = [
    # (ra, rb, rc, trans_a, trans_b): push- and pull-type patterns
    (8.0, 6.6, 14.6, False, False),   # X = L S (full range)
    (6.6, 14.6, 21.2, False, False),  # T = S X (full range)
    (8.0, 21.2, 14.6, False, False),  # Z = L T masked
    (14.6, 21.2, 8.0, True, True),    # W = X^T U^T masked
    (6.6, 14.6, 8.0, False, False),   # Q = H Z masked
    (8.0, 6.6, 14.6, True, False),    # transposed A, full range
    (6.6, 8.0, 5.0, False, True),     # transposed B, masked
    (8.0, 21.2, 14.6, False, True),   # Z = L T^T masked (as the evaluation forms it)
]


def _set_kernel_or_refused(plan, kernel, tb):
    """Select the kernel; the tensor-core kernel refuses plans without op(B) = B^T."""
    if kernel == "tensor" and not tb:
        with pytest.raises(LnvError) as e:
            plan.set_kernel(kernel)
        assert e.value.status == -5
        return False
    plan.set_kernel(kernel)
    return True


@pytest.mark.parametrize("kernel", ["default", "push", "pull", "pull-merge", "group", "group-sparse",
                                    "group-pipe", "group-mma", "triples", "group-pipe-half", "tensor",
                                    "tensor9", "tensor-tile"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nsf", [1, 2, 4, 9])
@pytest.mark.parametrize("case", PRODUCT_CASES)
def test_masked_product_matches_oracle(ctx, dtype, nsf, case, kernel):
    ra, rb, rc, ta, tb = case
    rng = np.random.default_rng(nsf * 7 + int(ta) + 2 * int(tb))
    ncell = 3 if nsf < 9 else 2
    pos, cell = synth.si_diamond_positions(ncell, rng)
    PA, PB, PC = (Pattern.build(ctx, pos, cell, r) for r in (ra, rb, rc))
    oa, ob, oc = (oracle.pattern(pos, cell, r) for r in (ra, rb, rc))
    A = oracle.csr(*oa, rng.standard_normal((oa[1].size, nsf, nsf)))
    B = oracle.csr(*ob, rng.standard_normal((ob[1].size, nsf, nsf)))
    A, B = rounded(A, dtype), rounded(B, dtype)
    plan = Plan(ctx, PA, PB, PC, trans_a=ta, trans_b=tb)
    if kernel != "default" and not _set_kernel_or_refused(plan, kernel, tb):
        return
    C = plan.multiply(to_dev(A["val"], dtype, ctx.device), to_dev(B["val"], dtype, ctx.device))
    ref = oracle.mprod(oracle.transpose(A) if ta else A, oracle.transpose(B) if tb else B, oc)
    err = rel_fro(C.cpu().numpy(), ref["val"])
    assert err <= TOL[dtype][0], (err, plan.mode)
    assert plan.triples > 0


@pytest.mark.parametrize("kernel", ["default", "push", "pull", "pull-merge", "group", "group-sparse",
                                    "group-pipe", "group-mma", "triples", "group-pipe-half", "tensor9",
                                    "tensor-tile"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nsf", [1, 4, 9])
def test_symmetric_product_formed_on_one_triangle(ctx, dtype, nsf, kernel):
    """T = S (L S) with symmetric S, L declared symmetric (LNV_SYM_C): the kernels
    form its upper triangle (the two-output form too: U = S (L H) alongside) and
    the lower triangle is mirrored.  Against the oracle's full product; the
    result is exactly symmetric."""
    ncell = 2 if nsf == 9 else 3
    w = synth.si_workload(ncell, nsf, 6.6, 8.0, nsf, oracle.pattern)
    pos, cell = w["pos"], w["cell"]
    S = rounded(oracle.csr(w["sh_row_ptr"], w["sh_col"], w["S"]), dtype)
    H = rounded(oracle.csr(w["sh_row_ptr"], w["sh_col"], w["H"]), dtype)
    L = rounded(oracle.csr(w["l_row_ptr"], w["l_col"], w["L"]), dtype)
    ox, ot = oracle.pattern(pos, cell, 14.6), oracle.pattern(pos, cell, 21.2)
    X = rounded(oracle.mprod(L, S, ox), dtype)
    Y = rounded(oracle.mprod(L, H, ox), dtype)
    PS, PX, PT = (Pattern.build(ctx, pos, cell, r) for r in (6.6, 14.6, 21.2))
    plan = Plan(ctx, PS, PX, PT, sym_c=True)
    if kernel != "default":
        plan.set_kernel(kernel)
    dev = ctx.device
    T = plan.multiply(to_dev(S["val"], dtype, dev), to_dev(X["val"], dtype, dev)).cpu().numpy()
    ref_t = oracle.mprod(S, X, ot)["val"]
    assert rel_fro(T, ref_t) <= TOL[dtype][0], plan.mode
    tr = PT.tr.cpu().numpy()
    assert np.array_equal(T, np.swapaxes(T[tr], 1, 2))
    # the fused pair through a system-style two-output call: T and U together
    sysm = System(ctx, nsf, PREC[dtype], pos, cell, 6.6, 8.0)
    if kernel != "default":
        sysm.set_stage_kernel("TU", kernel)
    Sd, Hd, Ld = (to_dev(M["val"], dtype, dev) for M in (S, H, L))
    ref = oracle_lnv(w, S, H, L)
    assert sysm.mirror
    for mirror in (True, False):
        sysm.set_mirror(mirror)
        out, G = sysm.energy_grad(Sd, Hd, Ld)
        assert rel_fro(G.cpu().numpy(), ref["G"]) <= TOL[dtype][0], mirror
        assert abs(out.cpu().numpy()[0][0] - ref["E"]) <= TOL[dtype][1] * abs(ref["E"]), mirror
        assert abs(out.cpu().numpy()[0][1] - ref["Ne"]) <= TOL[dtype][1] * abs(ref["Ne"]), mirror


def test_mirror_needs_exact_x(ctx):
    """With X truncated, T = S X is not symmetric: no mirror, and asking for it fails."""
    pos, cell = synth.si_diamond_positions(2, np.random.default_rng(1))
    s_exact = System(ctx, 4, "fp64", pos, cell, 6.6, 8.0, r_t=18.0)
    assert s_exact.mirror
    s_trunc = System(ctx, 4, "fp64", pos, cell, 6.6, 8.0, r_x=13.0)
    assert not s_trunc.mirror
    with pytest.raises(LnvError) as e:
        s_trunc.set_mirror(True)
    assert e.value.status == -5
    s_trunc.set_mirror(False)


def test_symmetric_product_needs_symmetric_pattern(ctx):
    pos, cell = synth.si_diamond_positions(2, np.random.default_rng(0))
    P = Pattern.build(ctx, pos, cell, 8.0)
    rp, col = P.row_ptr.cpu().numpy(), P.col.cpu().numpy()
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    keep = col >= rows  # upper triangle only: not symmetric
    nrp = np.concatenate([[0], np.cumsum(np.bincount(rows[keep], minlength=len(rp) - 1))])
    PU = Pattern.from_csr(ctx, nrp, col[keep])
    with pytest.raises(LnvError) as e:
        Plan(ctx, P, P, PU, sym_c=True)
    assert e.value.status == -4


def test_misaligned_value_arrays_are_refused(ctx):
    """Value arrays off a 16-byte boundary are refused on the host (LNV_ERR_ARG)
    before any kernel runs: the kernels move blocks in 16-byte pieces."""
    pos, cell = synth.si_diamond_positions(2, np.random.default_rng(3))
    P = Pattern.build(ctx, pos, cell, 6.6)
    n = P.nnzb * 16
    buf = torch.zeros(n + 4, dtype=torch.float32, device=ctx.device)
    A = buf[1:1 + n].view(P.nnzb, 4, 4)
    assert A.data_ptr() % 16 == 4
    B = torch.zeros((P.nnzb, 4, 4), dtype=torch.float32, device=ctx.device)
    with pytest.raises(LnvError) as e:
        Plan(ctx, P, P, P).multiply(A, B)
    assert e.value.status == -1
    sysm = System(ctx, 4, "fp32", pos, cell, 6.6, 8.0)
    L = torch.zeros((sysm.P_l.nnzb, 4, 4), dtype=torch.float32, device=ctx.device)
    with pytest.raises(LnvError) as e:
        sysm.energy_grad(A, B, L)
    assert e.value.status == -1


def test_plan_modes_follow_symbolic_counts(ctx):
    pos, cell = synth.si_diamond_positions(4, np.random.default_rng(0))
    P = {r: Pattern.build(ctx, pos, cell, r) for r in (6.6, 8.0, 14.6, 21.2)}
    # full-range products mostly miss on the dense table: hit lists
    assert Plan(ctx, P[8.0], P[6.6], P[14.6]).mode == "group-sparse"
    # masked products mostly hit: dense position table
    assert Plan(ctx, P[14.6], P[21.2], P[8.0], True, True).mode == "group"
    # a non-symmetric B pattern keeps the binary-search pull
    rp, col = P[21.2].row_ptr.cpu().numpy(), P[21.2].col.cpu().numpy()
    keep = col != np.repeat(np.arange(len(rp) - 1), np.diff(rp)) + 1  # drop (i, i+1) blocks
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))[keep]
    nrp = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=len(rp) - 1))])
    PB = Pattern.from_csr(ctx, nrp, col[keep])
    assert not PB.symmetric
    pl = Plan(ctx, P[8.0], PB, P[14.6])
    with pytest.raises(LnvError) as e:
        pl.set_kernel("pull-merge")
    assert e.value.status == -5


@pytest.mark.parametrize("kernel", ["default", "tensor", "tensor-tile"])
@pytest.mark.parametrize("n_atoms", [1, 7, 9, 42, 131])
def test_transposed_product_ragged_groups(ctx, kernel, n_atoms):
    """op(B) = B^T products on atom counts that leave a partial last row group
    (8-row groups of the tensor-core kernel, 4-row groups elsewhere) and
    partial 32-column tiles, with random clustered positions: FP32 against the
    oracle."""
    rng = np.random.default_rng(n_atoms)
    cell = np.array([20.0, 20.0, 20.0])
    pos = rng.uniform(0, 9.0, size=(n_atoms, 3))
    ra, rb, rc = 4.0, 7.0, 6.0
    PA, PB, PC = (Pattern.build(ctx, pos, cell, r) for r in (ra, rb, rc))
    oa, ob, oc = (oracle.pattern(pos, cell, r) for r in (ra, rb, rc))
    A = rounded(oracle.csr(*oa, rng.standard_normal((oa[1].size, 4, 4))), torch.float32)
    B = rounded(oracle.csr(*ob, rng.standard_normal((ob[1].size, 4, 4))), torch.float32)
    for ta in (False, True):
        plan = Plan(ctx, PA, PB, PC, trans_a=ta, trans_b=True)
        if kernel != "default":
            plan.set_kernel(kernel)
        C = plan.multiply(to_dev(A["val"], torch.float32, ctx.device), to_dev(B["val"], torch.float32, ctx.device))
        ref = oracle.mprod(oracle.transpose(A) if ta else A, oracle.transpose(B), oc)
        assert rel_fro(C.cpu().numpy(), ref["val"]) <= TOL[torch.float32][0], (ta, plan.mode)


@pytest.mark.parametrize("n_atoms", [1, 6, 7, 8, 15, 29, 61])
def test_tensor9_product_ragged_groups(ctx, n_atoms):
    """Kernel 10 (NSF = 9) on atom counts that leave a partial last 7-row group
    and partial 14-column tiles, random clustered positions, every operand
    transpose: FP32 against the oracle."""
    rng = np.random.default_rng(100 + n_atoms)
    cell = np.array([20.0, 20.0, 20.0])
    pos = rng.uniform(0, 9.0, size=(n_atoms, 3))
    ra, rb, rc = 4.0, 7.0, 6.0
    PA, PB, PC = (Pattern.build(ctx, pos, cell, r) for r in (ra, rb, rc))
    oa, ob, oc = (oracle.pattern(pos, cell, r) for r in (ra, rb, rc))
    A = rounded(oracle.csr(*oa, rng.standard_normal((oa[1].size, 9, 9))), torch.float32)
    B = rounded(oracle.csr(*ob, rng.standard_normal((ob[1].size, 9, 9))), torch.float32)
    for ta in (False, True):
        for tb in (False, True):
            plan = Plan(ctx, PA, PB, PC, trans_a=ta, trans_b=tb)
            plan.set_kernel("tensor9")
            C = plan.multiply(to_dev(A["val"], torch.float32, ctx.device),
                              to_dev(B["val"], torch.float32, ctx.device))
            ref = oracle.mprod(oracle.transpose(A) if ta else A, oracle.transpose(B) if tb else B, oc)
            assert rel_fro(C.cpu().numpy(), ref["val"]) <= TOL[torch.float32][0], (ta, tb)
    assert ctx.device_status() == 0


@pytest.mark.parametrize("n_atoms", [1, 7, 8, 9, 33, 42, 131])
def test_tensor_tile_product_ragged_groups(ctx, n_atoms):
    """Kernel 11 (tiles of 32 columns over their own k lists) on atom counts
    that leave a partial last 8-row group, partial tiles and tiles with few
    listed k's, random clustered positions, every operand transpose: FP32
    against the oracle."""
    rng = np.random.default_rng(200 + n_atoms)
    cell = np.array([20.0, 20.0, 20.0])
    pos = rng.uniform(0, 9.0, size=(n_atoms, 3))
    ra, rb, rc = 4.0, 7.0, 6.0
    PA, PB, PC = (Pattern.build(ctx, pos, cell, r) for r in (ra, rb, rc))
    oa, ob, oc = (oracle.pattern(pos, cell, r) for r in (ra, rb, rc))
    A = rounded(oracle.csr(*oa, rng.standard_normal((oa[1].size, 4, 4))), torch.float32)
    B = rounded(oracle.csr(*ob, rng.standard_normal((ob[1].size, 4, 4))), torch.float32)
    for ta in (False, True):
        for tb in (False, True):
            plan = Plan(ctx, PA, PB, PC, trans_a=ta, trans_b=tb)
            plan.set_kernel("tensor-tile")
            C = plan.multiply(to_dev(A["val"], torch.float32, ctx.device),
                              to_dev(B["val"], torch.float32, ctx.device))
            ref = oracle.mprod(oracle.transpose(A) if ta else A, oracle.transpose(B) if tb else B, oc)
            assert rel_fro(C.cpu().numpy(), ref["val"]) <= TOL[torch.float32][0], (ta, tb)
    assert ctx.device_status() == 0


# single-pass TF32 (operands rounded to TF32, FP32 sums): unit roundoff 2^-11,
# so products sit near 1e-4 relative and well below 3e-3; the FP32 bound of
# 2e-5 is out of its reach (the emulation in test_oracle measures it)
TOL_1PASS = 3e-3


@pytest.mark.parametrize("kernel", ["tensor-1pass", "tensor-tile-1pass"])
@pytest.mark.parametrize("n_atoms", [7, 33, 131])
def test_single_pass_tensor_kernels(ctx, kernel, n_atoms):
    """Kernels 12 and 13 (single-pass TF32 forms of 9 and 11) on ragged groups,
    every transpose they take, against the FP64 oracle: within the TF32 bound,
    and above the 3xTF32 kernels' error (they really run one pass)."""
    rng = np.random.default_rng(300 + n_atoms)
    cell = np.array([20.0, 20.0, 20.0])
    pos = rng.uniform(0, 9.0, size=(n_atoms, 3))
    ra, rb, rc = 4.0, 7.0, 6.0
    PA, PB, PC = (Pattern.build(ctx, pos, cell, r) for r in (ra, rb, rc))
    oa, ob, oc = (oracle.pattern(pos, cell, r) for r in (ra, rb, rc))
    A = rounded(oracle.csr(*oa, rng.standard_normal((oa[1].size, 4, 4))), torch.float32)
    B = rounded(oracle.csr(*ob, rng.standard_normal((ob[1].size, 4, 4))), torch.float32)
    for ta in (False, True):
        for tb in ((True,) if kernel == "tensor-1pass" else (False, True)):
            plan = Plan(ctx, PA, PB, PC, trans_a=ta, trans_b=tb)
            ref = oracle.mprod(oracle.transpose(A) if ta else A, oracle.transpose(B) if tb else B, oc)
            Ad, Bd = to_dev(A["val"], torch.float32, ctx.device), to_dev(B["val"], torch.float32, ctx.device)
            plan.set_kernel(kernel)
            e1 = rel_fro(plan.multiply(Ad, Bd).cpu().numpy(), ref["val"])
            plan.set_kernel(kernel.replace("-1pass", ""))
            e3 = rel_fro(plan.multiply(Ad, Bd).cpu().numpy(), ref["val"])
            assert e1 <= TOL_1PASS, (ta, tb, e1)
            assert e3 <= TOL[torch.float32][0] and e1 > 4 * e3, (ta, tb, e1, e3)
    assert ctx.device_status() == 0


def test_lnv_512_atoms_single_pass_products(ctx, si512):
    """The FP32 evaluation with Z, W on kernel 12 and TU, Q on kernel 13: E,
    N_e and G within the single-pass TF32 bound of the FP64 oracle."""
    w, ref = si512
    sysm = System(ctx, 4, "fp32", w["pos"], w["cell"], 6.6, 8.0)
    for st, k in dict(TU="tensor-tile-1pass", Z="tensor-1pass", Q="tensor-tile-1pass", W="tensor-1pass").items():
        sysm.set_stage_kernel(st, k)
    _, out, (G, _) = _gpu_lnv(ctx, w, torch.float32, sysm=sysm)
    assert abs(out[0, 0] - ref["E"]) <= TOL_1PASS * abs(ref["E"])
    assert abs(out[0, 1] - ref["Ne"]) <= TOL_1PASS * abs(ref["Ne"])
    assert rel_fro(G, ref["G"]) <= TOL_1PASS
    assert ctx.device_status() == 0


def test_tensor_tile_repeated_calls_are_identical(ctx):
    """Kernel 11 sums in a fixed order: two launches of T = S X (op(B) = B)
    give bit-identical output, within the FP32 bound of the oracle."""
    w, S, H, L = workload(3, 4, 6.6, 8.0, seed=7)
    pos, cell = w["pos"], w["cell"]
    PS, PX, PT = (Pattern.build(ctx, pos, cell, r) for r in (6.6, 14.6, 21.2))
    ox = oracle.pattern(pos, cell, 14.6)
    X = rounded(oracle.csr(*ox, np.random.default_rng(4).standard_normal((ox[1].size, 4, 4))), torch.float32)
    plan = Plan(ctx, PS, PX, PT)
    plan.set_kernel("tensor-tile")
    Sd, Xd = to_dev(S["val"], torch.float32, ctx.device), to_dev(X["val"], torch.float32, ctx.device)
    c1 = plan.multiply(Sd, Xd).cpu().numpy()
    c2 = plan.multiply(Sd, Xd).cpu().numpy()
    assert np.array_equal(c1, c2)
    ref = oracle.mprod(rounded(S, torch.float32), X, oracle.pattern(pos, cell, 21.2))
    assert rel_fro(c1, ref["val"]) <= TOL[torch.float32][0]
    assert ctx.device_status() == 0


def test_tensor9_repeated_calls_are_identical(ctx):
    """Kernel 10 sums in a fixed order: two launches give bit-identical output."""
    w, S, H, L = workload(2, 9, 6.6, 8.0, seed=6)
    pos, cell = w["pos"], w["cell"]
    PL, PT, PX = (Pattern.build(ctx, pos, cell, r) for r in (8.0, 21.2, 14.6))
    ot = oracle.pattern(pos, cell, 21.2)
    T = oracle.csr(*ot, np.random.default_rng(3).standard_normal((ot[1].size, 9, 9)))
    plan = Plan(ctx, PL, PT, PX, trans_b=True)
    plan.set_kernel("tensor9")
    Ld, Td = to_dev(L["val"], torch.float32, ctx.device), to_dev(T["val"], torch.float32, ctx.device)
    c1 = plan.multiply(Ld, Td).cpu().numpy()
    c2 = plan.multiply(Ld, Td).cpu().numpy()
    assert np.array_equal(c1, c2)
    ref = oracle.mprod(rounded(L, torch.float32), oracle.transpose(rounded(T, torch.float32)),
                       oracle.pattern(pos, cell, 14.6))
    assert rel_fro(c1, ref["val"]) <= TOL[torch.float32][0]
    assert ctx.device_status() == 0


def test_tensor_kernel_repeated_calls_are_identical(ctx):
    """Kernel 9 sums in a fixed order: two launches give bit-identical output."""
    w, S, H, L = workload(3, 4, 6.6, 8.0, seed=5)
    pos, cell = w["pos"], w["cell"]
    PL, PT, PX = (Pattern.build(ctx, pos, cell, r) for r in (8.0, 21.2, 14.6))
    ot = oracle.pattern(pos, cell, 21.2)
    T = oracle.csr(*ot, np.random.default_rng(2).standard_normal((ot[1].size, 4, 4)))
    plan = Plan(ctx, PL, PT, PX, trans_b=True)
    plan.set_kernel("tensor")
    Ld, Td = to_dev(L["val"], torch.float32, ctx.device), to_dev(T["val"], torch.float32, ctx.device)
    c1 = plan.multiply(Ld, Td).cpu().numpy()
    c2 = plan.multiply(Ld, Td).cpu().numpy()
    assert np.array_equal(c1, c2)
    assert ctx.device_status() == 0


def test_device_wait_that_runs_out_is_reported(ctx):
    """A bounded device-side wait that nothing completes gives up after the
    context's limit and raises LNV_ERR_TIMEOUT on the host; the context stays
    usable (no fault, no trap)."""
    assert ctx.device_status() == 0
    ctx.set_wait_limit(20_000_000)  # 20 ms
    try:
        ctx.debug_expire_wait()
        assert ctx.device_status() == -6
        assert ctx.device_status() == 0  # cleared by the read
        with pytest.raises(LnvError) as e:
            ctx.debug_expire_wait()
            ctx.check_device()
        assert e.value.status == -6
    finally:
        ctx.set_wait_limit(1_000_000_000)
    # the context still runs products afterwards
    pos, cell = synth.si_diamond_positions(2, np.random.default_rng(9))
    P = Pattern.build(ctx, pos, cell, 6.6)
    A = torch.ones((P.nnzb, 4, 4), dtype=torch.float32, device=ctx.device)
    C = Plan(ctx, P, P, P).multiply(A, A)
    assert torch.isfinite(C).all() and ctx.device_status() == 0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("kernel", ["default", "tensor"])
def test_multiply_alpha_beta(ctx, dtype, kernel):
    """lnv_bsr_multiply's C = alpha mask(op(A) op(B)) + beta C through the C
    ABI: beta = 0 overwrites C without reading it (NaN there does not leak),
    beta != 0 combines with the old C; against the oracle's product."""
    rng = np.random.default_rng(41)
    pos, cell = synth.si_diamond_positions(3, rng)
    PA, PB, PC = (Pattern.build(ctx, pos, cell, r) for r in (8.0, 21.2, 14.6))
    oa, ob, oc = (oracle.pattern(pos, cell, r) for r in (8.0, 21.2, 14.6))
    A = rounded(oracle.csr(*oa, rng.standard_normal((oa[1].size, 4, 4))), dtype)
    B = rounded(oracle.csr(*ob, rng.standard_normal((ob[1].size, 4, 4))), dtype)
    C0 = rounded(oracle.csr(*oc, rng.standard_normal((oc[1].size, 4, 4))), dtype)
    plan = Plan(ctx, PA, PB, PC, trans_b=True)
    if kernel != "default":
        plan.set_kernel(kernel)
    P = oracle.mprod(A, oracle.transpose(B), oc)["val"]
    Ad, Bd = to_dev(A["val"], dtype, ctx.device), to_dev(B["val"], dtype, ctx.device)
    for alpha, beta in [(1.0, 0.0), (0.5, 0.0), (0.5, -2.0), (-1.25, 1.0), (0.0, 3.0)]:
        C = to_dev(C0["val"], dtype, ctx.device)
        if beta == 0.0:
            C.fill_(float("nan"))
        plan.multiply(Ad, Bd, C, alpha=alpha, beta=beta)
        ref = alpha * P + (beta * C0["val"] if beta != 0.0 else 0.0)
        assert rel_fro(C.cpu().numpy(), ref) <= TOL[dtype][0], (alpha, beta)


def test_product_empty_and_ragged_rows(ctx):
    """Isolated atoms (rows holding only the diagonal) next to a dense cluster."""
    rng = np.random.default_rng(4)
    cluster = rng.uniform(0, 6.0, size=(40, 3))
    lone = np.array([[30.0, 30.0, 30.0], [45.0, 10.0, 20.0]])
    pos = np.concatenate([cluster, lone])
    cell = np.array([60.0, 60.0, 60.0])
    for dtype in (torch.float64, torch.float32):
        PA, PB, PC = (Pattern.build(ctx, pos, cell, r) for r in (3.0, 4.0, 5.0))
        oa, ob, oc = (oracle.pattern(pos, cell, r) for r in (3.0, 4.0, 5.0))
        A = rounded(oracle.csr(*oa, rng.standard_normal((oa[1].size, 4, 4))), dtype)
        B = rounded(oracle.csr(*ob, rng.standard_normal((ob[1].size, 4, 4))), dtype)
        C = Plan(ctx, PA, PB, PC).multiply(to_dev(A["val"], dtype, ctx.device),
                                           to_dev(B["val"], dtype, ctx.device))
        ref = oracle.mprod(A, B, oc)
        assert rel_fro(C.cpu().numpy(), ref["val"]) <= TOL[dtype][0]


# ------------------------------------------------------------------ a4 traces

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("nsf", [1, 4, 9])
def test_trace_matches_oracle(ctx, dtype, nsf):
    rng = np.random.default_rng(nsf)
    pos, cell = synth.si_diamond_positions(2, rng)
    P = Pattern.build(ctx, pos, cell, 7.0)
    op = oracle.pattern(pos, cell, 7.0)
    A = rounded(oracle.csr(*op, rng.standard_normal((op[1].size, nsf, nsf))), dtype)
    B = rounded(oracle.csr(*op, rng.standard_normal((op[1].size, nsf, nsf))), dtype)
    t = trace_product(ctx, P, to_dev(A["val"], dtype, ctx.device), to_dev(B["val"], dtype, ctx.device))
    ref = oracle.trace(A, B)
    assert abs(t.item() - ref) <= 1e-12 * np.sqrt(op[1].size) * nsf * nsf


# ------------------------------------------------------------------ a1-a7 LNV evaluation

def _gpu_lnv(ctx, w, dtype, grad=True, sysm=None):
    """One evaluation with dE/dL and dN_e/dL (when grad)."""
    if sysm is None:
        sysm = System(ctx, w["nsf"], PREC[dtype], w["pos"], w["cell"], w["r_sh"], w["r_l"])
    S, H, L = (to_dev(w[k], dtype, ctx.device) for k in ("S", "H", "L"))
    if grad:
        out, G, GN = sysm.energy_grad(S, H, L, grad=True, grad_ne=True)
        return sysm, out.cpu().numpy(), (G.cpu().numpy(), GN.cpu().numpy())
    out, _ = sysm.energy_grad(S, H, L, grad=False)
    return sysm, out.cpu().numpy(), None


def _check_lnv(out, G, ref, dtype):
    tm, ts = TOL[dtype]
    assert abs(out[0, 0] - ref["E"]) <= ts * abs(ref["E"]), (out[0, 0], ref["E"])
    assert abs(out[0, 1] - ref["Ne"]) <= ts * abs(ref["Ne"]), (out[0, 1], ref["Ne"])
    for k, t in enumerate(ref["traces"]):
        assert abs(out[0, 2 + k] - t) <= ts * max(abs(t), 1e-3)
    if G is not None:
        if isinstance(G, tuple):
            G, GN = G
            assert rel_fro(GN, ref["GN"]) <= tm
        assert rel_fro(G, ref["G"]) <= tm


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("ncell,nsf,r_sh,r_l", [(1, 1, 4.0, 5.0), (2, 2, 4.0, 5.0), (2, 4, 6.6, 8.0),
                                                (2, 9, 3.0, 4.0), (3, 4, 3.0, 4.5), (3, 9, 4.0, 5.0)])
def test_lnv_small_systems(ctx, dtype, ncell, nsf, r_sh, r_l):
    w, S, H, L = workload(ncell, nsf, r_sh, r_l, seed=ncell * 10 + nsf)
    sysm, out, G = _gpu_lnv(ctx, w, dtype)
    assert np.array_equal(sysm.P_l.col.cpu().numpy(), w["l_col"])
    ref = oracle_lnv(w, rounded(S, dtype), rounded(H, dtype), rounded(L, dtype))
    _check_lnv(out, G, ref, dtype)


@pytest.fixture(scope="module")
def si512():
    w, S, H, L = workload(4, 4, 6.6, 8.0, seed=0)
    return w, oracle_lnv(w, S, H, L)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_lnv_512_atoms(ctx, si512, dtype):
    """4x4x4 cells, NSF=4, R_L = 8 A (FP32 measured against the FP64 oracle)."""
    w, ref = si512
    _, out, G = _gpu_lnv(ctx, w, dtype)
    _check_lnv(out, G, ref, dtype)


@pytest.fixture(scope="module")
def si4096():
    w, S, H, L = workload(8, 4, 6.6, 8.0, seed=0)
    return w, oracle_lnv(w, S, H, L)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_lnv_4096_atoms_full(ctx, si4096, dtype):
    """The benchmark workload (8x8x8 cells, 4096 atoms, NSF=4, R_L = 8 A) with
    the plans' default kernels, every output against the oracle."""
    w, ref = si4096
    _, out, G = _gpu_lnv(ctx, w, dtype)
    _check_lnv(out, G, ref, dtype)


@pytest.mark.parametrize("stages", [("Z",), ("W",), ("Z", "W")])
def test_lnv_512_atoms_tensor_core_products(ctx, si512, stages):
    """FP32 evaluation with Z = L T^T and / or W = X^T U^T on the tcgen05
    kernel (9), every output against the FP64 oracle at the FP32 bound."""
    w, ref = si512
    sysm = System(ctx, 4, "fp32", w["pos"], w["cell"], 6.6, 8.0)
    for st in stages:
        sysm.set_stage_kernel(st, "tensor")
    assert all(sysm.stage_kernels()[st] == "tensor" for st in stages)
    _, out, G = _gpu_lnv(ctx, w, torch.float32, sysm=sysm)
    _check_lnv(out, G, ref, torch.float32)
    assert ctx.device_status() == 0


@pytest.mark.parametrize("ncell", [2, 3])
def test_lnv_nsf9_tensor_core_products(ctx, ncell):
    """NSF = 9 systems (s, p, d) with every product stage on the tcgen05 kernel
    (10), every output against the FP64 oracle at the FP32 bound."""
    w, S, H, L = workload(ncell, 9, 6.6, 8.0, seed=17 + ncell)
    sysm = System(ctx, 9, "fp32", w["pos"], w["cell"], 6.6, 8.0)
    for st in ("XY", "TU", "Z", "Q", "W"):
        sysm.set_stage_kernel(st, "tensor9")
    assert all(k == "tensor9" for k in sysm.stage_kernels().values())
    dev = ctx.device
    Sd, Hd, Ld = (to_dev(M["val"], torch.float32, dev) for M in (S, H, L))
    ref = oracle_lnv(w, rounded(S, torch.float32), rounded(H, torch.float32), rounded(L, torch.float32))
    for mirror in (True, False):
        sysm.set_mirror(mirror)
        out, G = sysm.energy_grad(Sd, Hd, Ld)
        _check_lnv(out.cpu().numpy(), G.cpu().numpy(), ref, torch.float32)
    assert ctx.device_status() == 0


@pytest.mark.parametrize("mirror", [True, False])
def test_lnv_512_atoms_tensor_tile_products(ctx, si512, mirror):
    """FP32 evaluation with every product stage on kernel 11 (T on the tiles of
    its upper part and mirrored, or formed whole), every output against the
    FP64 oracle at the FP32 bound."""
    w, ref = si512
    sysm = System(ctx, 4, "fp32", w["pos"], w["cell"], 6.6, 8.0)
    for st in ("XY", "TU", "Z", "Q", "W"):
        sysm.set_stage_kernel(st, "tensor-tile")
    assert all(k == "tensor-tile" for k in sysm.stage_kernels().values())
    sysm.set_mirror(mirror)
    _, out, G = _gpu_lnv(ctx, w, torch.float32, sysm=sysm)
    _check_lnv(out, G, ref, torch.float32)
    assert ctx.device_status() == 0


@pytest.mark.parametrize("tu", ["group-pipe", "tensor-tile"])
def test_lnv_4096_atoms_tensor_core_products(ctx, si4096, tu):
    """The benchmark workload with Z and W on the tcgen05 kernel 9 and TU on
    the SIMT kernel or on kernel 11."""
    w, ref = si4096
    sysm = System(ctx, 4, "fp32", w["pos"], w["cell"], 6.6, 8.0)
    sysm.set_stage_kernel("Z", "tensor")
    sysm.set_stage_kernel("W", "tensor")
    sysm.set_stage_kernel("TU", tu)
    _, out, G = _gpu_lnv(ctx, w, torch.float32, sysm=sysm)
    _check_lnv(out, G, ref, torch.float32)
    assert ctx.device_status() == 0


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_lnv_4096_atoms_bench_configuration(ctx, si4096, dtype):
    """The benchmark workload in the launch configuration bench.py times: the
    system autotuned the same way (kernel per product, T mirrored or whole),
    then every output against the oracle."""
    w, ref = si4096
    sysm = System(ctx, w["nsf"], PREC[dtype], w["pos"], w["cell"], w["r_sh"], w["r_l"])
    S, H, L = (to_dev(w[k], dtype, ctx.device) for k in ("S", "H", "L"))
    sysm.autotune(S, H, L, reps=2)
    _, out, G = _gpu_lnv(ctx, w, dtype, sysm=sysm)
    _check_lnv(out, G, ref, dtype)


@pytest.mark.parametrize("nsf", [4, 9])
def test_32768_atoms_sampled_rows_bench_configuration(ctx, nsf):
    """The 16x16x16-cell workloads (32768 atoms, R_SH = 6.6 A, R_L = 10 A,
    NSF = 4 and 9) in the configuration bench.py times them (FP32, autotuned):
    dE/dL and dN_e/dL on the rows of three atoms against the row-chain oracle
    (oracle/sampled.py), which forms those rows from the definition.  With
    NSF = 4, E and N_e are also checked against an FP64 evaluation of the same
    system on the GPU, at the FP32 bound (2e-5 relative); at NSF = 9 the FP64
    intermediates (about 160 GB) are not formed."""
    from oracle.sampled import lnv_grad_rows

    w = synth.si_workload(16, nsf, 6.6, 10.0, 0, oracle.pattern)
    sysm = System(ctx, nsf, "fp32", w["pos"], w["cell"], 6.6, 10.0)
    assert np.array_equal(sysm.P_l.col.cpu().numpy(), w["l_col"])
    Sd, Hd, Ld = (to_dev(w[k], torch.float32, ctx.device) for k in ("S", "H", "L"))
    sysm.autotune(Sd, Hd, Ld, reps=1)
    out, G, GN = sysm.energy_grad(Sd, Hd, Ld, grad=True, grad_ne=True)
    S, H, L = (oracle.csr(w[rp], w[c], w[k].astype(np.float32).astype(np.float64))
               for rp, c, k in (("sh_row_ptr", "sh_col", "S"), ("sh_row_ptr", "sh_col", "H"),
                                ("l_row_ptr", "l_col", "L")))
    assert ctx.device_status() == 0
    ref = lnv_grad_rows(S, H, L, [7, 16411, 32767])
    g = G.double().cpu().numpy()[ref["pos"]]
    gn = GN.double().cpu().numpy()[ref["pos"]]
    assert rel_fro(g, ref["G"]) <= TOL[torch.float32][0]
    assert rel_fro(gn, ref["GN"]) <= TOL[torch.float32][0]
    if nsf == 4:
        o32 = out.cpu().numpy()[0]
        del sysm, G, GN, out
        torch.cuda.empty_cache()
        s64 = System(ctx, nsf, "fp64", w["pos"], w["cell"], 6.6, 10.0)
        # the FP64 evaluation of the same (FP32-rounded) inputs
        o64, _ = s64.energy_grad(Sd.double(), Hd.double(), Ld.double(), grad=False)
        o64 = o64.cpu().numpy()[0]
        assert abs(o32[0] - o64[0]) <= TOL[torch.float32][1] * abs(o64[0]), (o32[0], o64[0])
        assert abs(o32[1] - o64[1]) <= TOL[torch.float32][1] * abs(o64[1]), (o32[1], o64[1])


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_energy_grad_from_host_buffers(ctx, dtype, pinned):
    """lnv_energy_grad_host (host arrays in, results in host memory) gives the
    device-pointer evaluation's results bit for bit, with pinned or pageable
    host memory, with and without the gradient; against the oracle too."""
    w, S, H, L = workload(2, 4, 6.6, 8.0, seed=12)
    sysm = System(ctx, 4, PREC[dtype], w["pos"], w["cell"], 6.6, 8.0)
    hs = [torch.from_numpy(np.ascontiguousarray(w[k])).to(dtype) for k in ("S", "H", "L")]
    if pinned:
        hs = [t.pin_memory() for t in hs]
    out_h, G_h = sysm.energy_grad_host(*hs)
    assert out_h.device.type == "cpu" and G_h.device.type == "cpu"
    out_d, G_d = sysm.energy_grad(*(t.to(ctx.device) for t in hs))
    assert torch.equal(out_h, out_d.cpu()) and torch.equal(G_h, G_d.cpu())
    out_e, G_e = sysm.energy_grad_host(*hs, grad=False)
    assert G_e is None and torch.equal(out_e[:, :2], out_h[:, :2])
    ref = oracle_lnv(w, rounded(S, dtype), rounded(H, dtype), rounded(L, dtype))
    _check_lnv(out_h.numpy(), G_h.numpy(), ref, dtype)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_autotuned_system_matches_oracle(ctx, dtype):
    """After the autotuner picks a kernel per product, results still match."""
    w, S, H, L = workload(3, 4, 6.6, 8.0, seed=31)
    sysm = System(ctx, 4, PREC[dtype], w["pos"], w["cell"], 6.6, 8.0)
    Sd, Hd, Ld = (to_dev(w[k], dtype, ctx.device) for k in ("S", "H", "L"))
    tuned = sysm.autotune(Sd, Hd, Ld, reps=1)
    assert set(tuned) == {"XY", "TU", "Z", "Q", "W"}
    out, G = sysm.energy_grad(Sd, Hd, Ld)
    ref = oracle_lnv(w, rounded(S, dtype), rounded(H, dtype), rounded(L, dtype))
    _check_lnv(out.cpu().numpy(), G.cpu().numpy(), ref, dtype)


def test_energy_only_matches_gradient_run(ctx):
    w, S, H, L = workload(2, 4, 6.6, 8.0, seed=3)
    sysm, out_g, (_, GN) = _gpu_lnv(ctx, w, torch.float64, grad=True)
    _, out_e, G = _gpu_lnv(ctx, w, torch.float64, grad=False, sysm=sysm)
    assert G is None
    assert np.array_equal(out_g, out_e)
    # dN_e/dL alone (no dE/dL) equals the one formed beside the gradient
    Sd, Hd, Ld = (to_dev(w[k], torch.float64, ctx.device) for k in ("S", "H", "L"))
    out_n, G_n, GN_n = sysm.energy_grad(Sd, Hd, Ld, grad=False, grad_ne=True)
    assert G_n is None
    assert np.array_equal(out_n.cpu().numpy(), out_e) and np.array_equal(GN_n.cpu().numpy(), GN)


def test_single_atom_closed_form(ctx):
    """NSF = 1, one atom: E = 2h(3 l^2 s - 2 l^3 s^2), dE/dl = 2h(6 l s - 6 l^2 s^2),
    dN_e/dl = 2(6 l s^2 - 6 l^2 s^3)."""
    s, h, l = 1.3, -0.7, 0.45
    sysm = System(ctx, 1, "fp64", np.zeros((1, 3)), [10.0, 10.0, 10.0], 3.0, 3.0)
    S, H, L = (torch.tensor([[[v]]], dtype=torch.float64, device=ctx.device) for v in (s, h, l))
    out, G, GN = sysm.energy_grad(S, H, L, grad_ne=True)
    out = out.cpu().numpy()[0]
    assert out[0] == pytest.approx(2 * h * (3 * l * l * s - 2 * l ** 3 * s * s), rel=1e-14)
    assert out[1] == pytest.approx(2 * (3 * l * l * s * s - 2 * l ** 3 * s ** 3), rel=1e-14)
    assert G.item() == pytest.approx(2 * h * (6 * l * s - 6 * l * l * s * s), rel=1e-14)
    assert GN.item() == pytest.approx(2 * (6 * l * s * s - 6 * l * l * s ** 3), rel=1e-14)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_deterministic_and_external_workspace(ctx, dtype):
    w, S, H, L = workload(3, 4, 6.6, 8.0, seed=9)
    sysm, out1, G1 = _gpu_lnv(ctx, w, dtype)
    _, out2, G2 = _gpu_lnv(ctx, w, dtype, sysm=sysm)
    assert np.array_equal(out1, out2) and np.array_equal(G1, G2)
    ws = torch.empty(sysm.workspace_size(True), dtype=torch.uint8, device=ctx.device)
    Sd, Hd, Ld = (to_dev(w[k], dtype, ctx.device) for k in ("S", "H", "L"))
    out3, G3, GN3 = sysm.energy_grad(Sd, Hd, Ld, workspace=ws, grad_ne=True)
    assert np.array_equal(out3.cpu().numpy(), out1) and np.array_equal(G3.cpu().numpy(), G1[0])
    assert np.array_equal(GN3.cpu().numpy(), G1[1])


# ------------------------------------------------------------------ a8 batched systems

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_systems_equal_single_runs(ctx, dtype):
    sizes = [2, 3, 2, 4]
    ws = [workload(n, 4, 6.6, 8.0, seed=1000 + k)[0] for k, n in enumerate(sizes)]
    off = [0]
    for w in ws:
        off.append(off[-1] + w["pos"].shape[0])
    sysb = System(ctx, 4, PREC[dtype], np.concatenate([w["pos"] for w in ws]), [w["cell"] for w in ws],
                  6.6, 8.0, seg_off=off)
    cat = {k: to_dev(np.concatenate([w[k] for w in ws]), dtype, ctx.device) for k in ("S", "H", "L")}
    out_b, G_b, GN_b = sysb.energy_grad(cat["S"], cat["H"], cat["L"], grad_ne=True)
    out_b, G_b, GN_b = out_b.cpu().numpy(), G_b.cpu().numpy(), GN_b.cpu().numpy()
    gofs = 0
    for k, w in enumerate(ws):
        _, out, (G, GN) = _gpu_lnv(ctx, w, dtype)
        assert np.array_equal(out_b[k], out[0])
        assert np.array_equal(G_b[gofs:gofs + G.shape[0]], G)
        assert np.array_equal(GN_b[gofs:gofs + G.shape[0]], GN)
        gofs += G.shape[0]


def test_argument_errors(ctx):
    w, S, H, L = workload(1, 4, 4.0, 5.0)
    sysm = System(ctx, 4, "fp64", w["pos"], w["cell"], 4.0, 5.0)
    S32 = to_dev(w["S"], torch.float32, ctx.device)
    Sd, Hd, Ld = (to_dev(w[k], torch.float64, ctx.device) for k in ("S", "H", "L"))
    with pytest.raises(ValueError):
        sysm.energy_grad(S32, Hd, Ld)
    with pytest.raises(ValueError):
        sysm.energy_grad(Sd[:-1], Hd, Ld)
    with pytest.raises(LnvError) as e:
        System(ctx, 3, "fp64", w["pos"], w["cell"], 4.0, 5.0)
    assert e.value.status == -1
    ws = torch.empty(16, dtype=torch.uint8, device=ctx.device)
    with pytest.raises(LnvError):
        sysm.energy_grad(Sd, Hd, Ld, workspace=ws)


# ------------------------------------------------------------------ autograd (recompute backward)

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_autograd_energy_gradient_matches_oracle(ctx, dtype):
    from paper_0911_3584_gb300 import lnv_energy
    w, S, H, L = workload(2, 4, 6.6, 8.0, seed=41)
    sysm = System(ctx, 4, PREC[dtype], w["pos"], w["cell"], 6.6, 8.0)
    Sd, Hd = (to_dev(w[k], dtype, ctx.device) for k in ("S", "H"))
    Ld = to_dev(w["L"], dtype, ctx.device).requires_grad_(True)
    E, Ne = lnv_energy(Ld, sysm, Sd, Hd)
    (3.0 * E).backward()
    ref = oracle_lnv(w, rounded(S, dtype), rounded(H, dtype), rounded(L, dtype))
    tm, ts = TOL[dtype]
    assert abs(E.item() - ref["E"]) <= ts * abs(ref["E"])
    assert abs(Ne.item() - ref["Ne"]) <= ts * abs(ref["Ne"])
    assert rel_fro(Ld.grad.cpu().numpy(), 3.0 * ref["G"]) <= tm


def test_autograd_gradient_against_central_differences(ctx):
    """Central differences of E(L + tD) in FP64 (step 1e-6) on 20 random blocks
    against <dE/dL, D> from the recompute backward."""
    from paper_0911_3584_gb300 import lnv_energy
    w, S, H, L = workload(3, 4, 6.6, 8.0, seed=43)
    sysm = System(ctx, 4, "fp64", w["pos"], w["cell"], 6.6, 8.0)
    Sd, Hd = (to_dev(w[k], torch.float64, ctx.device) for k in ("S", "H"))
    L0 = to_dev(w["L"], torch.float64, ctx.device)
    Lg = L0.clone().requires_grad_(True)
    E, _ = lnv_energy(Lg, sysm, Sd, Hd)
    E.backward()
    G = Lg.grad
    rp, col = w["l_row_ptr"], w["l_col"]
    n = rp.size - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    key = rows * n + col
    rng = np.random.default_rng(5)
    h = 1e-6
    for p in rng.choice(col.size, size=20, replace=False):
        i, j = rows[p], col[p]
        D = torch.zeros_like(L0)
        blk = torch.from_numpy(rng.standard_normal((4, 4))).to(ctx.device)
        if i == j:
            blk = 0.5 * (blk + blk.T)
        D[p] = blk
        D[int(np.searchsorted(key, j * n + i))] = blk.T
        ep = sysm.energy_grad(Sd, Hd, L0 + h * D, grad=False)[0][0, 0].item()
        em = sysm.energy_grad(Sd, Hd, L0 - h * D, grad=False)[0][0, 0].item()
        fd = (ep - em) / (2 * h)
        an = float((G * D).sum())
        # central differences of a cubic: error h^2 E'''/6 plus rounding eps |E| / h
        assert fd == pytest.approx(an, rel=1e-6, abs=1e-7)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_graph_captured_batched_evaluation(ctx, dtype):
    """Many systems in one block-diagonal evaluation captured in a CUDA graph:
    replays equal direct evaluations, including after L changes in place."""
    sizes = [2, 3, 2]
    ws = [workload(n, 4, 6.6, 8.0, seed=1000 + k)[0] for k, n in enumerate(sizes)]
    off = [0]
    for w in ws:
        off.append(off[-1] + w["pos"].shape[0])
    sysb = System(ctx, 4, PREC[dtype], np.concatenate([w["pos"] for w in ws]), [w["cell"] for w in ws],
                  6.6, 8.0, seg_off=off)
    cat = {k: to_dev(np.concatenate([w[k] for w in ws]), dtype, ctx.device) for k in ("S", "H", "L")}
    sysb.autotune(cat["S"], cat["H"], cat["L"], reps=1)
    graph, out_g, G_g = sysb.capture(cat["S"], cat["H"], cat["L"])
    for scale in (1.0, 0.9):
        cat["L"].mul_(scale)
        graph.replay()
        torch.cuda.synchronize()
        out_d, G_d = sysb.energy_grad(cat["S"], cat["H"], cat["L"])
        assert torch.equal(out_g, out_d) and torch.equal(G_g, G_d)
    # every system against the oracle at the stated bounds: E, N_e and dE/dL,
    # with the oracle given exactly the L values the device holds after the
    # in-place scaling (and the S, H values of the device's precision)
    L_dev = cat["L"].double().cpu().numpy()
    G_dev = G_g.double().cpu().numpy()
    lb = 0
    for k, w in enumerate(ws):
        nl = w["l_col"].size
        Lk = L_dev[lb:lb + nl]
        ref = oracle.lnv_energy_grad(w["pos"], w["cell"], 6.6, 8.0,
                                     rounded(oracle.csr(w["sh_row_ptr"], w["sh_col"], w["S"]), dtype),
                                     rounded(oracle.csr(w["sh_row_ptr"], w["sh_col"], w["H"]), dtype),
                                     oracle.csr(w["l_row_ptr"], w["l_col"], Lk))
        o = out_g[k].cpu().numpy()
        tm, ts = TOL[dtype]
        assert abs(o[0] - ref["E"]) <= ts * abs(ref["E"]), (k, o[0], ref["E"])
        assert abs(o[1] - ref["Ne"]) <= ts * abs(ref["Ne"]), (k, o[1], ref["Ne"])
        assert rel_fro(G_dev[lb:lb + nl], ref["G"]) <= tm, k
        lb += nl
    assert lb == G_dev.shape[0]


@pytest.mark.parametrize("kernels", [
    dict(XY="triples", TU="tensor-tile", Z="tensor", Q="tensor-tile", W="tensor"),
    dict(XY="triples", TU="tensor-tile-1pass", Z="tensor-1pass", Q="tensor-tile-1pass", W="tensor-1pass")])
def test_graph_captured_tensor_core_kernels(ctx, kernels):
    """The batched FP32 evaluation with the tcgen05 kernels pinned (the bench's
    choice, and its single-pass form) captured in a CUDA graph: replays equal
    direct evaluations bit for bit after L changes in place, and every system
    stays within its bound of the oracle (FP32, or single-pass TF32)."""
    sizes = [3, 2, 4]
    ws = [workload(n, 4, 6.6, 8.0, seed=2000 + k)[0] for k, n in enumerate(sizes)]
    off = [0]
    for w in ws:
        off.append(off[-1] + w["pos"].shape[0])
    sysb = System(ctx, 4, "fp32", np.concatenate([w["pos"] for w in ws]), [w["cell"] for w in ws],
                  6.6, 8.0, seg_off=off)
    for st, k in kernels.items():
        sysb.set_stage_kernel(st, k)
    assert sysb.stage_kernels() == kernels
    cat = {k: to_dev(np.concatenate([w[k] for w in ws]), torch.float32, ctx.device) for k in ("S", "H", "L")}
    graph, out_g, G_g = sysb.capture(cat["S"], cat["H"], cat["L"])
    for scale in (1.0, 0.9):
        cat["L"].mul_(scale)
        graph.replay()
        torch.cuda.synchronize()
        out_d, G_d = sysb.energy_grad(cat["S"], cat["H"], cat["L"])
        assert torch.equal(out_g, out_d) and torch.equal(G_g, G_d)
    assert ctx.device_status() == 0
    one = kernels["Z"].endswith("1pass")
    tm, ts = (TOL_1PASS, TOL_1PASS) if one else TOL[torch.float32]
    L_dev = cat["L"].double().cpu().numpy()
    G_dev = G_g.double().cpu().numpy()
    lb = 0
    for k, w in enumerate(ws):
        nl = w["l_col"].size
        ref = oracle.lnv_energy_grad(w["pos"], w["cell"], 6.6, 8.0,
                                     rounded(oracle.csr(w["sh_row_ptr"], w["sh_col"], w["S"]), torch.float32),
                                     rounded(oracle.csr(w["sh_row_ptr"], w["sh_col"], w["H"]), torch.float32),
                                     oracle.csr(w["l_row_ptr"], w["l_col"], L_dev[lb:lb + nl]))
        o = out_g[k].cpu().numpy()
        assert abs(o[0] - ref["E"]) <= ts * abs(ref["E"]), (k, o[0], ref["E"])
        assert abs(o[1] - ref["Ne"]) <= ts * abs(ref["Ne"]), (k, o[1], ref["Ne"])
        assert rel_fro(G_dev[lb:lb + nl], ref["G"]) <= tm, k
        lb += nl


# ------------------------------------------------------------------ minimisation (next row)

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n", [0, 1, 1000, 300001])
def test_vector_kernels(ctx, dtype, n):
    from paper_0911_3584_gb300 import vec_axpby, vec_dot
    rng = np.random.default_rng(n)
    x64, y64 = rng.standard_normal(n), rng.standard_normal(n)
    x, y = to_dev(x64, dtype, ctx.device), to_dev(y64, dtype, ctx.device)
    xr, yr = x.cpu().double().numpy(), y.cpu().double().numpy()
    a, b = 0.75, -1.3
    z = vec_axpby(ctx, a, x, b, y).cpu().double().numpy()
    ref = a * xr + b * yr
    ulp = np.finfo(np.float64 if dtype == torch.float64 else np.float32).eps
    assert np.all(np.abs(z - ref) <= 2 * ulp * (np.abs(a * xr) + np.abs(b * yr)) + 1e-300)
    # y is not read when its factor is 0 (NaN there must not leak)
    if n:
        ynan = torch.full_like(y, float("nan"))
        assert torch.equal(vec_axpby(ctx, 2.0, x, 0.0, ynan), (2.0 * x.double()).to(dtype))
    d = vec_dot(ctx, x, y).item()
    assert d == pytest.approx(float(xr @ yr), rel=1e-13, abs=1e-13 * np.sqrt(max(n, 1)))
    assert vec_dot(ctx, x, y).item() == d  # fixed reduction order


def _dense_min_system(ctx, dtype, m):
    """Untruncated 8-atom system (every range past the box), mu in the gap
    above the m-th generalised eigenvalue of (H, S), L = S^-1 / 2."""
    linalg = pytest.importorskip("scipy.linalg")
    from tests.dense_ref import from_dense, to_dense
    w, S, H, L = workload(1, 4, 5.0, 5.0, seed=12)
    Sd = to_dense(S["rp"], S["col"], S["val"])
    Hd = to_dense(H["rp"], H["col"], H["val"])
    eps = linalg.eigh(Hd, Sd, eigvals_only=True)
    mu = 0.5 * (eps[m - 1] + eps[m])
    L0 = from_dense(0.5 * np.linalg.inv(Sd), L["rp"], L["col"], 4)
    return w, S, H, oracle.csr(L["rp"], L["col"], L0), eps, mu


@pytest.mark.parametrize("m", [5, 16, 24])
def test_minimisation_reaches_ground_state(ctx, m):
    """lnv_minimize (FP64) reaches E = 2 sum eps_1..m and N_e = 2m, as the
    oracle's loop does."""
    w, S, H, L0, eps, mu = _dense_min_system(ctx, torch.float64, m)
    sysm = System(ctx, 4, "fp64", w["pos"], w["cell"], 5.0, 5.0)
    Sd, Hd, Ld = (to_dev(v, torch.float64, ctx.device) for v in (S["val"], H["val"], L0["val"]))
    iters, hist = sysm.minimize(Sd, Hd, Ld, mu, max_iter=400, tol=1e-8)
    assert iters < 400
    E, Ne = hist[-1, 1], hist[-1, 2]
    assert E == pytest.approx(2 * eps[:m].sum(), rel=1e-10, abs=1e-10)
    assert Ne == pytest.approx(2 * m, rel=1e-10)
    assert np.all(np.diff(hist[:, 0]) <= 1e-12 * abs(hist[-1, 0]))
    # the evaluation of the returned L agrees with the history's last row
    out, _ = sysm.energy_grad(Sd, Hd, Ld, grad=False)
    assert out[0, 1].item() == pytest.approx(Ne, rel=1e-12)


def test_minimisation_fp32(ctx):
    """FP32 products: the loop stops at the rounding of Omega, within 1e-5 of
    the ground-state energy."""
    m = 16
    w, S, H, L0, eps, mu = _dense_min_system(ctx, torch.float32, m)
    sysm = System(ctx, 4, "fp32", w["pos"], w["cell"], 5.0, 5.0)
    Sd, Hd, Ld = (to_dev(v, torch.float32, ctx.device) for v in (S["val"], H["val"], L0["val"]))
    _, hist = sysm.minimize(Sd, Hd, Ld, mu, max_iter=400, tol=1e-6)
    assert hist[-1, 1] == pytest.approx(2 * eps[:m].sum(), rel=1e-5)
    assert hist[-1, 2] == pytest.approx(2 * m, rel=1e-5)


def test_minimisation_truncated_matches_oracle(ctx):
    """64 atoms with R_L = 4.5 A inside the 10.9 A box: the truncated minimum
    found on the GPU equals the oracle loop's."""
    from oracle.minimize import lnv_minimize as oracle_minimize
    linalg = pytest.importorskip("scipy.linalg")
    from tests.dense_ref import to_dense
    w, S, H, L = workload(2, 4, 3.0, 4.5, seed=5)
    Sd = to_dense(S["rp"], S["col"], S["val"])
    Hd = to_dense(H["rp"], H["col"], H["val"])
    eps = linalg.eigh(Hd, Sd, eigvals_only=True)
    m = 64
    mu = 0.5 * (eps[m - 1] + eps[m])
    # start from the diagonal blocks of S^-1 / 2 (inside L's pattern)
    Sinv = np.linalg.inv(Sd)
    rows = np.repeat(np.arange(w["pos"].shape[0]), np.diff(L["rp"]))
    L0 = np.zeros_like(L["val"])
    for p, (i, j) in enumerate(zip(rows, L["col"])):
        if i == j:
            L0[p] = 0.5 * Sinv[4 * i:4 * i + 4, 4 * j:4 * j + 4]
    Lo, ho = oracle_minimize(w["pos"], w["cell"], 3.0, 4.5, S, H, oracle.csr(L["rp"], L["col"], L0), mu,
                             max_iter=300, tol=1e-8)
    sysm = System(ctx, 4, "fp64", w["pos"], w["cell"], 3.0, 4.5)
    Sg, Hg, Lg = (to_dev(v, torch.float64, ctx.device) for v in (S["val"], H["val"], L0))
    _, hg = sysm.minimize(Sg, Hg, Lg, mu, max_iter=300, tol=1e-8)
    assert hg[-1, 0] == pytest.approx(ho[-1, 0], rel=1e-9)
    assert hg[-1, 2] == pytest.approx(ho[-1, 2], rel=1e-7)
    assert hg[-1, 0] >= 2 * (eps[:m] - mu).sum() - 1e-9  # truncation cannot beat the exact minimum


# ------------------------------------------------------------------ truncated intermediates (next row)

@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("r_x,r_t", [(4.5, 4.5), (5.0, 6.0), (6.0, 8.0), (None, 8.0), (None, None)])
def test_truncated_system_matches_oracle(ctx, dtype, r_x, r_t):
    """512 atoms, R_SH = 3, R_L = 4.5: X, Y, Z kept within r_x and T, U within
    r_t, against the oracle's definition of the same truncation."""
    w, S, H, L = workload(4, 4, 3.0, 4.5, seed=6)
    sysm = System(ctx, 4, PREC[dtype], w["pos"], w["cell"], 3.0, 4.5, r_x=r_x, r_t=r_t)
    Sd, Hd, Ld = (to_dev(w[k], dtype, ctx.device) for k in ("S", "H", "L"))
    out, G = sysm.energy_grad(Sd, Hd, Ld)
    ref = oracle.lnv_energy_grad_truncated(w["pos"], w["cell"], 3.0, 4.5, r_x or 7.5, r_t or 10.5,
                                           rounded(S, dtype), rounded(H, dtype), rounded(L, dtype))
    _check_lnv(out.cpu().numpy(), G.cpu().numpy(), ref, dtype)


def test_truncation_ranges_are_checked(ctx):
    w, S, H, L = workload(2, 4, 3.0, 4.5)
    for r_x, r_t in [(4.0, None), (8.0, None), (None, 4.0), (None, 11.0)]:
        with pytest.raises(LnvError):
            System(ctx, 4, "fp64", w["pos"], w["cell"], 3.0, 4.5, r_x=r_x, r_t=r_t)


# ------------------------------------------------------------------ L carried between geometries (next row)

def _remap_ref(rp_f, col_f, vals, rp_t, col_t):
    n = len(rp_f) - 1
    where = {}
    for i in range(n):
        for q in range(rp_f[i], rp_f[i + 1]):
            where[(i, int(col_f[q]))] = q
    out = np.zeros((len(col_t),) + vals.shape[1:], vals.dtype)
    for i in range(n):
        for p in range(rp_t[i], rp_t[i + 1]):
            q = where.get((i, int(col_t[p])))
            if q is not None:
                out[p] = vals[q]
    return out


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("r_from,r_to", [(5.0, 5.0), (5.0, 6.5), (6.5, 4.0)])
def test_pattern_remap_is_exact(ctx, dtype, r_from, r_to):
    rng = np.random.default_rng(int(10 * r_from + r_to))
    pos, cell = synth.si_diamond_positions(2, rng)
    Pf = Pattern.build(ctx, pos, cell, r_from)
    Pt = Pattern.build(ctx, pos, cell, r_to)
    vals = torch.from_numpy(rng.standard_normal((Pf.nnzb, 4, 4))).to(ctx.device, dtype)
    got = Pf.remap(vals, Pt).cpu().numpy()
    ref = _remap_ref(Pf.row_ptr.cpu().numpy(), Pf.col.cpu().numpy(), vals.cpu().numpy(),
                     Pt.row_ptr.cpu().numpy(), Pt.col.cpu().numpy())
    assert np.array_equal(got, ref)


def test_warm_start_after_a_geometry_step(ctx):
    """Minimise at one geometry, move the atoms by ~0.01 A (L's pattern changes),
    and start the next minimisation from the previous L carried onto the new
    pattern: it reaches the cold start's minimum in fewer iterations."""
    linalg = pytest.importorskip("scipy.linalg")
    from tests.dense_ref import to_dense
    d = np.random.default_rng(1).normal(0.0, 0.01, (64, 3))
    w0 = synth.si_workload(2, 4, 3.0, 4.5, 5, oracle.pattern)
    w1 = synth.si_workload(2, 4, 3.0, 4.5, 5, oracle.pattern, displace=d)
    assert not np.array_equal(w0["l_col"], w1["l_col"])
    Sd = to_dense(w0["sh_row_ptr"], w0["sh_col"], w0["S"])
    Hd = to_dense(w0["sh_row_ptr"], w0["sh_col"], w0["H"])
    eps = linalg.eigh(Hd, Sd, eigvals_only=True)
    mu = 0.5 * (eps[63] + eps[64])

    def cold_start(w, sysm):
        Sinv = np.linalg.inv(to_dense(w["sh_row_ptr"], w["sh_col"], w["S"]))
        P = sysm.P_l
        rows = np.repeat(np.arange(64), np.diff(P.row_ptr.cpu().numpy()))
        L0 = np.zeros((P.nnzb, 4, 4))
        for p, (i, j) in enumerate(zip(rows, P.col.cpu().numpy())):
            if i == j:
                L0[p] = 0.5 * Sinv[4 * i:4 * i + 4, 4 * j:4 * j + 4]
        return to_dev(L0, torch.float64, ctx.device)

    s0 = System(ctx, 4, "fp64", w0["pos"], w0["cell"], 3.0, 4.5)
    S0, H0 = (to_dev(w0[k], torch.float64, ctx.device) for k in ("S", "H"))
    L0 = cold_start(w0, s0)
    s0.minimize(S0, H0, L0, mu, max_iter=400, tol=1e-8)

    s1 = System(ctx, 4, "fp64", w1["pos"], w1["cell"], 3.0, 4.5)
    S1, H1 = (to_dev(w1[k], torch.float64, ctx.device) for k in ("S", "H"))
    Lc = cold_start(w1, s1)
    it_cold, h_cold = s1.minimize(S1, H1, Lc, mu, max_iter=400, tol=1e-8)
    Lw = s0.P_l.remap(L0, s1.P_l)
    it_warm, h_warm = s1.minimize(S1, H1, Lw, mu, max_iter=400, tol=1e-8)
    assert h_warm[-1, 0] == pytest.approx(h_cold[-1, 0], rel=1e-9)
    assert it_warm < it_cold, (it_warm, it_cold)
    # the carried L starts far closer to the minimum than the cold start
    assert h_warm[0, 0] - h_warm[-1, 0] < 1e-2 * (h_cold[0, 0] - h_cold[-1, 0])
