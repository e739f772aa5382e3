"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2).

Each rank evaluates its own independent system (weak scaling); the job time
is the slowest rank's and the throughput counts every rank's atoms.  No GPU
and no collective in the data path: only the timing all-reduce.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        value, tmax = bench.aggregate(times[rank], atoms_per_rank=4096, steps=10, dist=dist, device="cpu")
        q.put((rank, value, tmax))
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(1.0, 2.0), (0.5, 0.25)])
def test_weak_scaling_aggregate_over_two_gloo_ranks(times):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    tmax = max(times)
    for rank, value, t in out:
        assert t == pytest.approx(tmax)
        assert value == pytest.approx(4096 * 2 * 10 / tmax)


def test_single_rank_aggregate():
    import bench
    value, t = bench.aggregate(2.0, atoms_per_rank=4096, steps=10, dist=None, device="cpu")
    assert t == 2.0 and value == pytest.approx(4096 * 10 / 2.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the oracle arm runs (and prints) on rank 0 only."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    called = []
    monkeypatch.setattr(bench, "reference_arm", lambda args: called.append(args))
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference"])
    bench.main()
    assert called == [] and capsys.readouterr().out == ""


# ---------------------------------------------------------------- work distribution (shard.py)

def test_lpt_assignment_properties():
    """Every system exactly once; the largest load within Graham's bound for
    list scheduling (total / m + max), and no worse than a round-robin deal."""
    from paper_0911_3584_gb300.shard import assign_lpt, lpt_loads
    rng = np.random.default_rng(3)
    for m in (1, 2, 3, 4, 8):
        w = rng.integers(1, 1000, size=37).astype(float)
        a = assign_lpt(w, m)
        assert sorted(i for part in a for i in part) == list(range(37))
        loads = lpt_loads(w, a)
        assert max(loads) <= w.sum() / m + w.max() + 1e-9
        rr = [w[r::m].sum() for r in range(m)]
        assert max(loads) <= max(rr) + 1e-9
    assert assign_lpt([5, 4, 3, 3, 2, 2, 1], 3) == [[0, 5], [1, 4, 6], [2, 3]]


def _small_systems():
    # independent periodic Si systems of uneven size (1^3 to 2^3 cells, NSF = 2)
    import oracle
    import synth
    specs = [(1, 11), (2, 12), (1, 13), (2, 14), (2, 15), (1, 16)]
    return [synth.si_workload(n, 2, 4.0, 5.0, seed, oracle.pattern) for n, seed in specs]


def _eval_system(w):
    import oracle
    S, H, L = (oracle.csr(w[r], w[c], w[k]) for r, c, k in
               (("sh_row_ptr", "sh_col", "S"), ("sh_row_ptr", "sh_col", "H"), ("l_row_ptr", "l_col", "L")))
    o = oracle.lnv_energy_grad(w["pos"], w["cell"], w["r_sh"], w["r_l"], S, H, L)
    return o["E"], o["Ne"], o["G"]


def _batched_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_0911_3584_gb300.shard import assign_lpt
        ws = _small_systems()
        work = [w["pos"].shape[0] * w["l_col"].size for w in ws]
        mine = assign_lpt(work, world)[rank]
        res = {s: _eval_system(ws[s]) for s in mine}
        allres = [None] * world
        dist.all_gather_object(allres, res)
        if rank == 0:
            union = {}
            for d in allres:
                assert not set(d) & set(union)
                union.update(d)
            q.put({s: (e, n, g.tobytes()) for s, (e, n, g) in union.items()})
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _spawn(target, world, *extra):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, world, port, q) + extra) for r in range(world)]
    for p in procs:
        p.start()
    out = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("world", [2, 4])
def test_batched_systems_split_over_gloo_ranks(world):
    """The batched workload's split: whole systems to ranks by work (LPT),
    each rank evaluating its own with no data exchange; the gathered union
    equals the single-rank evaluation of every system, bit for bit."""
    out = _spawn(_batched_worker, world)
    ws = _small_systems()
    assert sorted(out) == list(range(len(ws)))
    for s, w in enumerate(ws):
        e, n, g = _eval_system(w)
        assert out[s][0] == e and out[s][1] == n and out[s][2] == g.tobytes()


def _touched(A_pat, B_pat, C_pat, owned, own_mask):
    """Non-owned rows k with A_ik, B_kj and C_ij all in their patterns for some
    owned i: the rows of B a product over the owned rows really reads."""
    (arp, acol), (brp, bcol), (crp, ccol) = A_pat, B_pat, C_pat
    out = set()
    for i in owned:
        cset = set(ccol[crp[i]:crp[i + 1]].tolist())
        for k in acol[arp[i]:arp[i + 1]]:
            if own_mask[k] or k in out:
                continue
            if cset.intersection(bcol[brp[k]:brp[k + 1]].tolist()):
                out.add(int(k))
    return out


def _partition_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        import synth
        from paper_0911_3584_gb300.shard import halo_rows, local_rows, lnv_partitioned, row_parts
        w = synth.si_workload(4, 2, 3.0, 4.5, 21, oracle.pattern)
        n = w["pos"].shape[0]
        full = {k: oracle.csr(w[r], w[c], w[k]) for r, c, k in
                (("sh_row_ptr", "sh_col", "S"), ("sh_row_ptr", "sh_col", "H"), ("l_row_ptr", "l_col", "L"))}
        parts = row_parts(np.arange(n), world)  # atoms are cell-ordered: contiguous runs are compact
        mine = parts[rank]
        loc = {k: local_rows(v, mine) for k, v in full.items()}
        res = lnv_partitioned(dist, parts, oracle.pattern, w["pos"], w["cell"], 3.0, 4.5, loc["S"], loc["H"],
                              loc["L"], lambda A, B, pat, rows: oracle.mprod(A, B, pat, rows),
                              lambda A, B, rows: oracle.trace(A, B, rows=rows))
        # halo sets: exactly the rows the owned products touch
        own = np.zeros(n, bool)
        own[mine] = True
        px, pt = oracle.pattern(w["pos"], w["cell"], 7.5), oracle.pattern(w["pos"], w["cell"], 10.5)
        psh = (w["sh_row_ptr"], w["sh_col"])
        pl = (w["l_row_ptr"], w["l_col"])
        for A_pat, B_pat, C_pat in [(pl, psh, px), (psh, px, pt), (pl, pt, px), (px, pt, pl), (psh, px, pl)]:
            h = set(halo_rows(A_pat[0], A_pat[1], mine).tolist())
            assert h == _touched(A_pat, B_pat, C_pat, mine, own)
        rows = np.concatenate([np.arange(w["l_row_ptr"][i], w["l_row_ptr"][i + 1]) for i in mine])
        q_out = {"E": res["E"], "Ne": res["Ne"], "rows": rows, "G": res["G"][rows],
                 "recv": res["values_received"], "halo": res["halo_rows"]}
        allres = [None] * world
        dist.all_gather_object(allres, q_out)
        if rank == 0:
            q.put(allres)
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_row_partition_with_halo_exchange_over_gloo_ranks(world):
    """One 512-atom system split into spatially compact row parts over 2 or 4
    gloo ranks, each product formed on the owned rows after a point-to-point
    halo exchange, the four traces all-reduced: E and N_e equal the
    single-rank oracle to rounding, each rank's rows of dE/dL exactly, and
    the halo sets equal the rows the owned products touch (checked in the
    ranks).  Only a part of the matrices moves between ranks."""
    import oracle
    import synth
    allres = _spawn(_partition_worker, world)
    w = synth.si_workload(4, 2, 3.0, 4.5, 21, oracle.pattern)
    S, H, L = (oracle.csr(w[r], w[c], w[k]) for r, c, k in
               (("sh_row_ptr", "sh_col", "S"), ("sh_row_ptr", "sh_col", "H"), ("l_row_ptr", "l_col", "L")))
    ref = oracle.lnv_energy_grad(w["pos"], w["cell"], 3.0, 4.5, S, H, L)
    covered = np.zeros(ref["G"].shape[0], bool)
    for r in allres:
        assert r["E"] == pytest.approx(ref["E"], rel=1e-13)
        assert r["Ne"] == pytest.approx(ref["Ne"], rel=1e-13)
        assert np.array_equal(r["G"], ref["G"][r["rows"]])
        covered[r["rows"]] = True
        assert 0 < r["recv"]
    assert covered.all()
