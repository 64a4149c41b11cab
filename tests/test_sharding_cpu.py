"""Multi-rank logic on CPU process groups (gloo, world sizes 2, 3 and 4, and
5 where some ranks own no rows).

Each rank computes its share with the oracle; the gathered results must equal
the single-rank oracle: the Jacobi field and every per-sweep residual bit for
bit (§5: a reduction's partials combined across the teams of an SPMD region,
§3.1), matvec rows and the GEMM's 2D output tiles (panels broadcast along
process rows and columns) exactly on integer data and to FP64 rounding on
random data, AXPY's y bit for bit and its sum within the FP32 tolerance, and
every region of a batch run exactly once."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import upir_inputs as I
from oracle import upir_oracle as O
from paper_2209_10643_b300.sharding import (AxpyBlocks, GemmPanels, JacobiRowBlocks, MatvecRowBlocks,
                                            aggregate_throughput, block_range, rank_grid, region_bytes,
                                            shard_lpt)


def test_shard_lpt_partitions_every_item_once():
    costs = [5, 1, 9, 3, 3, 7, 2, 8, 1, 4]
    for world in (1, 2, 3, 4, 16):
        parts = shard_lpt(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        if world <= len(costs):
            assert max(loads) - min(loads) <= max(costs)
    assert shard_lpt([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        shard_lpt([1.0], 0)


def test_block_range_is_the_static_blocked_schedule():
    # the same owner map as the oracle's static schedule without chunk
    for n in range(0, 23):
        for world in range(1, 8):
            owner = O.static_owner_map(n, world, 0)
            for r in range(world):
                lo, hi = block_range(5, 5 + n, world, r)
                assert list(np.nonzero(owner == r)[0] + 5) == list(range(lo, hi))
    with pytest.raises(ValueError):
        block_range(0, 4, 2, 2)


def test_jacobi_plan_geometry():
    p = [JacobiRowBlocks(10, 7, 3, r) for r in range(3)]
    assert [(q.lo, q.hi) for q in p] == [(1, 4), (4, 7), (7, 9)]
    assert [q.local_rows for q in p] == [5, 5, 4]
    assert [(q.up, q.down) for q in p] == [(None, 1), (0, 2), (1, None)]
    q = [JacobiRowBlocks(5, 7, 5, r) for r in range(5)]  # 3 interior rows, 5 ranks
    assert [x.local_rows for x in q] == [3, 3, 3, 0, 0]
    assert q[2].down is None and q[3].up is None


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spawn(fn, world, *args):
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(fn, args=(world, port, out, *args), nprocs=world, start_method="spawn", join=True)
    return dict(out)


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _aggregate_worker(rank, world, port, out):
    _init(rank, world, port)
    try:
        out[rank] = aggregate_throughput(100.0 * (rank + 1), 0.5 + rank)
    finally:
        dist.destroy_process_group()


def test_aggregate_throughput_gloo_world2():
    out = _spawn(_aggregate_worker, 2)
    assert out[0] == out[1] == (300.0, 1.5)


def test_aggregate_without_group_is_identity():
    assert aggregate_throughput(7.0, 2.0) == (7.0, 2.0)


# ---------------------------------------------------------------- Jacobi --

def _jacobi_worker(rank, world, port, out, rows, cols, sweeps):
    _init(rank, world, port)
    try:
        u0 = I.jacobi_grid(rows, cols, seed=3)
        plan = JacobiRowBlocks(rows, cols, world, rank)
        a = torch.from_numpy(plan.slab(u0).copy())
        b = a.clone()
        res = torch.full((sweeps,), -np.inf, dtype=torch.float32)

        def sweep(src, dst, k):
            # this rank's rows by the oracle's FP32 mirror of one sweep
            v, r = O.jacobi_sweep_f32(src.numpy())
            dst.numpy()[1:-1, 1:-1] = v[1:-1, 1:-1]
            res[k] = float(r)

        final = plan.run(sweep, a, b, sweeps, res)
        full = plan.gather(final if plan.local_rows else torch.zeros((0, cols)))
        out[rank] = (full.numpy().copy(), res.numpy().copy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,rows,cols,sweeps", [(2, 37, 29, 6), (3, 40, 33, 5), (3, 6, 9, 4),
                                                    (5, 5, 8, 3)])
def test_jacobi_row_blocks_equal_single_rank_oracle(world, rows, cols, sweeps):
    out = _spawn(_jacobi_worker, world, rows, cols, sweeps)
    um, rm = O.jacobi_run(I.jacobi_grid(rows, cols, seed=3), sweeps, mirror_f32=True)
    for r in range(world):
        u, res = out[r]
        assert np.array_equal(u.view(np.uint32), um.view(np.uint32)), r
        assert np.array_equal(res.view(np.uint32), rm.view(np.uint32)), r


def test_jacobi_without_exchange_differs():
    """The halo exchange matters: skipping it (planted in the test, on the
    CPU) changes the field after two sweeps."""
    rows, cols, world = 12, 9, 2
    u0 = I.jacobi_grid(rows, cols, seed=3)
    plans = [JacobiRowBlocks(rows, cols, world, r) for r in range(world)]
    slabs = [[p.slab(u0).copy(), p.slab(u0).copy()] for p in plans]
    for k in range(2):
        for p, s in zip(plans, slabs):
            v, _ = O.jacobi_sweep_f32(s[k % 2])
            s[(k + 1) % 2][1:-1, 1:-1] = v[1:-1, 1:-1]
    full = np.concatenate([u0[:1]] + [p.owned(s[0]) for p, s in zip(plans, slabs)] + [u0[-1:]])
    um, _ = O.jacobi_run(u0, 2, mirror_f32=True)
    assert not np.array_equal(full, um)


# ---------------------------------------------------------------- matvec --

def _matvec_worker(rank, world, port, out, rows, cols, integer):
    _init(rank, world, port)
    try:
        if integer:
            a = I.small_int_matrix(rows, cols, -4, 4, seed=5)
            x = I.small_int_matrix(1, cols, -3, 3, seed=6)[0]
        else:
            a, x = I.matvec_inputs(rows, cols)
        plan = MatvecRowBlocks(rows, cols, world, rank)
        xt = torch.from_numpy(x.copy()) if rank == 0 else torch.zeros(cols, dtype=torch.float32)
        plan.replicate_x(xt)
        y = torch.from_numpy(O.matvec(plan.block(a), xt.numpy()))
        out[rank] = plan.gather(y).numpy().copy()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,rows,cols,integer", [(2, 33, 17, True), (3, 50, 41, False), (3, 2, 5, True)])
def test_matvec_row_blocks_equal_single_rank_oracle(world, rows, cols, integer):
    out = _spawn(_matvec_worker, world, rows, cols, integer)
    if integer:
        a = I.small_int_matrix(rows, cols, -4, 4, seed=5)
        x = I.small_int_matrix(1, cols, -3, 3, seed=6)[0]
    else:
        a, x = I.matvec_inputs(rows, cols)
    want = O.matvec(a, x)
    for r in range(world):
        if integer:
            assert np.array_equal(out[r], want)
        else:
            assert np.max(np.abs(out[r] - want)) <= 1e-12 * np.max(np.abs(want))


# ------------------------------------------------------------ AXPY + sum --

def _axpy_worker(rank, world, port, out, n):
    _init(rank, world, port)
    try:
        x, y = I.axpy_inputs(n, seed=2)
        plan = AxpyBlocks(n, world, rank)
        lo, hi = plan.lo, plan.hi
        yb = O.axpy(2.5, x[lo:hi], y[lo:hi])
        local = torch.tensor([np.float32(O.reduce_f64(O.RED_ADD, 0.0, yb))], dtype=torch.float32)
        def fold(parts, init):
            # the oracle's sum of the rank-ordered partials and the prior value
            return torch.tensor([np.float32(O.reduce_f64(O.RED_ADD, init, parts.numpy()))])

        total = plan.combine_sum(local, 0.75, fold)
        imod = torch.tensor([O.reduce_i64(O.RED_ADD, 0, O.imod_terms(lo, 1, hi - lo, 3, 1000))],
                            dtype=torch.int64)
        plan.combine_int(imod)
        parts = [torch.zeros(n, dtype=torch.float32) for _ in range(world)]
        mine = torch.zeros(n, dtype=torch.float32)
        mine[lo:hi] = torch.from_numpy(yb)
        dist.all_gather(parts, mine)
        out[rank] = (sum(p.numpy() for p in parts), float(total.item()), int(imod.item()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n", [(2, 10007), (3, 4099)])
def test_axpy_blocks_equal_single_rank_oracle(world, n):
    out = _spawn(_axpy_worker, world, n)
    x, y = I.axpy_inputs(n, seed=2)
    want_y = O.axpy(2.5, x, y)
    want_s = O.reduce_f64(O.RED_ADD, 0.75, want_y)
    for r in range(world):
        yg, s, i = out[r]
        assert np.array_equal(yg, want_y)
        assert abs(s - want_s) <= 1e-5 * abs(want_s)
        assert i == O.imod_sum_closed_form(n, 3, 1000)
    assert len({out[r][1] for r in range(world)}) == 1  # every rank folds the same value


# ---------------------------------------------------------------- batches --

def _batch_worker(rank, world, port, out):
    _init(rank, world, port)
    try:
        specs = I.batched_region_specs(40, seed=6, t_hi=2e4, max_side=120, max_rows=300, max_cols=300)
        mine = shard_lpt([region_bytes(s) for s in specs], world)[rank]
        res = {}
        for i in mine:
            arr = I.region_arrays(specs[i])
            if specs[i]["op"] == I.OP_AXPY_DOT:
                res[i] = float(np.sum(O.axpy(2.5, arr["x"], arr["y"]), dtype=np.float64))
            elif specs[i]["op"] == I.OP_JACOBI:
                res[i] = float(O.jacobi_sweep_f32(arr["u0"])[1])
            else:
                res[i] = float(np.sum(O.matvec(arr["A"], arr["x"])))
        gathered = [None] * world
        dist.all_gather_object(gathered, res)
        out[rank] = gathered
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_batch_lpt_runs_every_region_once(world):
    out = _spawn(_batch_worker, world)
    specs = I.batched_region_specs(40, seed=6, t_hi=2e4, max_side=120, max_rows=300, max_cols=300)
    got = out[0]
    keys = [k for part in got for k in part]
    assert sorted(keys) == list(range(len(specs)))
    loads = [sum(region_bytes(specs[k]) for k in part) for part in got]
    assert max(loads) - min(loads) <= max(region_bytes(s) for s in specs)
    merged = {k: v for part in got for k, v in part.items()}
    for i, sp in enumerate(specs):
        arr = I.region_arrays(sp)
        if sp["op"] == I.OP_AXPY_DOT:
            want = float(np.sum(O.axpy(2.5, arr["x"], arr["y"]), dtype=np.float64))
        elif sp["op"] == I.OP_JACOBI:
            want = float(O.jacobi_sweep_f32(arr["u0"])[1])
        else:
            want = float(np.sum(O.matvec(arr["A"], arr["x"])))
        assert merged[i] == want


# ------------------------------------------------------------------ GEMM --

def test_rank_grid_and_panels():
    assert [rank_grid(w) for w in (1, 2, 3, 4, 6, 9)] == [(1, 1), (2, 1), (3, 1), (2, 2), (6, 1), (3, 3)]
    g = [GemmPanels(10, 7, 9, 4, r) for r in range(4)]
    assert [(x.i, x.j, x.rows, x.cols) for x in g] == [(0, 0, (0, 5), (0, 4)), (0, 1, (0, 5), (4, 7)),
                                                      (1, 0, (5, 10), (0, 4)), (1, 1, (5, 10), (4, 7))]
    assert [g[0].panel(p) for p in range(2)] == [(0, 5), (5, 9)]


def _gemm_worker(rank, world, port, out, m, n, k, integer):
    _init(rank, world, port)
    try:
        if integer:
            a = I.small_int_matrix(m, k, -5, 5, seed=21)
            b = I.small_int_matrix(k, n, -5, 5, seed=22)
        else:
            a, b = I.gemm_inputs(m, n, k)
        plan = GemmPanels(m, n, k, world, rank)
        plan.make_groups()
        a_mine = torch.from_numpy(plan.a_local(a).astype(np.float64).copy())
        b_mine = torch.from_numpy(plan.b_local(b).astype(np.float64).copy())
        c = torch.zeros((plan.rows[1] - plan.rows[0], plan.cols[1] - plan.cols[0]), dtype=torch.float64)

        def gemm_acc(ap, bp, cc, first):
            prod = torch.from_numpy(O.gemm(ap.numpy(), bp.numpy()))
            if first:
                cc.copy_(prod)
            else:
                cc.add_(prod)

        plan.run(gemm_acc, a_mine, b_mine, c, lambda shape, like: torch.empty(shape, dtype=like.dtype))
        out[rank] = plan.gather(c).numpy().copy()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,m,n,k,integer", [(4, 37, 29, 23, True), (4, 40, 33, 50, False),
                                                 (2, 21, 19, 17, True), (3, 30, 20, 10, False),
                                                 (4, 1, 3, 1, True), (3, 2, 4, 5, True)])
def test_gemm_panels_equal_single_rank_oracle(world, m, n, k, integer):
    out = _spawn(_gemm_worker, world, m, n, k, integer)
    if integer:
        a = I.small_int_matrix(m, k, -5, 5, seed=21)
        b = I.small_int_matrix(k, n, -5, 5, seed=22)
    else:
        a, b = I.gemm_inputs(m, n, k)
    want = O.gemm(a, b)
    for r in range(world):
        if integer:
            assert np.array_equal(out[r], want), r
        else:
            assert np.max(np.abs(out[r] - want)) <= 1e-12 * np.max(np.abs(want)), r
