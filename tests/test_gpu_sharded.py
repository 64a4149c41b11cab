"""The row-block partition of one Jacobi problem (the multi-GPU path) with its
per-rank sweeps on the GPU.  Only one GPU is used: every rank's share runs
on it, one rank after another under the host's control (no kernel waits on
another), with the halo rows moved by device copies instead of messages and
the residuals combined by an elementwise max.  Field and per-sweep residuals
must equal the single-rank oracle bit for bit."""
import numpy as np
import pytest

import upir_inputs as I
from oracle import upir_oracle as O

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")
torch = pytest.importorskip("torch")
from paper_2209_10643_b300.sharding import (JacobiRowBlocks, UpirJacobiSweeper,  # noqa: E402
                                            exchange_in_process)


@pytest.fixture()
def ctx():
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    c = U.upir_init(0, stream.cuda_stream)
    yield c
    U.upir_finalize(c)
    torch.cuda.set_stream(torch.cuda.default_stream())


@pytest.mark.parametrize("world,rows,cols,sweeps", [(1, 130, 260, 5), (3, 131, 264, 6), (4, 70, 129, 4),
                                                    (2, 1030, 1024, 3)])
def test_row_blocks_on_gpu_equal_single_rank_oracle(ctx, world, rows, cols, sweeps):
    u0 = I.jacobi_grid(rows, cols, seed=7)
    plans = [JacobiRowBlocks(rows, cols, world, r) for r in range(world)]
    slabs, sweepers, res = [], [], []
    for p in plans:
        a = torch.from_numpy(p.slab(u0).copy()).cuda()
        b = a.clone()
        rv = torch.full((sweeps,), -np.inf, dtype=torch.float32, device="cuda")
        torch.cuda.current_stream().synchronize()
        slabs.append((a, b))
        res.append(rv)
        sweepers.append(UpirJacobiSweeper(ctx, p, a, b, rv, sweeps))
    try:
        for k in range(sweeps):
            for p, (a, b), sw in zip(plans, slabs, sweepers):
                src, dst = (a, b) if k % 2 == 0 else (b, a)
                sw(src, dst, k)
            exchange_in_process(plans, [s[(k + 1) % 2] for s in slabs])
        U.upir_ctx_wait(ctx)
        torch.cuda.synchronize()
    finally:
        for sw in sweepers:
            sw.close()
    final = [s[sweeps % 2] for s in slabs]
    full = np.concatenate([u0[:1]] + [p.owned(f).cpu().numpy() for p, f in zip(plans, final)] + [u0[-1:]])
    resid = torch.stack(res).max(dim=0).values.cpu().numpy()
    um, rm = O.jacobi_run(u0, sweeps, mirror_f32=True)
    assert np.array_equal(full.view(np.uint32), um.view(np.uint32))
    assert np.array_equal(resid.view(np.uint32), rm.view(np.uint32))


@pytest.mark.parametrize("world,m,n,k", [(4, 300, 260, 200), (2, 130, 96, 64), (9, 200, 136, 96)])
def test_gemm_panels_on_gpu_equal_oracle(ctx, world, m, n, k):
    """The 2D-tile GEMM partition with every rank's panel steps on the GPU
    (the FP32 GEMM loop for the first panel, the GEMM into a temporary and an
    AXPY with a = 1 for the others), the panel broadcasts replaced by slicing
    the full operands in one process; C within the FP32 GEMM tolerance."""
    from paper_2209_10643_b300.sharding import GemmPanels, UpirGemmAcc
    a, b = I.gemm_inputs(m, n, k)
    acc = UpirGemmAcc(ctx)
    c = np.zeros((m, n), np.float32)
    for r in range(world):
        plan = GemmPanels(m, n, k, world, r)
        (r0, r1), (c0, c1) = plan.rows, plan.cols
        cd = torch.zeros((r1 - r0, c1 - c0), dtype=torch.float32, device="cuda")
        for p in range(plan.q):
            k0, k1 = plan.panel(p) if plan.q > 1 else (0, k)
            ap = torch.from_numpy(a[r0:r1, k0:k1].copy()).cuda()
            bp = torch.from_numpy(b[k0:k1, c0:c1].copy()).cuda()
            torch.cuda.current_stream().synchronize()
            acc(ap, bp, cd, p == 0)
        c[r0:r1, c0:c1] = cd.cpu().numpy()
    want = O.gemm(a, b)
    assert np.linalg.norm(c - want) <= 1e-5 * np.linalg.norm(want)


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_rank_partials_folded_by_the_runtime(ctx, world):
    """The cross-rank fold of per-rank FP32 sums (the AXPY partition) runs as
    the runtime's own compensated reduction: the ranks' sums of an AXPY
    problem, folded with a prior value, match the oracle's sum of the whole
    problem within the FP32 tolerance."""
    from paper_2209_10643_b300.sharding import AxpyBlocks, UpirSumFold
    n = 100_003
    x, y = I.axpy_inputs(n, seed=31)
    want_y = O.axpy(2.5, x, y)
    parts = []
    for r in range(world):
        lo, hi = AxpyBlocks(n, world, r).lo, AxpyBlocks(n, world, r).hi
        parts.append(np.float32(O.reduce_f64(O.RED_ADD, 0.0, want_y[lo:hi])))
    fold = UpirSumFold(ctx)
    got = float(fold(torch.tensor(parts, dtype=torch.float32, device="cuda"), -3.25).item())
    want = O.reduce_f64(O.RED_ADD, -3.25, want_y)
    assert abs(got - want) <= 1e-5 * abs(want)


@pytest.mark.parametrize("sweeps", [5, 6])
def test_single_rank_run_submits_every_sweep_at_once(ctx, sweeps):
    """A rank with no neighbour runs its sweeps as one submission
    (``JacobiRowBlocks.run`` through the sweeper's whole region); field and
    residuals bit-exact against the oracle, for odd and even sweep counts."""
    u0 = I.jacobi_grid(260, 392, seed=13)
    plan = JacobiRowBlocks(260, 392, 1, 0)
    a = torch.from_numpy(plan.slab(u0).copy()).cuda()
    b = a.clone()
    res = torch.full((sweeps,), -np.inf, dtype=torch.float32, device="cuda")
    torch.cuda.current_stream().synchronize()
    sw = UpirJacobiSweeper(ctx, plan, a, b, res, sweeps)
    try:
        final = plan.run(sw, a, b, sweeps, res)
        U.upir_ctx_wait(ctx)
    finally:
        sw.close()
    um, rm = O.jacobi_run(u0, sweeps, mirror_f32=True)
    assert np.array_equal(final.cpu().numpy().view(np.uint32), um.view(np.uint32))
    assert np.array_equal(res.cpu().numpy().view(np.uint32), rm.view(np.uint32))
