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
