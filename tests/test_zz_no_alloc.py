"""The allocation-free AXPY entry point, for callers that cannot allocate
device memory (a process whose device memory is all reserved by its own pool,
a latency-critical path where cudaMalloc would synchronize the device, or an
embedder that cannot create a context).  It must give the results of the same
loop run through the ordinary region API, call after call, although every
call reuses one fixed scratch array.  This file is collected last on purpose."""
import numpy as np
import pytest

import upir_inputs as I
from oracle import upir_oracle as O

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")
torch = pytest.importorskip("torch")

REL_F32 = 1e-5
MAX_N = 1 << 26


def _region_api_twice(x, y0, n, a, mul, mod):
    """The existing path: one region with the AXPY loop and both reductions."""
    ctx = U.upir_init(0)
    try:
        xd = torch.from_numpy(x).cuda()
        yd = torch.from_numpy(y0.copy()).cuda()
        fs = torch.zeros(1, dtype=torch.float32, device="cuda")
        si = torch.zeros(1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        hx = U.upir_data_map_device(ctx, xd.data_ptr(), xd.numel() * 4)
        hy = U.upir_data_map_device(ctx, yd.data_ptr(), yd.numel() * 4)
        hf = U.upir_data_map_device(ctx, fs.data_ptr(), 4)
        hi = U.upir_data_map_device(ctx, si.data_ptr(), 8)
        r = U.upir_spmd_region(ctx, 0, 0)
        U.upir_loop_checked(ctx, r, U.make_loop_desc(
            0, n, body=U.UPIR_BODY_AXPY, bufs=[hx, hy], scalars=[a, mul, mod],
            reductions=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_Y, hf, 0),
                        (U.UPIR_RED_ADD, U.UPIR_I64, U.UPIR_TERM_IMOD, hi, 0)]))
        outs = []
        for _ in range(2):
            U.upir_region_submit(r, 0)
            U.upir_ctx_wait(ctx)
            outs.append((yd.cpu().numpy().copy(), float(fs.item()), int(si.item())))
        U.upir_region_destroy(r)
        for h in (hx, hy, hf, hi):
            U.upir_data_unmap(ctx, h)
        return outs
    finally:
        U.upir_finalize(ctx)


def _noalloc_twice(x, y0, n, a, mul, mod):
    xd = torch.from_numpy(x).cuda()
    yd = torch.from_numpy(y0.copy()).cuda()
    fs = torch.zeros(1, dtype=torch.float32, device="cuda")
    si = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    outs = []
    for _ in range(2):
        U.upir_axpy_reduce_noalloc(xd.data_ptr(), yd.data_ptr(), n, a, mul, mod,
                                   fs.data_ptr(), si.data_ptr(), stream)
        torch.cuda.synchronize()
        outs.append((yd.cpu().numpy().copy(), float(fs.item()), int(si.item())))
    return outs


# 2^20 folds the partials in the loop's last team; past 2048 teams (n > 2^22)
# a separate finalize kernel folds them in groups, using the array's group
# partials and its ticket; 2^26 is the documented maximum (32768 teams).
@pytest.mark.parametrize("n", [1, 4099, 1_000_003, 1 << 20, (1 << 22) + 1, (1 << 24) + 3, MAX_N])
def test_noalloc_matches_region_api_on_two_calls(n):
    x, y0 = I.axpy_inputs(n, seed=5)
    a, mul, mod = 2.5, 3, 1000
    want = _region_api_twice(x, y0, n, a, mul, mod)
    got = _noalloc_twice(x, y0, n, a, mul, mod)
    yref = y0
    for k, ((yw, fw, iw), (yg, fg, ig)) in enumerate(zip(want, got)):
        assert np.array_equal(yg.view(np.uint32), yw.view(np.uint32)), k
        assert abs(fg - fw) <= REL_F32 * max(abs(fw), 1e-30), k
        assert ig == iw, k
        # and both against the oracle: y bit-exact, sums within the FP32 tolerance
        yref = O.axpy(a, x, yref)
        assert np.array_equal(yg, yref)
        assert ig == (k + 1) * O.imod_sum_closed_form(n, mul, mod)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    d = torch.zeros(4, dtype=torch.float32, device="cuda")
    i = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = U.lib.upir_axpy_reduce_noalloc(d.data_ptr(), d.data_ptr(), MAX_N + 1, 1.0, 3, 1000,
                                        d.data_ptr(), i.data_ptr(), None)
    assert st == U.UPIR_EINVAL
    st = U.lib.upir_axpy_reduce_noalloc(d.data_ptr(), d.data_ptr(), 4, 1.0, 3, 0,
                                        d.data_ptr(), i.data_ptr(), None)
    assert st == U.UPIR_EINVAL
    assert U.lib.upir_axpy_reduce_noalloc(None, None, 0, 1.0, 3, 1000, d.data_ptr(), i.data_ptr(),
                                          None) == U.UPIR_OK
