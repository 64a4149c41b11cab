"""Asynchronous data movement and the two-step (arrive-compute / wait-release)
sync: copies on the copy stream stay ordered with the computation that uses
the buffers, results equal the oracle's, and a context can wait for another's
work on the device."""
import numpy as np
import pytest

import upir_inputs as I
from oracle import upir_oracle as O

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")
torch = pytest.importorskip("torch")
from upir_helpers import axpy_loop  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = U.upir_init(0)
    yield c
    U.upir_finalize(c)


def pinned(a: np.ndarray):
    t = torch.empty(a.shape, dtype=torch.float32, pin_memory=True)
    t.numpy()[...] = a
    return t


def run(ctx, loops, keep=False):
    r = U.upir_spmd_region(ctx, 0, 0)
    for lp in loops:
        U.upir_loop_checked(ctx, r, U.make_loop_desc(**lp))
    U.upir_region_submit(r, 0)
    if keep:
        return r
    U.upir_region_destroy(r)
    return None


@pytest.mark.parametrize("use_pinned", [True, False])
def test_map_async_then_compute(ctx, use_pinned):
    n = 1 << 22
    x, y = I.axpy_inputs(n)
    hx_host = pinned(x) if use_pinned else x.copy()
    hy_host = pinned(y) if use_pinned else y.copy()
    ptr = (lambda t: t.data_ptr()) if use_pinned else (lambda a: a.ctypes.data)
    hx = U.upir_data_map_async(ctx, ptr(hx_host), 4 * n, U.UPIR_MAP_TO)
    hy = U.upir_data_map_async(ctx, ptr(hy_host), 4 * n, U.UPIR_MAP_TOFROM)
    run(ctx, [axpy_loop(hx, hy, n)])
    U.upir_data_unmap(ctx, hx)
    U.upir_data_unmap(ctx, hy)
    got = hy_host.numpy() if use_pinned else hy_host
    assert np.array_equal(got, O.axpy(2.5, x, y))


def test_update_async_to_is_ordered_after_earlier_work(ctx):
    """y += a x_old (long region), then x is replaced asynchronously, then
    y += a x_new: the first region must have read x_old, the second x_new."""
    n = 1 << 24
    x_old, y0 = I.axpy_inputs(n, seed=1)
    x_new, _ = I.axpy_inputs(n, seed=2)
    xh = pinned(x_old)
    yh = pinned(y0)
    hx = U.upir_data_map(ctx, xh.data_ptr(), 4 * n, U.UPIR_MAP_TO)
    hy = U.upir_data_map(ctx, yh.data_ptr(), 4 * n, U.UPIR_MAP_TOFROM)
    # several passes make the first region long enough for a racing copy to show
    run(ctx, [axpy_loop(hx, hy, n, a=0.0) for _ in range(6)] + [axpy_loop(hx, hy, n)])
    xh.numpy()[...] = x_new  # the copy below runs after the work above
    U.upir_data_update_async(ctx, hx, U.UPIR_MAP_TO)
    run(ctx, [axpy_loop(hx, hy, n)])
    U.upir_data_unmap(ctx, hx)
    U.upir_data_unmap(ctx, hy)
    want = O.axpy(2.5, x_new, O.axpy(2.5, x_old, y0))
    assert np.array_equal(yh.numpy(), want)


def test_update_async_from_snapshot_precedes_later_writes(ctx):
    n = 1 << 22
    x, y = I.axpy_inputs(n, seed=3)
    xh, yh = pinned(x), pinned(y)
    hx = U.upir_data_map(ctx, xh.data_ptr(), 4 * n, U.UPIR_MAP_TO)
    hy = U.upir_data_map(ctx, yh.data_ptr(), 4 * n, U.UPIR_MAP_TOFROM)
    run(ctx, [axpy_loop(hx, hy, n)])
    U.upir_data_update_async(ctx, hy, U.UPIR_MAP_FROM)   # snapshot of y after one update
    run(ctx, [axpy_loop(hx, hy, n) for _ in range(4)])    # later writes wait for the snapshot's read
    U.upir_buf_wait(ctx, hy)
    snap = yh.numpy().copy()
    U.upir_data_unmap(ctx, hx)
    U.upir_data_unmap(ctx, hy)
    once = O.axpy(2.5, x, y)
    assert np.array_equal(snap, once)
    want = once
    for _ in range(4):
        want = O.axpy(2.5, x, want)
    assert np.array_equal(yh.numpy(), want)


def test_pipelined_regions(ctx):
    """Region k + 1's input is mapped while region k computes; every region's
    result is the oracle's."""
    n = 1 << 21
    ins = [I.axpy_inputs(n, seed=10 + k) for k in range(4)]
    hosts = [(pinned(x), pinned(y)) for x, y in ins]
    bufs = []
    for k, (xh, yh) in enumerate(hosts):
        hx = U.upir_data_map_async(ctx, xh.data_ptr(), 4 * n, U.UPIR_MAP_TO)
        hy = U.upir_data_map_async(ctx, yh.data_ptr(), 4 * n, U.UPIR_MAP_TOFROM)
        bufs.append((hx, hy))
        run(ctx, [axpy_loop(hx, hy, n) for _ in range(3)])
    for hx, hy in bufs:
        U.upir_data_unmap(ctx, hx)
        U.upir_data_unmap(ctx, hy)
    for (x, y), (_, yh) in zip(ins, hosts):
        want = y
        for _ in range(3):
            want = O.axpy(2.5, x, want)
        assert np.array_equal(yh.numpy(), want)


def test_arrive_and_wait_release_across_contexts(ctx):
    """Context A writes a device buffer, arrives; context B waits for that
    event on the device and then reads the buffer."""
    n = 1 << 24
    a_ctx, b_ctx = ctx, U.upir_init(0)
    try:
        x, y = I.axpy_inputs(n, seed=5)
        dx = torch.from_numpy(x).cuda()
        dy = torch.from_numpy(y).cuda()
        dz = torch.zeros(n, device="cuda")
        torch.cuda.synchronize()
        ax, ay = (U.upir_data_map_device(a_ctx, t.data_ptr(), 4 * n) for t in (dx, dy))
        bx, by = (U.upir_data_map_device(b_ctx, t.data_ptr(), 4 * n) for t in (dy, dz))
        # A: y <- y + 2.5 x, five times (long)
        run(a_ctx, [axpy_loop(ax, ay, n) for _ in range(5)])
        ev = U.upir_ctx_arrive(a_ctx)
        U.upir_ctx_wait_event(b_ctx, ev)
        # B: z <- z + 1.0 * y (reads A's result)
        run(b_ctx, [axpy_loop(bx, by, n, a=1.0)])
        U.upir_event_wait(ev)
        assert U.upir_event_query(ev)
        U.upir_ctx_wait(b_ctx)
        U.upir_ctx_wait(a_ctx)
        want = y
        for _ in range(5):
            want = O.axpy(2.5, x, want)
        assert np.array_equal(dz.cpu().numpy(), O.axpy(1.0, want, np.zeros(n, np.float32)))
        U.upir_event_destroy(ev)
        for h in (ax, ay):
            U.upir_data_unmap(a_ctx, h)
        for h in (bx, by):
            U.upir_data_unmap(b_ctx, h)
    finally:
        U.upir_finalize(b_ctx)


def test_async_argument_errors(ctx):
    with pytest.raises(U.UpirError) as e:
        U.upir_data_map_async(ctx, 0, 16, U.UPIR_MAP_TO)
    assert e.value.status == U.UPIR_EINVAL
    h = U.upir_data_map_async(ctx, 0, 16, U.UPIR_MAP_ALLOC)
    with pytest.raises(U.UpirError) as e:
        U.upir_data_update_async(ctx, h, U.UPIR_MAP_TO)   # no host copy
    assert e.value.status == U.UPIR_EINVAL
    U.upir_buf_wait(ctx, h)
    U.upir_data_unmap(ctx, h)
    with pytest.raises(U.UpirError) as e:
        U.upir_buf_wait(ctx, h)
    assert e.value.status == U.UPIR_ENOTMAPPED


def test_buf_copy_seeds_a_second_buffer_on_the_device(ctx):
    """One host grid mapped asynchronously, copied on the device into a
    buffer mapped FROM, then one Jacobi sweep from the copy: the copy waits
    for the host->device transfer, and the sweep for the copy."""
    u0 = I.jacobi_grid(96, seed=2)
    host = pinned(u0)
    back = np.full_like(u0, -1.0)
    out = np.full_like(u0, -1.0)
    ha = U.upir_data_map_async(ctx, host.data_ptr(), u0.nbytes, U.UPIR_MAP_TO)
    hb = U.upir_data_map(ctx, back.ctypes.data, u0.nbytes, U.UPIR_MAP_FROM)
    ho = U.upir_data_map(ctx, out.ctypes.data, u0.nbytes, U.UPIR_MAP_FROM)
    U.upir_buf_copy(ctx, hb, ha)
    U.upir_buf_copy(ctx, ho, hb)
    run(ctx, [dict(lb=1, ub=95, step=1, collapse=2, body=U.UPIR_BODY_JACOBI5, bufs=[hb, ho], scalars=[96, 96])])
    for h in (ha, hb, ho):
        U.upir_data_unmap(ctx, h)
    assert np.array_equal(back, u0)
    want, _ = O.jacobi_run(u0, 1, mirror_f32=True)
    assert np.array_equal(out, want)


def test_buf_copy_argument_errors(ctx):
    big = np.zeros(64, np.float32)
    small = np.zeros(16, np.float32)
    hbig = U.upir_data_map(ctx, big.ctypes.data, big.nbytes, U.UPIR_MAP_TO)
    hsmall = U.upir_data_map(ctx, small.ctypes.data, small.nbytes, U.UPIR_MAP_TO)
    with pytest.raises(U.UpirError) as e:
        U.upir_buf_copy(ctx, hsmall, hbig)
    assert e.value.status == U.UPIR_EINVAL
    U.upir_buf_copy(ctx, hbig, hsmall)   # the first 64 bytes of big
    U.upir_buf_copy(ctx, hbig, hbig)     # nothing to do
    U.upir_data_unmap(ctx, hsmall)
    with pytest.raises(U.UpirError) as e:
        U.upir_buf_copy(ctx, hbig, hsmall)
    assert e.value.status == U.UPIR_ENOTMAPPED
    U.upir_data_unmap(ctx, hbig)


def test_stream_of_recorded_regions_with_async_copies(ctx):
    """Three slots, each with buffers mapped once (bound to pinned host
    arrays) and a recorded two-sweep Jacobi region; two passes of: upload the
    grid and residual start values, seed the second grid on the device, run
    the region as a graph, download the field and residuals.  Each copy waits
    only for the work that uses its buffer, yet every result is the oracle's;
    the second pass, with other grids, reuses the slots behind the first
    pass's downloads."""
    side = 72
    slots = []
    for k in range(3):
        pa = pinned(np.zeros((side, side), np.float32))
        pr = pinned(np.zeros(2, np.float32))
        ha = U.upir_data_map(ctx, pa.data_ptr(), pa.numel() * 4, U.UPIR_MAP_ALLOC)
        hb = U.upir_data_map(ctx, 0, pa.numel() * 4, U.UPIR_MAP_ALLOC)
        hr = U.upir_data_map(ctx, pr.data_ptr(), 8, U.UPIR_MAP_ALLOC)
        loops = [dict(lb=1, ub=side - 1, step=1, collapse=2, body=U.UPIR_BODY_JACOBI5, bufs=[src, dst],
                      scalars=[side, side], reductions=[(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_RESID, hr, s)])
                 for s, (src, dst) in enumerate([(ha, hb), (hb, ha)])]
        r = U.upir_spmd_region(ctx, 0, 0)
        for lp in loops:
            U.upir_loop_checked(ctx, r, U.make_loop_desc(**lp))
        slots.append((pa, pr, ha, hb, hr, r))
    for p in range(2):
        grids = [I.jacobi_grid(side, seed=10 * p + k) for k in range(3)]
        for (pa, pr, ha, hb, hr, r), g in zip(slots, grids):
            U.upir_buf_wait(ctx, ha)  # the previous pass's download has left pa
            U.upir_buf_wait(ctx, hr)
            pa.numpy()[...] = g
            pr.numpy()[...] = -np.inf
            U.upir_data_update_async(ctx, ha, U.UPIR_MAP_TO)
            U.upir_data_update_async(ctx, hr, U.UPIR_MAP_TO)
            U.upir_buf_copy(ctx, hb, ha)
            U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH)
            U.upir_data_update_async(ctx, ha, U.UPIR_MAP_FROM)
            U.upir_data_update_async(ctx, hr, U.UPIR_MAP_FROM)
        for (pa, pr, ha, hb, hr, r), g in zip(slots, grids):
            U.upir_buf_wait(ctx, ha)
            U.upir_buf_wait(ctx, hr)
            want, res = O.jacobi_run(g, 2, mirror_f32=True)
            assert np.array_equal(pa.numpy(), want)
            assert np.array_equal(pr.numpy(), np.asarray(res, np.float32))
    for pa, pr, ha, hb, hr, r in slots:
        U.upir_region_destroy(r)
        for h in (ha, hb, hr):
            U.upir_data_unmap(ctx, h)
