"""Runtime behaviour on the GPU: mapping semantics (§4.1), argument checks,
ownership errors, graphs, batches, timing and the bounded device wait."""
import numpy as np
import pytest

import upir_inputs as I
from oracle import upir_oracle as O

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")
from upir_helpers import Session, axpy_loop, jacobi_loop  # noqa: E402


@pytest.fixture()
def s():
    sess = Session()
    yield sess
    sess.close()


def test_map_kinds(s):
    host = np.arange(8, dtype=np.float32)
    h_to = s.map(host, U.UPIR_MAP_TO)
    out = np.zeros(8, np.float32)
    h_from = s.map(out, U.UPIR_MAP_FROM)
    # y = 1 * x + y on the FROM buffer would read undefined data; copy through AXPY with a=1 on TOFROM
    y = np.zeros(8, np.float32)
    h_y = s.map(y, U.UPIR_MAP_TOFROM)
    s.run([axpy_loop(h_to, h_y, 8, a=1.0)])
    s.unmap(h_y)
    assert np.array_equal(y, host)
    # TO is not copied back
    s.unmap(h_to)
    assert np.array_equal(host, np.arange(8, dtype=np.float32))
    s.unmap(h_from)  # FROM copies whatever the device holds; size and call must succeed


def test_data_update_round_trip(s):
    x = np.ones(16, np.float32)
    y = np.zeros(16, np.float32)
    hx, hy = s.map(x, U.UPIR_MAP_TO), s.map(y, U.UPIR_MAP_ALLOC)
    y[:] = 5.0
    U.upir_data_update(s.ctx, hy, U.UPIR_MAP_TO)
    s.run([axpy_loop(hx, hy, 16, a=2.0)])
    y[:] = 0
    U.upir_data_update(s.ctx, hy, U.UPIR_MAP_FROM)
    assert np.all(y == 7.0)
    s.unmap(hx)
    s.unmap(hy)


def test_validation_errors(s):
    x = np.ones(10, np.float32)
    hx, hy = s.map(x, U.UPIR_MAP_TO), s.map(x.copy(), U.UPIR_MAP_TOFROM)
    r = U.upir_spmd_region(s.ctx, 0, 0)
    bad = [
        dict(axpy_loop(hx, hy, 10), step=0),                       # step 0
        dict(axpy_loop(hx, hy, 11)),                               # past the end of x
        dict(axpy_loop(hx, hy, 10), chunk=-1),
        dict(axpy_loop(hx, hy, 10), sched=7),
        dict(axpy_loop(hx, hy, 10), body=99),
        dict(axpy_loop(hx, hy, 10), lb=-(1 << 63), ub=(1 << 63) - 1),  # trip overflow
        dict(axpy_loop(hx, hy, 10), hints=[(77, 1)]),
        dict(axpy_loop(hx, hy, 10), bufs=[hx]),
        dict(axpy_loop(hx, hy, 10), reductions=[(9, U.UPIR_F32, U.UPIR_TERM_Y, hy, 0)]),
        dict(axpy_loop(hx, hy, 10), reductions=[(1, U.UPIR_F32, U.UPIR_TERM_Y, hy, 10)]),
        dict(axpy_loop(hx, hy, 10), reductions=[(1, U.UPIR_I64, U.UPIR_TERM_RESID, hy, 0)]),
    ]
    for d in bad:
        with pytest.raises(U.UpirError) as e:
            U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**d))
        assert e.value.status == U.UPIR_EINVAL, d
    with pytest.raises(U.UpirError) as e:
        U.upir_spmd_region(s.ctx, 1, 2048)
    assert e.value.status == U.UPIR_EINVAL
    U.upir_region_destroy(r)
    s.unmap(hx)
    s.unmap(hy)


def test_unmap_while_in_use_and_stale_handles(s):
    x = np.ones(10, np.float32)
    hx, hy = s.map(x, U.UPIR_MAP_TO), s.map(x.copy(), U.UPIR_MAP_TOFROM)
    r = U.upir_spmd_region(s.ctx, 0, 0)
    U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**axpy_loop(hx, hy, 10)))
    with pytest.raises(U.UpirError) as e:
        U.upir_data_unmap(s.ctx, hx)
    assert e.value.status == U.UPIR_EBUSY
    U.upir_region_destroy(r)
    s.unmap(hx)
    with pytest.raises(U.UpirError) as e:
        U.upir_data_unmap(s.ctx, hx)
    assert e.value.status == U.UPIR_ENOTMAPPED
    r = U.upir_spmd_region(s.ctx, 0, 0)
    with pytest.raises(U.UpirError) as e:
        U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**axpy_loop(hx, hy, 10)))
    assert e.value.status == U.UPIR_ENOTMAPPED
    U.upir_region_destroy(r)
    s.unmap(hy)


def test_bounded_wait_times_out_and_context_survives(s):
    U.upir_selftest_bounded_wait(s.ctx, 1 << 12)
    with pytest.raises(U.UpirError) as e:
        U.upir_ctx_wait(s.ctx)
    assert e.value.status == U.UPIR_ETIMEDOUT
    U.upir_ctx_wait(s.ctx)  # error word cleared
    x, y = I.axpy_inputs(1000)
    want = O.axpy(2.5, x, y)
    hx, hy = s.map(x, U.UPIR_MAP_TO), s.map(y, U.UPIR_MAP_TOFROM)
    s.run([axpy_loop(hx, hy, 1000)])
    s.unmap(hx)
    s.unmap(hy)
    assert np.array_equal(y, want)


def test_region_resubmit_graph_and_timing(s):
    n = 100_000
    x, y = I.axpy_inputs(n)
    y0 = y.copy()
    hx, hy = s.map(x, U.UPIR_MAP_TO), s.map(y, U.UPIR_MAP_TOFROM)
    r = U.upir_spmd_region(s.ctx, 0, 0)
    U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**axpy_loop(hx, hy, n, a=1.0)))
    U.upir_ctx_set_timing(s.ctx, True)
    U.upir_region_submit(r, 0)
    U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH)
    U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH)
    t = U.upir_ctx_timings(s.ctx)
    U.upir_ctx_set_timing(s.ctx, False)
    assert len(t) == 3 and t[0][0] == U.UPIR_BODY_AXPY and all(ms > 0 for _, ms in t)
    U.upir_region_destroy(r)
    s.unmap(hx)
    s.unmap(hy)
    want = y0
    for _ in range(3):
        want = O.axpy(1.0, x, want)
    assert np.array_equal(y, want)


@pytest.mark.parametrize("mode,tune", [(0, False), (1, False), (2, False), (2, True)])
def test_batch_of_regions_equals_each_region(s, mode, tune):
    specs = I.batched_region_specs(24, seed=6, t_hi=3e5, max_side=300, max_rows=600, max_cols=600)
    regions, checks, keep = [], [], []
    for sp in specs:
        arr = I.region_arrays(sp)
        r = U.upir_spmd_region(s.ctx, 0, 0)
        if sp["op"] == I.OP_AXPY_DOT:
            dot = np.zeros(1, np.float32)
            arr["y0"] = arr["y"].copy()
            hx, hy, hd = s.map(arr["x"], 0), s.map(arr["y"], 2), s.map(dot, 2)
            U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**axpy_loop(
                hx, hy, sp["n"], reds=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_XY, hd, 0)])))
            want = O.axpy(2.5, arr["x"], arr["y"])
            checks.append(("axpy", arr, want, dot, (hx, hy, hd)))
        elif sp["op"] == I.OP_JACOBI:
            res = np.full(1, -np.inf, np.float32)
            side = sp["side"]
            h0, h1, hr = s.map(arr["u0"], 0), s.map(arr["u1"], 2), s.map(res, 2)
            U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**jacobi_loop(h0, h1, side, side, hres=hr)))
            checks.append(("jacobi", arr, O.jacobi_sweep_f32(arr["u0"]), res, (h0, h1, hr)))
        else:
            y = np.zeros(sp["rows"], np.float32)
            ha, hx, hy = s.map(arr["A"], 0), s.map(arr["x"], 0), s.map(y, 2)
            U.upir_loop_checked(s.ctx, r, U.make_loop_desc(
                lb=0, ub=sp["rows"], body=U.UPIR_BODY_MATVEC, bufs=[ha, hx, hy],
                scalars=[sp["rows"], sp["cols"]]))
            checks.append(("matvec", arr, O.matvec(arr["A"], arr["x"]), y, (ha, hx, hy)))
        regions.append(r)
    b = U.upir_batch_create(s.ctx, regions, mode)
    if tune:
        # autotuning runs the batch many times: undo its in-place AXPY updates
        tiles = U.upir_batch_autotune(b, 1)
        assert tiles[0] in (4096, 8192, 16384, 32768) and tiles[1] in (8, 16, 32)
        for kind, arr, want, out, hs in checks:
            if kind == "axpy":
                arr["y"][:] = arr["y0"]
                U.upir_data_update(s.ctx, hs[1], U.UPIR_MAP_TO)
                out[0] = 0.0
                U.upir_data_update(s.ctx, hs[2], U.UPIR_MAP_TO)
    U.upir_batch_submit(b)
    U.upir_ctx_wait(s.ctx)
    U.upir_batch_destroy(b)
    for r in regions:
        U.upir_region_destroy(r)
    for kind, arr, want, out, hs in checks:
        for h in hs:
            s.unmap(h)
        if kind == "axpy":
            assert np.array_equal(arr["y"], want)
            ref = O.reduce_f64(O.RED_ADD, 0.0, arr["x"].astype(np.float64) * want)
            assert abs(out[0] - ref) <= 1e-5 * abs(ref)
        elif kind == "jacobi":
            v, r0 = want
            assert np.array_equal(arr["u1"], v) and out[0] == r0
        else:
            assert np.linalg.norm(out - want) <= 1e-5 * np.linalg.norm(want)


@pytest.mark.parametrize("op,init", [(U.UPIR_RED_MAX, -np.inf), (U.UPIR_RED_MAX, 0.3), (U.UPIR_RED_MAX, np.nan),
                                     (U.UPIR_RED_MIN, np.inf), (U.UPIR_RED_MIN, 1e-6)])
def test_persistent_batch_jacobi_residual_ops(s, op, init):
    """Jacobi regions of widths of every residue mod 4 in one persistent
    batch, each residual folded over its tiles and then into the variable's
    prior value (maxNum / minNum)."""
    sides = [(67, 64), (130, 301), (45, 258), (33, 131), (200, 75)]
    regions, checks = [], []
    for k, (rows, cols) in enumerate(sides):
        u0 = I.jacobi_grid(rows, cols, seed=20 + k)
        a, b = u0.copy(), u0.copy()
        res = np.array([init], np.float32)
        ha, hb, hr = s.map(a, U.UPIR_MAP_TO), s.map(b, U.UPIR_MAP_TOFROM), s.map(res, U.UPIR_MAP_TOFROM)
        r = U.upir_spmd_region(s.ctx, 0, 0)
        U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**jacobi_loop(ha, hb, rows, cols, hres=hr, op=op)))
        regions.append(r)
        checks.append((u0, b, res, (ha, hb, hr)))
    bt = U.upir_batch_create(s.ctx, regions, U.UPIR_BATCH_PERSISTENT)
    U.upir_batch_submit(bt)
    U.upir_ctx_wait(s.ctx)
    U.upir_batch_destroy(bt)
    for r in regions:
        U.upir_region_destroy(r)
    for u0, b, res, hs in checks:
        for h in hs:
            s.unmap(h)
        v, _ = O.jacobi_sweep_f32(u0)
        assert np.array_equal(b, v)
        d = np.abs(v[1:-1, 1:-1] - u0[1:-1, 1:-1])
        r = float(d.max() if op == U.UPIR_RED_MAX else d.min())
        want = r if np.isnan(init) else (max(init, r) if op == U.UPIR_RED_MAX else min(init, r))
        assert float(res[0]) == np.float32(want)


def test_persistent_batch_rejects_unsupported_regions(s):
    x = np.ones(64, np.float32)
    hx, hy = s.map(x, U.UPIR_MAP_TO), s.map(x.copy(), U.UPIR_MAP_TOFROM)
    r = U.upir_spmd_region(s.ctx, 0, 0)
    U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**axpy_loop(hx, hy, 64, step=2)))
    with pytest.raises(U.UpirError) as e:
        U.upir_batch_create(s.ctx, [r], U.UPIR_BATCH_PERSISTENT)
    assert e.value.status == U.UPIR_EUNSUPPORTED
    b = U.upir_batch_create(s.ctx, [r], U.UPIR_BATCH_GRAPH)
    with pytest.raises(U.UpirError) as e:
        U.upir_region_destroy(r)
    assert e.value.status == U.UPIR_EBUSY
    U.upir_batch_destroy(b)
    U.upir_region_destroy(r)
    s.unmap(hx)
    s.unmap(hy)


def test_allocator_failure_is_reported_without_leaks():
    """Host-side fault injection: a caller-supplied allocator that fails on
    its k-th call; the failing call returns UPIR_ENOMEM and every allocation
    made is released by the time the context is finalized."""
    import ctypes as C
    import torch

    live, calls = {}, [0]
    fail_at = 4

    @C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
    def alloc(nbytes, stream, user):
        calls[0] += 1
        if calls[0] == fail_at:
            return None
        t = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    @C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
    def free(ptr, nbytes, stream, user):
        live.pop(ptr, None)

    a = U.upir_allocator(alloc, free, None)
    h = C.c_void_p()
    torch.cuda.synchronize()
    assert U.lib.upir_init(C.byref(h), 0, None, C.byref(a)) == U.UPIR_OK  # call 1: error word
    ctx = h.value
    x = np.ones(1024, np.float32)
    bufs = []
    statuses = []
    for _ in range(4):  # calls 2, 3, 4 (fails), 5
        b = C.c_void_p()
        st = U.lib.upir_data_map(ctx, x.ctypes.data, x.nbytes, U.UPIR_MAP_TO, C.byref(b))
        statuses.append(st)
        if st == U.UPIR_OK:
            bufs.append(b.value)
    assert statuses == [U.UPIR_OK, U.UPIR_OK, U.UPIR_ENOMEM, U.UPIR_OK]
    assert b"allocation" in U.lib.upir_last_error(ctx)
    assert len(live) == 4  # error word + three mapped buffers
    for b in bufs[:1]:
        assert U.lib.upir_data_unmap(ctx, b) == U.UPIR_OK
    assert len(live) == 3
    U.lib.upir_finalize(ctx)  # frees the rest
    assert len(live) == 0


def test_nowait_loops_and_the_barrier_after_them(s):
    """§5 nowait: a loop marked nowait may run beside the next one, but the
    implicit barrier after that next loop covers both.  Loop 1 (nowait) is a
    long AXPY on y1, loop 2 a short independent one, loop 3 reads y1 (an
    AXPY with x = y1): it must see loop 1's finished update.  Then eight
    independent nowait AXPY loops with their own reductions, each checked."""
    n1, n2 = 1 << 25, 1024
    x1, y1 = I.axpy_inputs(n1, seed=41)
    x2, y2 = I.axpy_inputs(n2, seed=42)
    y3 = np.zeros(n1, np.float32)
    y1_0, y2_0 = y1.copy(), y2.copy()
    h = [s.map(a, U.UPIR_MAP_TOFROM) for a in (x1, y1, x2, y2, y3)]
    loops = [axpy_loop(h[0], h[1], n1), axpy_loop(h[2], h[3], n2), axpy_loop(h[1], h[4], n1, a=1.0)]
    loops[0]["nowait"] = 1
    for flags in (0, U.UPIR_SUBMIT_GRAPH):
        y1[:] = y1_0
        y2[:] = y2_0
        y3[:] = 0.0
        for hh in h:
            U.upir_data_update(s.ctx, hh, U.UPIR_MAP_TO)
        s.run(loops, flags=flags)
        for hh in h:
            U.upir_data_update(s.ctx, hh, U.UPIR_MAP_FROM)
        want1 = O.axpy(2.5, x1, y1_0)
        assert np.array_equal(y1, want1)
        assert np.array_equal(y2, O.axpy(2.5, x2, y2_0))
        assert np.array_equal(y3, O.axpy(1.0, want1, np.zeros(n1, np.float32)))
    for hh in h:
        s.unmap(hh)

    n = 300_007
    sets = []
    for k in range(8):
        x, y = I.axpy_inputs(n, seed=50 + k)
        sm = np.zeros(1, np.float32)
        im = np.zeros(1, np.int64)
        sets.append((x, y, y.copy(), sm, im, [s.map(x, U.UPIR_MAP_TO), s.map(y, U.UPIR_MAP_TOFROM),
                                               s.map(sm, U.UPIR_MAP_TOFROM), s.map(im, U.UPIR_MAP_TOFROM)]))
    loops = []
    for k, (x, y, y0, sm, im, hs) in enumerate(sets):
        lp = axpy_loop(hs[0], hs[1], n, reds=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_Y, hs[2], 0),
                                              (U.UPIR_RED_ADD, U.UPIR_I64, U.UPIR_TERM_IMOD, hs[3], 0)])
        lp["nowait"] = 1 if k < 7 else 0
        loops.append(lp)
    s.run(loops, flags=U.UPIR_SUBMIT_GRAPH)
    for x, y, y0, sm, im, hs in sets:
        for hh in hs:
            s.unmap(hh)
        want = O.axpy(2.5, x, y0)
        assert np.array_equal(y, want)
        ref = O.reduce_f64(O.RED_ADD, 0.0, want)
        assert abs(float(sm[0]) - ref) <= 1e-5 * abs(ref)
        assert int(im[0]) == O.imod_sum_closed_form(n, 3, 1000)
