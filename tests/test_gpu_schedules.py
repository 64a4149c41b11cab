"""The schedule policies beyond static and dynamic (guided, runtime, auto) and
the taskloop parallelization, against the oracle: chunk boundaries exactly as
the oracle's readings fix them, every iteration run exactly once by a single
worker per chunk, and loop results equal to those of the static schedule."""
import numpy as np
import pytest

import upir_inputs as I
from oracle import upir_oracle as O

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")
from upir_helpers import Session, axpy_loop, jacobi_loop  # noqa: E402


@pytest.fixture(scope="module")
def s():
    sess = Session()
    yield sess
    sess.close()


def run_coverage(s, trip, sched, chunk=0, teams=0, units=0, hints=()):
    owner = np.full(max(trip, 1), -1, np.int64)
    count = np.zeros(max(trip, 1), np.int64)
    ho, hc = s.map(owner, U.UPIR_MAP_TOFROM), s.map(count, U.UPIR_MAP_TOFROM)
    r = s.run([dict(lb=0, ub=trip, step=1, body=U.UPIR_BODY_COVERAGE, bufs=[ho, hc], chunk=chunk, sched=sched,
                    hints=list(hints))], teams, units, keep=True)
    t, u = U.upir_region_loop_geometry(r, 0)
    got = U.upir_region_loop_schedule(r, 0)
    U.upir_region_submit(r)  # a second run reuses the reset counters
    U.upir_ctx_wait(s.ctx)
    U.upir_region_destroy(r)
    s.unmap(ho)
    s.unmap(hc)
    return owner[:trip], count[:trip] // 2, count[:trip] % 2, t * u, got


@pytest.mark.parametrize("trip", [0, 1, 1000, 100003])
@pytest.mark.parametrize("chunk,teams,units", [(0, 0, 0), (3, 5, 64), (64, 0, 0), (1, 2, 32)])
def test_guided_chunks_and_coverage(s, trip, chunk, teams, units):
    owner, count, odd, W, (sc, ch, n) = run_coverage(s, trip, U.UPIR_SCHED_GUIDED, chunk, teams, units)
    want = O.guided_chunks(trip, W, chunk)
    assert (sc, ch) == (U.UPIR_SCHED_GUIDED, chunk) and n == len(want)
    assert not odd.any()
    assert O.check_chunked_assignment(trip, want, owner, count, W)


@pytest.mark.parametrize("trip", [1, 10, 4099, 100003])
@pytest.mark.parametrize("grain,ntasks", [(0, 0), (3, 0), (0, 4), (2, 3), (5000, 0), (0, 100000)])
def test_taskloop_tasks_and_coverage(s, trip, grain, ntasks):
    hints = ([(U.UPIR_HINT_GRAINSIZE, grain)] if grain else []) + ([(U.UPIR_HINT_NUM_TASKS, ntasks)] if ntasks else [])
    owner, count, odd, W, (sc, ch, n) = run_coverage(s, trip, U.UPIR_SCHED_TASKLOOP, hints=hints)
    want = O.taskloop_chunks(trip, grain, ntasks) if (grain or ntasks) else O.taskloop_chunks(trip, 0, 8 * 148)
    assert sc == U.UPIR_SCHED_TASKLOOP and n == len(want)
    assert not odd.any()
    assert O.check_chunked_assignment(trip, want, owner, count, W)


@pytest.mark.parametrize("sched,chunk,hints", [(U.UPIR_SCHED_GUIDED, 0, ()), (U.UPIR_SCHED_GUIDED, 512, ()),
                                               (U.UPIR_SCHED_TASKLOOP, 0, ((U.UPIR_HINT_GRAINSIZE, 1000),)),
                                               (U.UPIR_SCHED_TASKLOOP, 0, ((U.UPIR_HINT_NUM_TASKS, 77),))])
def test_axpy_reductions_under_guided_and_taskloop(s, sched, chunk, hints):
    n = 300007
    x, y = I.axpy_inputs(n)
    yy = y.copy()
    var = np.array([0.0], np.float32)
    ivar = np.array([0], np.int64)
    hx, hy = s.map(x, U.UPIR_MAP_TO), s.map(yy, U.UPIR_MAP_TOFROM)
    hv, hi = s.map(var, U.UPIR_MAP_TOFROM), s.map(ivar, U.UPIR_MAP_TOFROM)
    lp = axpy_loop(hx, hy, n, reds=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_Y, hv, 0),
                                    (U.UPIR_RED_ADD, U.UPIR_I64, U.UPIR_TERM_IMOD, hi, 0)], sched=sched, chunk=chunk)
    lp["hints"] = list(hints)
    s.run([lp])
    for h in (hx, hy, hv, hi):
        s.unmap(h)
    want = O.axpy(2.5, x, y)
    assert np.array_equal(yy, want)
    assert ivar[0] == sum(O.imod_terms(0, 1, n, 3, 1000))
    exact = float(np.sum(want.astype(np.float64)))
    assert abs(float(var[0]) - exact) <= 2 * 2.0 ** -24 * abs(exact) + 1e-6 * float(np.sum(np.abs(want)))


def test_tiled_and_row_bodies_match_static(s):
    """Guided schedules and taskloops over tiles (tiled JACOBI5, FILTER7) and
    rows (MATVEC) and the per-tile GEMM_F32 give the static schedule's results
    bit for bit: the arithmetic of each point, row or tile does not depend on
    who runs it."""
    u0 = I.jacobi_grid(300, seed=1)[:, :296].copy()
    rows, cols = u0.shape
    a, x = I.matvec_inputs(700, 333)
    ga, gb = I.gemm_inputs(300, 260, 96)
    w = np.random.default_rng(2).random(49).astype(np.float32)
    scheds = [(U.UPIR_SCHED_STATIC, 0, ()), (U.UPIR_SCHED_GUIDED, 0, ()), (U.UPIR_SCHED_GUIDED, 2, ()),
              (U.UPIR_SCHED_TASKLOOP, 0, ((U.UPIR_HINT_NUM_TASKS, 5),)),
              (U.UPIR_SCHED_TASKLOOP, 0, ((U.UPIR_HINT_GRAINSIZE, 2),))]
    outs = []
    for sched, chunk, hints in scheds:
        b = u0.copy()
        res = np.full(1, -np.inf, np.float32)
        f = np.zeros_like(u0)
        y = np.zeros(700, np.float32)
        c = np.zeros((300, 260), np.float32)
        h = {k: s.map(v, U.UPIR_MAP_TOFROM) for k, v in
             dict(u=u0.copy(), b=b, res=res, f=f, a=a, x=x, y=y, ga=ga, gb=gb, c=c).items()}
        jl = jacobi_loop(h["u"], h["b"], rows, cols, hres=h["res"], sched=sched, chunk=chunk, hints=hints)
        fl = dict(lb=3, ub=rows - 3, collapse=2, body=U.UPIR_BODY_FILTER7, bufs=[h["u"], h["f"]],
                  scalars=[rows, cols] + [float(v) for v in w], sched=sched, chunk=chunk, hints=list(hints))
        ml = dict(lb=0, ub=700, body=U.UPIR_BODY_MATVEC, bufs=[h["a"], h["x"], h["y"]], scalars=[700, 333],
                  sched=sched, chunk=chunk, hints=list(hints))
        gl = dict(lb=0, ub=300, collapse=2, body=U.UPIR_BODY_GEMM_F32, bufs=[h["ga"], h["gb"], h["c"]],
                  scalars=[300, 260, 96], sched=sched, chunk=chunk, hints=list(hints))
        s.run([jl, fl, ml, gl])
        for hh in h.values():
            s.unmap(hh)
        outs.append((b, res, f, y, c))
    for o in outs[1:]:
        for got, want in zip(o, outs[0]):
            assert np.array_equal(got, want)
    want_b, want_res = O.jacobi_run(u0, 1, mirror_f32=True)
    assert np.array_equal(outs[0][0], want_b) and outs[0][1][0] == want_res[0]


def test_time_blocked_jacobi_under_guided_and_taskloop(s):
    u0 = I.jacobi_grid(400, seed=3)[:, :388].copy()
    rows, cols = u0.shape
    want, terms = O.jacobi_tb(u0, 1, rows - 1, 3, mirror_f32=True)
    for sched, hints in [(U.UPIR_SCHED_GUIDED, ()), (U.UPIR_SCHED_TASKLOOP, ((U.UPIR_HINT_NUM_TASKS, 3),))]:
        b = np.zeros_like(u0)
        res = np.full(3, -np.inf, np.float32)
        ha, hb, hr = s.map(u0.copy(), U.UPIR_MAP_TO), s.map(b, U.UPIR_MAP_TOFROM), s.map(res, U.UPIR_MAP_TOFROM)
        s.run([dict(lb=1, ub=rows - 1, collapse=2, body=U.UPIR_BODY_JACOBI5_TB, bufs=[ha, hb],
                    scalars=[rows, cols, 3], sched=sched, hints=list(hints),
                    reductions=[(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_RESID, hr, 0)])])
        for h in (ha, hb, hr):
            s.unmap(h)
        assert np.array_equal(b[1:-1, 1:-1], want[1:-1, 1:-1])
        assert np.array_equal(res, np.array([t.max() for t in terms], np.float32))


def test_runtime_schedule_from_context_and_environment(s, monkeypatch):
    ho = s.map(np.zeros(5000, np.int64), U.UPIR_MAP_TO)
    hc = s.map(np.zeros(5000, np.int64), U.UPIR_MAP_TO)
    loop = dict(lb=0, ub=5000, body=U.UPIR_BODY_COVERAGE, bufs=[ho, hc], sched=U.UPIR_SCHED_RUNTIME)

    def resolved(sess):
        r = U.upir_spmd_region(sess.ctx, 0, 0)
        U.upir_loop_checked(sess.ctx, r, U.make_loop_desc(**loop))
        out = U.upir_region_loop_schedule(r, 0)
        U.upir_region_destroy(r)
        return out

    assert resolved(s)[:2] == (U.UPIR_SCHED_STATIC, 0)  # the default run schedule
    U.upir_ctx_set_run_schedule(s.ctx, U.UPIR_SCHED_GUIDED, 16)
    sc, ch, n = resolved(s)
    assert (sc, ch) == (U.UPIR_SCHED_GUIDED, 16) and n > 0
    U.upir_ctx_set_run_schedule(s.ctx, U.UPIR_SCHED_STATIC, 0)
    for bad in [(U.UPIR_SCHED_TASKLOOP, 0), (U.UPIR_SCHED_AUTO, 0), (U.UPIR_SCHED_DYNAMIC, -1)]:
        with pytest.raises(U.UpirError):
            U.upir_ctx_set_run_schedule(s.ctx, *bad)
    s.unmap(ho)
    s.unmap(hc)
    monkeypatch.setenv("UPIR_SCHEDULE", "dynamic,32")
    s2 = Session()
    try:
        ho = s2.map(np.zeros(5000, np.int64), U.UPIR_MAP_TO)
        hc = s2.map(np.zeros(5000, np.int64), U.UPIR_MAP_TO)
        loop["bufs"] = [ho, hc]
        assert resolved(s2) == (U.UPIR_SCHED_DYNAMIC, 32, 157)
        s2.unmap(ho)
        s2.unmap(hc)
    finally:
        s2.close()


def test_auto_schedule_with_and_without_model(s):
    n = 200000
    x, y = I.axpy_inputs(n)
    p = np.zeros(U.UPIR_MLP_NPARAM, np.float32)
    p[9] = 1.0                       # W1[0][9]: the log2(chunk + 1) feature
    p[64 * 12 + 64] = 1.0            # W2[0][0]
    p[64 * 12 + 64 + 64 * 64 + 64] = -1.0  # W3[0]: predicted time falls as the chunk grows
    for model, want in [(None, (U.UPIR_SCHED_STATIC, 0)), (p, (U.UPIR_SCHED_DYNAMIC, 65536))]:
        if model is None:
            U.upir_ctx_set_cost_model(s.ctx, None)
        else:
            U.upir_ctx_set_cost_model(s.ctx, model, np.zeros(12), np.ones(12))
        yy = y.copy()
        hx, hy = s.map(x, U.UPIR_MAP_TO), s.map(yy, U.UPIR_MAP_TOFROM)
        r = s.run([axpy_loop(hx, hy, n, sched=U.UPIR_SCHED_AUTO)], keep=True)
        sc, ch, _ = U.upir_region_loop_schedule(r, 0)
        _, units = U.upir_region_loop_geometry(r, 0)
        U.upir_region_destroy(r)
        s.unmap(hx)
        s.unmap(hy)
        assert (sc, ch) == want
        if model is not None:
            assert units == 128
        assert np.array_equal(yy, O.axpy(2.5, x, y))
    U.upir_ctx_set_cost_model(s.ctx, None)


def test_schedule_validation(s):
    hx = s.map(np.zeros(64, np.float32), U.UPIR_MAP_TO)
    hy = s.map(np.zeros(64, np.float32), U.UPIR_MAP_TO)
    cases = [(dict(sched=6), U.UPIR_EINVAL),
             (dict(sched=U.UPIR_SCHED_TASKLOOP, chunk=4), U.UPIR_EINVAL),
             (dict(sched=U.UPIR_SCHED_STATIC, hints=[(U.UPIR_HINT_GRAINSIZE, 4)]), U.UPIR_EINVAL),
             (dict(sched=U.UPIR_SCHED_TASKLOOP, hints=[(U.UPIR_HINT_NUM_TASKS, 0)]), U.UPIR_EINVAL)]
    for extra, want in cases:
        lp = axpy_loop(hx, hy, 64)
        lp.update(extra)
        r = U.upir_spmd_region(s.ctx, 0, 0)
        with pytest.raises(U.UpirError) as e:
            U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**lp))
        assert e.value.status == want, extra
        U.upir_region_destroy(r)
    s.unmap(hx)
    s.unmap(hy)
