"""Parity of the stencil loop nests beyond one 5-point sweep against the oracle:
the time-blocked Jacobi body (several sweeps per loop) and the 7 x 7 filter.
Both are bit-exact against the oracle's FP32 mirrors, which apply the same IEEE
operations in the same order; untouched points of the output keep their
previous contents."""
import numpy as np
import pytest

import upir_inputs as I
from oracle import upir_oracle as O

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")
from upir_helpers import Session, jacobi_loop  # noqa: E402

SENTINEL = -7.0


@pytest.fixture(scope="module")
def s():
    sess = Session()
    yield sess
    sess.close()


def tb_loop(h_in, h_out, rows, cols, sweeps, hres=None, res_index=0, op=U.UPIR_RED_MAX, lb=1, ub=None,
            sched=U.UPIR_SCHED_STATIC, chunk=0, hints=()):
    reds = [] if hres is None else [(op, U.UPIR_F32, U.UPIR_TERM_RESID, hres, res_index)]
    return dict(lb=lb, ub=rows - 1 if ub is None else ub, step=1, collapse=2, body=U.UPIR_BODY_JACOBI5_TB,
                bufs=[h_in, h_out], scalars=[rows, cols, sweeps], reductions=reds, sched=sched, chunk=chunk,
                hints=list(hints))


def run_tb(s, u0, sweeps, lb=1, ub=None, op=U.UPIR_RED_MAX, teams=0, units=0, sched=0, chunk=0, hints=()):
    rows, cols = u0.shape
    ub = rows - 1 if ub is None else ub
    a = u0.copy()
    b = np.full_like(u0, SENTINEL)
    res = np.full(sweeps + 2, np.inf if op == U.UPIR_RED_MIN else -np.inf, np.float32)
    ha, hb, hr = s.map(a, U.UPIR_MAP_TO), s.map(b, U.UPIR_MAP_TOFROM), s.map(res, U.UPIR_MAP_TOFROM)
    s.run([tb_loop(ha, hb, rows, cols, sweeps, hres=hr, res_index=1, op=op, lb=lb, ub=ub, sched=sched,
                   chunk=chunk, hints=hints)], teams, units)
    for h in (ha, hb, hr):
        s.unmap(h)
    return b, res


def check_tb(u0, sweeps, b, res, lb=1, ub=None, op=U.UPIR_RED_MAX):
    rows = u0.shape[0]
    ub = rows - 1 if ub is None else ub
    want, terms = O.jacobi_tb(u0, lb, ub, sweeps, mirror_f32=True)
    upd = np.zeros(u0.shape, bool)
    upd[lb:ub, 1:-1] = True
    assert np.array_equal(b[upd], want[upd])
    assert np.all(b[~upd] == SENTINEL)
    fold = np.max if op == U.UPIR_RED_MAX else np.min
    ident = np.float32(-np.inf if op == U.UPIR_RED_MAX else np.inf)
    for k, t in enumerate(terms):
        assert res[1 + k] == (np.float32(fold(t)) if t.size else ident), k
    assert res[0] == ident and res[sweeps + 1] == ident
    # and within the FP64 oracle's forward bound
    w64, _ = O.jacobi_tb(u0, lb, ub, sweeps)
    assert np.max(np.abs(b[upd] - w64[upd])) <= sweeps * 3 * 2.0 ** -24 + 1e-12


@pytest.mark.parametrize("rows,cols", [(5, 8), (130, 260), (257, 516), (300, 132)])
@pytest.mark.parametrize("sweeps", [1, 2, 3, 4, 8])
def test_jacobi_tb_bit_exact(s, rows, cols, sweeps):
    u0 = I.jacobi_grid(max(rows, cols), seed=1)[:rows, :cols].copy()
    b, res = run_tb(s, u0, sweeps)
    check_tb(u0, sweeps, b, res)


@pytest.mark.parametrize("lb,ub", [(2, 3), (7, 150), (100, 199)])
def test_jacobi_tb_row_subrange(s, lb, ub):
    u0 = I.jacobi_grid(200, seed=3)[:, :196].copy()
    b, res = run_tb(s, u0, 4, lb=lb, ub=ub)
    check_tb(u0, 4, b, res, lb=lb, ub=ub)


@pytest.mark.parametrize("sched,chunk,teams", [(U.UPIR_SCHED_STATIC, 1, 0), (U.UPIR_SCHED_STATIC, 3, 5),
                                               (U.UPIR_SCHED_DYNAMIC, 1, 0), (U.UPIR_SCHED_DYNAMIC, 2, 7)])
def test_jacobi_tb_schedules_and_min(s, sched, chunk, teams):
    u0 = I.jacobi_grid(400, seed=5)[:, :388].copy()
    for op in (U.UPIR_RED_MAX, U.UPIR_RED_MIN):
        b, res = run_tb(s, u0, 3, op=op, teams=teams, sched=sched, chunk=chunk)
        check_tb(u0, 3, b, res, op=op)


def test_jacobi_tb_tiles_and_units_hints(s):
    u0 = I.jacobi_grid(333, seed=6)[:, :324].copy()
    b, res = run_tb(s, u0, 5, units=512, hints=[(U.UPIR_HINT_TILE_M, 40), (U.UPIR_HINT_TILE_N, 112)])
    check_tb(u0, 5, b, res)
    # few warps: strips longer than the unrolled path
    b, res = run_tb(s, u0, 2, units=96, hints=[(U.UPIR_HINT_TILE_M, 13)])
    check_tb(u0, 2, b, res)
    b, res = run_tb(s, u0, 7, units=64)
    check_tb(u0, 7, b, res)


def test_jacobi_tb_chain_equals_single_sweeps(s):
    """24 sweeps as six loops of 4 sweeps each (ping-pong) give bit for bit the
    field and residuals of 24 one-sweep JACOBI5 loops."""
    u0 = I.jacobi_grid(520, seed=7)[:, :516].copy()
    rows, cols = u0.shape
    outs = []
    for tb in (False, True):
        a, b = u0.copy(), u0.copy()
        res = np.full(24, -np.inf, np.float32)
        ha, hb, hr = s.map(a, U.UPIR_MAP_TOFROM), s.map(b, U.UPIR_MAP_TOFROM), s.map(res, U.UPIR_MAP_TOFROM)
        loops = []
        if tb:
            for g in range(6):
                src, dst = (ha, hb) if g % 2 == 0 else (hb, ha)
                loops.append(tb_loop(src, dst, rows, cols, 4, hres=hr, res_index=4 * g))
        else:
            for k in range(24):
                src, dst = (ha, hb) if k % 2 == 0 else (hb, ha)
                loops.append(jacobi_loop(src, dst, rows, cols, hres=hr, res_index=k))
        s.run(loops, flags=U.UPIR_SUBMIT_GRAPH)
        for h in (ha, hb, hr):
            s.unmap(h)
        outs.append((a, res))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    want, wres = O.jacobi_run(u0, 24, mirror_f32=True)
    assert np.array_equal(outs[1][0], want) and np.array_equal(outs[1][1], wres)


def test_jacobi_tb_full_size_4096(s):
    u0 = I.jacobi_grid(4096, seed=1)
    b, res = run_tb(s, u0, 4)
    check_tb(u0, 4, b, res)


def test_jacobi_tb_rejects_bad_loops(s):
    u = np.zeros((16, 16), np.float32)
    ha, hb = s.map(u.copy(), U.UPIR_MAP_TO), s.map(u.copy(), U.UPIR_MAP_TO)
    hr = s.map(np.zeros(4, np.float32), U.UPIR_MAP_TO)
    u2 = np.zeros((16, 18), np.float32)
    hc, hd = s.map(u2.copy(), U.UPIR_MAP_TO), s.map(u2.copy(), U.UPIR_MAP_TO)
    cases = [(tb_loop(ha, hb, 16, 16, 9), U.UPIR_EINVAL),
             (tb_loop(ha, hb, 16, 16, 0), U.UPIR_EINVAL),
             (tb_loop(ha, hb, 16, 16, 5, hres=hr, res_index=0), U.UPIR_EINVAL),  # 5 residuals, 4 elements
             (tb_loop(ha, hb, 16, 16, 2, lb=0), U.UPIR_EINVAL),
             (tb_loop(ha, ha, 16, 16, 2), U.UPIR_EINVAL),
             (tb_loop(hc, hd, 16, 18, 2), U.UPIR_EUNSUPPORTED),
             (tb_loop(ha, hb, 16, 16, 4, hints=[(U.UPIR_HINT_TILE_N, 112)]), U.UPIR_EINVAL)]
    for lp, want in cases:
        r = U.upir_spmd_region(s.ctx, 0, 0)
        with pytest.raises(U.UpirError) as e:
            U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**lp))
        assert e.value.status == want
        U.upir_region_destroy(r)
    for h in (ha, hb, hr, hc, hd):
        s.unmap(h)


# --- FILTER7 -------------------------------------------------------------------

def filter_loop(h_in, h_out, rows, cols, w, lb=3, ub=None, sched=U.UPIR_SCHED_STATIC, chunk=0, hints=()):
    return dict(lb=lb, ub=rows - 3 if ub is None else ub, step=1, collapse=2, body=U.UPIR_BODY_FILTER7,
                bufs=[h_in, h_out], scalars=[rows, cols] + [float(v) for v in np.asarray(w, np.float32).ravel()],
                sched=sched, chunk=chunk, hints=list(hints))


def run_filter(s, x, w, lb=3, ub=None, teams=0, sched=0, chunk=0, hints=()):
    rows, cols = x.shape
    out = np.full_like(x, SENTINEL)
    hx, ho = s.map(x, U.UPIR_MAP_TO), s.map(out, U.UPIR_MAP_TOFROM)
    s.run([filter_loop(hx, ho, rows, cols, w, lb=lb, ub=ub, sched=sched, chunk=chunk, hints=hints)], teams)
    s.unmap(hx)
    s.unmap(ho)
    return out


def filter_weights(seed):
    w = np.random.default_rng(seed).random((7, 7)).astype(np.float32)
    return (w / w.sum()).astype(np.float32)


def check_filter(x, w, out, lb=3, ub=None):
    rows = x.shape[0]
    ub = rows - 3 if ub is None else ub
    upd = np.zeros(x.shape, bool)
    upd[lb:ub, 3:-3] = True
    assert np.array_equal(out[lb:ub, 3:-3], O.filter7_f32(x, w, lb, ub))
    assert np.all(out[~upd] == SENTINEL)


@pytest.mark.parametrize("rows,cols", [(7, 8), (64, 132), (131, 260), (300, 516)])
def test_filter7_bit_exact(s, rows, cols):
    x = I.jacobi_grid(max(rows, cols), seed=8)[:rows, :cols].copy()
    w = filter_weights(9)
    check_filter(x, w, run_filter(s, x, w))


def test_filter7_single_taps_and_signed_weights(s):
    x = I.jacobi_grid(100, seed=10)
    for i, j in [(3, 3), (0, 6), (6, 0)]:
        w = np.zeros((7, 7), np.float32)
        w[i, j] = 1.0
        out = run_filter(s, x, w)
        assert np.array_equal(out[3:-3, 3:-3], x[i:i + 94, j:j + 94])
    w = np.random.default_rng(11).standard_normal((7, 7)).astype(np.float32)
    check_filter(x, w, run_filter(s, x, w))


@pytest.mark.parametrize("lb,ub,sched,chunk,teams,hints", [
    (3, 4, 0, 0, 0, ()), (10, 77, 0, 0, 0, ()), (3, 197, 0, 2, 3, ()), (5, 190, 1, 1, 0, ()),
    (3, 197, 1, 3, 6, ()), (3, 197, 0, 0, 0, ((U.UPIR_HINT_TILE_M, 8), (U.UPIR_HINT_TILE_N, 32))),
    # one team walking every tile, and two teams on one-tile chunks with a
    # three-stage ring (long runs of refills of each stage)
    (3, 197, 0, 0, 1, ((U.UPIR_HINT_TILE_M, 8), (U.UPIR_HINT_TILE_N, 32))),
    (3, 197, 0, 1, 2, ((U.UPIR_HINT_TILE_M, 8), (U.UPIR_HINT_TILE_N, 32), (U.UPIR_HINT_STAGES, 3)))])
def test_filter7_ranges_schedules_tiles(s, lb, ub, sched, chunk, teams, hints):
    x = I.jacobi_grid(200, seed=12)[:, :196].copy()
    w = filter_weights(13)
    check_filter(x, w, run_filter(s, x, w, lb=lb, ub=ub, sched=sched, chunk=chunk, teams=teams, hints=hints),
                 lb=lb, ub=ub)


F7_VARIANTS = [
    # (tile_m, tile_n, stages, variant): fixed-shape kernels, 3-stage ring,
    # runtime-shape kernel; two output rows per paired FMA with 4- and 8-row
    # strips (variants 0 and 1), one FMA per output with 4- and 8-row strips
    # (variants 2 and 3)
    (32, 128, 2, 0), (64, 128, 2, 0), (32, 128, 3, 0), (32, 128, 2, 1), (64, 128, 3, 1),
    (16, 64, 2, 0), (40, 64, 3, 0), (24, 32, 2, 1),
    (32, 128, 2, 2), (32, 128, 3, 2), (64, 128, 2, 2), (32, 128, 2, 3), (16, 64, 2, 2), (40, 64, 3, 2),
    (24, 32, 2, 3), (64, 128, 3, 3)]


@pytest.mark.parametrize("tm,tn,stages,variant", F7_VARIANTS)
@pytest.mark.parametrize("rows,cols,lb,ub", [(200, 196, 3, 197), (301, 520, 40, 290)])
def test_filter7_variants_bit_exact(s, tm, tn, stages, variant, rows, cols, lb, ub):
    x = I.jacobi_grid(max(rows, cols), seed=17)[:rows, :cols].copy()
    w = filter_weights(18)
    hints = ((U.UPIR_HINT_TILE_M, tm), (U.UPIR_HINT_TILE_N, tn), (U.UPIR_HINT_STAGES, stages),
             (U.UPIR_HINT_VARIANT, variant))
    check_filter(x, w, run_filter(s, x, w, lb=lb, ub=ub, hints=hints), lb=lb, ub=ub)


def test_filter7_full_size_4096_sampled_rows(s):
    x = I.jacobi_grid(4096, seed=14)
    w = filter_weights(15)
    out = run_filter(s, x, w)
    for r in np.random.default_rng(16).integers(3, 4093, 48):
        assert np.array_equal(out[r, 3:-3], O.filter7_f32(x, w, r, r + 1)[0]), r
    assert np.all(out[:3] == SENTINEL) and np.all(out[-3:] == SENTINEL)
    assert np.all(out[:, :3] == SENTINEL) and np.all(out[:, -3:] == SENTINEL)


def test_filter7_rejects_bad_loops(s):
    x = np.zeros((16, 16), np.float32)
    hx, ho = s.map(x.copy(), U.UPIR_MAP_TO), s.map(x.copy(), U.UPIR_MAP_TO)
    hr = s.map(np.zeros(4, np.float32), U.UPIR_MAP_TO)
    w = np.ones((7, 7), np.float32)
    bad_red = filter_loop(hx, ho, 16, 16, w)
    bad_red["reductions"] = [(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_RESID, hr, 0)]
    short = filter_loop(hx, ho, 16, 16, w)
    short["scalars"] = short["scalars"][:40]
    cases = [(filter_loop(hx, ho, 16, 16, w, lb=2), U.UPIR_EINVAL),
             (filter_loop(hx, ho, 16, 16, w, ub=14), U.UPIR_EINVAL),
             (filter_loop(hx, hx, 16, 16, w), U.UPIR_EINVAL),
             (bad_red, U.UPIR_EINVAL), (short, U.UPIR_EINVAL),
             (filter_loop(hx, ho, 16, 16, w, hints=[(U.UPIR_HINT_TILE_M, 6)]), U.UPIR_EINVAL)]
    for lp, want in cases:
        r = U.upir_spmd_region(s.ctx, 0, 0)
        with pytest.raises(U.UpirError) as e:
            U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**lp))
        assert e.value.status == want
        U.upir_region_destroy(r)
    for h in (hx, ho, hr):
        s.unmap(h)
