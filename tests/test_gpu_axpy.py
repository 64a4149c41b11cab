"""Parity of the element-granular loops (AXPY, IMOD, COVERAGE) against the
oracle: schedules, reductions, edge sizes and the full AXPY workload."""
import numpy as np
import pytest

import upir_inputs as I
from oracle import upir_oracle as O

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")
from upir_helpers import Session, axpy_loop  # noqa: E402

REL_F32 = 1e-5  # FP32 loops against the FP64 oracle


@pytest.fixture(scope="module")
def s():
    sess = Session()
    yield sess
    sess.close()


def run_axpy(s, n, reds_spec, teams=0, units=0, sched=0, chunk=0, a=2.5, seed=0,
             finit=0.0, iinit=0, lb=0, ub=None, step=1, hints=(), imod=(3, 1000)):
    x, y = I.axpy_inputs(n, seed=seed)
    y0 = y.copy()
    fvar = np.array([finit], np.float32)
    ivar = np.array([iinit], np.int64)
    hx, hy = s.map(x, U.UPIR_MAP_TO), s.map(y, U.UPIR_MAP_TOFROM)
    hf, hi = s.map(fvar, U.UPIR_MAP_TOFROM), s.map(ivar, U.UPIR_MAP_TOFROM)
    reds = []
    for kind, op, term in reds_spec:
        reds.append((op, kind, term, hf if kind == U.UPIR_F32 else hi, 0))
    s.run([axpy_loop(hx, hy, n, a=a, reds=reds, sched=sched, chunk=chunk, lb=lb, ub=ub, step=step,
                     hints=hints, imod=imod)], teams, units)
    for h in (hx, hy, hf, hi):
        s.unmap(h)
    return x, y0, y, float(fvar[0]), int(ivar[0])


def expected_y(x, y0, a, lb, ub, step):
    idx = np.arange(lb, ub, step) if step > 0 else np.arange(lb, ub, step)
    want = y0.copy()
    if idx.size:
        want[idx] = O.axpy(a, x[idx], y0[idx])
    return want, idx


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 1000, 4099, 1 << 20])
def test_axpy_sum_and_imod_default_geometry(s, n):
    x, y0, y, fs, isum = run_axpy(s, n, [(U.UPIR_F32, U.UPIR_RED_ADD, U.UPIR_TERM_Y),
                                         (U.UPIR_I64, U.UPIR_RED_ADD, U.UPIR_TERM_IMOD)])
    want = O.axpy(2.5, x, y0)
    assert np.array_equal(y.view(np.uint32), want.view(np.uint32))  # bit-exact (single rounding)
    ref = O.reduce_f64(O.RED_ADD, 0.0, want)
    assert abs(fs - ref) <= REL_F32 * max(abs(ref), 1e-30) or (n == 0 and fs == 0.0)
    # compensated summation reaches the FP32 rounding of the exact sum to within 2 ulps
    if n:
        assert abs(fs - ref) <= 2 * np.spacing(np.float32(abs(ref))) + 1e-30
    assert isum == O.imod_sum_closed_form(n, 3, 1000)


def test_axpy_full_workload_matches_closed_forms(s):
    n = 1 << 20
    _, _, _, _, isum = run_axpy(s, n, [(U.UPIR_I64, U.UPIR_RED_ADD, U.UPIR_TERM_IMOD)])
    assert isum == 523730800
    _, _, _, _, ivsum = run_axpy(s, n, [(U.UPIR_I64, U.UPIR_RED_ADD, U.UPIR_TERM_IV)])
    assert ivsum == 549755289600


@pytest.mark.parametrize("teams,units,sched,chunk", [
    (1, 1, 0, 0), (3, 32, 0, 0), (7, 96, 0, 5), (2, 64, 0, 1), (13, 128, 0, 1000),
    (5, 64, 1, 0), (9, 256, 1, 7), (0, 0, 1, 64), (0, 0, 0, 4), (0, 0, 0, 4096),
])
def test_axpy_schedules_reach_the_same_result(s, teams, units, sched, chunk):
    n = 50_003
    x, y0, y, fs, isum = run_axpy(s, n, [(U.UPIR_F32, U.UPIR_RED_ADD, U.UPIR_TERM_XY),
                                         (U.UPIR_I64, U.UPIR_RED_ADD, U.UPIR_TERM_IMOD)],
                                  teams=teams, units=units, sched=sched, chunk=chunk)
    want = O.axpy(2.5, x, y0)
    assert np.array_equal(y, want)
    ref = O.reduce_f64(O.RED_ADD, 0.0, x.astype(np.float64) * want.astype(np.float64))
    assert abs(fs - ref) <= REL_F32 * abs(ref)
    assert isum == O.imod_sum_closed_form(n, 3, 1000)


# Unit-step ranges whose x and y share a 32-byte phase run in groups of eight
# iterations with 256-bit accesses after a scalar prologue up to the boundary;
# (+, y) pairs even and odd iterations in paired FP32 accumulators and
# (+, mul*iv mod m) sums groups in 32 bits when m < 2^28.  Ranges of every
# alignment and length, with each accumulation variant.
@pytest.mark.parametrize("lb,n,teams,units,vec", [
    (5, 100_003, 3, 32, 0), (3, 4099, 1, 32, 32), (0, 1 << 20, 0, 0, 32), (7, 300_001, 0, 0, 16),
    (1, 1000, 2, 64, 8), (0, 64, 1, 1, 32), (6, 23, 1, 1, 32), (0, 1 << 22, 0, 0, 0),
])
@pytest.mark.parametrize("fterm,mod", [(U.UPIR_TERM_Y, 1000), (U.UPIR_TERM_XY, 1000), (U.UPIR_TERM_Y, (1 << 30) + 3)])
def test_axpy_256bit_groups(s, lb, n, teams, units, vec, fterm, mod):
    hints = [(U.UPIR_HINT_VEC, vec)] if vec else []
    x, y0, y, fs, isum = run_axpy(s, n, [(U.UPIR_F32, U.UPIR_RED_ADD, fterm),
                                         (U.UPIR_I64, U.UPIR_RED_ADD, U.UPIR_TERM_IMOD)],
                                  teams=teams, units=units, lb=lb, hints=hints, imod=(7, mod))
    want, idx = expected_y(x, y0, 2.5, lb, n, 1)
    assert np.array_equal(y.view(np.uint32), want.view(np.uint32))
    terms = want[idx].astype(np.float64)
    if fterm == U.UPIR_TERM_XY:
        terms = terms * x[idx].astype(np.float64)
    ref = O.reduce_f64(O.RED_ADD, 0.0, terms)
    tol = 2 * np.spacing(np.float32(abs(ref))) if fterm == U.UPIR_TERM_Y else REL_F32 * abs(ref)
    assert abs(fs - ref) <= tol
    assert isum == sum(O.imod_terms(lb, 1, n - lb, 7, mod))


@pytest.mark.parametrize("op", [U.UPIR_RED_MAX, U.UPIR_RED_MIN])
def test_axpy_256bit_groups_min_max(s, op):
    x, y0, y, fs, isum = run_axpy(s, 100_003, [(U.UPIR_F32, op, U.UPIR_TERM_Y),
                                               (U.UPIR_I64, op, U.UPIR_TERM_IMOD)],
                                  lb=3, hints=[(U.UPIR_HINT_VEC, 32)], iinit=500 if op == U.UPIR_RED_MIN else 0)
    want, idx = expected_y(x, y0, 2.5, 3, 100_003, 1)
    assert np.array_equal(y, want)
    assert fs == O.reduce_f64(op, 0.0, want[idx])
    assert isum == O.reduce_i64(op, 500 if op == U.UPIR_RED_MIN else 0, O.imod_terms(3, 1, 100_000, 3, 1000))


# Partials of up to 2048 teams (static) or chunks (dynamic) are folded by the
# loop's last team; more take the separate finalize kernel.  Both sides of the
# boundary reach the oracle's result.
@pytest.mark.parametrize("n,teams,units,sched,chunk", [
    (300_001, 2048, 32, 0, 0), (300_001, 2049, 32, 0, 0), (300_001, 5000, 32, 0, 0),
    (299_008, 0, 0, 1, 146), (299_009, 0, 0, 1, 146), (1 << 20, 0, 0, 1, 1),
])
def test_axpy_reduction_fold_sizes(s, n, teams, units, sched, chunk):
    x, y0, y, fs, isum = run_axpy(s, n, [(U.UPIR_F32, U.UPIR_RED_ADD, U.UPIR_TERM_Y),
                                         (U.UPIR_I64, U.UPIR_RED_ADD, U.UPIR_TERM_IMOD)],
                                  teams=teams, units=units, sched=sched, chunk=chunk)
    want = O.axpy(2.5, x, y0)
    assert np.array_equal(y, want)
    ref = O.reduce_f64(O.RED_ADD, 0.0, want)
    assert abs(fs - ref) <= 2 * np.spacing(np.float32(abs(ref)))
    assert isum == O.imod_sum_closed_form(n, 3, 1000)


@pytest.mark.parametrize("sched,chunk,flags", [(0, 0, 0), (1, 97, 0), (0, 0, 1), (1, 97, 1)])
def test_resubmitted_region_folds_every_time(s, sched, chunk, flags):
    """The same recorded loop submitted four times (directly or as a CUDA
    graph): each submission folds its partials once into the variables."""
    n = 100_003
    x, y = I.axpy_inputs(n, seed=4)
    fvar = np.zeros(1, np.float32)
    ivar = np.zeros(1, np.int64)
    hx, hy = s.map(x, U.UPIR_MAP_TO), s.map(y.copy(), U.UPIR_MAP_TOFROM)
    hf, hi = s.map(fvar, U.UPIR_MAP_TOFROM), s.map(ivar, U.UPIR_MAP_TOFROM)
    r = U.upir_spmd_region(s.ctx, 0, 0)
    U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**axpy_loop(
        hx, hy, n, a=0.0, sched=sched, chunk=chunk,
        reds=[(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_Y, hf, 0), (U.UPIR_RED_ADD, U.UPIR_I64, U.UPIR_TERM_IMOD, hi, 0)])))
    for _ in range(4):
        U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH if flags else 0)
    U.upir_ctx_wait(s.ctx)
    U.upir_region_destroy(r)
    for h in (hx, hy, hf, hi):
        s.unmap(h)
    assert int(ivar[0]) == 4 * O.imod_sum_closed_form(n, 3, 1000)
    assert float(fvar[0]) == float(y.max())


@pytest.mark.parametrize("sched,chunk", [(0, 0), (1, 3)])
def test_axpy_reductions_are_bitwise_repeatable(s, sched, chunk):
    outs = set()
    for _ in range(3):
        *_, fs, _ = run_axpy(s, 300_001, [(U.UPIR_F32, U.UPIR_RED_ADD, U.UPIR_TERM_Y)],
                             sched=sched, chunk=chunk, teams=40, units=128)
        outs.add(np.float32(fs).view(np.uint32).item())
    assert len(outs) == 1


@pytest.mark.parametrize("op,init", [(U.UPIR_RED_MAX, 0.5), (U.UPIR_RED_MAX, 9.0),
                                     (U.UPIR_RED_MIN, -0.5), (U.UPIR_RED_MIN, -9.0), (U.UPIR_RED_ADD, 10.0)])
def test_axpy_float_ops_combine_initial_value(s, op, init):
    n = 2049
    x, y0, y, fs, _ = run_axpy(s, n, [(U.UPIR_F32, op, U.UPIR_TERM_Y)], finit=init, seed=3)
    want = O.axpy(2.5, x, y0)
    ref = O.reduce_f64(op, init, want)
    assert abs(fs - ref) <= REL_F32 * abs(ref)


# Teams whose size is not a multiple of the 32-lane warp: the missing lanes
# of the last warp take no part in the team's reduction tree.
@pytest.mark.parametrize("op", [U.UPIR_RED_MAX, U.UPIR_RED_MIN, U.UPIR_RED_ADD])
@pytest.mark.parametrize("teams,units", [(3, 45), (1, 1), (2, 17), (5, 1000)])
def test_axpy_partial_warp_teams(s, op, teams, units):
    x, y0, y, fs, isum = run_axpy(s, 20_011, [(U.UPIR_F32, op, U.UPIR_TERM_Y),
                                              (U.UPIR_I64, U.UPIR_RED_MAX, U.UPIR_TERM_IMOD)],
                                  teams=teams, units=units, finit=0.0, iinit=-1)
    want = O.axpy(2.5, x, y0)
    assert np.array_equal(y, want)
    ref = O.reduce_f64(op, 0.0, want)
    if op == U.UPIR_RED_ADD:
        assert abs(fs - ref) <= 2 * np.spacing(np.float32(abs(ref)))
    else:
        assert fs == ref  # max / min are exact
    assert isum == 999


def test_mul_reduction_short_loop(s):
    n = 40
    x = np.full(n, 0.25, np.float32)
    y = np.full(n, 1.0, np.float32)  # y_new = 1 + 2.5 * 0.25 = 1.625
    fvar = np.array([2.0], np.float32)
    hx, hy, hf = s.map(x, U.UPIR_MAP_TO), s.map(y, U.UPIR_MAP_TOFROM), s.map(fvar, U.UPIR_MAP_TOFROM)
    s.run([axpy_loop(hx, hy, n, reds=[(U.UPIR_RED_MUL, U.UPIR_F32, U.UPIR_TERM_Y, hf, 0)])], 3, 32)
    for h in (hx, hy, hf):
        s.unmap(h)
    ref = 2.0 * 1.625 ** n
    assert abs(float(fvar[0]) - ref) <= 1e-5 * ref


@pytest.mark.parametrize("lb,ub,step", [(7, 1000, 3), (999, -1, -1), (998, 3, -7), (5, 5, 1), (10, 0, 2)])
def test_axpy_strided_and_reverse_loops(s, lb, ub, step):
    n = 1000
    x, y0, y, _, isum = run_axpy(s, n, [(U.UPIR_I64, U.UPIR_RED_ADD, U.UPIR_TERM_IV)],
                                 lb=lb, ub=ub, step=step, teams=2, units=64)
    want, idx = expected_y(x, y0, 2.5, lb, ub, step)
    assert np.array_equal(y, want)
    assert isum == int(idx.sum())


@pytest.mark.parametrize("op,init", [(U.UPIR_RED_ADD, 5), (U.UPIR_RED_MAX, -10), (U.UPIR_RED_MIN, 10 ** 6),
                                     (U.UPIR_RED_MUL, 1)])
def test_imod_int64_ops_exact(s, op, init):
    trip_lb, trip_ub, step = -500, 2000, 3  # no term is 0 in this range
    mul, mod = 7, 1013
    ivar = np.array([init], np.int64)
    hi = s.map(ivar, U.UPIR_MAP_TOFROM)
    s.run([dict(lb=trip_lb, ub=trip_ub, step=step, body=U.UPIR_BODY_IMOD, scalars=[mul, mod],
                reductions=[(op, U.UPIR_I64, U.UPIR_TERM_IMOD, hi, 0)])], 4, 64)
    s.unmap(hi)
    trip = O.trip_count(trip_lb, trip_ub, step)
    terms = O.imod_terms(trip_lb, step, trip, mul, mod)
    assert int(ivar[0]) == O.reduce_i64(op, init, terms)


def test_int64_add_wraps(s):
    ivar = np.array([(1 << 63) - 10], np.int64)
    hi = s.map(ivar, U.UPIR_MAP_TOFROM)
    s.run([dict(lb=0, ub=100, step=1, body=U.UPIR_BODY_IMOD, scalars=[1, 1000],
                reductions=[(U.UPIR_RED_ADD, U.UPIR_I64, U.UPIR_TERM_IV, hi, 0)])], 2, 32)
    s.unmap(hi)
    assert int(ivar[0]) == O.reduce_i64(O.RED_ADD, (1 << 63) - 10, range(100))


@pytest.mark.parametrize("trip,teams,units,chunk", [
    (10, 1, 3, 0), (10, 1, 3, 2), (10, 1, 2, 3), (7, 1, 4, 0), (2, 1, 4, 0), (0, 1, 3, 0),
    (100_003, 3, 96, 0), (100_003, 7, 64, 17), (65, 2, 32, 9), (4096, 0, 0, 0),
])
def test_coverage_static_owner_map_bit_exact(s, trip, teams, units, chunk):
    owner = np.full(max(trip, 1), -1, np.int64)
    count = np.zeros(max(trip, 1), np.int64)
    ho, hc = s.map(owner, U.UPIR_MAP_TOFROM), s.map(count, U.UPIR_MAP_TOFROM)
    r = s.run([dict(lb=0, ub=trip, step=1, body=U.UPIR_BODY_COVERAGE, bufs=[ho, hc], chunk=chunk)],
              teams, units, keep=True)
    t, u = U.upir_region_loop_geometry(r, 0)
    U.upir_region_destroy(r)
    s.unmap(ho)
    s.unmap(hc)
    if teams:
        assert (t, u) == (teams, units)  # the requested geometry is honoured exactly
    want = O.static_owner_map(trip, t * u, chunk)
    assert np.array_equal(owner[:trip], want)
    assert np.all(count[:trip] == 1)


@pytest.mark.parametrize("trip,teams,units,chunk", [(10_007, 4, 64, 1), (10_007, 0, 0, 13), (257, 3, 32, 0)])
def test_coverage_dynamic_assignment_valid(s, trip, teams, units, chunk):
    owner = np.full(trip, -1, np.int64)
    count = np.zeros(trip, np.int64)
    ho, hc = s.map(owner, U.UPIR_MAP_TOFROM), s.map(count, U.UPIR_MAP_TOFROM)
    r = s.run([dict(lb=0, ub=trip, step=1, body=U.UPIR_BODY_COVERAGE, bufs=[ho, hc], chunk=chunk,
                    sched=U.UPIR_SCHED_DYNAMIC)], teams, units, keep=True)
    t, u = U.upir_region_loop_geometry(r, 0)
    U.upir_region_submit(r)  # a second run reuses the reset chunk counter
    U.upir_ctx_wait(s.ctx)
    U.upir_region_destroy(r)
    s.unmap(ho)
    s.unmap(hc)
    assert np.all(count == 2)
    assert O.check_dynamic_assignment(trip, chunk, owner, count // 2, t * u)
