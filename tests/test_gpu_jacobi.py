"""Parity of the 5-point Jacobi sweep loops against the oracle: the field and
the per-sweep max residual are bit-exact against the FP32 mirror (the kernel
applies the same IEEE operations in the same order) and within 1e-5 of the
FP64 oracle."""
import json
import os

import numpy as np
import pytest

import upir_inputs as I
from oracle import upir_oracle as O

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")
from upir_helpers import Session, jacobi_loop  # noqa: E402

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ABS_F64 = 1e-5


@pytest.fixture(scope="module")
def s():
    sess = Session()
    yield sess
    sess.close()


def run_sweeps(s, u0, sweeps, teams=0, units=0, hints=(), sched=0, chunk=0, graph=False):
    rows, cols = u0.shape
    a = u0.copy()
    b = u0.copy()
    res = np.full(max(sweeps, 1), -np.inf, np.float32)
    ha, hb = s.map(a, U.UPIR_MAP_TOFROM), s.map(b, U.UPIR_MAP_TOFROM)
    hr = s.map(res, U.UPIR_MAP_TOFROM)
    loops = []
    for k in range(sweeps):
        src, dst = (ha, hb) if k % 2 == 0 else (hb, ha)
        loops.append(jacobi_loop(src, dst, rows, cols, hres=hr, res_index=k, hints=hints,
                                 sched=sched, chunk=chunk))
    s.run(loops, teams, units, flags=U.UPIR_SUBMIT_GRAPH if graph else 0)
    for h in (ha, hb, hr):
        s.unmap(h)
    return (a if sweeps % 2 == 0 else b), res[:sweeps]


def test_hand_worked_5x5():
    with open(os.path.join(GOLD, "jacobi_5x5.json")) as f:
        g = json.load(f)
    sess = Session()
    try:
        u, res = run_sweeps(sess, np.array(g["initial"], np.float32), 2)
    finally:
        sess.close()
    assert np.array_equal(u.astype(np.float64), np.array(g["after_sweep_2"]))
    assert res.tolist() == [g["residual_1"], g["residual_2"]]


@pytest.mark.parametrize("rows,cols,sweeps,hints", [
    (64, 64, 7, ()),
    (131, 260, 5, ()),                                  # several tiles, ragged in both directions
    (37, 61, 4, ()),                                    # cols % 4 != 0: one copy per halo row
    (131, 259, 5, ()), (70, 1022, 3, ()), (45, 129, 4, ((U.UPIR_HINT_TILE_M, 5), (U.UPIR_HINT_TILE_N, 12))),
    # row copies ending 3 and 2 elements short of a 16-byte boundary at the
    # grid's end (the last elements come by plain loads), three and four stages
    (33, 67, 4, ((U.UPIR_HINT_TILE_M, 8), (U.UPIR_HINT_TILE_N, 32), (U.UPIR_HINT_STAGES, 3))),
    (34, 67, 3, ((U.UPIR_HINT_TILE_M, 3), (U.UPIR_HINT_TILE_N, 64), (U.UPIR_HINT_STAGES, 4))),
    (33, 61, 3, ((U.UPIR_HINT_VARIANT, 1),)),           # per-point variant forced on an unaligned width
    (200, 516, 3, ((U.UPIR_HINT_TILE_M, 7), (U.UPIR_HINT_TILE_N, 20))),
    (300, 300, 3, ((U.UPIR_HINT_VARIANT, 1),)),         # per-point variant forced
    (3, 3, 2, ()), (3, 8, 2, ()), (8, 3, 2, ()),        # degenerate grids
])
def test_field_and_residuals_bit_exact_vs_fp32_mirror(s, rows, cols, sweeps, hints):
    u0 = I.jacobi_grid(rows, cols, seed=1)
    u, res = run_sweeps(s, u0, sweeps, hints=hints)
    um, rm = O.jacobi_run(u0, sweeps, mirror_f32=True)
    assert np.array_equal(u.view(np.uint32), um.view(np.uint32))
    assert np.array_equal(res.view(np.uint32), rm.view(np.uint32))


@pytest.mark.parametrize("teams,units,sched,chunk", [(5, 256, 0, 0), (3, 64, 0, 2), (7, 128, 1, 1),
                                                     (0, 0, 1, 3), (1, 32, 0, 0),
                                                     (4, 100, 0, 0), (2, 20, 0, 0), (3, 1, 1, 1)])
def test_schedules_over_tiles(s, teams, units, sched, chunk):
    u0 = I.jacobi_grid(150, 332, seed=4)
    u, res = run_sweeps(s, u0, 3, teams=teams, units=units, sched=sched, chunk=chunk)
    um, rm = O.jacobi_run(u0, 3, mirror_f32=True)
    assert np.array_equal(u, um) and np.array_equal(res, rm)


@pytest.mark.parametrize("teams,units,sched,chunk", [(5, 256, 0, 0), (3, 64, 0, 2), (7, 128, 1, 1),
                                                     (0, 0, 1, 3), (4, 100, 0, 0), (3, 1, 1, 1)])
@pytest.mark.parametrize("cols", [331, 330, 329])
def test_unaligned_widths_over_tiles(s, teams, units, sched, chunk, cols):
    u0 = I.jacobi_grid(150, cols, seed=4)
    u, res = run_sweeps(s, u0, 3, teams=teams, units=units, sched=sched, chunk=chunk)
    um, rm = O.jacobi_run(u0, 3, mirror_f32=True)
    assert np.array_equal(u, um) and np.array_equal(res, rm)


def test_unaligned_width_4095_ten_sweeps(s):
    u0 = I.jacobi_grid(4095, seed=1)
    u, res = run_sweeps(s, u0, 10)
    um, rm = O.jacobi_run(u0, 10, mirror_f32=True)
    assert np.array_equal(u.view(np.uint32), um.view(np.uint32))
    assert np.array_equal(res.view(np.uint32), rm.view(np.uint32))


def test_graph_submission_matches(s):
    u0 = I.jacobi_grid(96, 128, seed=2)
    u, res = run_sweeps(s, u0, 6, graph=True)
    um, rm = O.jacobi_run(u0, 6, mirror_f32=True)
    assert np.array_equal(u, um) and np.array_equal(res, rm)


def test_full_workload_4096_100_sweeps(s):
    u0 = I.jacobi_grid(4096, seed=1)
    u, res = run_sweeps(s, u0, 100)
    um, rm = O.jacobi_run(u0, 100, mirror_f32=True)
    assert np.array_equal(u.view(np.uint32), um.view(np.uint32))
    assert np.array_equal(res.view(np.uint32), rm.view(np.uint32))
    u64, r64 = O.jacobi_run(u0, 100)
    assert np.max(np.abs(u.astype(np.float64) - u64)) <= ABS_F64
    assert np.max(np.abs(res.astype(np.float64) - r64)) <= 4e-5


def test_harmonic_field_fixed_point(s):
    r, c = np.meshgrid(np.arange(40), np.arange(64), indexing="ij")
    u0 = ((3 + 2 * r + 5 * c + r * c) * 2.0 ** -12).astype(np.float32)
    u, res = run_sweeps(s, u0, 2)
    assert np.array_equal(u, u0) and np.all(res == 0.0)


def test_min_reduction_and_partial_row_range(s):
    u0 = I.jacobi_grid(70, 72, seed=5)
    a, b = u0.copy(), u0.copy()
    res = np.array([np.inf], np.float32)
    ha, hb, hr = s.map(a, U.UPIR_MAP_TO), s.map(b, U.UPIR_MAP_TOFROM), s.map(res, U.UPIR_MAP_TOFROM)
    s.run([jacobi_loop(ha, hb, 70, 72, hres=hr, op=U.UPIR_RED_MIN, lb=10, ub=50)])
    for h in (ha, hb, hr):
        s.unmap(h)
    v, _ = O.jacobi_sweep_f32(u0)
    want = u0.copy()
    want[10:50, 1:-1] = v[10:50, 1:-1]
    assert np.array_equal(b, want)
    assert res[0] == np.min(np.abs(v[10:50, 1:-1] - u0[10:50, 1:-1]))


def test_grid_8192_beyond_l2(s):
    """8192^2 (a 537 MB ping-pong set, four times the L2): the sweep kernel
    streams from HBM; field and residuals bit-exact against the FP32 mirror."""
    u0 = I.jacobi_grid(8192, seed=1)
    u, res = run_sweeps(s, u0, 4)
    um, rm = O.jacobi_run(u0, 4, mirror_f32=True)
    assert np.array_equal(u.view(np.uint32), um.view(np.uint32))
    assert np.array_equal(res.view(np.uint32), rm.view(np.uint32))


def test_beyond_l2_tiles_on_ragged_grid(s):
    """5124 x 5128 (the two grids outgrow the L2, so the planner takes 64 x 64
    tiles; neither side a multiple of the tile): 3 sweeps bit-exact against
    the FP32 mirror."""
    u0 = I.jacobi_grid(5124, 5128, seed=9)
    u, res = run_sweeps(s, u0, 3)
    um, rm = O.jacobi_run(u0, 3, mirror_f32=True)
    assert np.array_equal(u.view(np.uint32), um.view(np.uint32))
    assert np.array_equal(res.view(np.uint32), rm.view(np.uint32))


ASC = (U.UPIR_HINT_TILE_ORDER, 1)  # every team walks its tiles ascending
DESC = (U.UPIR_HINT_TILE_ORDER, 2)  # every team walks its tiles descending


@pytest.mark.parametrize("rows,cols,sweeps,teams,units", [
    (131, 260, 5, 0, 0), (131, 259, 5, 0, 0),          # 2D boxes / row copies, ragged tiles
    (300, 516, 4, 7, 256),                              # explicit teams: uneven runs of tiles
    (150, 333, 3, 500, 256),                            # more teams than tiles: empty runs
    (1030, 1030, 6, 0, 0), (1027, 1029, 6, 0, 0),
])
def test_alternating_tile_order_bit_exact(s, rows, cols, sweeps, teams, units):
    """The planner's default walks every other sweep's tiles descending; the
    field and residuals equal those of the ascending and descending walks and
    the FP32 mirror's bit for bit."""
    u0 = I.jacobi_grid(rows, cols, seed=12)
    u, res = run_sweeps(s, u0, sweeps, teams=teams, units=units)
    ua, ra = run_sweeps(s, u0, sweeps, teams=teams, units=units, hints=(ASC,))
    ud, rd = run_sweeps(s, u0, sweeps, teams=teams, units=units, hints=(DESC,))
    um, rm = O.jacobi_run(u0, sweeps, mirror_f32=True)
    for got, want in ((u, um), (ua, um), (ud, um), (res, rm), (ra, rm), (rd, rm)):
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_tile_order_hint_values(s):
    a = np.zeros((40, 64), np.float32)
    ha, hb = s.map(a, U.UPIR_MAP_TO), s.map(a.copy(), U.UPIR_MAP_TOFROM)
    r = U.upir_spmd_region(s.ctx, 0, 0)
    with pytest.raises(U.UpirError) as e:
        U.upir_loop_checked(s.ctx, r, U.make_loop_desc(**jacobi_loop(ha, hb, 40, 64,
                                                                  hints=[(U.UPIR_HINT_TILE_ORDER, 3)])))
    assert e.value.status == U.UPIR_EINVAL
    U.upir_region_destroy(r)
    s.unmap(ha)
    s.unmap(hb)


@pytest.mark.parametrize("n", [4500, 4600])
def test_l2_policy_threshold_bit_exact(s, n):
    """Grids on either side of the size up to which the 2D-box kernel keeps
    its output in L2 (the two grids within 1.25 L2: 4500^2 is, 4600^2 is
    not): three sweeps bit-exact against the FP32 mirror."""
    u0 = I.jacobi_grid(n, seed=13)
    u, res = run_sweeps(s, u0, 3)
    um, rm = O.jacobi_run(u0, 3, mirror_f32=True)
    assert np.array_equal(u.view(np.uint32), um.view(np.uint32))
    assert np.array_equal(res.view(np.uint32), rm.view(np.uint32))
