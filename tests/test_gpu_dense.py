"""Parity of the dense loop nests (matvec, FP32 GEMM, bfloat16 split) against
the FP64 oracle."""
import numpy as np
import pytest

import upir_inputs as I
from oracle import upir_oracle as O

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")
from upir_helpers import Session  # noqa: E402


@pytest.fixture(scope="module")
def s():
    sess = Session()
    yield sess
    sess.close()


def run_matvec(s, a, x, teams=0, units=0, sched=0, chunk=0, lb=0, ub=None, step=1):
    rows, cols = a.shape
    y = np.full(rows, -7.0, np.float32)
    ha, hx, hy = s.map(a, U.UPIR_MAP_TO), s.map(x, U.UPIR_MAP_TO), s.map(y, U.UPIR_MAP_TOFROM)
    s.run([dict(lb=lb, ub=rows if ub is None else ub, step=step, body=U.UPIR_BODY_MATVEC,
                bufs=[ha, hx, hy], scalars=[rows, cols], sched=sched, chunk=chunk)], teams, units)
    for h in (ha, hx, hy):
        s.unmap(h)
    return y


def check_matvec(a, x, y):
    ref = O.matvec(a, x)
    absax = np.abs(a.astype(np.float64)) @ np.abs(x.astype(np.float64))
    assert np.linalg.norm(y - ref) <= 1e-5 * np.linalg.norm(ref)
    assert np.all(np.abs(y - ref) <= 1e-5 * absax + 1e-30)


@pytest.mark.parametrize("rows,cols", [(1, 1), (5, 3), (33, 517), (1000, 1003), (257, 4096), (64, 20000),
                                       (3, 2), (17, 130), (40, 5501), (300, 2481), (9, 642)])
def test_matvec_shapes(s, rows, cols):
    a, x = I.matvec_inputs(rows, cols)
    check_matvec(a, x, run_matvec(s, a, x))


@pytest.mark.parametrize("teams,units,sched,chunk", [(3, 64, 0, 0), (2, 32, 0, 5), (4, 128, 1, 2), (0, 0, 1, 0)])
def test_matvec_schedules(s, teams, units, sched, chunk):
    a, x = I.matvec_inputs(301, 700, seed_a=11)
    check_matvec(a, x, run_matvec(s, a, x, teams, units, sched, chunk))


def test_matvec_exact_structured(s):
    n = 513
    x = (np.arange(n) - 200).astype(np.float32)
    perm = np.random.default_rng(3).permutation(n)
    p = np.eye(n, dtype=np.float32)[perm]
    assert np.array_equal(run_matvec(s, p, x), x[perm])
    ones = np.ones((7, n), np.float32)
    assert np.all(run_matvec(s, ones, x) == float(x.astype(np.float64).sum()))


def test_matvec_strided_rows_only_touch_their_rows(s):
    a, x = I.matvec_inputs(100, 64)
    y = run_matvec(s, a, x, lb=97, ub=0, step=-4)
    rows = np.arange(97, 0, -4)
    ref = O.matvec(a, x)
    assert np.allclose(y[rows], ref[rows], rtol=1e-5, atol=1e-6)
    other = np.setdiff1d(np.arange(100), rows)
    assert np.all(y[other] == -7.0)


def test_matvec_full_workload_16384(s):
    a, x = I.matvec_inputs(16384, 16384)
    check_matvec(a, x, run_matvec(s, a, x))


def run_gemm(s, a, b, teams=0, sched=0, chunk=0, lb=0, ub=None, variant=0):
    m, k = a.shape
    n = b.shape[1]
    c = np.full((m, n), -3.0, np.float32)
    ha, hb, hc = s.map(a, U.UPIR_MAP_TO), s.map(b, U.UPIR_MAP_TO), s.map(c, U.UPIR_MAP_TOFROM)
    s.run([dict(lb=lb, ub=m if ub is None else ub, step=1, collapse=2, body=U.UPIR_BODY_GEMM_F32,
                bufs=[ha, hb, hc], scalars=[m, n, k], sched=sched, chunk=chunk,
                hints=[(U.UPIR_HINT_VARIANT, variant)] if variant else [])], teams, 0)
    for h in (ha, hb, hc):
        s.unmap(h)
    return c


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (300, 200, 130), (128, 256, 64), (129, 127, 17), (1024, 1024, 1024)])
def test_gemm_f32_vs_fp64(s, m, n, k):
    a, b = I.gemm_inputs(m, n, k)
    c = run_gemm(s, a, b)
    ref = O.gemm(a, b)
    assert np.linalg.norm(c - ref) <= 1e-5 * np.linalg.norm(ref)


def test_gemm_f32_exact_integers_and_schedules(s):
    a = I.small_int_matrix(200, 77, -8, 8, seed=1)
    b = I.small_int_matrix(77, 150, -8, 8, seed=2)
    ref = O.gemm(a, b)
    for teams, sched, chunk in [(0, 0, 0), (3, 0, 1), (2, 1, 1)]:
        assert np.array_equal(run_gemm(s, a, b, teams, sched, chunk), ref)


@pytest.mark.parametrize("n", [2250, 2252])
def test_gemm_f32_split_tail_exact_and_close(s, n):
    """A 2300 x n output has 18 x 18 = 324 tiles: 296 resident teams take
    whole tiles and the last 28 tiles are split in four shares of k (520, a
    ragged last k tile).  Small integers give the exact product whatever the
    split; random inputs stay within the FP32 bound.  n = 2250 runs the
    register-staged kernel, n = 2252 (rows on 16-byte boundaries) the TMA-fed
    one."""
    a = I.small_int_matrix(2300, 520, -8, 8, seed=3)
    b = I.small_int_matrix(520, n, -8, 8, seed=4)
    assert np.array_equal(run_gemm(s, a, b), O.gemm(a, b))
    a, b = I.gemm_inputs(2300, n, 520)
    c = run_gemm(s, a, b)
    ref = O.gemm(a, b)
    assert np.linalg.norm(c - ref) <= 1e-5 * np.linalg.norm(ref)
    tail = slice(2048, 2300)
    assert np.linalg.norm(c[tail] - ref[tail]) <= 1e-5 * np.linalg.norm(ref[tail])


@pytest.mark.parametrize("m,n,k,teams,sched,chunk", [
    (300, 260, 96, 0, 0, 0), (1000, 1004, 520, 0, 0, 0), (129, 132, 20, 0, 0, 0), (2300, 2252, 520, 0, 0, 0),
    (700, 516, 64, 5, 0, 2), (700, 516, 64, 0, 1, 3), (4, 4, 4, 0, 0, 0)])
def test_gemm_f32_tma_and_register_kernels_agree(s, m, n, k, teams, sched, chunk):
    """Both FP32 kernels run every element as one FMA chain in increasing k
    (and split the same tiles the same way): their results agree bit for bit,
    and match the FP64 product within the FP32 bound."""
    a, b = I.gemm_inputs(m, n, k)
    c_tma = run_gemm(s, a, b, teams, sched, chunk)
    c_reg = run_gemm(s, a, b, teams, sched, chunk, variant=1)
    assert np.array_equal(c_tma, c_reg)
    ref = O.gemm(a, b)
    assert np.linalg.norm(c_tma - ref) <= 1e-5 * np.linalg.norm(ref)


@pytest.mark.parametrize("variant", [0, 1])
def test_gemm_f32_row_subrange_touches_only_its_rows(s, variant):
    """Rows [70, 1030) of a 1100 x 5120 product, both kernels (the TMA boxes
    of the first and last tile rows cover rows outside the range, which are
    read but not written); the range's 8 x 40 tiles outnumber the 296
    resident teams, so the default plan splits the last 24 in k."""
    a, b = I.gemm_inputs(1100, 5120, 256)
    c = run_gemm(s, a, b, lb=70, ub=1030, variant=variant)
    ref = O.gemm(a, b)
    inside = slice(70, 1030)
    assert np.linalg.norm(c[inside] - ref[inside]) <= 1e-5 * np.linalg.norm(ref[inside])
    assert np.all(c[:70] == -3.0) and np.all(c[1030:] == -3.0)


def test_gemm_f32_empty_k_writes_zeros(s):
    a = np.zeros((40, 0), np.float32)
    b = np.zeros((0, 36), np.float32)
    assert np.all(run_gemm(s, a, b) == 0.0)


def test_gemm_f32_split_tail_resubmitted(s):
    """Each submission of a recorded split GEMM writes every tile: the shares'
    tickets are ready again for the next one (C is changed in between by an
    AXPY loop of the same region, C += 1 in place)."""
    m, n, k = 2300, 2250, 520
    a = I.small_int_matrix(m, k, -8, 8, seed=5)
    b = I.small_int_matrix(k, n, -8, 8, seed=6)
    c = np.zeros((m, n), np.float32)
    ones = np.ones(m * n, np.float32)
    ha, hb, hc, ho = (s.map(a, U.UPIR_MAP_TO), s.map(b, U.UPIR_MAP_TO), s.map(c, U.UPIR_MAP_TOFROM),
                      s.map(ones, U.UPIR_MAP_TO))
    r = U.upir_spmd_region(s.ctx, 0, 0)
    U.upir_loop_checked(s.ctx, r, U.make_loop_desc(lb=0, ub=m, step=1, collapse=2, body=U.UPIR_BODY_GEMM_F32,
                                                   bufs=[ha, hb, hc], scalars=[m, n, k]))
    U.upir_loop_checked(s.ctx, r, U.make_loop_desc(lb=0, ub=m * n, step=1, body=U.UPIR_BODY_AXPY,
                                                   bufs=[ho, hc], scalars=[1.0, 3, 1000]))
    for _ in range(3):
        U.upir_region_submit(r, 0)
    U.upir_ctx_wait(s.ctx)
    U.upir_region_destroy(r)
    for h in (ha, hb, hc, ho):
        s.unmap(h)
    assert np.array_equal(c, O.gemm(a, b) + 1.0)


def test_gemm_f32_full_size_sampled_and_freivalds(s):
    a, b = I.gemm_inputs(4096, 4096, 4096)
    c = run_gemm(s, a, b)
    g = np.random.default_rng(12)
    rows, cols = g.integers(0, 4096, 4096), g.integers(0, 4096, 4096)
    ref = np.einsum("ik,ki->i", a[rows].astype(np.float64), b[:, cols].astype(np.float64))
    assert np.linalg.norm(c[rows, cols] - ref) <= 1e-5 * np.linalg.norm(ref)
    r = g.choice([-1.0, 1.0], 4096)
    lhs = c.astype(np.float64) @ r
    rhs = a.astype(np.float64) @ (b.astype(np.float64) @ r)
    assert np.linalg.norm(lhs - rhs) <= 1e-5 * np.linalg.norm(rhs)


@pytest.mark.parametrize("rows,cols,transpose", [(64, 96, 0), (65, 97, 1), (1, 5, 1), (300, 40, 0)])
def test_split_bf16_bit_exact(s, rows, cols, transpose):
    a, _ = I.gemm_inputs(rows, 4, cols)
    hi = np.zeros(rows * cols, np.uint16)
    lo = np.zeros(rows * cols, np.uint16)
    hs, hh, hl = s.map(a, U.UPIR_MAP_TO), s.map(hi, U.UPIR_MAP_TOFROM), s.map(lo, U.UPIR_MAP_TOFROM)
    s.run([dict(lb=0, ub=rows, body=U.UPIR_BODY_SPLIT_BF16, bufs=[hs, hh, hl],
                scalars=[rows, cols, transpose])])
    for h in (hs, hh, hl):
        s.unmap(h)
    wh, wl = O.split_bf16(a)
    wh = (wh.view(np.uint32) >> 16).astype(np.uint16)
    wl = (wl.view(np.uint32) >> 16).astype(np.uint16)
    if transpose:
        wh, wl = wh.T.copy(), wl.T.copy()
    assert np.array_equal(hi, wh.ravel()) and np.array_equal(lo, wl.ravel())


# --- tensor-core GEMM (tcgen05): bfloat16 and split-bfloat16 -----------------------

def run_gemm_tc(s, a, b, x3=False, teams=0, chunk=0, lb=0, ub=None, variant=0, seg_kb=0):
    m, k = a.shape
    n = b.shape[1]
    ah, al = np.zeros(m * k, np.uint16), np.zeros(m * k, np.uint16)
    bh, bl = np.zeros(n * k, np.uint16), np.zeros(n * k, np.uint16)
    c = np.full((m, n), -3.0, np.float32)
    ha, hb = s.map(a, U.UPIR_MAP_TO), s.map(b, U.UPIR_MAP_TO)
    hah, hal, hbh, hbl = (s.map(v, U.UPIR_MAP_ALLOC) for v in (ah, al, bh, bl))
    hc = s.map(c, U.UPIR_MAP_TOFROM)
    # split A (row-major [m][k]) and B^T ([n][k], from B [k][n] transposed)
    s.run([dict(lb=0, ub=m, body=U.UPIR_BODY_SPLIT_BF16, bufs=[ha, hah, hal], scalars=[m, k, 0]),
           dict(lb=0, ub=k, body=U.UPIR_BODY_SPLIT_BF16, bufs=[hb, hbh, hbl], scalars=[k, n, 1])])
    body = U.UPIR_BODY_GEMM_BF16X3 if x3 else U.UPIR_BODY_GEMM_BF16
    bufs = [hah, hal, hbh, hbl, hc] if x3 else [hah, hbh, hc]
    hints = ([(U.UPIR_HINT_VARIANT, variant)] if variant else []) + ([(U.UPIR_HINT_TILE_M, seg_kb)] if seg_kb else [])
    s.run([dict(lb=lb, ub=m if ub is None else ub, collapse=2, body=body, bufs=bufs, scalars=[m, n, k],
                chunk=chunk, hints=hints)], teams, 0)
    for h in (ha, hb, hah, hal, hbh, hbl, hc):
        s.unmap(h)
    return c


@pytest.mark.parametrize("x3", [False, True])
def test_gemm_tc_exact_small_integers(s, x3):
    # integers in [-8, 8] are exact in bfloat16 and every partial sum is exact in FP32
    a = I.small_int_matrix(200, 136, -8, 8, seed=1)
    b = I.small_int_matrix(136, 300, -8, 8, seed=2)
    assert np.array_equal(run_gemm_tc(s, a, b, x3), O.gemm(a, b))


@pytest.mark.parametrize("x3", [False, True])
def test_gemm_tc_half_tiles_exact(s, x3):
    # 19 x 8 = 152 tiles of 128 x 256: one whole wave on 148 SMs, then 4 tiles
    # cut into 128-column halves; the last row and column of tiles are ragged
    a = I.small_int_matrix(2382, 64, -8, 8, seed=3)
    b = I.small_int_matrix(64, 1948, -8, 8, seed=4)
    assert np.array_equal(run_gemm_tc(s, a, b, x3), O.gemm(a, b))


@pytest.mark.parametrize("x3", [False, True])
def test_gemm_tc_k_split_exact_and_repeatable(s, x3):
    # 4 tiles on 148 SMs: every tile is cut into K parts that the last
    # finishing part adds up in part order
    a = I.small_int_matrix(256, 1024, -8, 8, seed=5)
    b = I.small_int_matrix(1024, 512, -8, 8, seed=6)
    assert np.array_equal(run_gemm_tc(s, a, b, x3), O.gemm(a, b))
    a, b = I.gemm_inputs(256, 512, 1024)
    c1 = run_gemm_tc(s, a, b, x3)
    c2 = run_gemm_tc(s, a, b, x3)
    assert np.array_equal(c1, c2)


# The CTA-pair kernel (tcgen05 cta_group::2, 256 x 256 tiles): the planner's
# choice for large bfloat16 GEMMs, forced here (variant 2) on small and ragged
# shapes; variant 1 is the one-SM kernel.
@pytest.mark.parametrize("x3", [False, True])
@pytest.mark.parametrize("m,n,k", [(200, 300, 136), (2382, 1948, 64), (513, 257, 72), (256, 256, 64), (1, 9, 8)])
def test_gemm_tc_pair_exact_small_integers(s, m, n, k, x3):
    a = I.small_int_matrix(m, k, -8, 8, seed=7)
    b = I.small_int_matrix(k, n, -8, 8, seed=8)
    assert np.array_equal(run_gemm_tc(s, a, b, x3, variant=2), O.gemm(a, b))


@pytest.mark.parametrize("x3,seg_kb", [(False, 3), (True, 5), (True, 32)])
def test_gemm_tc_pair_k_segments(s, x3, seg_kb):
    # K in accumulation segments of seg_kb k-blocks (64 or 32 deep), the
    # segments added in FP32 by the epilogue; the last segment is partial
    a = I.small_int_matrix(520, 1000, -8, 8, seed=11)
    b = I.small_int_matrix(1000, 300, -8, 8, seed=12)
    assert np.array_equal(run_gemm_tc(s, a, b, x3, variant=2, seg_kb=seg_kb), O.gemm(a, b))
    a, b = I.gemm_inputs(512, 512, 2048)
    c = run_gemm_tc(s, a, b, x3, variant=2, seg_kb=seg_kb)
    absab = np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64))
    if x3:
        check_tc(c, O.gemm(a, b), absab, 2048)
    else:
        check_tc(c, O.gemm_bf16(a, b), absab, 2048, tc_accum_tol(2048))


def test_gemm_tc_pair_half_tiles_exact(s):
    # 12 x 7 = 84 pair tiles: one wave on the resident clusters (fewer than 84
    # on a B300), then the rest cut into 128-column halves; ragged edges
    a = I.small_int_matrix(3055, 64, -8, 8, seed=9)
    b = I.small_int_matrix(64, 1787, -8, 8, seed=10)
    assert np.array_equal(run_gemm_tc(s, a, b), O.gemm(a, b))


def test_gemm_tc_pair_matches_one_sm_kernel(s):
    # the same K16 MMA sequence per output; the tensor core's own (not
    # round-to-nearest) accumulation differs between M = 128 and M = 256
    # instructions in the last bits only
    a, b = I.gemm_inputs(1024, 768, 1000)
    c1 = run_gemm_tc(s, a, b, variant=1)
    c2 = run_gemm_tc(s, a, b, variant=2)
    refb = O.gemm_bf16(a, b)
    absab = np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64))
    check_tc(c2, refb, absab, 1000, tc_accum_tol(1000))
    assert np.linalg.norm(c2 - c1) <= tc_accum_tol(1000) * np.linalg.norm(refb)
    assert np.array_equal(c2, run_gemm_tc(s, a, b, variant=2))  # repeatable


def test_gemm_tc_pair_row_subrange(s):
    a, b = I.gemm_inputs(600, 300, 64)
    c = run_gemm_tc(s, a, b, False, lb=70, ub=530, variant=2)
    ref = O.gemm_bf16(a, b)
    assert np.linalg.norm(c[70:530] - ref[70:530]) <= tc_accum_tol(64) * np.linalg.norm(ref[70:530])
    assert np.all(c[:70] == -3.0) and np.all(c[530:] == -3.0)


def tc_accum_tol(k):
    """Normwise tolerance for a single-segment tensor-core accumulation over K
    terms.  Its additions are not rounded to nearest, so the error grows
    linearly with K (measured 1.45e-5 at K = 4096 on N(0, 1/K) data);
    1.5e-5 per 1024 of K bounds it, and FP32 rounding (1e-5) below that."""
    return max(1e-5, 1.5e-5 * k / 1024)


def check_tc(c, ref, absab, k, tol=1e-5):
    """Normwise `tol` where the Frobenius norm averages many entries; for tiny
    outputs the componentwise bound of the split-bfloat16 products
    (3 * 2^-16 per product) plus the accumulation, relative to |A||B|."""
    if c.size >= 4096:
        assert np.linalg.norm(c - ref) <= tol * np.linalg.norm(ref)
    else:
        assert np.all(np.abs(c - ref) <= (3 * 2.0 ** -16 + k * 2.0 ** -22) * absab)


@pytest.mark.parametrize("m,n,k,teams,chunk", [(1, 1, 8, 0, 0), (129, 257, 72, 0, 0), (256, 512, 64, 3, 1),
                                                (384, 256, 200, 2, 0), (300, 700, 1032, 0, 0)])
def test_gemm_tc_ragged_shapes_and_schedules(s, m, n, k, teams, chunk):
    a, b = I.gemm_inputs(m, n, k)
    absab = np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64))
    c = run_gemm_tc(s, a, b, False, teams, chunk)
    check_tc(c, O.gemm_bf16(a, b), absab, k, tc_accum_tol(k))
    c3 = run_gemm_tc(s, a, b, True, teams, chunk)
    check_tc(c3, O.gemm(a, b), absab, k)


def test_gemm_tc_row_subrange_touches_only_its_rows(s):
    a, b = I.gemm_inputs(300, 256, 64)
    c = run_gemm_tc(s, a, b, False, lb=50, ub=250)
    ref = O.gemm_bf16(a, b)
    assert np.linalg.norm(c[50:250] - ref[50:250]) <= tc_accum_tol(64) * np.linalg.norm(ref[50:250])
    assert np.all(c[:50] == -3.0) and np.all(c[250:] == -3.0)


def test_gemm_tc_1024_accuracy_bounds(s):
    a, b = I.gemm_inputs(1024, 1024, 1024)
    ref64 = O.gemm(a, b)
    c = run_gemm_tc(s, a, b, False)
    # tensor-core accumulation of exact bfloat16 products: close to the exactly summed product
    refb = O.gemm_bf16(a, b)
    assert np.linalg.norm(c - refb) <= tc_accum_tol(1024) * np.linalg.norm(refb)
    # stated bound for the bfloat16 path against FP64
    assert np.linalg.norm(c - ref64) <= 1e-2 * np.linalg.norm(ref64)
    c3 = run_gemm_tc(s, a, b, True)
    assert np.linalg.norm(c3 - ref64) <= 1e-5 * np.linalg.norm(ref64)


def test_gemm_tc_full_size_sampled_and_freivalds(s):
    a, b = I.gemm_inputs(4096, 4096, 4096)
    g = np.random.default_rng(13)
    rows, cols = g.integers(0, 4096, 4096), g.integers(0, 4096, 4096)
    r = g.choice([-1.0, 1.0], 4096)
    for x3 in (False, True):
        c = run_gemm_tc(s, a, b, x3)
        if x3:
            ref = np.einsum("ik,ki->i", a[rows].astype(np.float64), b[:, cols].astype(np.float64))
            rhs = a.astype(np.float64) @ (b.astype(np.float64) @ r)
        else:
            ab, bb = O.bf16_round(a).astype(np.float64), O.bf16_round(b).astype(np.float64)
            ref = np.einsum("ik,ki->i", ab[rows], bb[:, cols])
            rhs = ab @ (bb @ r)
        tol = 1e-5 if x3 else tc_accum_tol(4096)
        assert np.linalg.norm(c[rows, cols] - ref) <= tol * np.linalg.norm(ref)
        assert np.linalg.norm(c.astype(np.float64) @ r - rhs) <= tol * np.linalg.norm(rhs)


def test_gemm_tc_rejects_unaligned_k(s):
    a = np.zeros(64 * 12, np.uint16)
    c = np.zeros(64 * 64, np.float32)
    ha, hc = s.map(a, U.UPIR_MAP_TO), s.map(c, U.UPIR_MAP_TO)
    r = U.upir_spmd_region(s.ctx, 0, 0)
    with pytest.raises(U.UpirError) as e:
        U.upir_loop_checked(s.ctx, r, U.make_loop_desc(0, 64, collapse=2, body=U.UPIR_BODY_GEMM_BF16,
                                                       bufs=[ha, ha, hc], scalars=[64, 64, 12]))
    assert e.value.status == U.UPIR_EUNSUPPORTED
    U.upir_region_destroy(r)
    s.unmap(ha)
    s.unmap(hc)
