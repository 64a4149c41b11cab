"""Pins for the CPU oracle: each check ties an oracle function to something other
than itself (hand-worked examples, closed forms, exact rational arithmetic,
brute force, an independent library routine, invariants of the mathematics)."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import upir_oracle as O
import upir_inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# --- canonical loop trip count (§3.2) -------------------------------------------

def test_trip_count_matches_python_range_brute_force():
    for lb in range(-7, 8):
        for ub in range(-7, 8):
            for step in [s for s in range(-4, 5) if s != 0]:
                assert O.trip_count(lb, ub, step) == len(range(lb, ub, step)), (lb, ub, step)


def test_trip_count_large_and_zero_step():
    assert O.trip_count(0, 1 << 40, 3) == len(range(0, 1 << 40, 3))
    with pytest.raises(ValueError):
        O.trip_count(0, 10, 0)


# --- schedules (§3.2 worksharing) ------------------------------------------------

def test_static_owner_hand_tables():
    for case in gold("schedule_tables.json")["cases"]:
        got = O.static_owner_map(case["trip"], case["workers"], case["chunk"])
        assert got.tolist() == case["owner"], case


def test_static_blocked_invariants_brute_force():
    for trip in range(0, 65):
        for w in range(1, 10):
            own = O.static_owner_map(trip, w, 0)
            assert np.all(own >= 0) and np.all(own < w)
            assert np.all(np.diff(own) >= 0)  # contiguous blocks in worker order
            counts = np.bincount(own, minlength=w)
            assert counts.sum() == trip
            assert counts.max() - counts.min() <= 1
            assert np.all(np.diff(counts) <= 0)  # the longer blocks come first


def test_static_chunked_invariants_brute_force():
    for trip in range(0, 65):
        for c in range(1, 10):
            for w in range(1, 10):
                own = O.static_owner_map(trip, w, c)
                assert np.all((own >= 0) & (own < w))
                starts = list(range(0, trip, c))
                for j, s in enumerate(starts):
                    blk = own[s:s + c]
                    assert np.all(blk == blk[0])
                    if j:
                        assert blk[0] == (own[starts[j - 1]] + 1) % w


def test_dynamic_chunks_and_validity_checker():
    for trip in range(0, 40):
        for c in range(0, 6):
            ch = O.dynamic_chunks(trip, c)
            flat = [k for s, e in ch for k in range(s, e)]
            assert flat == list(range(trip))
    trip, c, w = 23, 4, 3
    g = np.random.default_rng(0)
    owner = np.empty(trip, np.int64)
    for s, e in O.dynamic_chunks(trip, c):
        owner[s:e] = g.integers(0, w)
    count = np.ones(trip, np.int64)
    assert O.check_dynamic_assignment(trip, c, owner, count, w)
    bad = count.copy()
    bad[5] = 2
    assert not O.check_dynamic_assignment(trip, c, owner, bad, w)
    split = owner.copy()
    split[1] = (owner[0] + 1) % w
    assert not O.check_dynamic_assignment(trip, c, split, count, w)


# --- reductions (§5) ---------------------------------------------------------------

def test_integer_reduction_closed_forms():
    g = gold("closed_forms.json")
    n = g["n"]
    terms = O.imod_terms(0, 1, n, 3, 1000)
    assert O.reduce_i64(O.RED_ADD, 0, terms) == g["sum_3i_mod_1000"]
    assert O.imod_sum_closed_form(n, 3, 1000) == g["sum_3i_mod_1000"]
    iv = [O.induction_value(0, 1, k) for k in range(n)]
    assert O.reduce_i64(O.RED_ADD, 0, iv) == g["sum_i"] == n * (n - 1) // 2


def test_integer_reduction_ops_and_wrap():
    assert O.reduce_i64(O.RED_ADD, (1 << 63) - 1, [1]) == -(1 << 63)
    assert O.reduce_i64(O.RED_MUL, 1, range(1, 21)) == math.factorial(20)
    assert O.reduce_i64(O.RED_MUL, 1, [1 << 32, 1 << 32]) == 0  # 2^64 wraps to 0
    assert O.reduce_i64(O.RED_MAX, -5, [3, -9, 7, 1]) == 7
    assert O.reduce_i64(O.RED_MIN, 100, [3, -9, 7, 1]) == -9
    assert O.reduce_i64(O.RED_ADD, 17, []) == 17  # init combined exactly once


def test_imod_negative_induction_values():
    # (3 * iv) mod 7 with a non-negative remainder, iv = 5, 3, 1, -1, -3
    assert O.imod_terms(5, -2, 5, 3, 7) == [1, 2, 3, 4, 5]


def test_float_reduction_exact_cases():
    n = 1 << 20
    x = (np.arange(n, dtype=np.float64) * 2.0 ** -20).astype(np.float32)
    assert np.all(x.astype(np.float64) == np.arange(n) * 2.0 ** -20)
    assert O.reduce_f64(O.RED_ADD, 0.0, x) == (n * (n - 1) // 2) * 2.0 ** -20
    ints = np.arange(-5000, 5001, dtype=np.float32)
    assert O.reduce_f64(O.RED_ADD, 0.5, ints) == 0.5
    assert O.reduce_f64(O.RED_MAX, -np.inf, np.array([1, np.nan, 3], np.float32)) == 3.0
    assert O.reduce_f64(O.RED_MIN, np.inf, np.array([1, np.nan, -3], np.float32)) == -3.0
    assert O.reduce_f64(O.RED_MUL, 1.0, np.array([2, 0.5, -4], np.float32)) == -4.0
    # cancellation that a naive FP32 sum gets wrong
    v = np.array([1e8, 1.0, -1e8, 1.0], np.float32)
    assert O.reduce_f64(O.RED_ADD, 0.0, v) == 2.0


# --- AXPY body (§6 AXPY) ----------------------------------------------------------

def rn32_exact(q: Fraction) -> np.float32:
    """Nearest-even FP32 to the rational q, by comparing the candidates."""
    f = np.float32(float(q))
    cands = [np.nextafter(f, np.float32(-np.inf)), f, np.nextafter(f, np.float32(np.inf))]
    best = None
    for c in cands:
        d = abs(Fraction(float(c)) - q)
        key = (d, int(np.asarray(c).view(np.uint32)) & 1)
        if best is None or key < best[0]:
            best = (key, c)
    return np.float32(best[1])


def test_axpy_single_rounding_exact_rational():
    g = np.random.default_rng(1)
    x = np.concatenate([
        g.standard_normal(500).astype(np.float32),
        (g.standard_normal(300) * 1e-20).astype(np.float32),
        (g.standard_normal(300) * 1e20).astype(np.float32),
    ])
    y = np.concatenate([
        (g.standard_normal(500) * 1e15).astype(np.float32),
        g.standard_normal(300).astype(np.float32),
        (g.standard_normal(300) * 1e-3).astype(np.float32),
    ])
    for a in (2.5, -0.3, 3.0):
        got = O.axpy(a, x, y)
        a32 = Fraction(float(np.float32(a)))
        for i in range(0, len(x), 3):
            want = rn32_exact(Fraction(float(y[i])) + a32 * Fraction(float(x[i])))
            assert got[i].view(np.uint32) == want.view(np.uint32), (a, x[i], y[i])


def test_axpy_is_fused_not_mul_then_add():
    x = np.array([np.float32(1.0 + 2.0 ** -23)], np.float32)
    y = np.array([-2.5], np.float32)
    got = O.axpy(2.5, x, y)
    assert float(got[0]) == 2.0 ** -22 + 2.0 ** -24
    unfused = np.float32(np.float32(2.5) * x[0]) + y[0]
    assert float(unfused) == 2.0 ** -22


def test_axpy_workload_grid_is_exact_in_fp64():
    x, y = I.axpy_inputs(4096, seed=0)
    got = O.axpy(2.5, x, y)
    # on the 2^-23 grid a x + y is exact in FP64, so one FP32 rounding of it is the answer
    plain = (2.5 * x.astype(np.float64) + y.astype(np.float64))
    hi, lo = O.two_sum(2.5 * x.astype(np.float64), y.astype(np.float64))
    assert np.all(lo == 0)
    assert np.array_equal(got, plain.astype(np.float32))


# --- Jacobi body ------------------------------------------------------------------

def test_jacobi_hand_worked_5x5():
    g = gold("jacobi_5x5.json")
    u0 = np.array(g["initial"], np.float32)
    for mirror in (False, True):
        u, res = O.jacobi_run(u0, 2, mirror_f32=mirror)
        u1, r1 = O.jacobi_run(u0, 1, mirror_f32=mirror)
        assert np.array_equal(u1.astype(np.float64), np.array(g["after_sweep_1"]))
        assert np.array_equal(u.astype(np.float64), np.array(g["after_sweep_2"]))
        assert float(res[0]) == g["residual_1"] and float(res[1]) == g["residual_2"]
        assert float(r1[0]) == g["residual_1"]


def test_jacobi_harmonic_field_is_exact_fixed_point():
    r, c = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    u = ((3 + 2 * r + 5 * c + r * c) * 2.0 ** -12).astype(np.float32)
    v32, res32 = O.jacobi_sweep_f32(u)
    v64, res64 = O.jacobi_sweep_f64(u)
    assert np.array_equal(v32, u) and res32 == 0.0
    assert np.array_equal(v64, u.astype(np.float64)) and res64 == 0.0


def discrete_laplace_solution(n: int) -> np.ndarray:
    """Separation of variables for the discrete Laplace equation on an n x n
    grid with top edge 1 and the other edges 0."""
    m = n - 1
    u = np.zeros((n, n))
    u[0, :] = 1.0
    cc = np.arange(1, m)
    for k in range(1, m):
        th = k * math.pi / m
        lam = math.acosh(2.0 - math.cos(th))
        bk = (2.0 / m) * np.sum(np.sin(th * cc))
        for r in range(1, m):
            u[r, 1:m] += bk * np.sin(th * cc) * math.sinh(lam * (m - r)) / math.sinh(lam * m)
    return u


@pytest.mark.parametrize("n,sweeps", [(17, 3000), (33, 9000)])
def test_jacobi_converges_to_discrete_harmonic_solution(n, sweeps):
    u0 = np.zeros((n, n), np.float32)
    u0[0, :] = 1.0
    u, res = O.jacobi_run(u0, sweeps)
    exact = discrete_laplace_solution(n)
    assert np.max(np.abs(u[1:-1, 1:-1] - exact[1:-1, 1:-1])) <= 1e-10
    assert res[-1] < 1e-10 and np.all(np.diff(res[10:]) <= 1e-15)


def test_jacobi_fp32_mirror_within_forward_bound():
    u0 = I.jacobi_grid(64, seed=1)
    u32, r32 = O.jacobi_run(u0, 20, mirror_f32=True)
    u64, r64 = O.jacobi_run(u0, 20)
    bound = 20 * 3 * 2.0 ** -24
    assert np.max(np.abs(u32.astype(np.float64) - u64)) <= bound
    assert np.max(np.abs(r32.astype(np.float64) - r64)) <= 2 * bound


# --- matvec and GEMM bodies ------------------------------------------------------

def test_matvec_exact_structured_cases():
    n = 37
    x = np.arange(n, dtype=np.float32) - 11
    assert np.array_equal(O.matvec(np.eye(n, dtype=np.float32), x), x.astype(np.float64))
    perm = np.random.default_rng(2).permutation(n)
    p = np.eye(n, dtype=np.float32)[perm]
    assert np.array_equal(O.matvec(p, x), x[perm].astype(np.float64))
    ones = np.ones((5, n), np.float32)
    assert np.all(O.matvec(ones, x) == float(sum(range(-11, n - 11))))


def test_matvec_and_gemm_brute_force_integers():
    a = I.small_int_matrix(9, 13, -20, 20, seed=3)
    b = I.small_int_matrix(13, 7, -20, 20, seed=4)
    x = b[:, 0].copy()
    want_y = [sum(int(a[i, j]) * int(x[j]) for j in range(13)) for i in range(9)]
    assert O.matvec(a, x).tolist() == want_y
    want_c = [[sum(int(a[i, k]) * int(b[k, j]) for k in range(13)) for j in range(7)] for i in range(9)]
    assert O.gemm(a, b).tolist() == want_c
    # integers up to 256 are exact in bfloat16, so every variant is exact here
    assert O.gemm_bf16(a, b).tolist() == want_c
    assert O.gemm_bf16x3(a, b).tolist() == want_c


def test_bf16_round_matches_torch_conversion():
    g = np.random.default_rng(5)
    v = np.concatenate([
        g.standard_normal(20000).astype(np.float32),
        (g.standard_normal(2000) * 1e-39).astype(np.float32),  # subnormals
        np.array([0.0, -0.0, np.inf, -np.inf, 3.4e38, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8,
                  1.0 + 2 ** -8 + 2 ** -20], np.float32),
        np.random.default_rng(6).integers(0, 2 ** 32, 20000, dtype=np.uint64)
        .astype(np.uint32).view(np.float32),
    ])
    v = v[~np.isnan(v)]
    want = torch.from_numpy(v.copy()).to(torch.bfloat16).to(torch.float32).numpy()
    got = O.bf16_round(v)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
    assert np.isnan(O.bf16_round(np.array([np.nan], np.float32))[0])


def test_bf16_split_reconstructs_to_2pow_minus_16():
    # bfloat16 keeps 8 significant bits, so each rounding is within 2^-8 relative:
    # |v - hi| <= 2^-8 |v| and |(v - hi) - lo| <= 2^-8 |v - hi| <= 2^-16 |v|.
    a, _ = I.gemm_inputs(64, 64, 64)
    hi, lo = O.split_bf16(a)
    err = np.abs(a.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -16 * np.abs(a.astype(np.float64)))
    assert np.array_equal(O.bf16_round(hi), hi) and np.array_equal(O.bf16_round(lo), lo)


def test_gemm_freivalds_and_split_accuracy():
    a, b = I.gemm_inputs(96, 80, 112)
    c = O.gemm(a, b)
    r = np.random.default_rng(7).choice([-1.0, 1.0], size=80)
    lhs = c @ r
    rhs = a.astype(np.float64) @ (b.astype(np.float64) @ r)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(rhs))
    rel = np.linalg.norm(O.gemm_bf16x3(a, b) - c) / np.linalg.norm(c)
    assert rel < 2e-5
    rel16 = np.linalg.norm(O.gemm_bf16(a, b) - c) / np.linalg.norm(c)
    assert 1e-4 < rel16 < 1e-2


# --- data mapping (§4.1) -----------------------------------------------------------

def test_map_semantics_copy_and_poison():
    dev = O.Device()
    host = np.arange(6, dtype=np.float32)
    h_to = dev.map(host, O.MAP_TO)
    h_from = dev.map(np.zeros(6, np.float32), O.MAP_FROM)
    h_alloc = dev.map(np.zeros(4, np.int64), O.MAP_ALLOC)
    assert np.array_equal(dev.array(h_to), host)
    assert np.all(np.isnan(dev.array(h_from)))
    assert np.all(dev.array(h_alloc).view(np.uint8) == 0x5A)
    dev.array(h_to)[:] = -1
    dev.unmap(h_to)
    assert np.array_equal(host, np.arange(6, dtype=np.float32))  # 'to' is not copied back
    out = np.zeros(3, np.float32)
    h = dev.map(out, O.MAP_TOFROM)
    dev.array(h)[:] = 7
    dev.unmap(h)
    assert np.all(out == 7)
    with pytest.raises(ValueError):
        dev.map(host, 9)


# --- region interpreter (§3.1, §3.2, §5) -----------------------------------------

def test_region_axpy_with_two_reductions_closed_form():
    n = 1 << 16
    dev = O.Device()
    x = (np.arange(n, dtype=np.float64) * 2.0 ** -16).astype(np.float32)
    y = np.zeros(n, np.float32)
    sf = np.zeros(1, np.float32)
    si = np.array([5], np.int64)
    hx, hy = dev.map(x, O.MAP_TO), dev.map(y, O.MAP_TOFROM)
    hs, hi = dev.map(sf, O.MAP_TOFROM), dev.map(si, O.MAP_TOFROM)
    loop = O.Loop(O.BODY_AXPY, 0, n, 1, bufs=[hx, hy], scalars=[1.0, 3, 1000],
                  reductions=[O.Reduction(O.RED_ADD, O.DT_F32, hs, 0, O.TERM_Y),
                              O.Reduction(O.RED_ADD, O.DT_I64, hi, 0, O.TERM_IMOD)])
    O.run_region(dev, 4, 256, [loop])
    for h in (hx, hy, hs, hi):
        dev.unmap(h)
    assert np.array_equal(y, x)
    assert float(sf[0]) == (n * (n - 1) // 2) * 2.0 ** -16
    assert int(si[0]) == 5 + O.imod_sum_closed_form(n, 3, 1000)


def test_region_strided_axpy_touches_only_its_iterations():
    dev = O.Device()
    x = np.ones(10, np.float32)
    y = np.zeros(10, np.float32)
    hx, hy = dev.map(x, O.MAP_TO), dev.map(y, O.MAP_TOFROM)
    O.run_region(dev, 1, 2, [O.Loop(O.BODY_AXPY, 9, 0, -3, bufs=[hx, hy], scalars=[2.0])])
    dev.unmap(hy)
    assert y.tolist() == [0, 0, 0, 2, 0, 0, 2, 0, 0, 2]


def test_region_coverage_body_static_owner():
    dev = O.Device()
    owner = np.full(10, -1, np.int64)
    count = np.zeros(10, np.int64)
    ho, hc = dev.map(owner, O.MAP_TOFROM), dev.map(count, O.MAP_TOFROM)
    O.run_region(dev, 1, 3, [O.Loop(O.BODY_COVERAGE, 0, 10, 1, chunk=2, bufs=[ho, hc])])
    dev.unmap(ho)
    dev.unmap(hc)
    assert owner.tolist() == [0, 0, 1, 1, 2, 2, 0, 0, 1, 1]
    assert count.tolist() == [1] * 10


def test_region_jacobi_rows_and_residual():
    g = gold("jacobi_5x5.json")
    dev = O.Device()
    u0 = np.array(g["initial"], np.float32)
    u1 = u0.copy()
    r = np.full(1, -np.inf, np.float32)
    h0, h1, hr = dev.map(u0, O.MAP_TOFROM), dev.map(u1, O.MAP_TOFROM), dev.map(r, O.MAP_TOFROM)
    O.run_region(dev, 1, 1, [O.Loop(O.BODY_JACOBI5, 1, 4, 1, bufs=[h0, h1],
                                    reductions=[O.Reduction(O.RED_MAX, O.DT_F32, hr, 0, O.TERM_RESID)])])
    for h in (h0, h1, hr):
        dev.unmap(h)
    assert np.array_equal(u1.astype(np.float64), np.array(g["after_sweep_1"]))
    assert float(r[0]) == g["residual_1"]


# --- MLP cost model ------------------------------------------------------------------

def test_mlp_backward_matches_central_differences():
    p = {k: v.astype(np.float64) for k, v in I.mlp_init(seed=9, hidden=8).items()}
    x, t = I.mlp_dataset(6, seed=8)
    yhat, cache = O.mlp_forward(p, x, bf16_weights=False)
    g = O.mlp_backward(cache, yhat, t)
    h = 1e-6
    for k in O.MLP_KEYS:
        flat = p[k].ravel()
        for idx in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[idx]
            flat[idx] = old + h
            lp = O.mlp_loss(O.mlp_forward(p, x, False)[0], t)
            flat[idx] = old - h
            lm = O.mlp_loss(O.mlp_forward(p, x, False)[0], t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].ravel()[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (k, idx, fd, an)


def test_mlp_linear_layer_closed_form_gradient():
    # With all hidden units active and identity-like weights the net is linear:
    # yhat = w . x + b, and dL/dw = (2/B) X^T (X w + b - t).
    n_in = 12
    p = {"W1": np.eye(n_in * 1, n_in)[:n_in].astype(np.float64),
         "b1": np.full(n_in, 10.0), "W2": np.eye(n_in), "b2": np.zeros(n_in),
         "W3": np.arange(1, n_in + 1, dtype=np.float64)[None, :], "b3": np.array([0.5])}
    x, t = I.mlp_dataset(5, seed=3)
    x = x.astype(np.float64)
    yhat, cache = O.mlp_forward(p, x, bf16_weights=False)
    w = p["W3"][0]
    assert np.allclose(yhat, (x + 10.0) @ w + 0.5)
    g = O.mlp_backward(cache, yhat, t)
    resid = yhat - t
    assert np.allclose(g["W3"][0], (2 / 5) * (x + 10.0).T @ resid)
    assert np.allclose(g["b1"], (2 / 5) * resid.sum() * w)


def test_mlp_sgd_step_descends():
    p = I.mlp_init(seed=9)
    x, t = I.mlp_dataset(64, seed=8)
    y0, c0 = O.mlp_forward(p, x)
    l0 = O.mlp_loss(y0, t)
    p1 = O.mlp_sgd(p, O.mlp_backward(c0, y0, t), 1e-3)
    assert O.mlp_loss(O.mlp_forward(p1, x)[0], t) < l0


# --- time-blocked Jacobi body -------------------------------------------------

def test_jacobi_tb_hand_worked_5x5_two_sweeps():
    g = gold("jacobi_5x5.json")
    u0 = np.array(g["initial"], np.float32)
    u, terms = O.jacobi_tb(u0, 1, 4, 2)
    assert np.array_equal(u, np.array(g["after_sweep_2"]))
    assert [t.max() for t in terms] == [g["residual_1"], g["residual_2"]]
    um, tm = O.jacobi_tb(u0, 1, 4, 2, mirror_f32=True)
    assert np.array_equal(um, np.array(g["after_sweep_2"], np.float32))
    assert [np.float32(t.max()) for t in tm] == [np.float32(g["residual_1"]), np.float32(g["residual_2"])]


def test_jacobi_tb_row_subrange_keeps_other_rows_fixed():
    g = gold("jacobi_5x5_rows_1_to_2.json")
    u0 = np.array(g["initial"], np.float32)
    for mirror in (False, True):
        u, terms = O.jacobi_tb(u0, g["lb"], g["ub"], g["sweeps"], mirror_f32=mirror)
        assert np.array_equal(u, np.array(g["after"]))
        assert [float(t.max()) for t in terms] == g["residuals"]


@pytest.mark.parametrize("sweeps", [1, 3, 8])
def test_jacobi_tb_harmonic_field_is_fixed_point(sweeps):
    # u = (a + b r + c c' + d r c') / 2^k with small integers is discrete
    # harmonic and exact in FP32: every sweep reproduces it, residuals 0
    r, c = np.meshgrid(np.arange(17), np.arange(23), indexing="ij")
    u0 = ((3 + 2 * r - 5 * c + r * c) / 64.0).astype(np.float32)
    for mirror in (False, True):
        u, terms = O.jacobi_tb(u0, 1, 16, sweeps, mirror_f32=mirror)
        assert np.array_equal(u, u0)
        assert all(float(t.max()) == 0.0 for t in terms)


def test_jacobi_tb_no_rows_changes_nothing():
    u0 = I.jacobi_grid(9, seed=1)
    u, terms = O.jacobi_tb(u0, 4, 4, 3)
    assert np.array_equal(u, u0) and all(t.size == 0 for t in terms)


# --- 7 x 7 filter ---------------------------------------------------------------

def _delta(i, j, v=1.0):
    w = np.zeros((7, 7), np.float32)
    w[i, j] = v
    return w


@pytest.mark.parametrize("i,j", [(3, 3), (0, 0), (6, 1), (2, 5)])
def test_filter7_single_tap_is_a_shift(i, j):
    # a single unit weight at (i, j) copies x[r + i - 3][c + j - 3]: pins the
    # direction of both offsets and that the window is not transposed
    x = np.arange(400, dtype=np.float32).reshape(20, 20)
    want = x[3 + i - 3:17 + i - 3, j:j + 14]
    assert np.array_equal(O.filter7_f64(x, _delta(i, j), 3, 17), want)
    assert np.array_equal(O.filter7_f32(x, _delta(i, j), 3, 17), want)


def test_filter7_matches_library_correlation():
    from scipy.signal import correlate2d
    g = np.random.default_rng(21)
    x = g.standard_normal((40, 37))
    w = g.standard_normal((7, 7))
    want = correlate2d(x, w, mode="valid")          # [34, 31]: rows 3..36, cols 3..33
    assert np.allclose(O.filter7_f64(x, w, 3, 37), want, rtol=0, atol=1e-12)
    # a row sub-range takes the matching rows of the full result
    assert np.allclose(O.filter7_f64(x, w, 10, 20), want[7:17], rtol=0, atol=1e-12)


def test_filter7_linear_field_times_weight_sum():
    # a symmetric all-ones window maps a linear field f to 49 f exactly
    r, c = np.meshgrid(np.arange(16), np.arange(18), indexing="ij")
    x = (5 + 3 * r - 2 * c).astype(np.float32)
    w = np.ones((7, 7), np.float32)
    want = 49 * x[3:13, 3:15]
    assert np.array_equal(O.filter7_f64(x, w, 3, 13), want)
    assert np.array_equal(O.filter7_f32(x, w, 3, 13), want)


def test_filter7_mirror_rounds_each_tap_once():
    # taps (3,3) then (3,4): fma(1 + 2^-12, 1 + 2^-12, -(1 + 2^-11)) = 2^-24
    # exactly; a separately rounded product (a tie, to even) would give 0
    x = np.zeros((7, 8), np.float32)
    x[3, 3] = -(1 + 2.0 ** -11)
    x[3, 4] = 1 + 2.0 ** -12
    w = np.zeros((7, 7), np.float32)
    w[3, 3] = 1.0
    w[3, 3 + 1] = 1 + 2.0 ** -12
    out = O.filter7_f32(x, w, 3, 4)
    assert out[0, 0] == np.float32(2.0 ** -24)


def test_filter7_mirror_within_forward_bound():
    x = I.jacobi_grid(64, seed=3)
    w = np.random.default_rng(4).random((7, 7)).astype(np.float32)
    w /= w.sum()
    exact = O.filter7_f64(x, w, 3, 61)
    mirror = O.filter7_f32(x, w, 3, 61).astype(np.float64)
    absw = O.filter7_f64(np.abs(x), np.abs(w), 3, 61)
    assert np.all(np.abs(mirror - exact) <= 49 * 2.0 ** -24 * absw)


def test_filter7_mirror_exact_on_small_integers():
    g = np.random.default_rng(5)
    x = g.integers(-50, 50, (30, 33)).astype(np.float32)
    w = g.integers(-9, 10, (7, 7)).astype(np.float32)
    assert np.array_equal(O.filter7_f32(x, w, 3, 27), O.filter7_f64(x, w, 3, 27))


def test_region_interpreter_time_blocked_loop_reduces_per_sweep():
    dev = O.Device()
    u0 = I.jacobi_grid(12, seed=1)
    a, b = dev.map(u0.copy(), O.MAP_TOFROM), dev.map(u0.copy(), O.MAP_TOFROM)
    res = dev.map(np.full(6, -np.inf, np.float32), O.MAP_TOFROM)
    lp = O.Loop(O.BODY_JACOBI5_TB, 2, 9, bufs=[a, b], scalars=[12, 12, 4],
                reductions=[O.Reduction(O.RED_MAX, O.DT_F32, res, 1, O.TERM_RESID)])
    O.run_region(dev, 1, 1, [lp])
    want, terms = O.jacobi_tb(u0, 2, 9, 4)
    assert np.array_equal(dev.array(b)[2:9, 1:-1], want[2:9, 1:-1].astype(np.float32))
    assert np.array_equal(dev.array(b)[:2], u0[:2]) and np.array_equal(dev.array(a), u0)
    r = dev.array(res)
    assert r[0] == -np.inf and r[5] == -np.inf
    assert np.array_equal(r[1:5], np.array([t.max() for t in terms], np.float32))


# --- guided schedule and taskloop -------------------------------------------------

def test_guided_and_taskloop_hand_tables():
    g = gold("guided_taskloop_tables.json")
    for c in g["guided"]:
        ch = O.guided_chunks(c["trip"], c["workers"], c["chunk"])
        assert [e - s for s, e in ch] == c["sizes"], c
    for c in g["taskloop"]:
        ch = O.taskloop_chunks(c["trip"], c["grainsize"], c["num_tasks"])
        assert [e - s for s, e in ch] == c["sizes"], c


def test_guided_invariants_brute_force():
    for trip in range(0, 80):
        for workers in range(1, 7):
            for chunk in range(0, 6):
                ch = O.guided_chunks(trip, workers, chunk)
                sizes = [e - s for s, e in ch]
                assert sum(sizes) == trip and all(z > 0 for z in sizes)
                assert all(a >= b for a, b in zip(sizes, sizes[1:-1]))  # non-increasing but the last
                s = 0
                for a, b in ch:  # each chunk: max(c, ceil(remaining / W)), capped by what remains
                    assert a == s and b - a == min(trip - a, max(max(chunk, 1), -(-(trip - a) // workers)))
                    s = b


def test_taskloop_invariants_brute_force():
    for trip in range(0, 60):
        for gs in range(0, 8):
            for nt in range(0, 8):
                if gs == 0 and nt == 0:
                    continue
                ch = O.taskloop_chunks(trip, gs, nt)
                sizes = [e - s for s, e in ch]
                assert sum(sizes) == trip
                if trip == 0:
                    continue
                assert max(sizes) - min(sizes) <= 1
                if nt:
                    assert len(sizes) <= nt
                if gs and not nt:
                    assert min(sizes) >= min(gs, trip) and (trip < gs or max(sizes) < 2 * gs)


def test_chunked_assignment_checker_catches_violations():
    ch = O.guided_chunks(20, 3, 0)
    owner = np.zeros(20, np.int64)
    count = np.ones(20, np.int64)
    for k, (s, e) in enumerate(ch):
        owner[s:e] = k % 3
    assert O.check_chunked_assignment(20, ch, owner, count, 3)
    bad = owner.copy()
    bad[ch[0][0]] = (bad[ch[0][0]] + 1) % 3          # a chunk split over two workers
    assert not O.check_chunked_assignment(20, ch, bad, count, 3)
    twice = count.copy()
    twice[5] = 2                                        # an iteration run twice
    assert not O.check_chunked_assignment(20, ch, owner, twice, 3)
    assert not O.check_chunked_assignment(20, ch[:-1], owner, count, 3)   # chunks do not tile the range
