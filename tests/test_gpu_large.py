"""Iteration spaces and arrays past 2^31 elements (64-bit indexing on every
path of the element and matvec kernels), with structured device-resident
inputs whose results have closed forms: no oracle run at this size."""
import numpy as np
import pytest

from oracle import upir_oracle as O

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")
torch = pytest.importorskip("torch")
from upir_helpers import Session, axpy_loop  # noqa: E402

BIG = (1 << 31) + 4099


@pytest.fixture(scope="module")
def s():
    sess = Session()
    yield sess
    sess.close()
    torch.cuda.empty_cache()


def dev_map(s, t):
    return U.upir_data_map_device(s.ctx, t.data_ptr(), t.numel() * t.element_size())


def test_axpy_with_reductions_past_2p31_iterations(s):
    """y = 2.5 x + y over n = 2^31 + 4099 with x = 1, y = 0: every y is 2.5;
    the int64 reduction of (3 i mod 1000) equals its closed form exactly and
    the compensated FP32 sum of y is within two units in the last place of
    2.5 n.  A second loop over [2^31 - 8, n) checks ranges that start past
    the 32-bit boundary."""
    x = torch.ones(BIG, dtype=torch.float32, device="cuda")
    y = torch.zeros(BIG, dtype=torch.float32, device="cuda")
    fvar = np.zeros(2, np.float32)
    ivar = np.zeros(2, np.int64)
    torch.cuda.synchronize()
    hx, hy = dev_map(s, x), dev_map(s, y)
    hf, hi = s.map(fvar, U.UPIR_MAP_TOFROM), s.map(ivar, U.UPIR_MAP_TOFROM)
    lb2 = (1 << 31) - 8
    s.run([axpy_loop(hx, hy, BIG, reds=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_Y, hf, 0),
                                        (U.UPIR_RED_ADD, U.UPIR_I64, U.UPIR_TERM_IMOD, hi, 0)]),
           axpy_loop(hx, hy, BIG, lb=lb2, a=1.0, reds=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_Y, hf, 1),
                                                       (U.UPIR_RED_ADD, U.UPIR_I64, U.UPIR_TERM_IMOD, hi, 1)])])
    for h in (hx, hy, hf, hi):
        s.unmap(h)
    idx = torch.tensor([0, 1, 12345, lb2 - 1, lb2, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, BIG - 2, BIG - 1],
                       device="cuda")
    got = y[idx].cpu().numpy()
    want = np.array([2.5] * 4 + [3.5] * 6, np.float32)
    assert np.array_equal(got, want)
    assert int(ivar[0]) == O.imod_sum_closed_form(BIG, 3, 1000)
    assert int(ivar[1]) == O.imod_sum_closed_form(BIG, 3, 1000) - O.imod_sum_closed_form(lb2, 3, 1000)
    exact0 = 2.5 * BIG
    assert abs(float(fvar[0]) - exact0) <= 2 * np.spacing(np.float32(exact0))
    assert float(fvar[1]) == 3.5 * (BIG - lb2)
    del x, y
    torch.cuda.empty_cache()


@pytest.mark.parametrize("cols", [32772, 32771])
def test_matvec_past_2p31_elements(s, cols):
    """A 65536 x cols matrix (more than 2^31 elements; cols = 32771 puts
    three rows in four off the 16-byte grid) with A[r][c] = (r + c) mod 7 - 3
    and x = 1: y[r] depends on r mod 7 only and is an exact small integer."""
    rows = 65536
    a = torch.empty((rows, cols), dtype=torch.float32, device="cuda")
    cc = torch.arange(cols, device="cuda")[None, :]
    for r0 in range(0, rows, 4096):
        rr = torch.arange(r0, r0 + 4096, device="cuda")[:, None]
        a[r0:r0 + 4096] = ((rr + cc) % 7 - 3).to(torch.float32)
    del cc
    x = torch.ones(cols, dtype=torch.float32, device="cuda")
    y = torch.full((rows,), -7.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    ha, hx, hy = dev_map(s, a), dev_map(s, x), dev_map(s, y)
    s.run([dict(lb=0, ub=rows, body=U.UPIR_BODY_MATVEC, bufs=[ha, hx, hy], scalars=[rows, cols])])
    for h in (ha, hx, hy):
        s.unmap(h)
    per_residue = np.array([np.sum((k + np.arange(cols)) % 7 - 3) for k in range(7)], np.float32)
    want = per_residue[np.arange(rows) % 7]
    assert np.array_equal(y.cpu().numpy(), want)
    del a, x, y
    torch.cuda.empty_cache()


def test_jacobi_sweep_past_2p31_points(s):
    """One sweep of a 46342 x 46344 grid (more than 2^31 points) holding the
    discrete harmonic field u = r + 2 c, exact in FP32 at this size: the sweep
    returns it unchanged, point for point, and the max residual is 0."""
    rows, cols = 46342, 46344
    u = torch.empty((rows, cols), dtype=torch.float32, device="cuda")
    cc = 2 * torch.arange(cols, device="cuda", dtype=torch.float32)[None, :]
    for r0 in range(0, rows, 4096):
        r1 = min(rows, r0 + 4096)
        u[r0:r1] = torch.arange(r0, r1, device="cuda", dtype=torch.float32)[:, None] + cc
    del cc
    out = torch.full_like(u, -1.0)
    out[0] = u[0]
    out[-1] = u[-1]
    out[:, 0] = u[:, 0]
    out[:, -1] = u[:, -1]
    res = np.full(1, -np.inf, np.float32)
    torch.cuda.synchronize()
    hu, ho = dev_map(s, u), dev_map(s, out)
    hr = s.map(res, U.UPIR_MAP_TOFROM)
    s.run([dict(lb=1, ub=rows - 1, step=1, collapse=2, body=U.UPIR_BODY_JACOBI5, bufs=[hu, ho],
                scalars=[rows, cols], reductions=[(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_RESID, hr, 0)])])
    for h in (hu, ho, hr):
        s.unmap(h)
    assert bool(torch.equal(out, u))
    assert res[0] == 0.0
    del u, out
    torch.cuda.empty_cache()


def test_time_blocked_jacobi_past_2p31_points(s):
    """Eight sweeps in one time-blocked loop over the same 46342 x 46344
    harmonic field: the field comes back unchanged and all eight residuals
    are 0."""
    rows, cols = 46342, 46344
    u = torch.empty((rows, cols), dtype=torch.float32, device="cuda")
    cc = 2 * torch.arange(cols, device="cuda", dtype=torch.float32)[None, :]
    for r0 in range(0, rows, 4096):
        r1 = min(rows, r0 + 4096)
        u[r0:r1] = torch.arange(r0, r1, device="cuda", dtype=torch.float32)[:, None] + cc
    del cc
    out = u.clone()
    out[1:-1, 1:-1] = -1.0
    res = np.full(8, -np.inf, np.float32)
    torch.cuda.synchronize()
    hu, ho = dev_map(s, u), dev_map(s, out)
    hr = s.map(res, U.UPIR_MAP_TOFROM)
    s.run([dict(lb=1, ub=rows - 1, step=1, collapse=2, body=U.UPIR_BODY_JACOBI5_TB, bufs=[hu, ho],
                scalars=[rows, cols, 8], reductions=[(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_RESID, hr, 0)])])
    for h in (hu, ho, hr):
        s.unmap(h)
    assert bool(torch.equal(out, u))
    assert np.all(res == 0.0)
    del u, out
    torch.cuda.empty_cache()


@pytest.mark.parametrize("variant", [0, 1])
def test_gemm_f32_past_2p31_elements_of_a(s, variant):
    """C = A B with A 65536 x 32772 (more than 2^31 elements), A[r][k] =
    (r + k) mod 5 - 2 and B = 1 (32772 x 8): every C[r][j] is the exact
    integer sum over k, which depends on r mod 5 only; both FP32 kernels."""
    m, k, n = 65536, 32772, 8
    a = torch.empty((m, k), dtype=torch.float32, device="cuda")
    kk = torch.arange(k, device="cuda")[None, :]
    for r0 in range(0, m, 4096):
        rr = torch.arange(r0, r0 + 4096, device="cuda")[:, None]
        a[r0:r0 + 4096] = ((rr + kk) % 5 - 2).to(torch.float32)
    del kk
    b = torch.ones((k, n), dtype=torch.float32, device="cuda")
    c = torch.full((m, n), -3.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    ha, hb, hc = dev_map(s, a), dev_map(s, b), dev_map(s, c)
    s.run([dict(lb=0, ub=m, step=1, collapse=2, body=U.UPIR_BODY_GEMM_F32, bufs=[ha, hb, hc], scalars=[m, n, k],
                hints=[(U.UPIR_HINT_VARIANT, variant)] if variant else [])])
    for h in (ha, hb, hc):
        s.unmap(h)
    per_residue = np.array([np.sum((q + np.arange(k)) % 5 - 2) for q in range(5)], np.float32)
    want = np.repeat(per_residue[np.arange(m) % 5][:, None], n, axis=1)
    assert np.array_equal(c.cpu().numpy(), want)
    del a, b, c
    torch.cuda.empty_cache()
