"""The paper's four evaluation kernels (§6: AXPY, matrix multiplication,
matrix-vector multiplication and the size-7 stencil) at its problem sizes, run
as the paper's programs run them: map the host arrays, one offloaded loop,
unmap.  Each output is checked against the oracle: AXPY bit-exact (one
rounding per element), the stencil bit-exact against the oracle's FP32 mirror,
matmul and matvec normwise within 1e-5, and per element within the rounding
bound of an FP32 dot product of their length (matvec: 1e-5 of the absolute
products' sum, as in the full-size test).  The largest sizes (AXPY 10^7 and 10^8,
matrices beyond 1024 and grids beyond 1024) are left to the full-size parity
tests of each kernel."""
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


def offload(s, arrays, loop_of):
    hs = [s.map(a, kind) for a, kind in arrays]
    s.run([loop_of(hs)])
    for h in hs:
        s.unmap(h)


@pytest.mark.parametrize("n", [10240, 102400, 1024000])
def test_axpy_paper_sizes(s, n):
    x, y0 = I.axpy_inputs(n, seed=21)
    y = y0.copy()
    offload(s, [(x, U.UPIR_MAP_TO), (y, U.UPIR_MAP_TOFROM)],
            lambda hs: dict(lb=0, ub=n, body=U.UPIR_BODY_AXPY, bufs=hs, scalars=[2.0, 3, 1000]))
    assert np.array_equal(y.view(np.uint32), O.axpy(2.0, x, y0).view(np.uint32))


@pytest.mark.parametrize("n", [64, 128, 256, 512, 1024])
def test_matmul_paper_sizes(s, n):
    a, b = I.gemm_inputs(n, n, n, seed_a=22, seed_b=23)
    c = np.full((n, n), -3.0, np.float32)
    offload(s, [(a, U.UPIR_MAP_TO), (b, U.UPIR_MAP_TO), (c, U.UPIR_MAP_FROM)],
            lambda hs: dict(lb=0, ub=n, collapse=2, body=U.UPIR_BODY_GEMM_F32, bufs=hs, scalars=[n, n, n]))
    ref = O.gemm(a, b)
    # an FP32 dot product of length n by fused multiply-adds is within
    # gamma_(n + 2) = (n + 2) u / (1 - (n + 2) u) of the absolute products'
    # sum, u = 2^-24 (the k-split adds one more rounding)
    u = 2.0 ** -24
    gamma = (n + 2) * u / (1 - (n + 2) * u)
    bound = np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64))
    assert np.linalg.norm(c - ref) <= 1e-5 * np.linalg.norm(ref)
    assert np.all(np.abs(c - ref) <= gamma * bound + 1e-30)


@pytest.mark.parametrize("n", [1024, 2048, 4096])
def test_matvec_paper_sizes(s, n):
    a, x = I.matvec_inputs(n, n, seed_a=24, seed_x=25)
    y = np.full(n, -3.0, np.float32)
    offload(s, [(a, U.UPIR_MAP_TO), (x, U.UPIR_MAP_TO), (y, U.UPIR_MAP_FROM)],
            lambda hs: dict(lb=0, ub=n, body=U.UPIR_BODY_MATVEC, bufs=hs, scalars=[n, n]))
    ref = O.matvec(a, x)
    bound = np.abs(a.astype(np.float64)) @ np.abs(x.astype(np.float64))
    assert np.linalg.norm(y - ref) <= 1e-5 * np.linalg.norm(ref)
    assert np.all(np.abs(y - ref) <= 1e-5 * bound + 1e-30)


@pytest.mark.parametrize("n", [64, 128, 256, 512, 1024])
def test_stencil_paper_sizes(s, n):
    xg = I.jacobi_grid(n, seed=26)
    w = np.random.default_rng(27).random((7, 7)).astype(np.float32)
    w = (w / w.sum()).astype(np.float32)
    out = np.full_like(xg, -7.0)
    offload(s, [(xg, U.UPIR_MAP_TO), (out, U.UPIR_MAP_TOFROM)],
            lambda hs: dict(lb=3, ub=n - 3, step=1, collapse=2, body=U.UPIR_BODY_FILTER7, bufs=hs,
                            scalars=[n, n] + [float(v) for v in w.ravel()]))
    assert np.array_equal(out[3:n - 3, 3:n - 3].view(np.uint32),
                          O.filter7_f32(xg, w, 3, n - 3).view(np.uint32))
    edge = np.ones(out.shape, bool)
    edge[3:n - 3, 3:n - 3] = False
    assert np.all(out[edge] == -7.0)
