"""The batched uneven-regions workload at its full sizes (§3.1 SPMD regions
submitted together, §5 reduction syncs): 512 independent regions, seed 6,
trip counts log-uniform in [1e3, 1e7], Jacobi grids up to 2048^2, matvec up to
8192 x 8192.  Every region of the batch is compared with the oracle in all
three batch modes (one launch per loop, one CUDA graph of those launches, the
persistent executor after its tile autotuning):

- AXPY: y bit-exact; its dot reduction within 1e-5 of the FP64 exact sum;
- Jacobi: the field and the residual bit-exact against the FP32 mirror;
- matvec: within 1e-5 normwise and componentwise (against |A| |x|).

Outputs are poisoned (NaN) before each mode, so every point a region should
write is shown to be written."""
import numpy as np
import pytest

import upir_inputs as I
from oracle import upir_oracle as O

pytestmark = pytest.mark.gpu

U = pytest.importorskip("paper_2209_10643_b300")
from upir_helpers import Session  # noqa: E402

COUNT = 512
SEED = 6


class FullBatch:
    """The 512 regions mapped into one context, with the oracle's results."""

    def __init__(self):
        self.s = Session()
        self.specs = I.batched_region_specs(COUNT, seed=SEED)
        self.regions, self.items = [], []
        ctx = self.s.ctx
        for sp in self.specs:
            arr = I.region_arrays(sp)
            r = U.upir_spmd_region(ctx, 0, 0)
            if sp["op"] == I.OP_AXPY_DOT:
                y0 = arr["y"].copy()
                dot = np.zeros(1, np.float32)
                hx, hy, hd = self.s.map(arr["x"], 0), self.s.map(arr["y"], 2), self.s.map(dot, 2)
                U.upir_loop_checked(ctx, r, U.make_loop_desc(
                    lb=0, ub=sp["n"], body=U.UPIR_BODY_AXPY, bufs=[hx, hy], scalars=[2.5],
                    reductions=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_XY, hd, 0)]))
                want_y = O.axpy(2.5, arr["x"], y0)
                want_d = O.reduce_f64(O.RED_ADD, 0.0, arr["x"].astype(np.float64) * want_y)
                self.items.append(dict(kind="axpy", y=arr["y"], y0=y0, dot=dot, hy=hy, hd=hd,
                                       want_y=want_y, want_d=want_d))
            elif sp["op"] == I.OP_JACOBI:
                side = sp["side"]
                res = np.full(1, -np.inf, np.float32)
                h0, h1, hr = self.s.map(arr["u0"], 0), self.s.map(arr["u1"], 2), self.s.map(res, 2)
                U.upir_loop_checked(ctx, r, U.make_loop_desc(
                    lb=1, ub=side - 1, collapse=2, body=U.UPIR_BODY_JACOBI5, bufs=[h0, h1],
                    scalars=[side, side],
                    reductions=[(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_RESID, hr, 0)]))
                want_u, want_r = O.jacobi_sweep_f32(arr["u0"])
                self.items.append(dict(kind="jacobi", u1=arr["u1"], res=res, h1=h1, hr=hr,
                                       want_u=want_u, want_r=want_r))
            else:
                rows, cols = sp["rows"], sp["cols"]
                y = np.zeros(rows, np.float32)
                ha, hx, hy = self.s.map(arr["A"], 0), self.s.map(arr["x"], 0), self.s.map(y, 2)
                U.upir_loop_checked(ctx, r, U.make_loop_desc(
                    lb=0, ub=rows, body=U.UPIR_BODY_MATVEC, bufs=[ha, hx, hy], scalars=[rows, cols]))
                want = O.matvec(arr["A"], arr["x"])
                bound = np.abs(arr["A"]).astype(np.float64) @ np.abs(arr["x"]).astype(np.float64)
                self.items.append(dict(kind="matvec", y=y, hy=hy, want=want, bound=bound))
            self.regions.append(r)

    def reset(self):
        """Inputs back to their start values, outputs poisoned."""
        ctx = self.s.ctx
        for it in self.items:
            if it["kind"] == "axpy":
                it["y"][:] = it["y0"]
                it["dot"][0] = 0.0
                U.upir_data_update(ctx, it["hy"], U.UPIR_MAP_TO)
                U.upir_data_update(ctx, it["hd"], U.UPIR_MAP_TO)
            elif it["kind"] == "jacobi":
                it["u1"][1:-1, 1:-1] = np.nan
                it["res"][0] = -np.inf
                U.upir_data_update(ctx, it["h1"], U.UPIR_MAP_TO)
                U.upir_data_update(ctx, it["hr"], U.UPIR_MAP_TO)
            else:
                it["y"][:] = np.nan
                U.upir_data_update(ctx, it["hy"], U.UPIR_MAP_TO)

    def fetch(self):
        ctx = self.s.ctx
        for it in self.items:
            for key in ("hy", "hd", "h1", "hr"):
                if key in it:
                    U.upir_data_update(ctx, it[key], U.UPIR_MAP_FROM)

    def check(self):
        bad = []
        for k, it in enumerate(self.items):
            if it["kind"] == "axpy":
                if not np.array_equal(it["y"], it["want_y"]):
                    bad.append((k, "axpy y"))
                if not abs(float(it["dot"][0]) - it["want_d"]) <= 1e-5 * abs(it["want_d"]):
                    bad.append((k, "axpy dot", float(it["dot"][0]), it["want_d"]))
            elif it["kind"] == "jacobi":
                if not np.array_equal(it["u1"], it["want_u"]):
                    bad.append((k, "jacobi field"))
                if not it["res"][0] == it["want_r"]:
                    bad.append((k, "jacobi residual", float(it["res"][0]), float(it["want_r"])))
            else:
                y, want = it["y"].astype(np.float64), it["want"]
                if not np.linalg.norm(y - want) <= 1e-5 * np.linalg.norm(want):
                    bad.append((k, "matvec normwise"))
                if not np.all(np.abs(y - want) <= 1e-5 * it["bound"]):
                    bad.append((k, "matvec componentwise"))
        return bad

    def close(self):
        for r in self.regions:
            U.upir_region_destroy(r)
        self.s.close()


@pytest.fixture(scope="module")
def full():
    fb = FullBatch()
    yield fb
    fb.close()


def test_full_batch_spans_the_stated_ranges(full):
    sp = full.specs
    ops = [s["op"] for s in sp]
    assert len(sp) == COUNT
    assert ops.count(I.OP_AXPY_DOT) > 150 and ops.count(I.OP_JACOBI) > 100 and ops.count(I.OP_MATVEC) > 100
    assert max(s.get("n", 0) for s in sp) > 9_000_000
    assert max(s.get("side", 0) for s in sp) == 2048
    assert max(s.get("rows", 0) for s in sp) > 8000
    assert max(s.get("cols", 0) for s in sp) == 8192


@pytest.mark.parametrize("mode", ["launches", "graph", "persistent_autotuned"])
def test_full_batch_matches_oracle(full, mode):
    m = {"launches": U.UPIR_BATCH_LAUNCHES, "graph": U.UPIR_BATCH_GRAPH,
         "persistent_autotuned": U.UPIR_BATCH_PERSISTENT}[mode]
    b = U.upir_batch_create(full.s.ctx, full.regions, m)
    try:
        if m == U.UPIR_BATCH_PERSISTENT:
            tiles = U.upir_batch_autotune(b, 1)
            assert tiles[0] in (4096, 8192, 16384, 32768) and tiles[1] in (8, 16, 32)
        full.reset()
        U.upir_batch_submit(b)
        U.upir_ctx_wait(full.s.ctx)
    finally:
        U.upir_batch_destroy(b)
    full.fetch()
    bad = full.check()
    assert not bad, bad[:10]
