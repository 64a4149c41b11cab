"""Test-side conveniences over the C-ABI binding: map numpy arrays, build and
run one region, read results back.  Marshalling only."""
import numpy as np

import paper_2209_10643_b300 as U


class Session:
    """One upir context plus the numpy arrays mapped into it."""

    def __init__(self, device: int = 0):
        self.ctx = U.upir_init(device)
        self._bufs = {}

    def map(self, arr: np.ndarray, kind: int) -> int:
        assert arr.flags["C_CONTIGUOUS"]
        h = U.upir_data_map(self.ctx, arr.ctypes.data, arr.nbytes, kind)
        self._bufs[h] = arr
        return h

    def unmap(self, h: int) -> None:
        U.upir_data_unmap(self.ctx, h)
        self._bufs.pop(h, None)

    def run(self, loops, teams: int = 0, units: int = 0, flags: int = 0, keep: bool = False):
        """Record ``loops`` (kwargs dicts for make_loop_desc) in a region and submit it."""
        r = U.upir_spmd_region(self.ctx, teams, units)
        for lp in loops:
            U.upir_loop_checked(self.ctx, r, U.make_loop_desc(**lp))
        try:
            U.upir_region_submit(r, flags)
        except U.UpirError as e:
            raise U.UpirError(e.status, "upir_region_submit: " + U.lib.upir_last_error(self.ctx).decode())
        U.upir_ctx_wait(self.ctx)
        if keep:
            return r
        U.upir_region_destroy(r)
        return None

    def close(self):
        U.upir_finalize(self.ctx)
        self.ctx = None


def axpy_loop(hx, hy, n, a=2.5, reds=(), sched=U.UPIR_SCHED_STATIC, chunk=0, imod=(3, 1000),
              lb=0, step=1, ub=None, hints=()):
    return dict(lb=lb, ub=n if ub is None else ub, step=step, body=U.UPIR_BODY_AXPY, bufs=[hx, hy],
                scalars=[a, imod[0], imod[1]], reductions=list(reds), sched=sched, chunk=chunk,
                hints=list(hints))


def jacobi_loop(h_in, h_out, rows, cols, hres=None, res_index=0, op=U.UPIR_RED_MAX,
                sched=U.UPIR_SCHED_STATIC, chunk=0, hints=(), lb=1, ub=None):
    reds = [] if hres is None else [(op, U.UPIR_F32, U.UPIR_TERM_RESID, hres, res_index)]
    return dict(lb=lb, ub=rows - 1 if ub is None else ub, step=1, collapse=2,
                body=U.UPIR_BODY_JACOBI5, bufs=[h_in, h_out], scalars=[rows, cols],
                reductions=reds, sched=sched, chunk=chunk, hints=list(hints))
