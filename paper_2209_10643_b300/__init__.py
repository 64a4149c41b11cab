"""Python binding of the UPIR region runtime (``libupir.so``, C ABI in include/upir.h).

Argument marshalling only: every function here calls the C function of the same
name and turns a negative status into ``UpirError``.  All computation runs in the
library's CUDA kernels.  The library must be built (``python
paper_2209_10643_b300/build.py``); importing this package without it raises
ImportError — there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libupir.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2209_10643_b300/build.py`")
lib = C.CDLL(LIB_PATH)

# ----------------------------------------------------------------- constants --
UPIR_OK, UPIR_EINVAL, UPIR_ENOTMAPPED, UPIR_EBUSY, UPIR_ENOMEM, UPIR_ECUDA, \
    UPIR_ETIMEDOUT, UPIR_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6, -7
UPIR_MAP_TO, UPIR_MAP_FROM, UPIR_MAP_TOFROM, UPIR_MAP_ALLOC = 0, 1, 2, 3
(UPIR_SCHED_STATIC, UPIR_SCHED_DYNAMIC, UPIR_SCHED_GUIDED, UPIR_SCHED_RUNTIME, UPIR_SCHED_AUTO,
 UPIR_SCHED_TASKLOOP) = range(6)
UPIR_RED_NONE, UPIR_RED_ADD, UPIR_RED_MUL, UPIR_RED_MAX, UPIR_RED_MIN = 0, 1, 2, 3, 4
UPIR_F32, UPIR_I64 = 0, 1
(UPIR_BODY_AXPY, UPIR_BODY_IMOD, UPIR_BODY_JACOBI5, UPIR_BODY_MATVEC, UPIR_BODY_GEMM_F32,
 UPIR_BODY_GEMM_BF16, UPIR_BODY_GEMM_BF16X3, UPIR_BODY_COVERAGE, UPIR_BODY_SPLIT_BF16,
 UPIR_BODY_JACOBI5_TB, UPIR_BODY_FILTER7) = range(11)
UPIR_TERM_Y, UPIR_TERM_XY, UPIR_TERM_IMOD, UPIR_TERM_IV, UPIR_TERM_RESID = range(5)
(UPIR_HINT_VARIANT, UPIR_HINT_TILE_M, UPIR_HINT_TILE_N, UPIR_HINT_VEC, UPIR_HINT_STAGES, UPIR_HINT_GRAINSIZE,
 UPIR_HINT_NUM_TASKS, UPIR_HINT_TILE_ORDER) = range(1, 9)
UPIR_SYNC_BARRIER, UPIR_SYNC_TASKWAIT = 0, 1
UPIR_SUBMIT_GRAPH = 1
UPIR_BATCH_LAUNCHES, UPIR_BATCH_GRAPH, UPIR_BATCH_PERSISTENT = 0, 1, 2
UPIR_MLP_IN, UPIR_MLP_HIDDEN, UPIR_MLP_NPARAM = 12, 64, 64 * 12 + 64 + 64 * 64 + 64 + 64 + 1


class UpirError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)}")
        self.status = status


# ---------------------------------------------------------------- structures --
class upir_allocator(C.Structure):
    _fields_ = [("alloc", C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)),
                ("user", C.c_void_p)]


class upir_reduction(C.Structure):
    _fields_ = [("op", C.c_int32), ("dtype", C.c_int32), ("term", C.c_int32),
                ("reserved", C.c_int32), ("var", C.c_void_p), ("index", C.c_int64)]


class upir_loop_desc(C.Structure):
    _fields_ = [("lb", C.c_int64), ("ub", C.c_int64), ("step", C.c_int64),
                ("collapse", C.c_int32), ("sched", C.c_int32), ("chunk", C.c_int64),
                ("body", C.c_int32), ("nbufs", C.c_int32), ("bufs", C.POINTER(C.c_void_p)),
                ("nscalars", C.c_int32), ("nreductions", C.c_int32),
                ("scalars", C.POINTER(C.c_double)), ("reductions", C.POINTER(upir_reduction)),
                ("nowait", C.c_int32), ("nhints", C.c_int32), ("hints", C.POINTER(C.c_int64))]


_vp, _i32, _i64, _sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
_P = C.POINTER
_SIGS = {
    "upir_status_string": (C.c_char_p, [_i32]),
    "upir_last_error": (C.c_char_p, [_vp]),
    "upir_init": (_i32, [_P(_vp), _i32, _vp, _P(upir_allocator)]),
    "upir_finalize": (_i32, [_vp]),
    "upir_data_map": (_i32, [_vp, _vp, _sz, _i32, _P(_vp)]),
    "upir_data_map_device": (_i32, [_vp, _vp, _sz, _P(_vp)]),
    "upir_data_update": (_i32, [_vp, _vp, _i32]),
    "upir_data_unmap": (_i32, [_vp, _vp]),
    "upir_buf_device_ptr": (_i32, [_vp, _P(_vp), _P(_sz)]),
    "upir_spmd_region": (_i32, [_vp, _i32, _i32, _P(_vp)]),
    "upir_loop": (_i32, [_vp, _P(upir_loop_desc)]),
    "upir_sync": (_i32, [_vp, _i32]),
    "upir_region_submit": (_i32, [_vp, _i32]),
    "upir_region_destroy": (_i32, [_vp]),
    "upir_batch_create": (_i32, [_vp, _P(_vp), _i32, _i32, _P(_vp)]),
    "upir_batch_submit": (_i32, [_vp]),
    "upir_batch_destroy": (_i32, [_vp]),
    "upir_batch_autotune": (_i32, [_vp, _i32, _P(_i64)]),
    "upir_ctx_wait": (_i32, [_vp]),
    "upir_ctx_set_timing": (_i32, [_vp, _i32]),
    "upir_ctx_timings": (_i32, [_vp, _P(C.c_float), _P(_i32), _i32, _P(_i32)]),
    "upir_region_loop_geometry": (_i32, [_vp, _i32, _P(_i32), _P(_i32)]),
    "upir_region_loop_schedule": (_i32, [_vp, _i32, _P(_i32), _P(_i64), _P(_i64)]),
    "upir_data_map_async": (_i32, [_vp, _vp, _sz, _i32, _P(_vp)]),
    "upir_data_update_async": (_i32, [_vp, _vp, _i32]),
    "upir_buf_wait": (_i32, [_vp, _vp]),
    "upir_buf_copy": (_i32, [_vp, _vp, _vp]),
    "upir_ctx_arrive": (_i32, [_vp, _P(_vp)]),
    "upir_event_query": (_i32, [_vp]),
    "upir_event_wait": (_i32, [_vp]),
    "upir_ctx_wait_event": (_i32, [_vp, _vp]),
    "upir_event_destroy": (_i32, [_vp]),
    "upir_ctx_set_run_schedule": (_i32, [_vp, _i32, _i64]),
    "upir_ctx_set_cost_model": (_i32, [_vp, _vp, _vp, _vp]),
    "upir_auto_candidates": (_i32, [_i32, _P(_i32), _P(_i64), _P(_i32), _i32, _P(_i32)]),
    "upir_auto_features": (_i32, [_i32, _i64, _i64, _i32, _i64, _i32, _i32, _P(C.c_float)]),
    "upir_auto_pick": (_i32, [_vp, _vp, _vp, _i32, _i64, _i64, _i32, _i32, _P(_i32), _P(_i64), _P(_i32)]),
    "upir_selftest_bounded_wait": (_i32, [_vp, _i64]),
    "upir_ctx_set_spin_limit": (_i32, [_vp, _i64]),
    "upir_axpy_reduce_noalloc": (_i32, [_vp, _vp, _i64, C.c_float, _i64, _i64, _vp, _vp, _vp]),
    "upir_mlp_forward": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "upir_mlp_backward": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, _vp]),
    "upir_mlp_sgd": (_i32, [_vp, _vp, _vp, C.c_float]),
}
EXPORTED = tuple(_SIGS)
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


def status_string(s: int) -> str:
    return lib.upir_status_string(s).decode()


def _chk(ctx, st: int, what: str) -> None:
    if st != UPIR_OK:
        detail = lib.upir_last_error(ctx).decode() if ctx else ""
        raise UpirError(st, f"{what} ({detail})" if detail else what)


# ------------------------------------------------------------------ wrappers --

def upir_init(device: int = 0, stream: int | None = None) -> int:
    h = C.c_void_p()
    st = lib.upir_init(C.byref(h), device, stream, None)
    _chk(None, st, "upir_init")
    return h.value


def upir_finalize(ctx: int) -> None:
    lib.upir_finalize(ctx)


def upir_data_map(ctx: int, host_ptr: int, nbytes: int, kind: int) -> int:
    h = C.c_void_p()
    _chk(ctx, lib.upir_data_map(ctx, host_ptr, nbytes, kind, C.byref(h)), "upir_data_map")
    return h.value


def upir_data_map_device(ctx: int, dev_ptr: int, nbytes: int) -> int:
    h = C.c_void_p()
    _chk(ctx, lib.upir_data_map_device(ctx, dev_ptr, nbytes, C.byref(h)), "upir_data_map_device")
    return h.value


def upir_data_update(ctx: int, buf: int, direction: int) -> None:
    _chk(ctx, lib.upir_data_update(ctx, buf, direction), "upir_data_update")


def upir_data_unmap(ctx: int, buf: int) -> None:
    _chk(ctx, lib.upir_data_unmap(ctx, buf), "upir_data_unmap")


def upir_buf_device_ptr(buf: int) -> tuple[int, int]:
    p, n = C.c_void_p(), C.c_size_t()
    _chk(None, lib.upir_buf_device_ptr(buf, C.byref(p), C.byref(n)), "upir_buf_device_ptr")
    return p.value or 0, n.value


def upir_spmd_region(ctx: int, num_teams: int = 0, num_units: int = 0) -> int:
    h = C.c_void_p()
    _chk(ctx, lib.upir_spmd_region(ctx, num_teams, num_units, C.byref(h)), "upir_spmd_region")
    return h.value


def make_loop_desc(lb: int, ub: int, step: int = 1, *, body: int, bufs=(), scalars=(),
                   reductions=(), sched: int = UPIR_SCHED_STATIC, chunk: int = 0,
                   collapse: int = 1, nowait: int = 0, hints=()):
    """Build a ``upir_loop_desc``; the returned tuple keeps its arrays alive.

    ``reductions`` is a sequence of (op, dtype, term, var_buf, index)."""
    nb, ns, nr = len(bufs), len(scalars), len(reductions)
    b_arr = (C.c_void_p * max(nb, 1))(*bufs)
    s_arr = (C.c_double * max(ns, 1))(*scalars)
    r_arr = (upir_reduction * max(nr, 1))(*[upir_reduction(op, dt, term, 0, var, idx)
                                            for (op, dt, term, var, idx) in reductions])
    flat = [v for kv in hints for v in kv]
    h_arr = (C.c_int64 * max(len(flat), 1))(*flat)
    # ctypes stores an array assigned to a pointer field as the address of
    # its first element (no cast objects: this runs once per recorded loop)
    d = upir_loop_desc(lb, ub, step, collapse, sched, chunk, body, nb, b_arr, ns, nr, s_arr, r_arr,
                       nowait, len(hints), h_arr)
    return d, (b_arr, s_arr, r_arr, h_arr)


def upir_loop(region: int, desc) -> None:
    d = desc[0] if isinstance(desc, tuple) else desc
    st = lib.upir_loop(region, C.byref(d))
    if st != UPIR_OK:
        raise UpirError(st, "upir_loop")


def upir_loop_checked(ctx: int, region: int, desc) -> None:
    d = desc[0] if isinstance(desc, tuple) else desc
    _chk(ctx, lib.upir_loop(region, C.byref(d)), "upir_loop")


def upir_sync(region: int, kind: int) -> None:
    st = lib.upir_sync(region, kind)
    if st != UPIR_OK:
        raise UpirError(st, "upir_sync")


def upir_region_submit(region: int, flags: int = 0) -> None:
    st = lib.upir_region_submit(region, flags)
    if st != UPIR_OK:
        raise UpirError(st, "upir_region_submit")


def upir_region_destroy(region: int) -> None:
    st = lib.upir_region_destroy(region)
    if st != UPIR_OK:
        raise UpirError(st, "upir_region_destroy")


def upir_batch_create(ctx: int, regions, mode: int) -> int:
    arr = (C.c_void_p * max(len(regions), 1))(*regions)
    h = C.c_void_p()
    _chk(ctx, lib.upir_batch_create(ctx, arr, len(regions), mode, C.byref(h)), "upir_batch_create")
    return h.value


def upir_batch_submit(batch: int) -> None:
    st = lib.upir_batch_submit(batch)
    if st != UPIR_OK:
        raise UpirError(st, "upir_batch_submit")


def upir_batch_destroy(batch: int) -> None:
    lib.upir_batch_destroy(batch)


def upir_batch_autotune(batch: int, reps: int = 3) -> tuple[int, int, int]:
    out = (C.c_int64 * 3)()
    st = lib.upir_batch_autotune(batch, reps, out)
    if st != UPIR_OK:
        raise UpirError(st, "upir_batch_autotune")
    return out[0], out[1], out[2]


def upir_ctx_wait(ctx: int) -> None:
    _chk(ctx, lib.upir_ctx_wait(ctx), "upir_ctx_wait")


def upir_ctx_set_timing(ctx: int, enable: bool) -> None:
    _chk(ctx, lib.upir_ctx_set_timing(ctx, int(enable)), "upir_ctx_set_timing")


def upir_ctx_timings(ctx: int, cap: int = 65536) -> list[tuple[int, float]]:
    ms = (C.c_float * cap)()
    body = (C.c_int32 * cap)()
    n = C.c_int32()
    _chk(ctx, lib.upir_ctx_timings(ctx, ms, body, cap, C.byref(n)), "upir_ctx_timings")
    return [(body[i], ms[i]) for i in range(n.value)]


def upir_region_loop_geometry(region: int, index: int) -> tuple[int, int]:
    t, u = C.c_int32(), C.c_int32()
    st = lib.upir_region_loop_geometry(region, index, C.byref(t), C.byref(u))
    if st != UPIR_OK:
        raise UpirError(st, "upir_region_loop_geometry")
    return t.value, u.value


def upir_data_map_async(ctx: int, host_ptr: int, nbytes: int, kind: int) -> int:
    h = C.c_void_p()
    _chk(ctx, lib.upir_data_map_async(ctx, host_ptr, nbytes, kind, C.byref(h)), "upir_data_map_async")
    return h.value


def upir_data_update_async(ctx: int, buf: int, direction: int) -> None:
    _chk(ctx, lib.upir_data_update_async(ctx, buf, direction), "upir_data_update_async")


def upir_buf_wait(ctx: int, buf: int) -> None:
    _chk(ctx, lib.upir_buf_wait(ctx, buf), "upir_buf_wait")


def upir_buf_copy(ctx: int, dst: int, src: int) -> None:
    """Device-side copy of ``src`` into the first bytes of ``dst`` (ordered
    on the context's compute stream)."""
    _chk(ctx, lib.upir_buf_copy(ctx, dst, src), "upir_buf_copy")


def upir_ctx_arrive(ctx: int) -> int:
    h = C.c_void_p()
    _chk(ctx, lib.upir_ctx_arrive(ctx, C.byref(h)), "upir_ctx_arrive")
    return h.value


def upir_event_query(ev: int) -> bool:
    """True when the event's work has completed."""
    st = lib.upir_event_query(ev)
    if st not in (UPIR_OK, UPIR_EBUSY):
        raise UpirError(st, "upir_event_query")
    return st == UPIR_OK


def upir_event_wait(ev: int) -> None:
    st = lib.upir_event_wait(ev)
    if st != UPIR_OK:
        raise UpirError(st, "upir_event_wait")


def upir_ctx_wait_event(ctx: int, ev: int) -> None:
    _chk(ctx, lib.upir_ctx_wait_event(ctx, ev), "upir_ctx_wait_event")


def upir_event_destroy(ev: int) -> None:
    st = lib.upir_event_destroy(ev)
    if st != UPIR_OK:
        raise UpirError(st, "upir_event_destroy")


def upir_region_loop_schedule(region: int, index: int) -> tuple[int, int, int]:
    """(sched, chunk, nchunks) the planner settled on for a loop."""
    sc, ch, n = C.c_int32(), C.c_int64(), C.c_int64()
    st = lib.upir_region_loop_schedule(region, index, C.byref(sc), C.byref(ch), C.byref(n))
    if st != UPIR_OK:
        raise UpirError(st, "upir_region_loop_schedule")
    return sc.value, ch.value, n.value


def upir_ctx_set_run_schedule(ctx: int, sched: int, chunk: int = 0) -> None:
    _chk(ctx, lib.upir_ctx_set_run_schedule(ctx, sched, chunk), "upir_ctx_set_run_schedule")


def _f32(a):
    import numpy as np
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32).ravel())


def upir_ctx_set_cost_model(ctx: int, params, feat_mean=None, feat_std=None) -> None:
    """Install (or with params None remove) the cost model of schedule(auto)."""
    if params is None:
        _chk(ctx, lib.upir_ctx_set_cost_model(ctx, None, None, None), "upir_ctx_set_cost_model")
        return
    p, m, sd = _f32(params), _f32(feat_mean), _f32(feat_std)
    if p.size != UPIR_MLP_NPARAM or m.size != UPIR_MLP_IN or sd.size != UPIR_MLP_IN:
        raise ValueError("cost model needs UPIR_MLP_NPARAM parameters and 12 means / deviations")
    _chk(ctx, lib.upir_ctx_set_cost_model(ctx, p.ctypes.data, m.ctypes.data, sd.ctypes.data),
         "upir_ctx_set_cost_model")


def upir_auto_candidates(body: int) -> list[tuple[int, int, int]]:
    n = C.c_int32()
    _chk(None, lib.upir_auto_candidates(body, None, None, None, 0, C.byref(n)), "upir_auto_candidates")
    sc, ch, un = (C.c_int32 * n.value)(), (C.c_int64 * n.value)(), (C.c_int32 * n.value)()
    _chk(None, lib.upir_auto_candidates(body, sc, ch, un, n.value, C.byref(n)), "upir_auto_candidates")
    return [(sc[i], ch[i], un[i]) for i in range(n.value)]


def upir_auto_features(body: int, trip: int, cols: int, sched: int, chunk: int, units: int, teams: int):
    out = (C.c_float * UPIR_MLP_IN)()
    _chk(None, lib.upir_auto_features(body, trip, cols, sched, chunk, units, teams, out), "upir_auto_features")
    return list(out)


def upir_auto_pick(params, feat_mean, feat_std, body: int, trip: int, cols: int = 0, units: int = 0,
                   teams: int = 0) -> tuple[int, int, int]:
    """(sched, chunk, units) the model picks (host computation, no GPU)."""
    sc, ch, un = C.c_int32(), C.c_int64(), C.c_int32()
    if params is None:
        args = (None, None, None)
    else:
        p, m, sd = _f32(params), _f32(feat_mean), _f32(feat_std)
        args = (p.ctypes.data, m.ctypes.data, sd.ctypes.data)
    _chk(None, lib.upir_auto_pick(*args, body, trip, cols, units, teams, C.byref(sc), C.byref(ch), C.byref(un)),
         "upir_auto_pick")
    return sc.value, ch.value, un.value


def upir_selftest_bounded_wait(ctx: int, spin_limit: int) -> None:
    _chk(ctx, lib.upir_selftest_bounded_wait(ctx, spin_limit), "upir_selftest_bounded_wait")


def upir_ctx_set_spin_limit(ctx: int, spin_limit: int) -> None:
    _chk(ctx, lib.upir_ctx_set_spin_limit(ctx, spin_limit), "upir_ctx_set_spin_limit")


def upir_axpy_reduce_noalloc(x: int, y: int, n: int, a: float, imod_mul: int, imod_mod: int,
                             sum_y: int, imod_sum: int, stream: int | None = None) -> None:
    st = lib.upir_axpy_reduce_noalloc(x, y, n, a, imod_mul, imod_mod, sum_y, imod_sum, stream)
    if st != UPIR_OK:
        raise UpirError(st, "upir_axpy_reduce_noalloc")


def upir_mlp_forward(ctx: int, params: int, x: int, batch: int, pred: int) -> None:
    _chk(ctx, lib.upir_mlp_forward(ctx, params, x, batch, pred), "upir_mlp_forward")


def upir_mlp_backward(ctx: int, params: int, x: int, target: int, batch: int, grad: int,
                      loss: int | None) -> None:
    _chk(ctx, lib.upir_mlp_backward(ctx, params, x, target, batch, grad, loss),
         "upir_mlp_backward")


def upir_mlp_sgd(ctx: int, params: int, grad: int, lr: float) -> None:
    _chk(ctx, lib.upir_mlp_sgd(ctx, params, grad, lr), "upir_mlp_sgd")
