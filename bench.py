"""Benchmark of the UPIR region runtime on B300.

Headline workload: the 2D Jacobi 5-point region, a 4096 x 4096 FP32 grid
(top edge 1, other edges 0, interior uniform[0,1) from seed 1), 100 sweeps, a
per-sweep reduction(max) of |u_new - u| into its own variable, ping-pong
buffers mapped once.  One step = one submission of that 100-loop region.
Metric: parallel-loop HBM GB/s (algorithmic bytes: 8 B per interior point per
sweep) against the measured HBM copy peak.  The other loop regions (AXPY with
reductions, matvec, GEMM, batched regions) are measured after the headline
and reported under "extra".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own independent problem (weak scaling, no
data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

# The oracle is sequential by design and is timed on one host core: hold the
# host BLAS to one thread before numpy loads it (this process uses numpy only
# for input generation and the oracle).
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import upir_inputs as I  # noqa: E402

# Nothing from the package is imported at module level: importing it loads
# libupir.so, and the reference arm (the host oracle) must run without it.

N_GRID = 4096
SWEEPS = 100
JACOBI_BYTES_PER_SWEEP = 8 * (N_GRID - 2) ** 2
# the headline metric and the workload it is measured on (both arms)
METRIC = "Parallel-loop HBM GB/s vs peak; batched regions/s fused vs per-region launch"
WORKLOAD = f"jacobi5_{N_GRID}x{N_GRID}_{SWEEPS}sweeps_maxresidual"


def headline_config(world: int) -> dict:
    """The headline workload's description, printed unchanged by both arms."""
    return {"workload": WORKLOAD, "grid": [N_GRID, N_GRID], "sweeps": SWEEPS, "schedule": "static",
            "parallelism": f"independent problem per rank x{world}",
            "l2": "flushed before each step (256 MiB write, then 256 MiB read); working set 134 MB > 126 MB L2",
            "submission": "CUDA graph of the 100 sweep launches (programmatic dependent launch)"}


# DRAM bytes (read + write) of one launch of the sweep kernel on this grid, from
# an ncu capture of the current kernel in the middle of the 100-sweep graph
# (caches not flushed between launches, so each sweep finds what the previous
# one left in L2): mean of five consecutive launches, 6.9 MB read and 65.1 MB
# written (the sweep's output reaches DRAM once; its input comes from L2)
JACOBI_TRAFFIC_BYTES = 6_911_897 + 65_144_064
L2_FLUSH_BYTES = 256 << 20
L2_BYTES = 126 << 20  # the GPU's L2


def dist_env() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (1 process: 0, 0, 1)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def one_thread():
    """Context manager holding the host BLAS to one thread where threadpoolctl
    is available (the environment variables set above already do so when
    numpy is first loaded by this process)."""
    try:
        from threadpoolctl import threadpool_limits
        return threadpool_limits(limits=1)
    except ImportError:
        import contextlib
        return contextlib.nullcontext()


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "source": "measured"}
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (getattr(self, "out", "") or "").splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------- ours --

class Runtime:
    def __init__(self, device: int):
        import torch
        import paper_2209_10643_b300 as U
        self.U, self.torch = U, torch
        torch.cuda.set_device(device)
        # a dedicated stream, made torch's current one, so that torch events and
        # the library's launches share it (the legacy default stream has handle 0)
        self.stream = torch.cuda.Stream(device=device)
        torch.cuda.set_stream(self.stream)
        self.ctx = U.upir_init(device, self.stream.cuda_stream)
        self.flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        self.flush_rd = torch.zeros(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        self.host = []
        self.handles = []

    def map(self, arr, kind, track=False):
        self.host.append(arr)
        h = self.U.upir_data_map(self.ctx, arr.ctypes.data, arr.nbytes, kind)
        if track:
            self.handles.append(h)
        return h

    def flush_l2(self):
        # Write a buffer larger than L2, then read another one: the read
        # evicts the written lines (their write-back happens inside it), so
        # the timed work starts with an L2 that holds neither its inputs nor
        # dirty lines whose write-back it would pay for.  Stream-ordered and
        # not waited for: the GPU is still busy with the flush while the host
        # enqueues the timed work, so the timed region starts with the GPU's
        # own start of that work, not with the host's launch latency.
        self.flush_buf.fill_(1.0)
        self.flush_rd.sum()

    def region(self, loops, teams=0, units=0):
        r = self.U.upir_spmd_region(self.ctx, teams, units)
        for lp in loops:
            self.U.upir_loop_checked(self.ctx, r, self.U.make_loop_desc(**lp))
        return r

    def timed_submits(self, submit, reps, warmup=3, flush=True):
        """Mean per-rep device time (ms) of ``submit()``, measured with the
        library's per-launch CUDA events; also the per-rep times and the
        per-launch records.  The mean, not the median: event pairs around a
        launch that follows other work read in steps of 2.048 us on this GPU,
        and with the start's phase against those steps varying from rep to
        rep only the mean converges on the duration."""
        U = self.U
        for _ in range(warmup):
            submit()
        U.upir_ctx_wait(self.ctx)
        U.upir_ctx_timings(self.ctx)
        per_rep = []
        launches = []
        for _ in range(reps):
            if flush:
                self.flush_l2()
            U.upir_ctx_set_timing(self.ctx, True)
            submit()
            U.upir_ctx_set_timing(self.ctx, False)
            rec = U.upir_ctx_timings(self.ctx)
            per_rep.append(sum(ms for _, ms in rec))
            launches.extend(rec)
        return statistics.fmean(per_rep), per_rep, launches


def timed_whole(rt: Runtime, submit, reps: int, warmup: int = 3) -> tuple[float, list]:
    """Mean device time (ms) of ``submit()`` with ONE event pair around the
    whole submission (every launch it makes, and the gaps between them), on
    the context stream, with the L2 flushed before each repetition."""
    torch = rt.torch
    for _ in range(warmup):
        submit()
    rt.U.upir_ctx_wait(rt.ctx)
    times = []
    for _ in range(reps):
        rt.flush_l2()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        submit()
        ev1.record()
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
    return statistics.fmean(times), times


def jacobi_region_loops(U, ha, hb, hr):
    loops = []
    for k in range(SWEEPS):
        src, dst = (ha, hb) if k % 2 == 0 else (hb, ha)
        loops.append(dict(lb=1, ub=N_GRID - 1, step=1, collapse=2, body=U.UPIR_BODY_JACOBI5,
                          bufs=[src, dst], scalars=[N_GRID, N_GRID],
                          reductions=[(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_RESID, hr, k)]))
    return loops


def headline(rt: Runtime, steps: int, warmup: int, pk: dict, device: int):
    U, torch = rt.U, rt.torch
    u0 = I.jacobi_grid(N_GRID, seed=1)
    a, b = u0.copy(), u0.copy()
    res = np.full(SWEEPS, -np.inf, np.float32)
    ha, hb = rt.map(a, U.UPIR_MAP_TOFROM), rt.map(b, U.UPIR_MAP_TOFROM)
    hr = rt.map(res, U.UPIR_MAP_TOFROM)
    r = rt.region(jacobi_region_loops(U, ha, hb, hr))
    for _ in range(warmup):
        U.upir_region_submit(r, 0)
    U.upir_ctx_wait(rt.ctx)
    U.upir_ctx_timings(rt.ctx)

    import torch.distributed as dist
    if dist.is_initialized():
        dist.barrier()
    torch.cuda.synchronize()
    # timed region: graph submissions of the region (the runtime's fast path);
    # one CUDA graph holds the 100 sweep launches, so the average launch
    # duration of the sweep kernel is the step time / 100
    U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH)  # instantiate the graph outside the timed region
    torch.cuda.synchronize()
    step_ms = []
    with ClockSampler(device) as clk:
        for _ in range(steps):
            rt.flush_l2()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record()
            U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH)
            ev1.record()
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
        torch.cuda.synchronize()
    if dist.is_initialized():
        dist.barrier()
    total_s = sum(step_ms) / 1e3
    from paper_2209_10643_b300.sharding import aggregate_throughput
    units, secs = aggregate_throughput(steps * SWEEPS * JACOBI_BYTES_PER_SWEEP, total_s)
    value = units / secs / 1e9
    avg_kernel_s = statistics.mean(step_ms) / 1e3 / SWEEPS
    achieved = JACOBI_BYTES_PER_SWEEP / avg_kernel_s / 1e9

    # the same region launch by launch, each launch bracketed by its own events
    lms, _, launches = rt.timed_submits(lambda: U.upir_region_submit(r, 0), min(steps, 20), warmup)
    per_launch_us = statistics.mean(ms for _, ms in launches) * 1e3
    U.upir_region_destroy(r)
    for h in (ha, hb, hr):
        U.upir_data_unmap(rt.ctx, h)

    # end to end through the public API with host buffers (pinned)
    e2e = jacobi_e2e(rt, u0, max(3, min(steps, 32)))
    return {
        "value": value, "ms_per_step": statistics.mean(step_ms), "clocks": clk.summary(),
        "gpu_launches": steps * SWEEPS,
        "roofline": {"bound": "hbm", "kernel": "jacobi_tma_kernel", "achieved": achieved,
                     "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                     "peak_source": pk["source"] + " (burst copy)",
                     "algorithmic_bytes_per_launch": JACOBI_BYTES_PER_SWEEP,
                     "avg_launch_us": avg_kernel_s * 1e6, "traffic": JACOBI_TRAFFIC_BYTES,
                     # the same launch counted in DRAM bytes
                     "traffic_frac": (JACOBI_TRAFFIC_BYTES / avg_kernel_s / 1e9 / pk["hbm_gbs"]
                                      if JACOBI_TRAFFIC_BYTES else None),
                     "note": "achieved counts the algorithmic 8 B per point per sweep; a sweep reads "
                             "its input from L2, where the previous sweep (walking its tiles the other "
                             "way, its output stored with normal priority and its input read "
                             "evict-first) left it, so frac can pass 1; traffic is the DRAM bytes of "
                             "one launch in the sequence and traffic_frac that launch's DRAM rate"},
        "per_launch": {"ms_per_step": lms, "avg_launch_us_with_events": per_launch_us,
                       "value": SWEEPS * JACOBI_BYTES_PER_SWEEP / (lms / 1e3) / 1e9},
        "e2e": e2e, "residual_last": float(res[-1]),
    }


def jacobi_e2e(rt: Runtime, u0: np.ndarray, steps: int) -> dict:
    """The headline step end to end through the C ABI with host buffers
    (pinned): every step maps its grid and the residual variables to the
    device, seeds the second grid from the first with a device-side copy
    (both carry the boundary), runs the 100 sweeps and reads the field and
    the residuals back.  Two forms: one step after another (map, record,
    submit and unmap per step, synchronous copies), and a stream of steps
    whose buffers are mapped and regions recorded beforehand, with
    asynchronous copies per step: the host->device copies of step i + 1 and
    the device->host copies of step i - 1 (one copy stream per direction)
    overlap the sweeps of step i.  Both include every step's copies in the
    timed region; the stream is the reported value."""
    U, torch = rt.U, rt.torch
    nb = u0.nbytes

    def pinned(shape):
        return torch.empty(shape, dtype=torch.float32, pin_memory=True).numpy()

    sets = [(pinned(u0.shape), pinned(SWEEPS)) for _ in range(steps)]

    def refill():
        for pa, pr in sets:
            pa[...] = u0
            pr[...] = -np.inf

    def sequential(pa, pr):
        ha = U.upir_data_map(rt.ctx, pa.ctypes.data, nb, U.UPIR_MAP_TOFROM)
        hb = U.upir_data_map(rt.ctx, 0, nb, U.UPIR_MAP_ALLOC)
        U.upir_buf_copy(rt.ctx, hb, ha)
        # the residual variables start at -inf, so they are mapped tofrom
        hr = U.upir_data_map(rt.ctx, pr.ctypes.data, pr.nbytes, U.UPIR_MAP_TOFROM)
        r = rt.region(jacobi_region_loops(U, ha, hb, hr))
        U.upir_region_submit(r, 0)
        U.upir_region_destroy(r)
        U.upir_data_unmap(rt.ctx, hb)
        U.upir_data_unmap(rt.ctx, hr)
        U.upir_data_unmap(rt.ctx, ha)

    # the stream: each step's device buffers are mapped (bound to its pinned
    # host arrays, no copy) and its region recorded before the timed region;
    # a timed step uploads its grid and residual start values, seeds the
    # second grid on the device, runs the 100 sweeps as one graph and reads
    # the field and residuals back.  A copy waits only for the work that
    # uses its buffer, so the uploads of step i + 1 and the downloads of
    # step i - 1 overlap the sweeps of step i.
    slots = []
    for pa, pr in sets:
        ha = U.upir_data_map(rt.ctx, pa.ctypes.data, nb, U.UPIR_MAP_ALLOC)
        hb = U.upir_data_map(rt.ctx, 0, nb, U.UPIR_MAP_ALLOC)
        hr = U.upir_data_map(rt.ctx, pr.ctypes.data, pr.nbytes, U.UPIR_MAP_ALLOC)
        slots.append((ha, hb, hr, rt.region(jacobi_region_loops(U, ha, hb, hr))))

    def stream():
        for ha, hb, hr, r in slots:
            U.upir_data_update_async(rt.ctx, ha, U.UPIR_MAP_TO)
            U.upir_data_update_async(rt.ctx, hr, U.UPIR_MAP_TO)
            U.upir_buf_copy(rt.ctx, hb, ha)
            U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH)
            U.upir_data_update_async(rt.ctx, ha, U.UPIR_MAP_FROM)
            U.upir_data_update_async(rt.ctx, hr, U.UPIR_MAP_FROM)
        for ha, hb, hr, r in slots:
            U.upir_buf_wait(rt.ctx, ha)
            U.upir_buf_wait(rt.ctx, hr)
        U.upir_ctx_wait(rt.ctx)

    # one after another: the first step warms up, the median of the rest
    seq_times = []
    for i in range(min(steps, 5) + 1):
        pa, pr = sets[0]
        pa[...] = u0
        pr[...] = -np.inf
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sequential(pa, pr)
        t1 = time.perf_counter()
        if i:
            seq_times.append(t1 - t0)
    want_u, want_r = sets[0][0].copy(), sets[0][1].copy()
    t_seq = statistics.median(seq_times)

    refill()
    stream()  # warm-up: graph instantiation
    refill()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    stream()
    t_stream = (time.perf_counter() - t0) / steps
    same = all(np.array_equal(pa, want_u) and np.array_equal(pr, want_r) for pa, pr in sets)
    for ha, hb, hr, r in slots:
        U.upir_region_destroy(r)
        for h in (ha, hb, hr):
            U.upir_data_unmap(rt.ctx, h)
    if not same:
        raise RuntimeError("streamed end-to-end steps disagree with the sequential step")
    return {"value": SWEEPS * JACOBI_BYTES_PER_SWEEP / t_stream / 1e9, "unit": "GB/s",
            "h2d_bytes_per_step": nb + SWEEPS * 4, "d2h_bytes_per_step": nb + SWEEPS * 4,
            "ms_per_step": t_stream * 1e3,
            "mode": f"stream of {steps} steps, buffers mapped and regions recorded once, asynchronous "
                    "copies per step (they overlap the sweeps of the neighbouring steps); each step's "
                    "results checked against the sequential step",
            "sequential": {"value": SWEEPS * JACOBI_BYTES_PER_SWEEP / t_seq / 1e9, "ms_per_step": t_seq * 1e3}}


def extra_axpy(rt: Runtime, n: int, pk: dict) -> dict:
    U = rt.U
    x, y = I.axpy_inputs(n, seed=0)
    fs = np.zeros(1, np.float32)
    si = np.zeros(1, np.int64)
    hx, hy = rt.map(x, U.UPIR_MAP_TO), rt.map(y, U.UPIR_MAP_TOFROM)
    hf, hi = rt.map(fs, U.UPIR_MAP_TOFROM), rt.map(si, U.UPIR_MAP_TOFROM)
    r = rt.region([dict(lb=0, ub=n, body=U.UPIR_BODY_AXPY, bufs=[hx, hy], scalars=[2.5, 3, 1000],
                        reductions=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_Y, hf, 0),
                                    (U.UPIR_RED_ADD, U.UPIR_I64, U.UPIR_TERM_IMOD, hi, 0)])])
    ms, _, _ = rt.timed_submits(lambda: U.upir_region_submit(r, 0), 60)
    gms, _, _ = rt.timed_submits(lambda: U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH), 60)
    U.upir_region_destroy(r)
    out = {"n": n, "us": ms * 1e3, "GB/s": 12 * n / (ms / 1e3) / 1e9, "graph_us": gms * 1e3, "bytes": 12 * n}
    out["single_launch_GB/s"] = out["GB/s"]
    if 8 * n > 2 * L2_BYTES:
        # x and y outgrow the L2: ten loops back to back in one graph, one
        # event pair around them, give the loop's device time without the
        # per-launch event overhead (each loop does its full work)
        out.update(loops_in_graph(rt, [dict(lb=0, ub=n, body=U.UPIR_BODY_AXPY, bufs=[hx, hy],
                                            scalars=[2.5, 3, 1000],
                                            reductions=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_Y, hf, 0),
                                                        (U.UPIR_RED_ADD, U.UPIR_I64, U.UPIR_TERM_IMOD, hi, 0)])],
                                  12 * n, pk))
    else:
        out["frac_hbm"] = out["GB/s"] / pk["hbm_gbs"]
        out.update(axpy_stream(rt, n, pk))
    for h in (hx, hy, hf, hi):
        U.upir_data_unmap(rt.ctx, h)
    return out


def axpy_stream(rt: Runtime, n: int, pk: dict, count: int = 20) -> dict:
    """A stream of ``count`` independent single-loop AXPY regions of the same
    size, each on its own x, y and reduction variables (together more than
    the L2 holds, so each loop reads cold data), recorded as one graph and
    timed with one event pair: the per-region time when regions follow one
    another, next to the latency of one region alone."""
    U = rt.U
    loops = []
    for k in range(count):
        x, y = I.axpy_inputs(n, seed=100 + k)
        fs, si = np.zeros(1, np.float32), np.zeros(1, np.int64)
        hx, hy = rt.map(x, U.UPIR_MAP_TO, True), rt.map(y, U.UPIR_MAP_TOFROM, True)
        hf, hi = rt.map(fs, U.UPIR_MAP_TOFROM, True), rt.map(si, U.UPIR_MAP_TOFROM, True)
        loops.append(dict(lb=0, ub=n, body=U.UPIR_BODY_AXPY, bufs=[hx, hy], scalars=[2.5, 3, 1000],
                          reductions=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_Y, hf, 0),
                                      (U.UPIR_RED_ADD, U.UPIR_I64, U.UPIR_TERM_IMOD, hi, 0)]))
    out = {}
    # with the implicit barrier after each loop, and with nowait (independent
    # loops: the next may start while this one finishes)
    for key, nowait in (("stream", 0), ("stream_nowait", 1)):
        r = rt.region([dict(lp, nowait=nowait if k < count - 1 else 0) for k, lp in enumerate(loops)])
        U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH)
        ms, _ = timed_whole(rt, lambda: U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH), 20)
        U.upir_region_destroy(r)
        per = ms / count
        gbs = 12 * n / (per / 1e3) / 1e9
        out.update({f"{key}_us_per_region": per * 1e3, f"{key}_GB/s": gbs, f"{key}_frac_hbm": gbs / pk["hbm_gbs"]})
    for h in rt.handles:
        U.upir_data_unmap(rt.ctx, h)
    rt.handles.clear()
    out.update({"stream_regions": count,
                "stream_timing": f"{count} independent single-loop regions on their own buffers "
                                 f"({count * 8 * n / 1e6:.0f} MB, more than the L2) recorded as the loops of one "
                                 "region, one CUDA graph, one event pair around it, L2 flushed first; "
                                 "stream_nowait: the loops marked nowait"})
    return out


def loops_in_graph(rt: Runtime, loop: list, bytes_per_loop: float, pk: dict, count: int = 10,
                   reps: int = 10) -> dict:
    """``count`` copies of ``loop`` in one region submitted as a CUDA graph,
    one event pair around each submission (L2 flushed before each); the
    per-loop time and rate.  For loops whose data outgrow the L2."""
    U = rt.U
    r = rt.region(loop * count)
    U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH)
    ms, _ = timed_whole(rt, lambda: U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH), reps)
    U.upir_region_destroy(r)
    per = ms / count
    gbs = bytes_per_loop / (per / 1e3) / 1e9
    return {"loops_in_graph": count, "us_per_loop_in_graph": per * 1e3, "GB/s": gbs,
            "frac_hbm": gbs / pk["hbm_gbs"],
            "timing": f"{count} loops back to back in one CUDA graph, one event pair around it, "
                      f"L2 flushed before each of {reps} repetitions (the data outgrow the L2)"}


def extra_matvec(rt: Runtime, pk: dict) -> dict:
    U = rt.U
    n = 16384
    a, x = I.matvec_inputs(n, n)
    y = np.zeros(n, np.float32)
    ha, hx, hy = rt.map(a, U.UPIR_MAP_TO), rt.map(x, U.UPIR_MAP_TO), rt.map(y, U.UPIR_MAP_TOFROM)
    loop = dict(lb=0, ub=n, body=U.UPIR_BODY_MATVEC, bufs=[ha, hx, hy], scalars=[n, n])
    r = rt.region([loop])
    ms, _, _ = rt.timed_submits(lambda: U.upir_region_submit(r, 0), 20)
    U.upir_region_destroy(r)
    byts = 4 * n * n + 8 * n
    out = {"rows": n, "cols": n, "us": ms * 1e3, "single_launch_GB/s": byts / (ms / 1e3) / 1e9}
    # A (1.07 GB) outgrows the L2: the loop's device time from a graph of ten
    out.update(loops_in_graph(rt, [loop], byts, pk))
    for h in (ha, hx, hy):
        U.upir_data_unmap(rt.ctx, h)
    rt.host.clear()
    return out


def extra_jacobi_tb(rt: Runtime, pk: dict, sweeps_per_loop: int) -> dict:
    """The headline's 100 sweeps of the 4096^2 grid carried by 100 / T
    time-blocked loops of T sweeps each (one HBM pass per T sweeps), as one
    CUDA-graph submission; the same per-sweep residuals."""
    U, torch = rt.U, rt.torch
    T = sweeps_per_loop
    u0 = I.jacobi_grid(N_GRID, seed=1)
    a, b = u0.copy(), u0.copy()
    res = np.full(SWEEPS, -np.inf, np.float32)
    ha, hb = rt.map(a, U.UPIR_MAP_TOFROM), rt.map(b, U.UPIR_MAP_TOFROM)
    hr = rt.map(res, U.UPIR_MAP_TOFROM)
    loops, done = [], 0
    groups = [T] * (SWEEPS // T) + ([SWEEPS % T] if SWEEPS % T else [])
    for g, t in enumerate(groups):
        src, dst = (ha, hb) if g % 2 == 0 else (hb, ha)
        loops.append(dict(lb=1, ub=N_GRID - 1, step=1, collapse=2, body=U.UPIR_BODY_JACOBI5_TB,
                          bufs=[src, dst], scalars=[N_GRID, N_GRID, t],
                          reductions=[(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_RESID, hr, done)]))
        done += t
    r = rt.region(loops)
    U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH)
    U.upir_ctx_wait(rt.ctx)
    times = []
    for _ in range(8):
        rt.flush_l2()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH)
        ev1.record()
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
    tm, tn = U.upir_region_loop_geometry(r, 0)
    U.upir_region_destroy(r)
    for h in (ha, hb, hr):
        U.upir_data_unmap(rt.ctx, h)
    rt.host.clear()
    ms = statistics.median(times)
    alg = SWEEPS * JACOBI_BYTES_PER_SWEEP / (ms / 1e3) / 1e9
    return {"sweeps_per_loop": T, "loops": len(groups), "teams": tm, "units": tn, "ms_per_100_sweeps": ms,
            "us_per_sweep": ms * 1e3 / SWEEPS, "algorithmic_GB/s": alg,
            "algorithmic_over_measured_hbm": alg / pk["hbm_gbs"],
            "note": "algorithmic bytes count 8 B per point per sweep; the grid crosses HBM once per loop"}


def extra_jacobi_grid(rt: Runtime, pk: dict, n: int = 4095, sweeps: int = 20) -> dict:
    """Jacobi sweeps on an n x n grid, one CUDA-graph submission of `sweeps`
    loops, L2 flushed before each repetition.  n = 4095: a width that is not
    a multiple of 4 (rows off the 16-byte grid: the row-copy TMA kernel);
    n = 8192: a 537 MB ping-pong set, four times the L2, so every sweep
    streams its grid from HBM."""
    U, torch = rt.U, rt.torch
    u0 = I.jacobi_grid(n, seed=1)
    a, b = u0.copy(), u0.copy()
    res = np.full(sweeps, -np.inf, np.float32)
    ha, hb = rt.map(a, U.UPIR_MAP_TOFROM), rt.map(b, U.UPIR_MAP_TOFROM)
    hr = rt.map(res, U.UPIR_MAP_TOFROM)
    loops = []
    for k in range(sweeps):
        src, dst = (ha, hb) if k % 2 == 0 else (hb, ha)
        loops.append(dict(lb=1, ub=n - 1, step=1, collapse=2, body=U.UPIR_BODY_JACOBI5, bufs=[src, dst],
                          scalars=[n, n], reductions=[(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_RESID, hr, k)]))
    r = rt.region(loops)
    U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH)
    U.upir_ctx_wait(rt.ctx)
    times = []
    for _ in range(8):
        rt.flush_l2()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        U.upir_region_submit(r, U.UPIR_SUBMIT_GRAPH)
        ev1.record()
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
    tm, tn = U.upir_region_loop_geometry(r, 0)
    U.upir_region_destroy(r)
    for h in (ha, hb, hr):
        U.upir_data_unmap(rt.ctx, h)
    rt.host.clear()
    ms = statistics.median(times)
    gbs = sweeps * 8 * (n - 2) ** 2 / (ms / 1e3) / 1e9
    return {"grid": [n, n], "sweeps": sweeps, "teams": tm, "units": tn, "us_per_sweep": ms * 1e3 / sweeps,
            "algorithmic_GB/s": gbs, "frac_hbm": gbs / pk["hbm_gbs"]}


def rng_weights7() -> np.ndarray:
    """The size-7 filter's weights in the bench: seeded uniform [0, 1),
    normalised to sum 1."""
    w = np.random.default_rng(15).random((7, 7)).astype(np.float32)
    return (w / w.sum()).astype(np.float32)


def extra_filter7(rt: Runtime, pk: dict) -> dict:
    """The size-7 filter (7 x 7 window, FMA chain) over a 4096^2 grid."""
    U = rt.U
    x = I.jacobi_grid(N_GRID, seed=14)
    w = rng_weights7()
    out = np.zeros_like(x)
    hx, ho = rt.map(x, U.UPIR_MAP_TO), rt.map(out, U.UPIR_MAP_TOFROM)
    r = rt.region([dict(lb=3, ub=N_GRID - 3, step=1, collapse=2, body=U.UPIR_BODY_FILTER7, bufs=[hx, ho],
                        scalars=[N_GRID, N_GRID] + [float(v) for v in w.ravel()])])
    ms, _, _ = rt.timed_submits(lambda: U.upir_region_submit(r, 0), 30)
    tm, tn = U.upir_region_loop_geometry(r, 0)
    U.upir_region_destroy(r)
    for h in (hx, ho):
        U.upir_data_unmap(rt.ctx, h)
    rt.host.clear()
    pts = (N_GRID - 6) ** 2
    gbs = 8 * pts / (ms / 1e3) / 1e9
    tf = 2 * 49 * pts / (ms / 1e3) / 1e12
    props = rt.torch.cuda.get_device_properties(0)
    fp32_peak = props.multi_processor_count * 128 * 2 * 2.032e9 / 1e12
    ref = cublas_sgemm_rate(rt)
    return {"grid": [N_GRID, N_GRID], "teams": tm, "units": tn, "us": ms * 1e3, "GB/s": gbs,
            "frac_hbm": gbs / pk["hbm_gbs"], "TFLOP/s": tf, "fp32_fma_peak_tflops": fp32_peak,
            "frac_fp32_peak": tf / fp32_peak, "cublas_sgemm_TFLOP/s": ref["TFLOP/s"],
            "frac_of_cublas_sgemm": tf / ref["TFLOP/s"]}


def extra_pipeline(rt: Runtime, count: int = 6) -> dict:
    """Regions with host data: each maps a 4096^2 grid (two buffers, from
    page-locked host memory), runs the 100 Jacobi sweeps as time-blocked
    loops and copies the field back.  Synchronous mapping serialises copies
    and computation; asynchronous mapping (a copy stream per direction, the
    device ordering them with the computation) overlaps region k + 1's
    host->device copies and region k - 1's device->host copy with region k's
    sweeps."""
    U, torch = rt.U, rt.torch
    n = N_GRID * N_GRID
    u0 = I.jacobi_grid(N_GRID, seed=1)
    hosts = []
    for _ in range(count):
        a = torch.empty(n, dtype=torch.float32, pin_memory=True)
        b = torch.empty(n, dtype=torch.float32, pin_memory=True)
        a.numpy()[...] = u0.ravel()
        b.numpy()[...] = u0.ravel()
        hosts.append((a, b))

    def loops(ha, hb):
        out = []
        for g in range(SWEEPS // 8 + (1 if SWEEPS % 8 else 0)):
            t = min(8, SWEEPS - 8 * g)
            src, dst = (ha, hb) if g % 2 == 0 else (hb, ha)
            out.append(dict(lb=1, ub=N_GRID - 1, step=1, collapse=2, body=U.UPIR_BODY_JACOBI5_TB,
                            bufs=[src, dst], scalars=[N_GRID, N_GRID, t]))
        return out

    last = (SWEEPS + 7) // 8 % 2  # which buffer holds the field at the end

    def sequential():
        for a, b in hosts:
            ha = U.upir_data_map(rt.ctx, a.data_ptr(), 4 * n, U.UPIR_MAP_TO)
            hb = U.upir_data_map(rt.ctx, b.data_ptr(), 4 * n, U.UPIR_MAP_TO)
            r = rt.region(loops(ha, hb))
            U.upir_region_submit(r, 0)
            U.upir_data_update(rt.ctx, hb if last else ha, U.UPIR_MAP_FROM)
            U.upir_region_destroy(r)
            U.upir_data_unmap(rt.ctx, ha)
            U.upir_data_unmap(rt.ctx, hb)
        U.upir_ctx_wait(rt.ctx)

    def pipelined():
        live = []
        for a, b in hosts:
            ha = U.upir_data_map_async(rt.ctx, a.data_ptr(), 4 * n, U.UPIR_MAP_TO)
            hb = U.upir_data_map_async(rt.ctx, b.data_ptr(), 4 * n, U.UPIR_MAP_TO)
            r = rt.region(loops(ha, hb))
            U.upir_region_submit(r, 0)
            U.upir_data_update_async(rt.ctx, hb if last else ha, U.UPIR_MAP_FROM)
            live.append((r, ha, hb))
        for r, ha, hb in live:
            U.upir_buf_wait(rt.ctx, hb if last else ha)
            U.upir_region_destroy(r)
            U.upir_data_unmap(rt.ctx, ha)
            U.upir_data_unmap(rt.ctx, hb)
        U.upir_ctx_wait(rt.ctx)

    res = {}
    for name, fn in (("sequential", sequential), ("pipelined", pipelined)):
        fn()  # warm-up: planning paths, allocator pools
        times = []
        for _ in range(3):
            t0 = time.perf_counter()
            fn()
            times.append(time.perf_counter() - t0)
        t = statistics.median(times)
        res[name] = {"ms_per_region": 1e3 * t / count, "regions_per_s": count / t}
    want = hosts[0][1 if last else 0].numpy()
    rt.host.clear()
    h2d = 2 * 4 * n
    return {"regions": count, "grid": [N_GRID, N_GRID], "sweeps": SWEEPS, "sweeps_per_loop": 8,
            "h2d_bytes_per_region": h2d, "d2h_bytes_per_region": 4 * n, **res,
            "speedup_pipelined": res["sequential"]["ms_per_region"] / res["pipelined"]["ms_per_region"],
            "field_checksum": float(np.sum(want, dtype=np.float64))}


def extra_gemm_f32(rt: Runtime) -> dict:
    import torch
    U = rt.U
    m = n = k = 4096
    a, b = I.gemm_inputs(m, n, k)
    c = np.zeros((m, n), np.float32)
    ha, hb, hc = rt.map(a, U.UPIR_MAP_TO), rt.map(b, U.UPIR_MAP_TO), rt.map(c, U.UPIR_MAP_TOFROM)
    r = rt.region([dict(lb=0, ub=m, collapse=2, body=U.UPIR_BODY_GEMM_F32, bufs=[ha, hb, hc],
                        scalars=[m, n, k])])
    ms, _, _ = rt.timed_submits(lambda: U.upir_region_submit(r, 0), 5)
    U.upir_region_destroy(r)
    for h in (ha, hb, hc):
        U.upir_data_unmap(rt.ctx, h)
    rt.host.clear()
    props = torch.cuda.get_device_properties(0)
    fp32_peak = props.multi_processor_count * 128 * 2 * 2.032e9 / 1e12
    tf = 2 * m * n * k / (ms / 1e3) / 1e12
    ref = cublas_sgemm_rate(rt)
    return {"shape": [m, n, k], "ms": ms, "TFLOP/s": tf, "fp32_simt_peak_tflops": fp32_peak,
            "frac_fp32_peak": tf / fp32_peak, "cublas_sgemm": ref,
            "frac_of_cublas_sgemm": tf / ref["TFLOP/s"]}


_SGEMM_RATE = {}


def cublas_sgemm_rate(rt: Runtime) -> dict:
    """A measured FP32 FMA rate to set the FP32-bound kernels against: the
    library SGEMM (cuBLAS through torch.matmul, FP32 compute with TF32 off)
    on 4096^3, timed like the kernels (L2 flushed, one event pair per call,
    mean of 10).  Computed once per process."""
    if _SGEMM_RATE:
        return _SGEMM_RATE
    torch = rt.torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        g = torch.Generator(device="cuda").manual_seed(3)
        a = torch.randn(4096, 4096, device="cuda", generator=g)
        b = torch.randn(4096, 4096, device="cuda", generator=g)
        c = torch.empty(4096, 4096, device="cuda")
        ms, _ = timed_whole(rt, lambda: torch.matmul(a, b, out=c), 10)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    _SGEMM_RATE.update({"ms": ms, "TFLOP/s": 2 * 4096 ** 3 / (ms / 1e3) / 1e12,
                        "what": "cuBLAS SGEMM via torch.matmul, FP32 compute, TF32 off, 4096^3, "
                                "L2 flushed, one event pair per call, mean of 10"})
    return _SGEMM_RATE


def extra_gemm_tc(rt: Runtime, pk: dict) -> dict:
    """C = A B, 4096^3, A and B ~ N(0, 1/K): bfloat16 tensor cores with FP32
    accumulation, and the split-bfloat16 (3 products) form.  The bfloat16
    operands are prepared once by the SPLIT_BF16 loop, timed separately."""
    U = rt.U
    m = n = k = 4096
    a, b = I.gemm_inputs(m, n, k)
    ah, al = np.zeros(m * k, np.uint16), np.zeros(m * k, np.uint16)
    bh, bl = np.zeros(n * k, np.uint16), np.zeros(n * k, np.uint16)
    c = np.zeros((m, n), np.float32)
    ha, hb = rt.map(a, U.UPIR_MAP_TO), rt.map(b, U.UPIR_MAP_TO)
    hah, hal, hbh, hbl = (rt.map(v, U.UPIR_MAP_ALLOC) for v in (ah, al, bh, bl))
    hc = rt.map(c, U.UPIR_MAP_ALLOC)
    prep = rt.region([dict(lb=0, ub=m, body=U.UPIR_BODY_SPLIT_BF16, bufs=[ha, hah, hal], scalars=[m, k, 0]),
                      dict(lb=0, ub=k, body=U.UPIR_BODY_SPLIT_BF16, bufs=[hb, hbh, hbl], scalars=[k, n, 1])])
    pms, _, _ = rt.timed_submits(lambda: U.upir_region_submit(prep, 0), 5)
    out = {"shape": [m, n, k], "split_ms": pms}
    flops = 2.0 * m * n * k
    # bf16: the planner's kernel (CTA pairs at this size); bf16_one_sm: the
    # one-SM kernel (variant 1) for comparison
    for name, body, bufs, mult, hints in (
            ("bf16", U.UPIR_BODY_GEMM_BF16, [hah, hbh, hc], 1, []),
            ("bf16_one_sm", U.UPIR_BODY_GEMM_BF16, [hah, hbh, hc], 1, [(U.UPIR_HINT_VARIANT, 1)]),
            ("bf16x3", U.UPIR_BODY_GEMM_BF16X3, [hah, hal, hbh, hbl, hc], 3, [])):
        r = rt.region([dict(lb=0, ub=m, collapse=2, body=body, bufs=bufs, scalars=[m, n, k], hints=hints)])
        ms, _, _ = rt.timed_submits(lambda: U.upir_region_submit(r, 0), 30)
        U.upir_region_destroy(r)
        tf = flops / (ms / 1e3) / 1e12
        out[name] = {"ms": ms, "TFLOP/s": tf, "tensor_TFLOP/s": tf * mult,
                     "frac_bf16_peak": tf * mult / pk["bf16_tflops"]}
    U.upir_region_destroy(prep)
    for h in (ha, hb, hah, hal, hbh, hbl, hc):
        U.upir_data_unmap(rt.ctx, h)
    rt.host.clear()
    return out


def batch_oracle(specs: list, arrays: list) -> dict:
    """CPU-baseline leg of the batched-regions workload: the oracle (FP64
    numpy, one thread) runs all 512 regions, timed; its results also serve
    to check the GPU's outputs of every batch mode."""
    from oracle import upir_oracle as O
    want = []
    with one_thread():
        t0 = time.perf_counter()
        for sp, arr in zip(specs, arrays):
            if sp["op"] == I.OP_AXPY_DOT:
                y = O.axpy(2.5, arr["x"], arr["y"])
                want.append((y, O.reduce_f64(O.RED_ADD, 0.0, arr["x"].astype(np.float64) * y)))
            elif sp["op"] == I.OP_JACOBI:
                want.append(O.jacobi_sweep_f32(arr["u0"]))
            else:
                want.append((O.matvec(arr["A"], arr["x"]),
                             np.abs(arr["A"]).astype(np.float64) @ np.abs(arr["x"]).astype(np.float64)))
        dt = time.perf_counter() - t0
    return {"want": want, "seconds": dt,
            "cpu_baseline": {"value": len(specs) / dt, "unit": "regions/s", "cores": 1, "kind": "oracle",
                             "sample": f"all {len(specs)} regions (AXPY exact rounding + exact dot, "
                                       "FP32-mirror Jacobi sweep, FP64 matvec)", "seconds": dt}}


def extra_batch(rt: Runtime, count: int = 512, check: bool = True) -> dict:
    """512 uneven independent regions (40 % AXPY+dot, 30 % one Jacobi sweep,
    30 % matvec; trip counts log-uniform in [1e3, 1e7], seed 6): regions/s of
    one launch per loop, of those launches in one CUDA graph, and of the
    persistent executor (tile shapes autotuned), all with data resident.
    Every mode is timed the same way: one event pair around the whole batch,
    L2 flushed before each repetition.  Outside the timed region each mode
    runs once more from the start values with its outputs poisoned, and every
    region's results are compared with the oracle's (from the CPU-baseline
    leg): AXPY y bit-exact and its dot within 1e-5, the Jacobi field and
    residual bit-exact against the FP32 mirror, matvec within 1e-5 normwise
    and componentwise."""
    U = rt.U
    specs = I.batched_region_specs(count, seed=6)
    arrays = [I.region_arrays(sp) for sp in specs]
    oracle = batch_oracle(specs, arrays) if check else None
    regions, items, total_bytes = [], [], 0.0
    for sp, arr in zip(specs, arrays):
        r = U.upir_spmd_region(rt.ctx, 0, 0)
        if sp["op"] == I.OP_AXPY_DOT:
            dot = np.zeros(1, np.float32)
            y0 = arr["y"].copy()
            hx, hy, hd = rt.map(arr["x"], 0, True), rt.map(arr["y"], 2, True), rt.map(dot, 2, True)
            lp = dict(lb=0, ub=sp["n"], body=U.UPIR_BODY_AXPY, bufs=[hx, hy], scalars=[2.5],
                      reductions=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_XY, hd, 0)])
            total_bytes += 12 * sp["n"]
            items.append(("axpy", (arr["y"], y0, dot), (hy, hd)))
        elif sp["op"] == I.OP_JACOBI:
            side = sp["side"]
            res = np.full(1, -np.inf, np.float32)
            h0, h1, hr = rt.map(arr["u0"], 0, True), rt.map(arr["u1"], 2, True), rt.map(res, 2, True)
            lp = dict(lb=1, ub=side - 1, collapse=2, body=U.UPIR_BODY_JACOBI5, bufs=[h0, h1],
                      scalars=[side, side], reductions=[(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_RESID, hr, 0)])
            total_bytes += 8 * (side - 2) ** 2
            items.append(("jacobi", (arr["u1"], res), (h1, hr)))
        else:
            y = np.zeros(sp["rows"], np.float32)
            ha, hx, hy = rt.map(arr["A"], 0, True), rt.map(arr["x"], 0, True), rt.map(y, 2, True)
            lp = dict(lb=0, ub=sp["rows"], body=U.UPIR_BODY_MATVEC, bufs=[ha, hx, hy],
                      scalars=[sp["rows"], sp["cols"]])
            total_bytes += 4 * sp["rows"] * sp["cols"]
            items.append(("matvec", (y,), (hy,)))
        U.upir_loop_checked(rt.ctx, r, U.make_loop_desc(**lp))
        regions.append(r)

    def reset():
        for kind, host, hs in items:
            if kind == "axpy":
                host[0][:] = host[1]
                host[2][0] = 0.0
            elif kind == "jacobi":
                host[0][1:-1, 1:-1] = np.nan
                host[1][0] = -np.inf
            else:
                host[0][:] = np.nan
            for h in hs:
                U.upir_data_update(rt.ctx, h, U.UPIR_MAP_TO)

    def mismatches() -> int:
        bad = 0
        for (kind, host, hs), want in zip(items, oracle["want"]):
            for h in hs:
                U.upir_data_update(rt.ctx, h, U.UPIR_MAP_FROM)
            if kind == "axpy":
                ok = np.array_equal(host[0], want[0]) and abs(float(host[2][0]) - want[1]) <= 1e-5 * abs(want[1])
            elif kind == "jacobi":
                ok = np.array_equal(host[0], want[0]) and host[1][0] == want[1]
            else:
                y = host[0].astype(np.float64)
                ok = (np.linalg.norm(y - want[0]) <= 1e-5 * np.linalg.norm(want[0])
                      and bool(np.all(np.abs(y - want[0]) <= 1e-5 * want[1])))
            bad += 0 if ok else 1
        return bad

    out = {"regions": count, "algorithmic_GB": total_bytes / 1e9,
           "timing": "one CUDA event pair around the whole batch submission, L2 flushed before each of "
                     "10 repetitions, mean"}
    tiles = None
    for name, mode in (("launches", U.UPIR_BATCH_LAUNCHES), ("graph", U.UPIR_BATCH_GRAPH),
                       ("persistent", U.UPIR_BATCH_PERSISTENT)):
        b = U.upir_batch_create(rt.ctx, regions, mode)
        if mode == U.UPIR_BATCH_PERSISTENT:
            tiles = U.upir_batch_autotune(b, 3)
        ms, _ = timed_whole(rt, lambda: U.upir_batch_submit(b), 10)
        out[name] = {"ms": ms, "regions_per_s": count / (ms / 1e3), "GB/s": total_bytes / (ms / 1e3) / 1e9}
        if oracle is not None:
            reset()
            U.upir_batch_submit(b)
            U.upir_ctx_wait(rt.ctx)
            out[name]["regions_differing_from_oracle"] = mismatches()
        U.upir_batch_destroy(b)
    out["persistent_tiles"] = {"axpy_iters": tiles[0], "jacobi_rows": tiles[1], "matvec_rows": tiles[2]}
    out["speedup_persistent_vs_launches"] = out["launches"]["ms"] / out["persistent"]["ms"]
    out["speedup_persistent_vs_graph"] = out["graph"]["ms"] / out["persistent"]["ms"]
    if oracle is not None:
        out["cpu_baseline"] = oracle["cpu_baseline"]
        out["checked"] = "every region of every mode against the oracle"
    else:
        out["checked"] = "not checked (CPU-baseline leg skipped)"
    for r in regions:
        U.upir_region_destroy(r)
    for h in rt.handles:
        U.upir_data_unmap(rt.ctx, h)
    rt.handles.clear()
    return out


def extra_costmodel(rt: Runtime) -> dict:
    """Learned schedule cost model: trained on ~20k timed variants of 950
    AXPY/Jacobi/matvec regions and 120 FP32 GEMM loops, ranking the candidate
    schedules of 1000 unseen regions drawn like the batched-region workload
    (seed 7) and of 100 unseen GEMM loops."""
    from paper_2209_10643_b300 import costmodel as CM
    return CM.run_protocol(rt.ctx)


def cpu_baseline_jacobi(budget_s: float = 12.0) -> dict:
    """The oracle (FP64 numpy, single thread) on a bounded sample of the
    headline workload: the full 4096^2 grid for as many sweeps as fit the budget."""
    from oracle import upir_oracle as O
    u0 = I.jacobi_grid(N_GRID, seed=1)
    t0 = time.perf_counter()
    O.jacobi_run(u0, 1)
    one = time.perf_counter() - t0
    sweeps = max(1, min(SWEEPS, int(budget_s / max(one, 1e-3))))
    t0 = time.perf_counter()
    O.jacobi_run(u0, sweeps)
    dt = time.perf_counter() - t0
    return {"value": sweeps * JACOBI_BYTES_PER_SWEEP / dt / 1e9, "unit": "GB/s", "cores": 1,
            "kind": "oracle", "sample": f"{sweeps} of {SWEEPS} sweeps on the {N_GRID}x{N_GRID} grid, FP64 numpy",
            "seconds": dt, "host_cores_available": os.cpu_count()}


def cpu_baseline_axpy(n: int = 1 << 20) -> dict:
    """The oracle on the single-region AXPY workload in full: y = fma(2.5, x, y)
    exactly rounded, the FP64 exact sum of y and the int64 sum of (3 i mod 1000)."""
    from oracle import upir_oracle as O
    x, y = I.axpy_inputs(n, seed=0)
    with one_thread():
        t0 = time.perf_counter()
        w = O.axpy(2.5, x, y)
        O.reduce_f64(O.RED_ADD, 0.0, w)
        O.reduce_i64(O.RED_ADD, 0, O.imod_terms(0, 1, n, 3, 1000))
        dt = time.perf_counter() - t0
    return {"value": 12 * n / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"the whole workload, n = {n}", "seconds": dt}


def cpu_baseline_matvec(n: int = 16384) -> dict:
    """The oracle's FP64 matvec on the full 16384^2 workload."""
    from oracle import upir_oracle as O
    a, x = I.matvec_inputs(n, n)
    with one_thread():
        t0 = time.perf_counter()
        O.matvec(a, x)
        dt = time.perf_counter() - t0
    return {"value": (4 * n * n + 8 * n) / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"the whole workload, {n} x {n}", "seconds": dt}


def cpu_baseline_gemm() -> dict:
    """The oracle's FP64 GEMM: 1024^3 in full, and 4096^3 (the workload) once."""
    from oracle import upir_oracle as O
    out = {}
    for m in (1024, 4096):
        a, b = I.gemm_inputs(m, m, m)
        with one_thread():
            t0 = time.perf_counter()
            O.gemm(a, b)
            dt = time.perf_counter() - t0
        out[f"{m}^3"] = {"value": 2.0 * m ** 3 / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": f"one full {m}^3 product in FP64", "seconds": dt}
    return out


def with_cpu(fn, cpu_fn, cpu: bool):
    """Run an extra workload and, when the CPU-baseline leg is on, attach the
    oracle's timing of the same configuration."""
    def run():
        out = fn()
        if cpu:
            out["cpu_baseline"] = cpu_fn()
        return out
    return run


# Execution times the paper reports for the UPIR compiler's offloaded kernels
# (§6, the AXPY, matrix multiplication, matrix-vector multiplication and
# size-7 stencil figures: one V100, mean of 10 runs, the timed span not
# stated); context beside this machine's times, not targets.
PAPER_V100_MS = {
    "axpy": {10240: 13.85, 102400: 14.61, 1024000: 21.54, 10240000: 74.75, 102400000: 702.39},
    "matmul": {64: 13.91, 128: 17.49, 256: 27.6, 512: 135.03, 1024: 976.88},
    "matvec": {1024: 17.88, 2048: 20.7, 4096: 44.2, 8192: 145.74, 16384: 583.45},
    "stencil": {64: 13.69, 128: 15.14, 256: 15.7, 512: 20.32, 1024: 28.72, 2048: 56.47},
}


def extra_paper_workloads(rt: Runtime, runs: int = 10, warmup: int = 2) -> dict:
    """The paper's four evaluation kernels at its problem sizes, each run end
    to end through the C ABI from ordinary (pageable) host arrays: map the
    inputs to the device and the output back, record the one-loop region,
    submit it, unmap (the output comes back) and wait; host wall clock around
    all of it, the mean of ``runs`` runs after ``warmup``, as the paper times
    its kernels (10 runs)."""
    U = rt.U
    ctx = rt.ctx
    TO, FROM, TOFROM = U.UPIR_MAP_TO, U.UPIR_MAP_FROM, U.UPIR_MAP_TOFROM
    w7 = rng_weights7()

    def one(arrays, loop_of):
        hs = [U.upir_data_map(ctx, a.ctypes.data, a.nbytes, kind) for a, kind in arrays]
        r = rt.region([loop_of(hs)])
        U.upir_region_submit(r, 0)
        U.upir_region_destroy(r)
        for h in hs:
            U.upir_data_unmap(ctx, h)
        U.upir_ctx_wait(ctx)

    def timed(arrays, loop_of):
        for _ in range(warmup):
            one(arrays, loop_of)
        t = []
        for _ in range(runs):
            t0 = time.perf_counter()
            one(arrays, loop_of)
            t.append((time.perf_counter() - t0) * 1e3)
        return round(statistics.fmean(t), 4)

    out = {"protocol": f"host wall clock around map, region, submit, unmap and wait; mean of {runs} runs "
                       f"after {warmup}; pageable numpy host arrays",
           "paper_v100_ms": {k: {str(n): v for n, v in d.items()} for k, d in PAPER_V100_MS.items()}}
    res = {}
    for n in PAPER_V100_MS["axpy"]:
        x, y = I.axpy_inputs(n, seed=0)
        res.setdefault("axpy", {})[str(n)] = timed(
            [(x, TO), (y, TOFROM)],
            lambda hs, n=n: dict(lb=0, ub=n, body=U.UPIR_BODY_AXPY, bufs=hs, scalars=[2.0, 3, 1000]))
    for n in PAPER_V100_MS["matmul"]:
        a, b = I.gemm_inputs(n, n, n)
        c = np.zeros((n, n), np.float32)
        res.setdefault("matmul", {})[str(n)] = timed(
            [(a, TO), (b, TO), (c, FROM)],
            lambda hs, n=n: dict(lb=0, ub=n, collapse=2, body=U.UPIR_BODY_GEMM_F32, bufs=hs, scalars=[n, n, n]))
    for n in PAPER_V100_MS["matvec"]:
        a, xv = I.matvec_inputs(n, n)
        yv = np.zeros(n, np.float32)
        res.setdefault("matvec", {})[str(n)] = timed(
            [(a, TO), (xv, TO), (yv, FROM)],
            lambda hs, n=n: dict(lb=0, ub=n, body=U.UPIR_BODY_MATVEC, bufs=hs, scalars=[n, n]))
    for n in PAPER_V100_MS["stencil"]:
        xg = I.jacobi_grid(n, seed=14)
        og = np.zeros_like(xg)
        res.setdefault("stencil", {})[str(n)] = timed(
            [(xg, TO), (og, TOFROM)],
            lambda hs, n=n: dict(lb=3, ub=n - 3, step=1, collapse=2, body=U.UPIR_BODY_FILTER7, bufs=hs,
                                 scalars=[n, n] + [float(v) for v in w7.ravel()]))
    out["ms"] = res
    out["paper_over_this"] = {k: {m: round(PAPER_V100_MS[k][int(m)] / v, 1) for m, v in d.items()}
                              for k, d in res.items()}
    return out


def extra_workloads(rt: Runtime, pk: dict, cpu: bool = True) -> dict:
    return {"axpy_2^20": with_cpu(lambda: extra_axpy(rt, 1 << 20, pk), cpu_baseline_axpy, cpu),
            "axpy_2^26": lambda: extra_axpy(rt, 1 << 26, pk),
            "axpy_2^28": lambda: extra_axpy(rt, 1 << 28, pk),
            "matvec_16384": with_cpu(lambda: extra_matvec(rt, pk), cpu_baseline_matvec, cpu),
            "jacobi_tb4_4096": lambda: extra_jacobi_tb(rt, pk, 4),
            "jacobi_tb8_4096": lambda: extra_jacobi_tb(rt, pk, 8),
            "jacobi_4095": lambda: extra_jacobi_grid(rt, pk, 4095, 20),
            "jacobi_8192": lambda: extra_jacobi_grid(rt, pk, 8192, 20),
            "filter7_4096": lambda: extra_filter7(rt, pk),
            "pipelined_regions": lambda: extra_pipeline(rt),
            "gemm_f32_4096": with_cpu(lambda: extra_gemm_f32(rt), cpu_baseline_gemm, cpu),
            "gemm_tc_4096": lambda: extra_gemm_tc(rt, pk),
            "batch_512_regions": lambda: extra_batch(rt, check=cpu),
            "cost_model": lambda: extra_costmodel(rt),
            "paper_workloads": lambda: extra_paper_workloads(rt)}


def run_ours(args) -> None:
    rank, local_rank, world = dist_env()
    if args.extra_only:
        rt = Runtime(local_rank)
        print(json.dumps({args.extra_only: extra_workloads(rt, peaks(), not args.no_cpu)[args.extra_only]()}),
              flush=True)
        return
    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    pk = peaks()
    rt = Runtime(local_rank)
    h = headline(rt, args.steps, args.warmup, pk, local_rank)
    extra = {}
    if rank == 0 and not args.no_extra:
        for name, fn in extra_workloads(rt, pk, world == 1 and not args.no_cpu).items():
            try:
                extra[name] = fn()
            except Exception as e:  # report, keep the headline
                extra[name] = {"error": repr(e)}
            rt.host.clear()
    cpu = cpu_baseline_jacobi() if (rank == 0 and world == 1 and not args.no_cpu) else None
    if rank == 0:
        line = {
            "metric": METRIC,
            "value": round(h["value"], 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(h["ms_per_step"], 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": headline_config(world),
            "roofline": h["roofline"], "clocks": h["clocks"], "gpu_launches": h["gpu_launches"],
            "e2e": h["e2e"], "cpu_baseline": cpu,
            "per_launch_submission": h["per_launch"],
            "extra": extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_sharded(args) -> None:
    """Strong scaling: ONE 4096^2 Jacobi problem, 100 sweeps per step, split
    by rows over the ranks (halo row exchange with each neighbour every
    sweep, one allreduce(max) of the per-sweep residuals per step).  Value =
    the problem's algorithmic bytes per step x steps / the slowest rank's
    time.  At N = 1 there is no exchange and the slab is the whole grid."""
    import torch
    import torch.distributed as dist
    from paper_2209_10643_b300.sharding import JacobiRowBlocks, UpirJacobiSweeper

    rank, local_rank, world = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    rt = Runtime(local_rank)
    if world > 1:
        dist.barrier()  # a collective of every rank before the first point-to-point batch
    plan = JacobiRowBlocks(N_GRID, N_GRID, world, rank)
    u0 = I.jacobi_grid(N_GRID, seed=1)
    a = torch.from_numpy(plan.slab(u0).copy()).cuda()
    b = a.clone()
    res = torch.full((SWEEPS,), -np.inf, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    sweeper = UpirJacobiSweeper(rt.ctx, plan, a, b, res, SWEEPS)

    def step():
        res.fill_(-np.inf)
        plan.run(sweeper, a, b, SWEEPS, res)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ms = []
    with ClockSampler(local_rank) as clk:
        for _ in range(args.steps):
            rt.flush_l2()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            step()
            ev1.record()
            ev1.synchronize()
            ms.append(ev0.elapsed_time(ev1))
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    from paper_2209_10643_b300.sharding import aggregate_throughput
    local_s = sum(ms) / 1e3
    _, secs = aggregate_throughput(0.0, local_s)
    total = args.steps * SWEEPS * JACOBI_BYTES_PER_SWEEP
    resid_last = float(res[-1].item())
    sweeper.close()
    if rank == 0:
        value = total / secs / 1e9
        line = {
            "metric": METRIC,
            "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [N_GRID, N_GRID],
                       "sweeps": SWEEPS, "parallelism": f"row blocks x{world}, one halo row per neighbour "
                                                          "per sweep, allreduce(max) of the residuals",
                       "l2": "flushed before each step (256 MiB write, then 256 MiB read)",
                       "submission": "one CUDA graph per sweep and rank, halo messages between sweeps"},
            "clocks": clk.summary(), "gpu_launches": args.steps * SWEEPS,
            "residual_last": resid_last,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- reference --

def run_reference(args) -> None:
    """The oracle, as it stands, on the host cores: each step one bounded sample
    (2 FP64 sweeps of the 4096^2 grid) of the headline workload."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    from oracle import upir_oracle as O
    u0 = I.jacobi_grid(N_GRID, seed=1)
    per = 2
    for _ in range(args.warmup):
        O.jacobi_run(u0, 1)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.jacobi_run(u0, per)
        ts.append(time.perf_counter() - t0)
    dt = sum(ts)
    value = args.steps * per * JACOBI_BYTES_PER_SWEEP / dt / 1e9
    line = {"impl": "reference", "metric": METRIC,
            "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": headline_config(world),
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per} FP64 sweeps of the {N_GRID}x{N_GRID} grid per step"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extra", action="store_true", help="skip the extra workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--sharded", action="store_true",
                    help="strong scaling: one Jacobi problem split by rows over the ranks")
    ap.add_argument("--extra-only", default=None,
                    help="run only the named extra workload (e.g. gemm_tc_4096) and print its JSON")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    if args.impl == "reference":
        run_reference(args)
    elif args.sharded:
        run_sharded(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
