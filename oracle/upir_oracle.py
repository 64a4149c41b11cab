"""UPIR region oracle: a plain, sequential CPU restatement of what an offloaded
SPMD region with worksharing loops, reductions and explicit data mapping computes.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` may import or call this module.  The
CUDA library and its Python binding never do, and this module imports nothing
from them.  It shares no code with the CUDA path; only the seeded input
generators (``upir_inputs``) feed both.

Precision: floating-point results are computed in FP64 from the FP32 inputs
("FP64 mode", the reference for tolerances).  Where the CUDA path is required to
reproduce FP32 rounding exactly (the AXPY update, the Jacobi field and its
residuals, the 7 x 7 filter), an FP32 "mirror" applies the same IEEE
single-precision operations in the order the method's formula fixes.

Each function cites the passage of the paper it follows.  Where the paper is
silent the reading taken is stated in the docstring.  Every function here is
pinned by a CPU test against something other than itself (closed forms,
brute force, invariants, hand-worked examples, exact rational arithmetic);
none is "parity unpinned".
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ----------------------------------------------------------------------------
# Data mapping — §4.1 (the figure with the dialect of data attributes): the
# data-mapping property is one of to / from / tofrom / allocate.
# ----------------------------------------------------------------------------

MAP_TO, MAP_FROM, MAP_TOFROM, MAP_ALLOC = 0, 1, 2, 3

F32_POISON_BITS = np.uint32(0x7FA00000)  # a signalling NaN
INT_POISON_BYTE = 0x5A


class Device:
    """An arena standing in for device memory.

    ``to``/``tofrom`` copy the host bytes in; ``from``/``allocate`` give storage
    whose contents are undefined, which the oracle fills with a poison pattern
    (signalling NaN for FP32, 0x5A bytes otherwise) so that a read-before-write
    shows up.  Unmapping copies ``from``/``tofrom`` buffers back to the host
    array.  (The paper does not say what an ``allocate`` mapping holds; reading:
    undefined, hence poison.)
    """

    def __init__(self):
        self._bufs: dict[int, tuple[np.ndarray, np.ndarray, int]] = {}
        self._next = 1

    def map(self, host: np.ndarray, kind: int) -> int:
        if kind not in (MAP_TO, MAP_FROM, MAP_TOFROM, MAP_ALLOC):
            raise ValueError("unknown map kind")
        if kind in (MAP_TO, MAP_TOFROM):
            dev = host.copy()
        else:
            dev = np.empty_like(host)
            if dev.dtype == np.float32:
                dev.view(np.uint32)[...] = F32_POISON_BITS
            else:
                dev.view(np.uint8)[...] = INT_POISON_BYTE
        h = self._next
        self._next += 1
        self._bufs[h] = (host, dev, kind)
        return h

    def array(self, h: int) -> np.ndarray:
        return self._bufs[h][1]

    def unmap(self, h: int) -> None:
        host, dev, kind = self._bufs.pop(h)
        if kind in (MAP_FROM, MAP_TOFROM):
            host[...] = dev


# ----------------------------------------------------------------------------
# Canonical loop — §3.2 (the figure with the dialect of data parallelism):
# induction variable, lowerBound, upperBound, step.  The AXPY listings of §6
# (``for (i = 0; i < n; i++)`` lowered to ``lowerBound(0) upperBound(n)``) fix
# the upper bound as exclusive.
# ----------------------------------------------------------------------------

def trip_count(lb: int, ub: int, step: int) -> int:
    """Number of iterations of ``for (iv = lb; iv < ub (or > ub); iv += step)``.

    Reading (paper silent): step 0 is an error; a negative step counts down
    with an exclusive lower end.
    """
    if step == 0:
        raise ValueError("step must be non-zero")
    if step > 0:
        if ub <= lb:
            return 0
        return (ub - lb + step - 1) // step
    if lb <= ub:
        return 0
    return (lb - ub + (-step) - 1) // (-step)


def induction_value(lb: int, step: int, k: int) -> int:
    """Value of the induction variable at logical iteration k."""
    return lb + k * step


# ----------------------------------------------------------------------------
# Worksharing schedules — §3.2: ``loop_parallel worksharing`` with
# ``schedule(static|dynamic [, chunk])`` and ``distribute(teams, units)``.
# The paper gives no semantics; the OpenMP-like reading taken here:
#   * workers are the teams x units SPMD units, flattened w = t * units + u;
#   * static, chunk c > 0: logical chunk j = [j c, min((j+1) c, trip)) goes to
#     worker j mod W (round robin);
#   * static, no chunk: W contiguous blocks; the first (trip mod W) workers get
#     ceil(trip / W) iterations and the others floor(trip / W);
#   * dynamic, chunk c (0 means 1): chunks j = 0, 1, 2, ... are handed out in
#     increasing order to whichever worker asks next; any assignment is valid,
#     so only the chunk boundaries and "each chunk claimed exactly once" are
#     fixed.
# ----------------------------------------------------------------------------

SCHED_STATIC, SCHED_DYNAMIC, SCHED_GUIDED, SCHED_RUNTIME, SCHED_AUTO, SCHED_TASKLOOP = range(6)


def static_owner_map(trip: int, workers: int, chunk: int) -> np.ndarray:
    """Worker that owns each logical iteration under a static schedule."""
    if workers <= 0:
        raise ValueError("need at least one worker")
    owner = np.full(trip, -1, dtype=np.int64)
    if chunk > 0:
        j = 0
        while j * chunk < trip:
            start = j * chunk
            end = min(start + chunk, trip)
            for k in range(start, end):
                owner[k] = j % workers
            j += 1
    else:
        base, extra = divmod(trip, workers)
        k = 0
        for w in range(workers):
            n = base + (1 if w < extra else 0)
            for _ in range(n):
                owner[k] = w
                k += 1
    return owner


def dynamic_chunks(trip: int, chunk: int) -> list[tuple[int, int]]:
    """Chunk boundaries of a dynamic schedule, in hand-out order."""
    c = chunk if chunk > 0 else 1
    return [(s, min(s + c, trip)) for s in range(0, trip, c)]


def guided_chunks(trip: int, workers: int, chunk: int) -> list[tuple[int, int]]:
    """Chunk boundaries of ``schedule(guided, c)`` (§3.2 lists guided among
    the schedule policies without defining it).  Reading, after OpenMP: each
    chunk handed out holds max(c, ceil(R / W)) iterations, R being the
    iterations not yet handed out and W the workers (c = 0 means 1; the last
    chunk may be shorter); chunks go out in increasing iteration order to
    whichever worker asks next."""
    if workers <= 0:
        raise ValueError("need at least one worker")
    c = chunk if chunk > 0 else 1
    out, s = [], 0
    while s < trip:
        e = min(s + max(c, -(-(trip - s) // workers)), trip)
        out.append((s, e))
        s = e
    return out


def taskloop_chunks(trip: int, grainsize: int = 0, num_tasks: int = 0) -> list[tuple[int, int]]:
    """Tasks of ``loop_parallel taskloop(grainsize, num_tasks)`` (§3.2: the two
    fields control the granularity or the number of tasks).  Reading, after
    OpenMP: num_tasks(n) makes min(n, trip) tasks; grainsize(g) makes
    max(1, floor(trip / g)) tasks, so each holds between g and 2g - 1
    iterations (or all of them when trip < g); with both fields the smaller
    count wins.  The iterations are split into that many contiguous tasks, the
    first (trip mod n) one iteration longer; tasks run in any order on any
    worker, each exactly once."""
    if trip == 0:
        return []
    counts = []
    if num_tasks > 0:
        counts.append(min(num_tasks, trip))
    if grainsize > 0:
        counts.append(max(1, trip // grainsize))
    if not counts:
        raise ValueError("taskloop needs grainsize or num_tasks")
    n = min(counts)
    base, extra = divmod(trip, n)
    out, s = [], 0
    for t in range(n):
        e = s + base + (1 if t < extra else 0)
        out.append((s, e))
        s = e
    return out


def check_chunked_assignment(trip: int, chunks: list[tuple[int, int]], owner: np.ndarray,
                             count: np.ndarray, workers: int) -> bool:
    """True when (owner, count) is a valid execution of a schedule that hands
    out the given chunks to whichever worker asks: the chunks tile [0, trip),
    every iteration ran exactly once and each chunk ran on a single worker."""
    if owner.shape != (trip,) or count.shape != (trip,):
        return False
    if trip and (count.min() != 1 or count.max() != 1):
        return False
    s0 = 0
    for s, e in chunks:
        if s != s0 or e <= s:
            return False
        s0 = e
        w = owner[s]
        if w < 0 or w >= workers or np.any(owner[s:e] != w):
            return False
    return s0 == trip


def check_dynamic_assignment(trip: int, chunk: int, owner: np.ndarray,
                             count: np.ndarray, workers: int) -> bool:
    """True when (owner, count) is a valid dynamic-schedule execution:
    every iteration ran exactly once and each chunk ran on a single worker."""
    return check_chunked_assignment(trip, dynamic_chunks(trip, chunk), owner, count, workers)


# ----------------------------------------------------------------------------
# Reductions — §5 (the figure with the dialect of synchronization): a sync of
# kind ``reduction`` carries an operation and the data it reduces.  Reading
# (paper silent): identities + -> 0, * -> 1, max -> -inf, min -> +inf; the
# variable's value before the loop is combined exactly once; max/min ignore a
# NaN operand (IEEE maxNum/minNum); integer arithmetic wraps in two's
# complement at 64 bits.
# ----------------------------------------------------------------------------

RED_NONE, RED_ADD, RED_MUL, RED_MAX, RED_MIN = 0, 1, 2, 3, 4


def wrap_i64(v: int) -> int:
    v &= (1 << 64) - 1
    return v - (1 << 64) if v >= (1 << 63) else v


def reduce_i64(op: int, init: int, terms) -> int:
    """Exact integer reduction of ``init`` and ``terms`` with 64-bit wrap."""
    acc = int(init)
    for t in terms:
        t = int(t)
        if op == RED_ADD:
            acc = wrap_i64(acc + t)
        elif op == RED_MUL:
            acc = wrap_i64(acc * t)
        elif op == RED_MAX:
            acc = max(acc, t)
        elif op == RED_MIN:
            acc = min(acc, t)
        else:
            raise ValueError("unknown reduction op")
    return acc


def reduce_f64(op: int, init: float, terms: np.ndarray) -> float:
    """FP64-mode reduction of FP32 terms.

    ``+`` is the exact sum rounded once to FP64 (``math.fsum``); ``*`` is the
    sequential FP64 product; max/min follow IEEE maxNum/minNum.
    """
    vals = [float(init)] + [float(t) for t in np.asarray(terms).ravel()]
    if op == RED_ADD:
        return math.fsum(vals)
    if op == RED_MUL:
        p = 1.0
        for v in vals:
            p *= v
        return p
    if op in (RED_MAX, RED_MIN):
        finite = [v for v in vals if not math.isnan(v)]
        if not finite:
            return math.nan
        return max(finite) if op == RED_MAX else min(finite)
    raise ValueError("unknown reduction op")


# ----------------------------------------------------------------------------
# Exact FP32 rounding helpers (used by the AXPY body).
# ----------------------------------------------------------------------------

def two_sum(a: np.ndarray, b: np.ndarray):
    """Knuth's TwoSum in FP64: s + e == a + b exactly, s = fl(a + b)."""
    s = a + b
    bp = s - a
    ap = s - bp
    e = (a - ap) + (b - bp)
    return s, e


def round_f32_of_exact(hi: np.ndarray, lo: np.ndarray) -> np.ndarray:
    """Nearest-even FP32 value of the exact real hi + lo (|lo| <= ulp(hi)/2).

    Rounds hi + lo to 53 bits with round-to-odd, then to 24 bits with
    round-to-nearest-even; with 53 >= 2*24 + 2 the double rounding is innocuous
    (Boldo and Melquiond, "Emulation of FMA and correctly rounded sums: proved
    algorithms using rounding to odd", IEEE Trans. Computers, 2008).
    """
    hi = np.asarray(hi, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    odd_bit = (hi.view(np.uint64) & np.uint64(1)) != 0
    nudge = (lo != 0) & ~odd_bit
    toward = np.where(lo > 0, np.inf, -np.inf)
    ro = np.where(nudge, np.nextafter(hi, toward), hi)
    return ro.astype(np.float32)


# ----------------------------------------------------------------------------
# Loop bodies.
# ----------------------------------------------------------------------------

def axpy(a: float, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """AXPY update y_i <- y_i + a x_i (§6, AXPY listings), one rounding.

    The listings multiply by an ``int a``; the workload uses a = 2.5 in FP32.
    Reading (paper silent on contraction): the update is rounded once, as a
    fused multiply-add.  a x_i is exact in FP64 (24 + 24 significant bits), the
    FP64 sum's error is recovered with TwoSum, and the exact value is rounded
    once to FP32.
    """
    a32 = np.float64(np.float32(a))
    p = a32 * x.astype(np.float64)
    hi, lo = two_sum(p, y.astype(np.float64))
    return round_f32_of_exact(hi, lo)


def imod_terms(lb: int, step: int, trip: int, mul: int, mod: int) -> list[int]:
    """Integer reduction terms (mul * iv) mod m for every induction value iv.

    The product wraps at 64 bits; the remainder is the non-negative one (m > 0).
    """
    if mod <= 0:
        raise ValueError("modulus must be positive")
    return [wrap_i64(mul * induction_value(lb, step, k)) % mod for k in range(trip)]


def imod_sum_closed_form(n: int, mul: int, mod: int) -> int:
    """sum_{i<n} (mul*i mod m) when gcd(mul, m) == 1: each run of m consecutive
    i visits 0..m-1 once, so full runs contribute m(m-1)/2 each."""
    if math.gcd(mul, mod) != 1:
        raise ValueError("closed form needs gcd(mul, mod) == 1")
    full, rest = divmod(n, mod)
    return full * (mod * (mod - 1) // 2) + sum((mul * i) % mod for i in range(rest))


def jacobi_sweep_f64(u: np.ndarray) -> tuple[np.ndarray, float]:
    """One Jacobi sweep of the 5-point Laplace stencil in FP64.

    Interior points take the mean of their four neighbours; boundary values are
    copied unchanged.  Returns the new field and max |u_new - u| over the
    interior (the loop's reduction(max)).  (§6 evaluates a 2D stencil; the
    workload fixes the 5-point Jacobi form.)
    """
    u = np.asarray(u, dtype=np.float64)
    v = u.copy()
    if u.shape[0] > 2 and u.shape[1] > 2:
        v[1:-1, 1:-1] = 0.25 * ((u[:-2, 1:-1] + u[2:, 1:-1]) + (u[1:-1, :-2] + u[1:-1, 2:]))
        res = float(np.max(np.abs(v[1:-1, 1:-1] - u[1:-1, 1:-1])))
    else:
        res = -math.inf
    return v, res


def jacobi_sweep_f32(u: np.ndarray) -> tuple[np.ndarray, np.float32]:
    """The same sweep in IEEE FP32, with the operation order fixed:
    0.25 * ((north + south) + (west + east)), each step rounded to FP32,
    residual |new - old| in FP32."""
    u = np.asarray(u, dtype=np.float32)
    v = u.copy()
    if u.shape[0] > 2 and u.shape[1] > 2:
        ns = u[:-2, 1:-1] + u[2:, 1:-1]
        we = u[1:-1, :-2] + u[1:-1, 2:]
        v[1:-1, 1:-1] = np.float32(0.25) * (ns + we)
        res = np.max(np.abs(v[1:-1, 1:-1] - u[1:-1, 1:-1]))
    else:
        res = np.float32(-np.inf)
    return v, np.float32(res)


def jacobi_run(u0: np.ndarray, sweeps: int, mirror_f32: bool = False):
    """``sweeps`` Jacobi sweeps with ping-pong buffers and a barrier after each
    (implicit barrier after a worksharing loop, §5).  Returns the final field
    and the per-sweep residuals."""
    step = jacobi_sweep_f32 if mirror_f32 else jacobi_sweep_f64
    u = u0.astype(np.float32 if mirror_f32 else np.float64)
    res = []
    for _ in range(sweeps):
        u, r = step(u)
        res.append(r)
    return u, np.array(res, dtype=np.float32 if mirror_f32 else np.float64)


def jacobi_tb(uin: np.ndarray, lb: int, ub: int, sweeps: int, mirror_f32: bool = False):
    """Time-blocked Jacobi body: ``sweeps`` successive 5-point sweeps of u_in
    in which only rows [lb, ub) of the interior columns are updated and every
    other point keeps its u_in value (the time loop of the §6 stencil nest
    carried inside one loop body).

    Each sweep is the sweep of ``jacobi_sweep_f64`` (or the FP32 mirror), its
    values kept on the updated points only.  Returns the field after the last
    sweep and, per sweep, the array of |new - old| over the updated points (the
    terms of that sweep's reduction).
    """
    sweep = jacobi_sweep_f32 if mirror_f32 else jacobi_sweep_f64
    dt = np.float32 if mirror_f32 else np.float64
    u = np.asarray(uin).astype(dt)
    terms = []
    for _ in range(sweeps):
        v, _ = sweep(u)
        new = u.copy()
        new[lb:ub, 1:-1] = v[lb:ub, 1:-1]
        terms.append(np.abs(new[lb:ub, 1:-1] - u[lb:ub, 1:-1]).ravel())
        u = new
    return u, terms


def fmaf(a: np.ndarray, b: np.ndarray, c: np.ndarray) -> np.ndarray:
    """FP32 fused multiply-add, rounded once: a b is exact in FP64 (two 24-bit
    significands), TwoSum recovers the FP64 sum's error, and the exact value is
    rounded to FP32 once."""
    p = np.asarray(a, dtype=np.float64) * np.asarray(b, dtype=np.float64)
    hi, lo = two_sum(p, np.asarray(c, dtype=np.float64))
    return round_f32_of_exact(hi, lo)


def filter7_f64(x: np.ndarray, w: np.ndarray, r0: int, r1: int) -> np.ndarray:
    """The 2D stencil with a filter of size 7 (§6, stencil evaluation: "filter
    size = 7"), read as a 7 x 7 weighted window: for rows r in [r0, r1) and
    columns c in [3, cols - 3),
        out[r][c] = sum_{i=0..6} sum_{j=0..6} w[i][j] x[r + i - 3][c + j - 3]
    in FP64.  Returns the [r1 - r0, cols - 6] block of outputs."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64).reshape(7, 7)
    cols = x.shape[1]
    out = np.zeros((r1 - r0, max(cols - 6, 0)))
    for i in range(7):
        for j in range(7):
            out += w[i, j] * x[r0 + i - 3:r1 + i - 3, j:j + cols - 6]
    return out


def filter7_f32(x: np.ndarray, w: np.ndarray, r0: int, r1: int) -> np.ndarray:
    """The same filter in FP32 with the summation order fixed: the accumulator
    starts at 0 and takes w[i][j] x[...] by fused multiply-add, i outer and j
    inner (row-major over the window), each step rounded once."""
    x = np.asarray(x, dtype=np.float32)
    w = np.asarray(w, dtype=np.float32).reshape(7, 7)
    cols = x.shape[1]
    acc = np.zeros((r1 - r0, max(cols - 6, 0)), dtype=np.float32)
    for i in range(7):
        for j in range(7):
            acc = fmaf(w[i, j], x[r0 + i - 3:r1 + i - 3, j:j + cols - 6], acc)
    return acc


def matvec(a: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y_i = sum_j A_ij x_j in FP64 (§6, matrix-vector multiplication)."""
    return a.astype(np.float64) @ x.astype(np.float64)


def gemm(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """C = A B in FP64 (§6, matrix multiplication)."""
    return a.astype(np.float64) @ b.astype(np.float64)


def bf16_round(v: np.ndarray) -> np.ndarray:
    """Round FP32 to the nearest bfloat16 (ties to even), returned as FP32.

    bfloat16 keeps the top 16 bits of an FP32 word; rounding adds half an ulp of
    the kept part (0x7FFF plus the kept lsb, for ties-to-even) before
    truncating.  NaN stays NaN.
    """
    v = np.asarray(v, dtype=np.float32)
    bits = v.view(np.uint32).astype(np.uint64)
    rounded = ((bits + np.uint64(0x7FFF) + ((bits >> np.uint64(16)) & np.uint64(1)))
               >> np.uint64(16)) << np.uint64(16)
    out = (rounded & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    return np.where(np.isnan(v), v, out).astype(np.float32)


def split_bf16(v: np.ndarray):
    """Two-term bfloat16 split: hi = bf16(v), lo = bf16(v - hi).
    (v - hi is exact in FP32.)"""
    hi = bf16_round(v)
    lo = bf16_round((np.asarray(v, np.float32) - hi).astype(np.float32))
    return hi, lo


def gemm_bf16(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """The product of the bfloat16-rounded operands, exactly accumulated (FP64)."""
    return gemm(bf16_round(a), bf16_round(b))


def gemm_bf16x3(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Split-bfloat16 product A_hi B_hi + A_hi B_lo + A_lo B_hi (lo*lo dropped),
    exactly accumulated.  Reading: "bf16x3" is a two-term split with three
    products."""
    ah, al = split_bf16(a)
    bh, bl = split_bf16(b)
    return gemm(ah, bh) + gemm(ah, bl) + gemm(al, bh)


# ----------------------------------------------------------------------------
# Region interpreter — §3.1 (spmd num_teams / num_units), §3.2 (loop and
# worksharing), §4.1 (data), §5 (sync: reduction, barrier).
# ----------------------------------------------------------------------------

BODY_AXPY, BODY_IMOD, BODY_JACOBI5, BODY_MATVEC, BODY_GEMM_F32, \
    BODY_GEMM_BF16, BODY_GEMM_BF16X3, BODY_COVERAGE, BODY_SPLIT_BF16, \
    BODY_JACOBI5_TB, BODY_FILTER7 = range(11)

TERM_Y, TERM_XY, TERM_IMOD, TERM_IV, TERM_RESID = range(5)

DT_F32, DT_I64 = 0, 1


@dataclass
class Reduction:
    op: int
    dtype: int
    var: int            # device buffer handle
    index: int = 0
    term: int = TERM_Y


@dataclass
class Loop:
    body: int
    lb: int
    ub: int
    step: int = 1
    sched: int = SCHED_STATIC
    chunk: int = 0
    bufs: list = field(default_factory=list)
    scalars: list = field(default_factory=list)
    reductions: list = field(default_factory=list)


def run_loop(dev: Device, teams: int, units: int, loop: Loop) -> dict:
    """Execute one worksharing loop sequentially, in iteration order.

    Iterations have no cross-iteration dependences in any body here, so the
    sequential order gives the result every schedule must reach (up to the
    rounding order of floating-point reductions).  Returns the static owner map
    (when the schedule is static) for the coverage body.
    """
    trip = trip_count(loop.lb, loop.ub, loop.step)
    workers = teams * units
    out: dict = {"trip": trip}
    terms: dict[int, np.ndarray | list] = {}

    if loop.body == BODY_AXPY:
        x, y = dev.array(loop.bufs[0]), dev.array(loop.bufs[1])
        idx = np.array([induction_value(loop.lb, loop.step, k) for k in range(trip)],
                       dtype=np.int64) if loop.step != 1 else np.arange(loop.lb, loop.lb + trip)
        ynew = axpy(loop.scalars[0], x[idx], y[idx])
        y[idx] = ynew
        terms[TERM_Y] = ynew
        terms[TERM_XY] = x[idx].astype(np.float64) * ynew.astype(np.float64)
    elif loop.body == BODY_JACOBI5:
        uin, uout = dev.array(loop.bufs[0]), dev.array(loop.bufs[1])
        r0, r1 = loop.lb, loop.lb + trip * loop.step
        if loop.step != 1 or r0 < 1 or r1 > uin.shape[0] - 1:
            raise ValueError("Jacobi rows must be a unit-step sub-range of the interior")
        v, _ = jacobi_sweep_f64(uin)
        new = v[r0:r1, 1:-1]
        uout[r0:r1, 1:-1] = new.astype(np.float32)
        terms[TERM_RESID] = np.abs(new - uin[r0:r1, 1:-1].astype(np.float64)).ravel()
    elif loop.body == BODY_JACOBI5_TB:
        uin, uout = dev.array(loop.bufs[0]), dev.array(loop.bufs[1])
        r0, r1 = loop.lb, loop.lb + trip * loop.step
        if loop.step != 1 or r0 < 1 or r1 > uin.shape[0] - 1:
            raise ValueError("Jacobi rows must be a unit-step sub-range of the interior")
        u, sweep_terms = jacobi_tb(uin, r0, r1, int(loop.scalars[2]))
        uout[r0:r1, 1:-1] = u[r0:r1, 1:-1].astype(np.float32)
        terms["sweeps"] = sweep_terms
    elif loop.body == BODY_FILTER7:
        xin, xout = dev.array(loop.bufs[0]), dev.array(loop.bufs[1])
        r0, r1 = loop.lb, loop.lb + trip * loop.step
        if loop.step != 1 or r0 < 3 or r1 > xin.shape[0] - 3:
            raise ValueError("filter rows must be a unit-step range inside [3, rows - 3)")
        xout[r0:r1, 3:-3] = filter7_f64(xin, np.asarray(loop.scalars[2:51]), r0, r1).astype(np.float32)
    elif loop.body == BODY_MATVEC:
        a, x, y = (dev.array(h) for h in loop.bufs[:3])
        rows = [induction_value(loop.lb, loop.step, k) for k in range(trip)]
        vals = matvec(a[rows], x)
        y[rows] = vals.astype(np.float32)
        terms[TERM_Y] = vals
    elif loop.body in (BODY_GEMM_F32, BODY_GEMM_BF16, BODY_GEMM_BF16X3):
        a, b, c = (dev.array(h) for h in loop.bufs[:3])
        fn = {BODY_GEMM_F32: gemm, BODY_GEMM_BF16: gemm_bf16,
              BODY_GEMM_BF16X3: gemm_bf16x3}[loop.body]
        rows = [induction_value(loop.lb, loop.step, k) for k in range(trip)]
        c[rows] = fn(a[rows], b).astype(np.float32)
    elif loop.body == BODY_COVERAGE:
        owner_buf, count_buf = dev.array(loop.bufs[0]), dev.array(loop.bufs[1])
        if loop.sched == SCHED_STATIC:
            om = static_owner_map(trip, workers, loop.chunk)
            owner_buf[:trip] = om
            out["owner"] = om
        count_buf[:trip] += 1
    elif loop.body != BODY_IMOD:
        raise ValueError("unknown body")

    for red in loop.reductions:
        var = dev.array(red.var)
        if loop.body == BODY_JACOBI5_TB:
            # one reduction per sweep, into consecutive elements of the variable
            for k, t in enumerate(terms["sweeps"]):
                out.setdefault("f64", {})[(red.var, red.index + k)] = reduce_f64(
                    red.op, float(var[red.index + k]), np.asarray(t))
                var[red.index + k] = np.float32(out["f64"][(red.var, red.index + k)])
            continue
        if red.term in (TERM_IMOD, TERM_IV):
            if red.term == TERM_IMOD:
                t = imod_terms(loop.lb, loop.step, trip, int(loop.scalars[-2]),
                               int(loop.scalars[-1]))
            else:
                t = [induction_value(loop.lb, loop.step, k) for k in range(trip)]
        else:
            t = terms[red.term]
        if red.dtype == DT_I64:
            var[red.index] = reduce_i64(red.op, int(var[red.index]), t)
        else:
            out.setdefault("f64", {})[(red.var, red.index)] = reduce_f64(
                red.op, float(var[red.index]), np.asarray(t))
            var[red.index] = np.float32(out["f64"][(red.var, red.index)])
    return out


def run_region(dev: Device, teams: int, units: int, loops: list[Loop]) -> list[dict]:
    """An SPMD region (§3.1) whose loops run one after another; the implicit
    barrier at the end of each worksharing loop (§5) orders them."""
    return [run_loop(dev, teams, units, lp) for lp in loops]


# ----------------------------------------------------------------------------
# Learned cost model: the 12 -> 64 -> 64 -> 1 ReLU MLP trained on measured
# log2 times.  Not part of the paper; restated from its definition.
# Weights are used in bfloat16 in the forward pass (the master copy stays FP32);
# gradients are taken with respect to the rounded weights.
# ----------------------------------------------------------------------------

MLP_KEYS = ("W1", "b1", "W2", "b2", "W3", "b3")


def mlp_forward(p: dict, x: np.ndarray, bf16_weights: bool = True):
    """Forward pass in FP64.  Returns predictions [B] and the cached activations."""
    def w(k):
        v = p[k]
        return (bf16_round(v) if bf16_weights and k.startswith("W") else v).astype(np.float64)

    x = np.asarray(x, dtype=np.float64)
    z1 = x @ w("W1").T + p["b1"].astype(np.float64)
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w("W2").T + p["b2"].astype(np.float64)
    h2 = np.maximum(z2, 0.0)
    yhat = (h2 @ w("W3").T + p["b3"].astype(np.float64))[:, 0]
    cache = {"x": x, "z1": z1, "h1": h1, "z2": z2, "h2": h2,
             "W2": w("W2"), "W3": w("W3")}
    return yhat, cache


def mlp_loss(yhat: np.ndarray, t: np.ndarray) -> float:
    """Mean squared error over the batch."""
    d = np.asarray(yhat, np.float64) - np.asarray(t, np.float64)
    return float(np.mean(d * d))


def mlp_backward(cache: dict, yhat: np.ndarray, t: np.ndarray) -> dict:
    """Gradients of ``mlp_loss`` by the chain rule, written out layer by layer."""
    bsz = yhat.shape[0]
    dy = 2.0 * (yhat - np.asarray(t, np.float64)) / bsz         # [B]
    g = {}
    g["W3"] = dy[None, :] @ cache["h2"]                            # [1, 64]
    g["b3"] = np.array([dy.sum()])
    dh2 = dy[:, None] @ cache["W3"]                                # [B, 64]
    dz2 = dh2 * (cache["z2"] > 0)
    g["W2"] = dz2.T @ cache["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ cache["W2"]
    dz1 = dh1 * (cache["z1"] > 0)
    g["W1"] = dz1.T @ cache["x"]
    g["b1"] = dz1.sum(axis=0)
    return g


def mlp_sgd(p: dict, g: dict, lr: float) -> dict:
    """One plain SGD step on the FP32 master weights."""
    return {k: (p[k].astype(np.float64) - lr * g[k]).astype(np.float32) for k in MLP_KEYS}
