"""Running the hot path on several GPUs of one node: one process per GPU.

Two ways to use N ranks:

- **independent problems** (weak scaling): each rank runs its own problem, or
  its share of a batch of independent regions; the only collectives are the
  timing barrier and the max/sum that report whole-job throughput;
- **one problem partitioned** (strong scaling), following the SPMD region's
  teams (§3.1) one level up, with the partials combined as the reduction
  sync combines them (§5):
  - Jacobi: a block of grid rows per rank.  Every sweep a rank updates its
    rows, then exchanges one halo row with each neighbour; the per-sweep
    max residuals are combined with one allreduce(max);
  - matvec: a block of rows of A per rank, x replicated, y gathered;
  - GEMM: 2D output tiles on a grid of ranks, the A and B panels broadcast
    along process rows and columns one K panel at a time;
  - AXPY + sum: a block of iterations per rank, the per-rank FP32 sums
    gathered in rank order and folded by the runtime's own compensated
    reduction (deterministic for a given N);
  - batches: regions assigned by longest-processing-time over their
    predicted (cost-model) or algorithmic costs, no exchange.

Row and iteration blocks follow the static schedule without chunk: N
contiguous blocks, the first (count mod N) one longer.

The exchange steps work on torch tensors through ``torch.distributed``
(NCCL on GPUs, gloo on CPU) and take the per-rank compute as a callable, so
the same partition and exchange logic runs with the CUDA kernels on GPUs
and, in the tests, with any CPU implementation of a sweep on gloo ranks.
No TMA multicast and no peer-memory access is used: a halo row crosses
ranks as a point-to-point message copied into the receiver's own buffer.
"""
from __future__ import annotations

import os
from typing import Callable


def dist_env() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (1 process: 0, 0, 1)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


# ------------------------------------------------------------- partitions --

def block_range(lo: int, hi: int, world: int, rank: int) -> tuple[int, int]:
    """Rank ``rank``'s contiguous block of [lo, hi) split into ``world``
    blocks, the first ((hi - lo) mod world) one longer (the static schedule
    without chunk)."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    n = max(hi - lo, 0)
    q, r = divmod(n, world)
    start = lo + rank * q + min(rank, r)
    return start, start + q + (1 if rank < r else 0)


def shard_lpt(costs: list[float], world: int) -> list[list[int]]:
    """Longest-processing-time assignment of independent items to ``world`` ranks.

    Items are taken in decreasing cost (ties by index) and each goes to the rank
    with the least total so far (ties by rank), so every item lands on exactly
    one rank and the result is deterministic."""
    if world <= 0:
        raise ValueError("world must be positive")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    for lst in out:
        lst.sort()
    return out


def region_bytes(spec: dict) -> float:
    """Algorithmic bytes of one batched region (the fallback cost for LPT)."""
    if "n" in spec:
        return 12.0 * spec["n"]
    if "side" in spec:
        return 8.0 * (spec["side"] - 2) ** 2
    return 4.0 * spec["rows"] * spec["cols"] + 8.0 * spec["rows"]


# ----------------------------------------------------------- aggregation --

def aggregate_throughput(local_units: float, local_seconds: float, group=None) -> tuple[float, float]:
    """Whole-job (total units, max seconds) over the ranks of ``group``.

    With no process group initialised this is the identity.  Throughput is the
    units all ranks processed divided by the slowest rank's time."""
    import torch

    dist = _dist()
    if dist is None:
        return local_units, local_seconds
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(u.item()), float(t.item())


# ----------------------------------------------------------------- Jacobi --

class JacobiRowBlocks:
    """One rows x cols Jacobi problem split by rows over ``world`` ranks.

    Rank r owns the interior rows [lo, hi) of the block partition of
    [1, rows - 1) and holds a slab of the grid's rows [lo - 1, hi + 1): its
    own rows plus one halo row above and one below (the global boundary rows
    for the first and last rank).  Local row k is global row lo - 1 + k.
    A rank with no rows (more ranks than interior rows) holds no slab and
    takes part in the collectives only.

    A sweep on a rank computes its own rows of ``dst`` from ``src`` (local
    rows [1, local_rows - 1), all interior columns) and its local max
    residual; then ``exchange(dst)`` sends the first own row up and the last
    own row down and receives the neighbours' rows into the halo rows.  As
    in the one-rank region, both ping-pong buffers start as the same grid
    (boundary included), so the boundary never has to move."""

    def __init__(self, rows: int, cols: int, world: int, rank: int, group=None):
        self.rows, self.cols, self.world, self.rank, self.group = rows, cols, world, rank, group
        self.lo, self.hi = block_range(1, rows - 1, world, rank)
        self.active = min(world, max(rows - 2, 0))  # ranks that own rows: a prefix 0..active-1
        self.local_rows = self.hi - self.lo + 2 if self.hi > self.lo else 0
        self.up = rank - 1 if 0 < rank < self.active else None
        self.down = rank + 1 if rank + 1 < self.active else None

    # the slab of a full grid (host set-up and tests)
    def slab(self, grid):
        return grid[self.lo - 1:self.hi + 1] if self.local_rows else grid[0:0]

    def owned(self, local):
        """The slab's own rows (local rows [1, local_rows - 1))."""
        return local[1:self.local_rows - 1] if self.local_rows else local[0:0]

    def exchange(self, buf) -> None:
        """Halo exchange on a local slab (a contiguous 2D torch tensor): own
        first row to the rank above and own last row to the rank below, the
        neighbours' rows received in place into the halo rows.  All messages
        of a step are posted together."""
        dist = _dist()
        if dist is None or self.local_rows == 0:
            return
        ops = []
        last = self.local_rows - 2
        if self.up is not None:
            ops.append(dist.P2POp(dist.isend, buf[1].contiguous(), self.up, self.group))
            ops.append(dist.P2POp(dist.irecv, buf[0], self.up, self.group))
        if self.down is not None:
            ops.append(dist.P2POp(dist.isend, buf[last].contiguous(), self.down, self.group))
            ops.append(dist.P2POp(dist.irecv, buf[last + 1], self.down, self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()

    def combine_residuals(self, res) -> None:
        """Per-sweep residual maxima over all ranks, in place (a rank without
        rows contributes -inf, the identity of max).  One allreduce covers all
        sweeps: a residual does not steer the sweeps, and max does not depend
        on the order in which the ranks' maxima are combined."""
        dist = _dist()
        if dist is not None and self.world > 1:
            dist.all_reduce(res, op=dist.ReduceOp.MAX, group=self.group)

    def run(self, sweep: Callable, buf_a, buf_b, sweeps: int, res) -> object:
        """``sweeps`` sweeps with ping-pong slabs; ``sweep(src, dst, k)``
        updates the own rows of ``dst`` from ``src`` and writes this rank's
        max residual of sweep k into ``res[k]`` (a rank without rows is not
        called and leaves -inf there).  Returns the slab holding the result."""
        src, dst = buf_a, buf_b
        if self.up is None and self.down is None and self.local_rows and hasattr(sweep, "all_sweeps"):
            # no neighbour to exchange with: every sweep in one submission
            sweep.all_sweeps()
            if sweeps % 2:
                src, dst = dst, src
        else:
            for k in range(sweeps):
                if self.local_rows:
                    sweep(src, dst, k)
                self.exchange(dst)
                src, dst = dst, src
        self.combine_residuals(res)
        return src

    def gather(self, local, out=None):
        """The full grid on every rank from the own rows of every rank (plus
        the first and last boundary rows, taken from the first and last
        active ranks' halo rows).  Test and check helper, not a step."""
        import torch

        dist = _dist()
        if dist is None or self.world == 1:
            return local.clone() if out is None else out.copy_(local)
        blk = max(block_range(1, self.rows - 1, self.world, 0)[1] - 1, 0)
        piece = torch.zeros((blk + 2, self.cols), dtype=local.dtype, device=local.device)
        if self.local_rows:
            piece[:self.local_rows] = local
        parts = [torch.empty_like(piece) for _ in range(self.world)]
        dist.all_gather(parts, piece, group=self.group)
        full = torch.empty((self.rows, self.cols), dtype=local.dtype, device=local.device) if out is None else out
        for r in range(self.active):
            lo, hi = block_range(1, self.rows - 1, self.world, r)
            full[lo:hi] = parts[r][1:hi - lo + 1]
            if r == 0:
                full[0] = parts[r][0]
            if r == self.active - 1:
                full[self.rows - 1] = parts[r][hi - lo + 1]
        return full


# ----------------------------------------------------------------- matvec --

class MatvecRowBlocks:
    """y = A x with the rows of A split over the ranks and x replicated.

    Rank r owns rows [lo, hi) of the block partition of [0, rows) and
    computes those entries of y; ``gather`` assembles y on every rank."""

    def __init__(self, rows: int, cols: int, world: int, rank: int, group=None):
        self.rows, self.cols, self.world, self.rank, self.group = rows, cols, world, rank, group
        self.lo, self.hi = block_range(0, rows, world, rank)

    def block(self, a):
        return a[self.lo:self.hi]

    def replicate_x(self, x, src: int = 0):
        """x from rank ``src`` to every rank (when only one rank holds it)."""
        dist = _dist()
        if dist is not None and self.world > 1:
            dist.broadcast(x, src, group=self.group)
        return x

    def gather(self, y_local):
        import torch

        dist = _dist()
        if dist is None or self.world == 1:
            return y_local.clone()
        blk = block_range(0, self.rows, self.world, 0)[1]
        piece = torch.zeros(blk, dtype=y_local.dtype, device=y_local.device)
        piece[:self.hi - self.lo] = y_local
        parts = [torch.empty_like(piece) for _ in range(self.world)]
        dist.all_gather(parts, piece, group=self.group)
        out = torch.empty(self.rows, dtype=y_local.dtype, device=y_local.device)
        for r in range(self.world):
            lo, hi = block_range(0, self.rows, self.world, r)
            out[lo:hi] = parts[r][:hi - lo]
        return out


# ------------------------------------------------------------ AXPY + sum --

class AxpyBlocks:
    """AXPY + reduction(+) split into a block of iterations per rank.

    Each rank runs the loop on its block and reduces into its own FP32
    variable (starting from 0); ``combine_sum`` gathers the N per-rank sums
    in rank order and hands them to ``fold(parts, init)``, which adds them in
    that order, with compensation, to the variable's value from before the
    loop: the result does not depend on message timing.  On GPUs the fold is
    the runtime's own reduction (``UpirSumFold``).  Integer reductions
    combine exactly with one allreduce(sum)."""

    def __init__(self, n: int, world: int, rank: int, group=None):
        self.n, self.world, self.rank, self.group = n, world, rank, group
        self.lo, self.hi = block_range(0, n, world, rank)

    def combine_sum(self, local_sum, init: float, fold: Callable):
        """local_sum: a one-element FP32 tensor holding this rank's sum.
        Returns fold(the N sums as one tensor in rank order, init)."""
        import torch

        dist = _dist()
        if dist is None or self.world == 1:
            parts = local_sum.reshape(1)
        else:
            parts = torch.empty(self.world, dtype=local_sum.dtype, device=local_sum.device)
            dist.all_gather(list(parts.split(1)), local_sum.reshape(1), group=self.group)
        return fold(parts, init)

    def combine_int(self, local):
        dist = _dist()
        if dist is not None and self.world > 1:
            dist.all_reduce(local, op=dist.ReduceOp.SUM, group=self.group)
        return local


class UpirSumFold:
    """The fold of ``AxpyBlocks.combine_sum`` on the GPU, through the region
    runtime: the N per-rank sums as the y of an AXPY loop with a = 0 (which
    leaves them unchanged) whose reduction(+) of y, compensated and in a
    fixed order, lands in a one-element variable holding ``init``."""

    def __init__(self, ctx: int):
        import paper_2209_10643_b300 as U

        self.U, self.ctx = U, ctx

    def __call__(self, parts, init: float):
        import torch

        U = self.U
        n = parts.numel()
        zeros = torch.zeros(n, dtype=torch.float32, device=parts.device)
        var = torch.full((1,), float(init), dtype=torch.float32, device=parts.device)
        y = parts.to(torch.float32).contiguous().clone()
        torch.cuda.current_stream().synchronize()
        hs = [U.upir_data_map_device(self.ctx, t.data_ptr(), t.numel() * 4) for t in (zeros, y, var)]
        r = U.upir_spmd_region(self.ctx, 0, 0)
        try:
            U.upir_loop_checked(self.ctx, r, U.make_loop_desc(
                lb=0, ub=n, body=U.UPIR_BODY_AXPY, bufs=hs[:2], scalars=[0.0],
                reductions=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_Y, hs[2], 0)]))
            U.upir_region_submit(r, 0)
            U.upir_ctx_wait(self.ctx)
        finally:
            U.upir_region_destroy(r)
            for h in hs:
                U.upir_data_unmap(self.ctx, h)
        return var


# ------------------------------------------------- the GPU side of a rank --

class UpirJacobiSweeper:
    """The per-rank sweep of ``JacobiRowBlocks`` on the GPU, through the
    region runtime: one single-loop region per sweep (JACOBI5 over the
    slab's own rows, its residual into element k of the residual vector),
    recorded once and submitted as a CUDA graph per sweep.

    ``ta``, ``tb`` (the two slabs, local_rows x cols FP32, contiguous) and
    ``tres`` (FP32 [sweeps]) are device tensors that must outlive the sweeper
    (their memory is mapped, not copied); the context's stream must be
    torch's current stream when the exchange runs, so that the halo messages
    are ordered after the sweep that wrote the rows and before the next one."""

    def __init__(self, ctx: int, plan: JacobiRowBlocks, ta, tb, tres, sweeps: int, graph: bool = True):
        import paper_2209_10643_b300 as U

        self.U, self.ctx, self.graph = U, ctx, graph
        self.handles, self.regions, self.whole = [], [], None
        if not plan.local_rows:
            return
        nb = plan.local_rows * plan.cols * 4
        ha = U.upir_data_map_device(ctx, ta.data_ptr(), nb)
        hb = U.upir_data_map_device(ctx, tb.data_ptr(), nb)
        hr = U.upir_data_map_device(ctx, tres.data_ptr(), 4 * sweeps)
        self.handles = [ha, hb, hr]
        def desc(k, hints=()):
            src, dst = (ha, hb) if k % 2 == 0 else (hb, ha)
            return U.make_loop_desc(
                lb=1, ub=plan.local_rows - 1, collapse=2, body=U.UPIR_BODY_JACOBI5, bufs=[src, dst],
                scalars=[plan.local_rows, plan.cols],
                reductions=[(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_RESID, hr, k)], hints=list(hints))

        descs = [desc(k) for k in range(sweeps)]
        # a region per sweep: odd sweeps walk their tiles descending, so that
        # each starts where the previous one ended (what the planner does by
        # itself for consecutive sweeps inside one region)
        for k in range(sweeps):
            r = U.upir_spmd_region(ctx, 0, 0)
            U.upir_loop_checked(ctx, r, desc(k, [(U.UPIR_HINT_TILE_ORDER, 2)] if k % 2 else []))
            self.regions.append(r)
        # every sweep in one region, for a rank with no neighbour (one rank)
        if plan.up is None and plan.down is None:
            self.whole = U.upir_spmd_region(ctx, 0, 0)
            for d in descs:
                U.upir_loop_checked(ctx, self.whole, d)

    def __call__(self, src, dst, k: int) -> None:
        self.U.upir_region_submit(self.regions[k], self.U.UPIR_SUBMIT_GRAPH if self.graph else 0)

    def all_sweeps(self) -> None:
        if self.whole is None:
            raise RuntimeError("all_sweeps: this rank exchanges halo rows between sweeps")
        self.U.upir_region_submit(self.whole, self.U.UPIR_SUBMIT_GRAPH if self.graph else 0)

    def close(self) -> None:
        self.U.upir_ctx_wait(self.ctx)
        for r in self.regions + ([self.whole] if self.whole else []):
            self.U.upir_region_destroy(r)
        self.whole = None
        for h in self.handles:
            self.U.upir_data_unmap(self.ctx, h)
        self.regions, self.handles = [], []


def exchange_in_process(plans: list, bufs: list) -> None:
    """The halo exchange of ``JacobiRowBlocks`` between ranks held by one
    process (each rank's slab a tensor in ``bufs``): the same rows move as
    in ``exchange``, by copies.  For running every rank's share of a
    partitioned problem on one device, one rank after another."""
    for r in range(len(plans) - 1):
        a, b = plans[r], plans[r + 1]
        if not (a.local_rows and b.local_rows):
            continue
        last = a.local_rows - 2
        bufs[r + 1][0].copy_(bufs[r][last])
        bufs[r][last + 1].copy_(bufs[r + 1][1])


# ------------------------------------------------------------------- GEMM --

def rank_grid(world: int) -> tuple[int, int]:
    """(process rows, process columns) for ``world`` ranks: a square grid
    when ``world`` is a square, else one column (row panels)."""
    q = int(round(world ** 0.5))
    return (q, q) if q * q == world else (world, 1)


class GemmPanels:
    """C = A B over a pr x pc grid of ranks, 2D output tiles with A and B
    broadcast one panel at a time (SUMMA).

    Rank r = i pc + j owns C's block (rows block i of [0, M), columns block
    j of [0, N)).  K is split into q = pc panels (q = 1 on a one-column
    grid).  The inputs start distributed as 2D blocks: rank (i, j) holds
    A[rows_i, panel_j] and B[panel_i, cols_j] (on a one-column grid, A's row
    block and all of B).  Step p broadcasts A[rows_i, panel_p] from rank
    (i, p) along process row i and B[panel_p, cols_j] from rank (p, j) along
    process column j; every rank adds A_ip B_pj into its block.  The panels
    are added in order p = 0, 1, ..., so a rank's result does not depend on
    message timing."""

    def __init__(self, M: int, N: int, K: int, world: int, rank: int):
        self.M, self.N, self.K, self.world, self.rank = M, N, K, world, rank
        self.pr, self.pc = rank_grid(world)
        self.i, self.j = divmod(rank, self.pc)
        self.rows = block_range(0, M, self.pr, self.i)
        self.cols = block_range(0, N, self.pc, self.j)
        self.q = self.pc
        self.row_groups = self.col_groups = None

    def panel(self, p: int) -> tuple[int, int]:
        return block_range(0, self.K, self.q, p)

    def make_groups(self) -> None:
        """Process-row and process-column groups (every rank creates every
        group, in the same order)."""
        dist = _dist()
        if dist is None or self.world == 1:
            return
        rows = [dist.new_group([i * self.pc + j for j in range(self.pc)]) for i in range(self.pr)]
        cols = [dist.new_group([i * self.pc + j for i in range(self.pr)]) for j in range(self.pc)]
        self.row_groups, self.col_groups = rows, cols

    def a_local(self, A):
        k0, k1 = self.panel(self.j)
        return A[self.rows[0]:self.rows[1], k0:k1]

    def b_local(self, B):
        k0, k1 = self.panel(self.i) if self.q > 1 else (0, self.K)
        return B[k0:k1, self.cols[0]:self.cols[1]]

    def run(self, gemm_acc: Callable, a_mine, b_mine, c_local, new_panel: Callable) -> None:
        """``gemm_acc(a_p, b_p, c, first)`` computes c = a_p b_p (first) or
        c += a_p b_p; ``new_panel(shape, like)`` makes a receive buffer.  On a
        one-column grid there is one panel and no message."""
        dist = _dist()
        if self.q == 1 or dist is None:
            gemm_acc(a_mine, b_mine, c_local, True)
            return
        for p in range(self.q):
            k0, k1 = self.panel(p)
            a_p = a_mine if p == self.j else new_panel((self.rows[1] - self.rows[0], k1 - k0), a_mine)
            b_p = b_mine if p == self.i else new_panel((k1 - k0, self.cols[1] - self.cols[0]), b_mine)
            dist.broadcast(a_p, self.i * self.pc + p, group=self.row_groups[self.i])
            dist.broadcast(b_p, p * self.pc + self.j, group=self.col_groups[self.j])
            gemm_acc(a_p, b_p, c_local, p == 0)

    def gather(self, c_local):
        """The full C on every rank (test and check helper, not a step)."""
        import torch

        dist = _dist()
        if dist is None or self.world == 1:
            return c_local.clone()
        bm = block_range(0, self.M, self.pr, 0)[1]
        bn = block_range(0, self.N, self.pc, 0)[1]
        piece = torch.zeros((bm, bn), dtype=c_local.dtype, device=c_local.device)
        piece[:c_local.shape[0], :c_local.shape[1]] = c_local
        parts = [torch.empty_like(piece) for _ in range(self.world)]
        dist.all_gather(parts, piece)
        out = torch.empty((self.M, self.N), dtype=c_local.dtype, device=c_local.device)
        for r in range(self.world):
            i, j = divmod(r, self.pc)
            r0, r1 = block_range(0, self.M, self.pr, i)
            c0, c1 = block_range(0, self.N, self.pc, j)
            out[r0:r1, c0:c1] = parts[r][:r1 - r0, :c1 - c0]
        return out


class UpirGemmAcc:
    """The per-rank step of ``GemmPanels`` on the GPU, through the region
    runtime: c = a b by the FP32 GEMM loop, or for a later panel t = a b
    followed by c += t as an AXPY loop with a = 1 (one rounding per element,
    the panels added in order).  Tensors are FP32, row-major, contiguous, on
    the device of the context, whose stream must be torch's current stream."""

    def __init__(self, ctx: int):
        import paper_2209_10643_b300 as U

        self.U, self.ctx, self.tmp = U, ctx, None

    def _map(self, t):
        return self.U.upir_data_map_device(self.ctx, t.data_ptr(), t.numel() * 4)

    def __call__(self, a, b, c, first: bool) -> None:
        import torch

        U = self.U
        m, k = a.shape
        n = b.shape[1]
        out = c
        if not first:
            if self.tmp is None or self.tmp.numel() < m * n:
                self.tmp = torch.empty(m * n, dtype=torch.float32, device=c.device)
            out = self.tmp[:m * n].view(m, n)
        ha, hb, ho = self._map(a), self._map(b), self._map(out)
        hs = [ha, hb, ho]
        r = U.upir_spmd_region(self.ctx, 0, 0)
        try:
            U.upir_loop_checked(self.ctx, r, U.make_loop_desc(lb=0, ub=m, collapse=2, body=U.UPIR_BODY_GEMM_F32,
                                                              bufs=[ha, hb, ho], scalars=[m, n, k]))
            if not first:
                hc = self._map(c)
                hs.append(hc)
                U.upir_loop_checked(self.ctx, r, U.make_loop_desc(lb=0, ub=m * n, body=U.UPIR_BODY_AXPY,
                                                                  bufs=[ho, hc], scalars=[1.0]))
            U.upir_region_submit(r, 0)
            U.upir_ctx_wait(self.ctx)
        finally:
            U.upir_region_destroy(r)
            for h in hs:
                U.upir_data_unmap(self.ctx, h)
