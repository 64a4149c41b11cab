"""Learned schedule cost model for worksharing loops, built on the C ABI.

For a loop region the model scores candidate schedules (schedule kind, chunk,
units per team, teams) from 12 features and picks the one it predicts
fastest.  Its training data are timings the runtime measures itself
(exhaustive autotuning of candidate schedules with CUDA events); training runs
on the GPU through the library's MLP forward/backward/SGD kernels.  The
exhaustive autotuner remains the fallback and the reference the model's regret
is measured against.

Features (12): op one-hot (AXPY, JACOBI5, MATVEC, GEMM), log2 trip count,
bytes per iteration, flops per iteration, schedule one-hot (static, dynamic),
log2(chunk + 1), log2 units per team, log2 teams.  A GEMM loop's iterations
are its output elements (bytes per iteration K / 16: the 128 x 128 tile
kernel's operand reads per output; flops 2 K).  Units and teams are the
geometry the planner launches the candidate with; schedule(auto) computes the
same teams for every candidate by planning the loop without device scratch,
so the features the model is trained on are the features it is asked about.
"""
from __future__ import annotations

import math
import statistics

import numpy as np

import paper_2209_10643_b300 as U

OP_AXPY, OP_JACOBI, OP_MATVEC, OP_GEMM = range(4)
NFEAT = 12


def features(op: int, trip: int, bytes_per_iter: float, flops_per_iter: float, sched: int,
             chunk: int, units: int, teams: int) -> np.ndarray:
    f = np.zeros(NFEAT, np.float32)
    f[op] = 1.0
    f[4] = math.log2(max(trip, 1))
    f[5] = bytes_per_iter
    f[6] = flops_per_iter
    f[7 + sched] = 1.0
    f[9] = math.log2(chunk + 1)
    f[10] = math.log2(max(units, 1))
    f[11] = math.log2(max(teams, 1))
    return f


_OP_BODY = {OP_AXPY: U.UPIR_BODY_AXPY, OP_JACOBI: U.UPIR_BODY_JACOBI5, OP_MATVEC: U.UPIR_BODY_MATVEC,
            OP_GEMM: U.UPIR_BODY_GEMM_F32}


def candidates(op: int) -> list[dict]:
    """Candidate schedules per loop kind (teams = 0: the planner sizes the
    grid), the same list the runtime's schedule(auto) ranks."""
    return [dict(sched=sc, chunk=ch, units=un, teams=0) for sc, ch, un in U.upir_auto_candidates(_OP_BODY[op])]


def heuristic(op: int, trip: int) -> dict:
    """The paper's CUDA geometry: 256 units per team, one iteration per unit
    ((n + 255) / 256 teams), static schedule."""
    teams = max(1, min((trip + 255) // 256, 2 ** 31 - 1)) if op == OP_AXPY else 0
    return dict(sched=U.UPIR_SCHED_STATIC, chunk=0, units=256, teams=teams)


class Pool:
    """Device buffers large enough for every problem of a sweep; each problem
    runs on prefixes of them (their values are seeded uniform[-1, 1), which
    is all the timing needs).  GEMM operands take prefixes of the matrix
    buffer (A), the grid buffers (B) and the vector buffer (C)."""

    def __init__(self, ctx: int, max_vec: int, max_grid: int, max_mat: int, seed: int = 11):
        import torch
        g = torch.Generator(device="cuda").manual_seed(seed)

        def buf(n):
            return (torch.rand(max(n, 1), device="cuda", generator=g) * 2 - 1).contiguous()

        self.ctx = ctx
        self.x, self.y = buf(max_vec), buf(max_vec)
        self.u0, self.u1 = buf(max_grid), buf(max_grid)
        self.a = buf(max_mat)
        self.var = torch.zeros(16, device="cuda")
        torch.cuda.synchronize()

    def wrap(self, t, n: int, offset: int = 0) -> int:
        return U.upir_data_map_device(self.ctx, t.data_ptr() + 4 * offset, 4 * n)


class Problem:
    """One region's loop on pool prefixes, run under candidate schedules."""

    def __init__(self, pool: Pool, spec: dict):
        self.ctx, self.spec, self.handles = pool.ctx, spec, []
        op = spec["op"]
        w = lambda t, n, o=0: self._h(pool.wrap(t, n, o))  # noqa: E731
        if op == OP_AXPY:
            n = spec["n"]
            hx, hy, hd = w(pool.x, n), w(pool.y, n), w(pool.var, 1)
            self.loop = dict(lb=0, ub=n, body=U.UPIR_BODY_AXPY, bufs=[hx, hy], scalars=[2.5],
                             reductions=[(U.UPIR_RED_ADD, U.UPIR_F32, U.UPIR_TERM_XY, hd, 0)])
        elif op == OP_JACOBI:
            side = spec["side"]
            h0, h1, hr = w(pool.u0, side * side), w(pool.u1, side * side), w(pool.var, 1, 1)
            self.loop = dict(lb=1, ub=side - 1, collapse=2, body=U.UPIR_BODY_JACOBI5, bufs=[h0, h1],
                             scalars=[side, side],
                             reductions=[(U.UPIR_RED_MAX, U.UPIR_F32, U.UPIR_TERM_RESID, hr, 0)])
        elif op == OP_MATVEC:
            rows, cols = spec["rows"], spec["cols"]
            ha, hx, hy = w(pool.a, rows * cols), w(pool.x, cols), w(pool.y, rows)
            self.loop = dict(lb=0, ub=rows, body=U.UPIR_BODY_MATVEC, bufs=[ha, hx, hy],
                             scalars=[rows, cols])
        else:
            m, n, k = spec["m"], spec["n"], spec["k"]
            ha, hb, hc = w(pool.a, m * k), w(pool.u0, k * n), w(pool.x, m * n)
            self.loop = dict(lb=0, ub=m, collapse=2, body=U.UPIR_BODY_GEMM_F32, bufs=[ha, hb, hc],
                             scalars=[m, n, k])
        self.op, self.trip, self.bpi, self.fpi = spec_shape(spec)

    def _h(self, h):
        self.handles.append(h)
        return h

    def region(self, cand: dict) -> int:
        r = U.upir_spmd_region(self.ctx, cand["teams"], cand["units"])
        try:
            U.upir_loop_checked(self.ctx, r, U.make_loop_desc(**self.loop, sched=cand["sched"],
                                                              chunk=cand["chunk"]))
        except U.UpirError:
            U.upir_region_destroy(r)
            raise
        return r

    def measure(self, cand: dict, reps: int = 3) -> tuple[float, np.ndarray]:
        """Median device time (ms) of the loop under `cand`, and its features
        (with the units and teams the planner launched it with)."""
        r = self.region(cand)
        teams, units = U.upir_region_loop_geometry(r, 0)
        U.upir_region_submit(r, 0)  # warm-up
        U.upir_ctx_set_timing(self.ctx, True)
        for _ in range(reps):
            U.upir_region_submit(r, 0)
        U.upir_ctx_set_timing(self.ctx, False)
        rec = U.upir_ctx_timings(self.ctx)
        U.upir_region_destroy(r)
        ms = statistics.median(t for _, t in rec)
        return ms, features(self.op, self.trip, self.bpi, self.fpi, cand["sched"], cand["chunk"],
                            units, teams)

    def close(self):
        for h in self.handles:
            U.upir_data_unmap(self.ctx, h)
        self.handles.clear()


def sweep(pool: Pool, specs: list[dict], reps: int = 3):
    """Exhaustive autotuning of every candidate schedule of every region.

    Returns per region its (candidate, ms, features) rows and the heuristic's
    (ms, features)."""
    out = []
    for sp in specs:
        pb = Problem(pool, sp)
        rows = []
        for cand in candidates(sp["op"]):
            try:
                ms, f = pb.measure(cand, reps)
            except U.UpirError:
                continue
            rows.append((cand, ms, f))
        try:
            hms, hf = pb.measure(heuristic(sp["op"], pb.trip), reps)
        except U.UpirError:
            hms, hf = float("nan"), None
        pb.close()
        out.append({"spec": sp, "rows": rows, "heuristic": (hms, hf)})
    return out


def gemm_specs(count: int, seed: int) -> list[dict]:
    """FP32 GEMM loops C = A B like the dense workload at log-spaced sizes:
    M, N, K each 2^U(7, 11.5), N and K rounded to multiples of 4 (the tile
    kernel's TMA path), M to a multiple of 8."""
    g = np.random.Generator(np.random.Philox(seed))
    out = []
    for _ in range(count):
        m, n, k = (int(2 ** g.uniform(7, 11.5)) for _ in range(3))
        out.append({"op": OP_GEMM, "m": max(8, m // 8 * 8), "n": max(4, n // 4 * 4), "k": max(4, k // 4 * 4)})
    return out


def training_specs(count: int = 800, seed: int = 10, gemm: int = 0) -> list[dict]:
    """Regions like the AXPY, Jacobi and matvec workloads at log-spaced sizes,
    plus ``gemm`` GEMM loops (seed + 1)."""
    g = np.random.Generator(np.random.Philox(seed))
    specs = []
    for i in range(count):
        op = i % 3
        if op == OP_AXPY:
            specs.append({"op": OP_AXPY, "n": int(2 ** g.uniform(10, 25))})
        elif op == OP_JACOBI:
            specs.append({"op": OP_JACOBI, "side": int(2 ** g.uniform(6, 12))})
        else:
            rows = int(2 ** g.uniform(8, 14))
            cols = int(min(max(2 ** g.uniform(5, 24) // rows, 1), 16384))
            specs.append({"op": OP_MATVEC, "rows": rows, "cols": cols})
    return specs + gemm_specs(gemm, seed + 1)


def dataset(results) -> tuple[np.ndarray, np.ndarray]:
    """Features and log2(time in microseconds) of every measured variant."""
    f = np.stack([r[2] for res in results for r in res["rows"]])
    t = np.array([math.log2(r[1] * 1e3) for res in results for r in res["rows"]], np.float32)
    return f, t


class GpuMLP:
    """The 12-64-64-1 MLP, its parameters and data resident on the GPU,
    trained with the library's kernels.

    Tensors are made by torch on its current stream and consumed by the
    library on the context's stream (and the other way round), so every
    hand-over synchronises the producing stream first."""

    def __init__(self, ctx: int, params: dict):
        import torch
        self.ctx, self.torch = ctx, torch
        flat = np.concatenate([params[k].astype(np.float32).ravel()
                               for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
        assert flat.size == U.UPIR_MLP_NPARAM
        self.p = torch.from_numpy(flat).cuda()
        self.g = torch.zeros_like(self.p)
        self.loss = torch.zeros(1, device="cuda")
        torch.cuda.current_stream().synchronize()

    def params(self) -> dict:
        U.upir_ctx_wait(self.ctx)
        flat = self.p.cpu().numpy()
        sizes = {"W1": (64, 12), "b1": (64,), "W2": (64, 64), "b2": (64,), "W3": (1, 64), "b3": (1,)}
        out, o = {}, 0
        for k, shp in sizes.items():
            n = int(np.prod(shp))
            out[k] = flat[o:o + n].reshape(shp).copy()
            o += n
        return out

    def predict(self, x):
        x = self.torch.as_tensor(x, device="cuda", dtype=self.torch.float32).contiguous()
        y = self.torch.empty(x.shape[0], device="cuda")
        self.torch.cuda.current_stream().synchronize()
        U.upir_mlp_forward(self.ctx, self.p.data_ptr(), x.data_ptr(), x.shape[0], y.data_ptr())
        U.upir_ctx_wait(self.ctx)
        return y

    def full_loss(self, x, t) -> float:
        """Mean squared error over all rows (a backward pass; the gradient is discarded)."""
        self.torch.cuda.current_stream().synchronize()
        U.upir_mlp_backward(self.ctx, self.p.data_ptr(), x.data_ptr(), t.data_ptr(), x.shape[0],
                            self.g.data_ptr(), self.loss.data_ptr())
        U.upir_ctx_wait(self.ctx)
        return float(self.loss.item())

    def step(self, x, t, lr: float) -> None:
        U.upir_mlp_backward(self.ctx, self.p.data_ptr(), x.data_ptr(), t.data_ptr(), x.shape[0],
                            self.g.data_ptr(), self.loss.data_ptr())
        U.upir_mlp_sgd(self.ctx, self.p.data_ptr(), self.g.data_ptr(), lr)

    def train(self, x_np: np.ndarray, t_np: np.ndarray, epochs: int = 300, batch: int = 512,
              lr: float = 0.05, seed: int = 0, log_every: int = 10) -> list[float]:
        """Minibatch SGD with a cosine learning-rate decay.  Returns the
        full-data loss before training and every `log_every` epochs."""
        torch = self.torch
        x = torch.from_numpy(x_np.astype(np.float32)).cuda()
        t = torch.from_numpy(t_np.astype(np.float32)).cuda()
        g = np.random.Generator(np.random.Philox(seed))
        n = x.shape[0]
        losses = [self.full_loss(x, t)]
        for ep in range(epochs):
            perm = torch.from_numpy(g.permutation(n)).cuda()
            xs, ts = x[perm].contiguous(), t[perm].contiguous()
            torch.cuda.current_stream().synchronize()  # the shuffled copies exist
            lr_ep = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))  # cosine decay
            for s in range(0, n, batch):
                m = min(batch, n - s)
                U.upir_mlp_backward(self.ctx, self.p.data_ptr(), xs.data_ptr() + 4 * NFEAT * s,
                                    ts.data_ptr() + 4 * s, m, self.g.data_ptr(), self.loss.data_ptr())
                U.upir_mlp_sgd(self.ctx, self.p.data_ptr(), self.g.data_ptr(), lr_ep)
            U.upir_ctx_wait(self.ctx)  # xs, ts stay alive until the kernels are done
            if (ep + 1) % log_every == 0 or ep == epochs - 1:
                losses.append(self.full_loss(x, t))
        return losses


def install(ctx: int, model: "GpuMLP", mean: np.ndarray, std: np.ndarray) -> None:
    """Make a trained model the one the context's schedule(auto) consults."""
    p = model.params()
    flat = np.concatenate([p[k].astype(np.float32).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    U.upir_ctx_set_cost_model(ctx, flat, np.asarray(mean, np.float32),
                              np.where(np.asarray(std) > 0, std, 1.0).astype(np.float32))


def standardize(f: np.ndarray, mean=None, std=None):
    if mean is None:
        mean, std = f.mean(axis=0), f.std(axis=0)
        std = np.where(std > 0, std, 1.0)
    return ((f - mean) / std).astype(np.float32), mean, std


def regret_report(results, model: GpuMLP, mean, std) -> dict:
    """Per region: the model's pick (argmin of predictions over the measured
    candidates) against the exhaustive best, and the heuristic likewise."""
    regrets, h_regrets, ops = [], [], []
    for res in results:
        rows = res["rows"]
        if not rows:
            continue
        f = np.stack([r[2] for r in rows])
        pred = model.predict(standardize(f, mean, std)[0]).cpu().numpy()
        times = np.array([r[1] for r in rows])
        best = times.min()
        regrets.append(times[int(np.argmin(pred))] / best - 1.0)
        ops.append(res["spec"]["op"])
        hms = res["heuristic"][0]
        if not math.isnan(hms):
            h_regrets.append(hms / best - 1.0)
    r = np.array(regrets)
    h = np.array(h_regrets)
    ops = np.array(ops)

    def stats(v):
        return {"mean": float(v.mean()), "median": float(np.median(v)), "p90": float(np.quantile(v, 0.9))}

    names = {OP_AXPY: "axpy", OP_JACOBI: "jacobi", OP_MATVEC: "matvec", OP_GEMM: "gemm"}
    return {"regions": int(r.size),
            "model_regret": stats(r),
            "model_regret_by_op": {names[o]: dict(stats(r[ops == o]), regions=int((ops == o).sum()))
                                   for o in sorted(set(ops.tolist()))},
            "heuristic_regret": stats(h) if h.size else None}


def spec_shape(spec: dict) -> tuple[int, int, float, float]:
    """(op, trip, bytes per iteration, flops per iteration) of a region spec,
    as ``Problem`` and the runtime's features count them."""
    op = spec["op"]
    if op == OP_AXPY:
        return op, spec["n"], 12.0, 4.0
    if op == OP_JACOBI:
        return op, (spec["side"] - 2) ** 2, 8.0, 6.0
    if op == OP_MATVEC:
        return op, spec["rows"], 4.0 * spec["cols"], 2.0 * spec["cols"]
    return op, spec["m"] * spec["n"], spec["k"] / 16.0, 2.0 * spec["k"]


class Trained:
    """A trained model with the feature statistics and target offset it was
    trained with."""

    def __init__(self, model: "GpuMLP", mean, std, tmean: float):
        self.model, self.mean, self.std, self.tmean = model, mean, std, tmean

    def predict_us(self, specs: list[dict]) -> np.ndarray:
        """Predicted time (microseconds) of each region under its best
        candidate schedule: the time schedule(auto) expects for it."""
        rows, owner = [], []
        for k, sp in enumerate(specs):
            op, trip, bpi, fpi = spec_shape(sp)
            for c in candidates(op):
                rows.append(features(op, trip, bpi, fpi, c["sched"], c["chunk"], c["units"], c["teams"]))
                owner.append(k)
        pred = self.model.predict(standardize(np.stack(rows), self.mean, self.std)[0]).cpu().numpy() + self.tmean
        best = np.full(len(specs), np.inf)
        np.minimum.at(best, np.array(owner), pred)
        return np.exp2(best)


def pool_for(ctx: int, specs: list[dict]) -> Pool:
    """A pool large enough for every spec of ``specs``."""
    max_vec = max([sp.get("n", 0) for sp in specs] + [sp["m"] * sp["n"] for sp in specs if "m" in sp] + [16384])
    max_grid = max([sp.get("side", 0) ** 2 for sp in specs] + [sp["k"] * sp["n"] for sp in specs if "m" in sp] + [1])
    max_mat = max([sp.get("rows", 0) * sp.get("cols", 0) for sp in specs] +
                  [sp["m"] * sp["k"] for sp in specs if "m" in sp] + [1])
    return Pool(ctx, max_vec, max_grid, max_mat)


def train(ctx: int, pool: Pool, train_specs: list[dict], epochs: int = 300, reps: int = 3):
    """Exhaustive autotuning of the training regions, then the MLP trained
    on the GPU.  Returns the trained model, the training log and timings."""
    import time

    import upir_inputs as I

    t0 = time.perf_counter()
    results = sweep(pool, train_specs, reps)
    t1 = time.perf_counter()
    f, t = dataset(results)
    fs, mean, std = standardize(f)
    tmean = float(t.mean())
    model = GpuMLP(ctx, I.mlp_init(seed=9))
    losses = model.train(fs, t - tmean, epochs=epochs)
    pred = model.predict(fs).cpu().numpy() + tmean
    rmse = float(np.sqrt(np.mean((pred - t) ** 2)))
    t2 = time.perf_counter()
    log = {"variants": int(f.shape[0]), "losses": losses, "rmse_log2": rmse,
           "seconds": {"autotune_train": t1 - t0, "train": t2 - t1}}
    return Trained(model, mean, std, tmean), log


def run_protocol(ctx: int, n_train: int = 950, n_eval: int = 1000, epochs: int = 300, seed_eval: int = 7,
                 eval_t_hi: float = 1e7, reps: int = 3, n_train_gemm: int = 120, n_eval_gemm: int = 100) -> dict:
    """Autotune the training regions exhaustively, train the MLP on the GPU,
    then rank the candidate schedules of unseen regions (drawn like the
    batched-region workload, plus unseen GEMM loops, seed_eval + 5) and
    report its regret against the exhaustive autotuner, overall and per loop
    kind, next to the regret of the paper's default geometry."""
    import time

    import upir_inputs as I

    train_specs = training_specs(n_train, gemm=n_train_gemm)
    eval_specs = I.batched_region_specs(n_eval, seed=seed_eval, t_hi=eval_t_hi) + \
        gemm_specs(n_eval_gemm, seed_eval + 5)
    pool = pool_for(ctx, train_specs + eval_specs)
    tr, log = train(ctx, pool, train_specs, epochs, reps)
    t2 = time.perf_counter()
    ev = sweep(pool, eval_specs, reps)
    t3 = time.perf_counter()

    rep = regret_report(ev, tr.model, tr.mean, tr.std)
    fe, te = dataset(ev)
    pe = tr.model.predict(standardize(fe, tr.mean, tr.std)[0]).cpu().numpy() + tr.tmean
    rep.update({
        "train_regions": len(train_specs), "train_gemm_regions": n_train_gemm,
        "eval_gemm_regions": n_eval_gemm, "train_variants": log["variants"],
        "eval_variants": int(fe.shape[0]), "epochs": epochs,
        "loss_first": log["losses"][0], "loss_last": log["losses"][-1],
        "train_rmse_log2": log["rmse_log2"], "eval_rmse_log2": float(np.sqrt(np.mean((pe - te) ** 2))),
        "seconds": dict(log["seconds"], autotune_eval=t3 - t2),
    })
    return rep
