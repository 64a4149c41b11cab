"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and lays them out; it holds none of the
arithmetic of the method (no loop bodies, no schedules, no reductions).  Every
generator uses numpy's counter-based Philox bit generator with a fixed seed, so
the CUDA path and the CPU oracle read the very same host arrays.

Shapes and distributions follow the workloads of the paper's evaluation (§6:
AXPY, matrix-vector product, matrix multiplication and a 2D stencil, all dense
FP32 arrays of the stated sizes), scaled to the sizes the benchmark runs.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def uniform_pm1(n: int, gen: np.random.Generator) -> np.ndarray:
    """FP32 values uniform on [-1, 1), on the 2^-23 grid (exactly representable)."""
    u = gen.random(n, dtype=np.float32)  # multiples of 2^-24 in [0, 1)
    return (np.float32(2.0) * u - np.float32(1.0)).astype(np.float32)


def axpy_inputs(n: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """x then y, both uniform[-1, 1) FP32, drawn from one stream."""
    g = rng(seed)
    x = uniform_pm1(n, g)
    y = uniform_pm1(n, g)
    return x, y


def jacobi_grid(n_rows: int, n_cols: int | None = None, seed: int = 1) -> np.ndarray:
    """FP32 grid: top row (corners included) = 1.0, other edges = 0, interior uniform[0, 1)."""
    n_cols = n_rows if n_cols is None else n_cols
    g = rng(seed)
    u = np.zeros((n_rows, n_cols), dtype=np.float32)
    if n_rows > 2 and n_cols > 2:
        u[1:-1, 1:-1] = g.random((n_rows - 2, n_cols - 2), dtype=np.float32)
    u[0, :] = 1.0
    return u


def matvec_inputs(rows: int, cols: int, seed_a: int = 2, seed_x: int = 3):
    """A ~ N(0, 1) FP32 row-major [rows, cols]; x uniform[-1, 1) FP32 [cols]."""
    a = rng(seed_a).standard_normal((rows, cols), dtype=np.float32)
    x = uniform_pm1(cols, rng(seed_x))
    return a, x


def gemm_inputs(m: int, n: int, k: int, seed_a: int = 4, seed_b: int = 5):
    """A [m, k] and B [k, n] ~ N(0, 1/k) FP32, row-major."""
    s = np.float32(1.0 / math.sqrt(k))
    a = (rng(seed_a).standard_normal((m, k), dtype=np.float32) * s).astype(np.float32)
    b = (rng(seed_b).standard_normal((k, n), dtype=np.float32) * s).astype(np.float32)
    return a, b


def small_int_matrix(rows: int, cols: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """FP32 matrix of integers drawn uniformly from [lo, hi]."""
    return rng(seed).integers(lo, hi + 1, size=(rows, cols)).astype(np.float32)


# --- uneven batches of regions ------------------------------------------------

OP_AXPY_DOT, OP_JACOBI, OP_MATVEC = 0, 1, 2


def batched_region_specs(count: int = 512, seed: int = 6, t_lo: float = 1e3,
                         t_hi: float = 1e7, max_side: int = 2048,
                         max_rows: int = 8192, max_cols: int = 8192) -> list[dict]:
    """Uneven independent regions: 40 % AXPY+dot, 30 % one Jacobi sweep, 30 % matvec.

    The trip count T is log-uniform in [t_lo, t_hi].  AXPY uses n = T; a Jacobi
    sweep uses a square grid of side clamp(round(sqrt T), 64, max_side); a matvec
    draws rows log-uniform in [256, max_rows] and uses cols = clamp(round(T/rows),
    1, max_cols).
    """
    g = rng(seed)
    specs = []
    for r in range(count):
        p = g.random()
        t = int(round(math.exp(g.uniform(math.log(t_lo), math.log(t_hi)))))
        if p < 0.4:
            specs.append({"op": OP_AXPY_DOT, "n": t, "seed": 1000 + r})
        elif p < 0.7:
            side = int(min(max(round(math.sqrt(t)), 64), max_side))
            specs.append({"op": OP_JACOBI, "side": side, "seed": 1000 + r})
        else:
            rows = int(round(math.exp(g.uniform(math.log(256), math.log(max_rows)))))
            cols = int(min(max(round(t / rows), 1), max_cols))
            specs.append({"op": OP_MATVEC, "rows": rows, "cols": cols, "seed": 1000 + r})
    return specs


def region_arrays(spec: dict) -> dict:
    """Host arrays for one batched-region spec."""
    s = spec["seed"]
    if spec["op"] == OP_AXPY_DOT:
        x, y = axpy_inputs(spec["n"], seed=s)
        return {"x": x, "y": y}
    if spec["op"] == OP_JACOBI:
        u = jacobi_grid(spec["side"], seed=s)
        return {"u0": u, "u1": u.copy()}
    a, x = matvec_inputs(spec["rows"], spec["cols"], seed_a=s, seed_x=s + 50000)
    return {"A": a, "x": x}


def mlp_dataset(rows: int, seed: int = 8):
    """Random 12-feature rows and targets for MLP gradient checks."""
    g = rng(seed)
    x = g.standard_normal((rows, 12), dtype=np.float32)
    t = g.standard_normal(rows, dtype=np.float32)
    return x, t


def mlp_init(seed: int = 9, hidden: int = 64, n_in: int = 12) -> dict:
    """He-style random initial weights for the 12-64-64-1 ReLU MLP, FP32."""
    g = rng(seed)

    def w(o, i):
        return (g.standard_normal((o, i), dtype=np.float32)
                * np.float32(math.sqrt(2.0 / i))).astype(np.float32)

    return {
        "W1": w(hidden, n_in), "b1": np.zeros(hidden, np.float32),
        "W2": w(hidden, hidden), "b2": np.zeros(hidden, np.float32),
        "W3": w(1, hidden), "b3": np.zeros(1, np.float32),
    }
