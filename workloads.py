"""Seeded synthetic inputs for the blaz compressed-matrix hot path.

This module holds no arithmetic of the method: it only draws matrices and
request streams.  Both the CUDA library's tests/benchmark and the CPU oracle
consume exactly the arrays produced here.

Workloads (Sec. IV of the paper measures on discretised smooth functions; the
shapes and value distributions below stand in for them):

* ``plain_pair()``: two 256x256 smooth fields,
  A[i,j] = sin(2 pi i/64) cos(2 pi j/48) + 1e-3 N(0,1) (seed 0) and
  B[i,j] = sin(2 pi i/40) cos(2 pi j/72) + 1e-3 N(0,1) (seed 1).
* ``bump_field(n, seed)``: an n x n sum of 16 Gaussian bumps (centres uniform
  in [0,n)^2, widths uniform in [0.02, 0.2] n, amplitudes N(0,1)) plus
  1e-4 N(0,1) noise; seed n for A and n+1 for B.
* ``smoothed_normal(n, seed)``: N(0,1) entries smoothed by a 5x5 box filter
  with periodic wrap (dense right-hand operand of the matrix product).
* ``paper_function(k, n)``: the six test functions f1..f6 of Fig. 6 sampled
  on [-2,2]^2 (Table I).
* ``batch_ops(count, seed)``: mixed-operation batch descriptors.
* ``poisson_requests(...)``: a served request stream.
"""
from __future__ import annotations

import math

import numpy as np


def plain_pair():
    """The small two-field case (256 x 256)."""
    i = np.arange(256, dtype=np.float64)[:, None]
    j = np.arange(256, dtype=np.float64)[None, :]
    ra = np.random.default_rng(0)
    rb = np.random.default_rng(1)
    A = np.sin(2 * np.pi * i / 64) * np.cos(2 * np.pi * j / 48) + 1e-3 * ra.standard_normal((256, 256))
    B = np.sin(2 * np.pi * i / 40) * np.cos(2 * np.pi * j / 72) + 1e-3 * rb.standard_normal((256, 256))
    return np.ascontiguousarray(A), np.ascontiguousarray(B)


def _bump_params(n: int, seed: int, nbumps: int = 16):
    rng = np.random.default_rng(seed)
    cy = rng.uniform(0, n, nbumps)
    cx = rng.uniform(0, n, nbumps)
    w = rng.uniform(0.02, 0.2, nbumps) * n
    amp = rng.standard_normal(nbumps)
    return rng, cy, cx, w, amp


def bump_field(n: int, seed: int, rows: int | None = None, noise: float = 1e-4):
    """n x n (or rows x n) smooth field: 16 Gaussian bumps plus white noise.

    Each bump is separable, exp(-r^2/(2w^2)) = g(y) g(x), so the field is a
    sum of 16 outer products; evaluated in float64 on the host."""
    rows = n if rows is None else rows
    rng, cy, cx, w, amp = _bump_params(n, seed)
    y = np.arange(rows, dtype=np.float64)
    x = np.arange(n, dtype=np.float64)
    out = np.zeros((rows, n))
    for b in range(len(amp)):
        gy = amp[b] * np.exp(-((y - cy[b]) ** 2) / (2 * w[b] ** 2))
        gx = np.exp(-((x - cx[b]) ** 2) / (2 * w[b] ** 2))
        out += np.outer(gy, gx)
    out += noise * rng.standard_normal((rows, n))
    return out


def bump_field_torch(n: int, seed: int, device, rows: int | None = None, noise: float = 1e-4):
    """Same field law as ``bump_field`` drawn directly in device memory with
    torch (bump parameters from the same numpy stream; the white noise from a
    torch generator seeded with ``seed``).  Used for the large sizes where a
    host round trip would dominate set-up time."""
    import torch

    rows = n if rows is None else rows
    _, cy, cx, w, amp = _bump_params(n, seed)
    y = torch.arange(rows, dtype=torch.float64, device=device)
    x = torch.arange(n, dtype=torch.float64, device=device)
    out = torch.zeros((rows, n), dtype=torch.float64, device=device)
    for b in range(len(amp)):
        gy = float(amp[b]) * torch.exp(-((y - float(cy[b])) ** 2) / (2 * float(w[b]) ** 2))
        gx = torch.exp(-((x - float(cx[b])) ** 2) / (2 * float(w[b]) ** 2))
        out.addr_(gy, gx)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    out.add_(torch.randn((rows, n), generator=g, dtype=torch.float64, device=device), alpha=noise)
    return out


def smoothed_normal(rows: int, cols: int, seed: int = 7):
    """N(0,1) entries smoothed by a 5x5 box filter with periodic wrap."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal((rows, cols))
    acc = np.zeros_like(z)
    for di in range(-2, 3):
        for dj in range(-2, 3):
            acc += np.roll(np.roll(z, di, axis=0), dj, axis=1)
    return acc / 25.0


def paper_function(k: int, n: int):
    """M_k[i,j] = f_k(x_j, y_i) on an n x n grid of [-2,2]^2 (Fig. 6, Table I)."""
    t = np.linspace(-2.0, 2.0, n)
    x = t[None, :]
    y = t[:, None]
    r2 = x * x + y * y
    if k == 1:
        return x * y + 0 * y
    if k == 2:
        return x * y / (1 + r2)
    if k == 3:
        return x * x - y
    if k == 4:
        return (x * x) * (y * y)
    if k == 5:
        return np.cos(np.sqrt(r2))
    if k == 6:
        return np.cos(r2) * np.exp(-0.1 * r2)
    raise ValueError(k)


def random_block_matrix(rows: int, cols: int, seed: int, kind: str = "smooth"):
    """Small matrices for parity tests: smooth fields, rough noise, constant
    blocks, special values."""
    rng = np.random.default_rng(seed)
    if kind == "smooth":
        i = np.arange(rows)[:, None]
        j = np.arange(cols)[None, :]
        return np.sin(i / 7.0 + rng.uniform()) * np.cos(j / 11.0) + 1e-3 * rng.standard_normal((rows, cols))
    if kind == "noise":
        return rng.standard_normal((rows, cols)) * 10.0 ** rng.integers(-3, 4)
    if kind == "wide":
        return rng.standard_normal((rows, cols)) * 10.0 ** rng.integers(-30, 30, size=(rows, cols)).astype(float)
    raise ValueError(kind)


OP_MIX = (("compress", 0.40), ("add", 0.30), ("scale", 0.15), ("dot", 0.10), ("matmul", 0.05))


def _side(rng, lo: int, hi: int) -> int:
    v = math.exp(rng.uniform(math.log(lo), math.log(hi)))
    return int(max(lo, min(hi, 8 * round(v / 8))))


def batch_ops(count: int = 2000, seed: int = 11, lo: int = 64, hi: int = 2048):
    """Mixed-op batch: list of dicts {op, rows, cols, m (matmul), c (scale)}."""
    rng = np.random.default_rng(seed)
    names = [o for o, _ in OP_MIX]
    probs = np.array([p for _, p in OP_MIX])
    ops = []
    for _ in range(count):
        op = names[rng.choice(len(names), p=probs)]
        d = {"op": op, "rows": _side(rng, lo, hi), "cols": _side(rng, lo, hi), "seed": int(rng.integers(1 << 31))}
        if op == "matmul":
            d["m"] = _side(rng, lo, hi)
        if op == "scale":
            d["c"] = float(rng.uniform(-4, 4))
        ops.append(d)
    return ops


def poisson_requests(rate: float = 5000.0, duration_s: float = 1.0, seed: int = 13, lo: int = 64,
                     hi: int = 4096, max_requests: int = 50000):
    """Arrival times (s) and op descriptors of a Poisson request stream."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    names = [o for o, _ in OP_MIX]
    probs = np.array([p for _, p in OP_MIX])
    while len(out) < max_requests:
        t += rng.exponential(1.0 / rate)
        if t > duration_s:
            break
        op = names[rng.choice(len(names), p=probs)]
        d = {"t": t, "op": op, "rows": _side(rng, lo, hi), "cols": _side(rng, lo, hi),
             "seed": int(rng.integers(1 << 31))}
        if op == "matmul":
            d["m"] = _side(rng, lo, hi)
        if op == "scale":
            d["c"] = float(rng.uniform(-4, 4))
        out.append(d)
    return out
