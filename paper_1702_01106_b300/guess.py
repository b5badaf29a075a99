"""Training driver for the learned initial guess (host orchestration only).

Collects (features, targets) from converged stages of the library's own
float64 solver, fits the standardisation and runs the device Adam steps with
a step-decayed learning rate.  Every step of data generation and training
runs in libgrim's kernels.
"""
from __future__ import annotations

import torch

from .grim import MLP, Grim, GRIM_FP64


def collect(prob, P, dt: float, steps: int, device, tol: float = 1e-12, stride: int = 1):
    """Features [M, 32] and targets [M, 16] (float32, device) of both stages of
    every stride-th of steps * stride float64 steps from the state P (numpy
    [10, n3, n2, n1]), solved to `tol`; M = 2 * steps * zones.  A stride > 1
    spreads the samples over a longer stretch of the evolution.  Returns
    (X, Y, final state)."""
    g = Grim(prob.with_(tol=tol), precision=GRIM_FP64)
    a = torch.from_numpy(P).to(device)
    half = torch.empty_like(a)
    full = torch.empty_like(a)
    N = prob.zones
    X = torch.empty((2 * steps * N, 32), dtype=torch.float32, device=device)
    Y = torch.empty((2 * steps * N, 16), dtype=torch.float32, device=device)
    k = 0
    for s in range(steps * stride):
        sample = s % stride == 0
        for PE, dts, out in ((a, 0.5 * dt, half), (half, dt, full)):
            g.stage(a, PE, dts, out)
            if sample:
                g.mlp_sample(a, out, X[k * N:(k + 1) * N], Y[k * N:(k + 1) * N])
                k += 1
        a, full = full, a
    g.close()
    return X, Y, a


def drop_outliers(X, Y, limit: float, sample: int = 1 << 20, seed: int = 1):
    """Rows of (X, Y) whose every feature and target lies within `limit`
    spans of its column's median, the span being the width of the column's
    central 99.8 % (0.1 % to 99.9 % quantiles, over a seeded sample of
    rows).  Zones far outside the bulk (the surface of a torus, whose stage
    residuals reach 1e3) would otherwise set the standardisation and leave
    the bulk's features below bfloat16 resolution; at run time such zones
    fall back to the plain start.  A quantile span rather than the median
    absolute deviation: where most zones are at rest (the atmosphere around
    a torus) the deviation of a velocity or a change is near zero, and it
    would mark the whole torus as outlying."""
    g = torch.Generator(device=X.device).manual_seed(seed)
    idx = torch.randint(0, X.shape[0], (min(sample, X.shape[0]),), device=X.device, generator=g)
    keep = torch.ones(X.shape[0], dtype=torch.bool, device=X.device)
    for A in (X, Y):
        S = A[idx].double().sort(dim=0).values
        n = S.shape[0]
        med = S[n // 2]
        span = S[min(n - 1, int(0.999 * n))] - S[int(0.001 * n)]
        live = span > 0
        dev = ((A.double() - med).abs() / torch.where(live, span, torch.ones_like(span)))[:, live]
        keep &= (dev <= limit).all(dim=1)
    return X[keep].contiguous(), Y[keep].contiguous()


def train(X, Y, steps: int = 6000, batch: int = 4096, lr: float = 3e-3, halvings: int = 3, seed: int = 1):
    """A freshly initialised MLP trained with Adam; the learning rate halves
    `halvings` times at equal intervals.  Returns (mlp, losses per interval)."""
    m = MLP(seed=seed)
    m.fit_norm(X, Y)
    parts = halvings + 1
    losses = []
    for k in range(parts):
        losses.append(m.train(X, Y, steps=steps // parts, batch=batch, lr=lr * 0.5 ** k, seed=seed * 1000 + k))
    return m, losses
