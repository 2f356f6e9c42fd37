"""Training pipeline of the learned Newton guess, run on the GPU with the
library's own kernels.

1. Log traced interface states from the method's own runs:
   enzo_ppm_sweep_logged, FP32 path, plain guess.
2. Compute targets as the converged two-shock p* of those states:
   enzo_riemann_solve in FP64.
3. Compute the features with enzo_mlp_features and train with
   enzo_mlp_train_step (tcgen05 forward/backward, Adam).

PyTorch only holds the tensors, draws minibatch indices and reads scalars.
"""
from __future__ import annotations

import time

import numpy as np

from . import (FP32, FP64, MLP, PatchBatch, Params, mlp_features, patch_table, ppm_sweep_logged,
               riemann_solve, synth, timestep_cfl)


def log_states(batch: PatchBatch, params: Params, nsteps: int, stride: int, cap: int, step0: int = 0):
    """Advance `batch` nsteps steps (periodic patches), logging sampled states."""
    import torch
    log = torch.empty((cap, 6), dtype=torch.float32, device=batch.device)
    count = torch.zeros(1, dtype=torch.int64, device=batch.device)
    for s in range(nsteps):
        dt = timestep_cfl(batch, params)
        order = (0, 1, 2) if (step0 + s) % 2 == 0 else (2, 1, 0)
        for d in order:
            ppm_sweep_logged(batch, d, dt, 0, params, log, count, stride)
    n = min(int(count.item()), cap)
    return log[:n]


def dataset(states, gamma):
    """Features and targets ln(p*/sqrt(pL pR)) with FP64 two-shock roots."""
    import torch
    s64 = [states[:, i].double().contiguous() for i in range(6)]
    o = riemann_solve(*s64, Params(gamma=gamma, precision=FP64))
    ps = o["pstar"]
    scale = torch.maximum(s64[2], s64[5])
    keep = (ps > 1e-12 * scale) & (o["iters"] >= 0)
    s32 = [a[keep].float() for a in s64]
    x = mlp_features(*s32, gamma)
    y = torch.log(ps[keep] / torch.sqrt(s64[2][keep] * s64[5][keep])).float()
    return x, y, s32


def train(x, y, steps=2000, batch=8192, lr=2e-3, lr_final=3e-4, seed=0, holdout=0.05):
    """Adam on minibatches; returns (net, dict of losses)."""
    import torch
    n = x.shape[0]
    nte = max(1, int(holdout * n))
    ntr = n - nte
    net = MLP(seed=seed, device=x.device)
    g = torch.Generator(device=x.device).manual_seed(seed)
    perm = torch.randperm(n, device=x.device, generator=g)
    xtr, ytr = x[perm[:ntr]], y[perm[:ntr]]
    xte, yte = x[perm[ntr:]], y[perm[ntr:]]
    first = None
    t0 = time.perf_counter()
    for it in range(steps):
        frac = it / max(1, steps - 1)
        rate = lr * (lr_final / lr) ** frac
        idx = torch.randint(0, ntr, (min(batch, ntr),), device=x.device, generator=g)
        loss = net.train_step(xtr[idx], ytr[idx], rate)
        if first is None:
            first = float(loss.item())
    torch.cuda.synchronize(x.device)
    secs = time.perf_counter() - t0
    test = float(net.train_step(xte, yte, 0.0).item())
    return net, {"first_loss": first, "test_loss": test, "train_seconds": secs, "samples": n}


def default_training_set(gamma=5.0 / 3.0, device="cuda", stride=16, cap=4_000_000):
    """States logged from a 32^3 white-noise grid (rms Mach 1, 10 steps) and a
    96^3 k^-4 turbulent grid (rms Mach 3, 6 steps), the single-grid recipes at
    reduced size, FP32 path with the plain guess."""
    import torch
    out = []
    for n, recipe, steps, cfg in ((32, "white", 10, 1), (96, "turbulent", 6, 2)):
        U = synth.single_grid((n, n, n), recipe, config=cfg, gamma=gamma)
        table = patch_table([(n, n, n)], [0], [1.0 / n] * 3, flags=1)
        b = PatchBatch(table, [f.ravel() for f in U], device=device)
        out.append(log_states(b, Params(gamma=gamma, precision=FP32), steps, stride, cap))
    return torch.cat(out, dim=0)


def config_training_set(gamma=5.0 / 3.0, device="cuda", target=100_000_000):
    """About `target` states logged from the two single-grid recipes at their
    full sizes: the 32^3 white-noise grid (rms Mach 1, 10 steps, every
    interface) and the 256^3 k^-4 turbulent grid (rms Mach 3, 20 steps, every
    stride-th interface so that the total comes near the target)."""
    import torch
    out = []
    U = synth.single_grid((32, 32, 32), "white", config=1, gamma=gamma)
    b = PatchBatch(patch_table([(32, 32, 32)], [0], [1.0 / 32] * 3, flags=1), [f.ravel() for f in U], device=device)
    out.append(log_states(b, Params(gamma=gamma, precision=FP32), 10, 1, 4_000_000))
    del b
    n, steps = 256, 20
    per_run = 3 * steps * (n + 1) * n * n
    stride = max(1, per_run // max(1, target - out[0].shape[0]))
    U = synth.single_grid((n, n, n), "turbulent", config=2, gamma=gamma)
    b = PatchBatch(patch_table([(n, n, n)], [0], [1.0 / n] * 3, flags=1), [f.ravel() for f in U], device=device)
    del U
    out.append(log_states(b, Params(gamma=gamma, precision=FP32), steps, stride, int(1.2 * per_run / stride) + 1024))
    del b
    torch.cuda.empty_cache()
    return torch.cat(out, dim=0)
