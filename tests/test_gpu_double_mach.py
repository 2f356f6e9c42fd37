"""Double Mach reflection (the test of Sec. 11 of that name): a Mach-10 shock
at 30 degrees to a reflecting wall, gamma 1.4, pre-shock rho 1.4 and p 1,
domain 4 x 1, with contact steepening, flattening and the diffusive flux on, as
the paper runs it.  Boundaries as stated there: lower y and right x reflecting,
left x inflowing (post-shock state), upper y following the exact shock line
x_s(y, t) = 1/6 + (y + 20 t)/sqrt(3).  The ghost zones are the caller's
(Dirichlet ghosts, the paper's patch model): one numpy fill for both sides.

* FP64 GPU sweeps bit-identical to the oracle's over 25 steps (96 x 24).
* FP32 on 384 x 96 to t = 0.205: the shock's rightmost extent near x = 3,
  which the paper gives for that time (the incident shock reaches
  x_s(1, 0.205) = 3.11 on the upper boundary)."""
import math

import numpy as np
import pytest

import oracle
import paper_1307_2265_gb300 as ez
from gpu_helpers import batch_from_patches, gpu_patches
from paper_1307_2265_gb300 import synth

pytestmark = pytest.mark.gpu
G = 1.4
NG = 3
PRE = (1.4, 0.0, 0.0, 1.0)                                        # rho, u, v, p
POST = (8.0, 8.25 * math.cos(math.pi / 6), -8.25 * math.sin(math.pi / 6), 116.5)
OPT = 7                                                           # steepen | flatten | diffuse


def _cons(rho, u, v, p):
    w = np.zeros_like(rho)
    return synth.prims_to_conserved(rho, u, v, w, p, G)


def _state_where(mask, shape):
    out = []
    for a, b in zip(POST, PRE):
        out.append(np.where(mask, a, b) * np.ones(shape))
    return out


def _initial(nx, ny):
    dx = 4.0 / nx
    x = (np.arange(nx + 2 * NG) - NG + 0.5) * dx
    y = (np.arange(ny + 2 * NG) - NG + 0.5) * (1.0 / ny)
    X, Y = np.meshgrid(x, y, indexing="xy")
    post = X < 1.0 / 6.0 + Y / math.sqrt(3.0)
    prims = _state_where(post, X.shape)
    U = _cons(*[f.reshape(1, ny + 2 * NG, nx + 2 * NG) for f in prims])
    # one z cell: copy the plane into the z ghost layers
    return [np.repeat(f, 1 + 2 * NG, axis=0) for f in U], x, y


def _fill(U, x, y, t, nx, ny):
    """Ghosts of the double Mach problem at time t (x first, then y over the
    full x extent, then z as a copy of the plane)."""
    s = slice(NG, NG + ny)
    # left: inflow (post-shock); right: reflecting
    for f, val in zip(U, _cons(*[np.full((1, 1, 1), v) for v in POST])):
        f[:, s, :NG] = val[0, 0, 0]
    for g in range(NG):
        src = NG + nx - 1 - g
        for k, f in enumerate(U):
            f[:, s, NG + nx + g] = -f[:, s, src] if k == 1 else f[:, s, src]
    # bottom: reflecting
    for g in range(NG):
        for k, f in enumerate(U):
            f[:, NG - 1 - g, :] = -f[:, NG + g, :] if k == 2 else f[:, NG + g, :]
    # top: post-shock left of the exact shock line, pre-shock right of it
    for g in range(NG):
        row = NG + ny + g
        post = x < 1.0 / 6.0 + (y[row] + 20.0 * t) / math.sqrt(3.0)
        vals = _cons(*[v.reshape(1, 1, -1) for v in _state_where(post, x.shape)])
        for f, val in zip(U, vals):
            f[:, row, :] = val[0, 0]
    # z: single plane
    for f in U:
        f[:NG] = f[NG]
        f[NG + 1:] = f[NG]


def _sweeps(step):
    order = (0, 1, 2) if step % 2 == 0 else (2, 1, 0)
    done = 0
    for d in order:
        yield d, 7 & ~done & ~(1 << d)
        done |= 1 << d


def _coverage(d, cover, n):
    lo = [0 if (cover >> a) & 1 and a != d else NG for a in range(3)]
    hi = [n[a] + 2 * NG if (cover >> a) & 1 and a != d else NG + n[a] for a in range(3)]
    return lo, hi


def test_double_mach_fp64_matches_oracle():
    nx, ny = 96, 24
    U, x, y = _initial(nx, ny)
    dx = [4.0 / nx, 1.0 / ny, 1.0]
    P = oracle.Params(gamma=G, options=OPT)
    params = ez.Params(gamma=G, precision=ez.FP64, options=OPT)
    ora = [f.copy() for f in U]
    b = batch_from_patches([U], dx)
    t = 0.0
    for step in range(25):
        _fill(ora, x, y, t, nx, ny)
        dt = 0.4 / oracle.cfl_rate(ora, dx, P)
        for d, cover in _sweeps(step):
            lo, hi = _coverage(d, cover, (nx, ny, 1))
            oracle.sweep(ora, dx, d, dt, lo, hi, P)
        g = gpu_patches(b)[0]
        _fill(g, x, y, t, nx, ny)
        for dev, host in zip(b.patch_fields(0), g):
            dev.copy_(__import__("torch").from_numpy(host))
        for d, cover in _sweeps(step):
            ez.ppm_sweep(b, d, dt, cover, params)
        t += dt
    for a, c in zip(gpu_patches(b)[0], ora):
        assert np.array_equal(a[NG:NG + 1, NG:NG + ny, NG:NG + nx], c[NG:NG + 1, NG:NG + ny, NG:NG + nx])


def test_double_mach_shock_reaches_x3_at_t0205():
    import torch
    nx, ny = 384, 96
    U, x, y = _initial(nx, ny)
    dx = [4.0 / nx, 1.0 / ny, 1.0]
    params = ez.Params(gamma=G, precision=ez.FP32, options=OPT)
    b = batch_from_patches([U], dx)
    t, step, t_end = 0.0, 0, 0.205
    while t < t_end - 1e-12:
        g = gpu_patches(b)[0]
        _fill(g, x, y, t, nx, ny)
        for dev, host in zip(b.patch_fields(0), g):
            dev.copy_(torch.from_numpy(host))
        ez.timestep_cfl(b, params, out=b.dt_dev)
        dt = min(float(b.dt_dev.item()), t_end - t)
        for d, cover in _sweeps(step):
            ez.ppm_sweep(b, d, dt, cover, params)
        t += dt
        step += 1
    rho = gpu_patches(b)[0][0][NG, NG:NG + ny, NG:NG + nx]
    xs = x[NG:NG + nx]
    shocked = rho > 1.4 * 1.5
    rightmost = float(xs[np.max(np.nonzero(shocked.any(axis=0)))])
    expect = 1.0 / 6.0 + (1.0 + 20.0 * t_end) / math.sqrt(3.0)
    print(f"\ndouble Mach {nx}x{ny}, t = {t_end}: rightmost shocked cell x = {rightmost:.3f} "
          f"(exact incident shock on the upper boundary {expect:.3f}), {step} steps, max rho {rho.max():.2f}")
    assert abs(rightmost - expect) < 0.1
    assert np.all(np.isfinite(rho)) and rho.min() > 0.0 and rho.max() < 30.0
    assert b.read_status()["nan"] == 0
