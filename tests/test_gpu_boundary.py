"""External boundaries (Sec. 3.1: reflecting, outflow, periodic) on the GPU
against the oracle: the ghost fill bit for bit on uneven patches for every
combination of conditions, and FP64 steps of a closed (reflecting) box and an
outflow tube bit-identical to the oracle's; the FP32 path conserves mass and
energy in the closed box."""
import itertools

import numpy as np
import pytest

import oracle
import paper_1307_2265_gb300 as ez
from gpu_helpers import active, batch_from_patches, gpu_patches, l1_rel, white_patch
from paper_1307_2265_gb300 import synth

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0
BCS = (ez.BC_PERIODIC, ez.BC_REFLECT, ez.BC_OUTFLOW)


@pytest.mark.parametrize("bc", list(itertools.product(BCS, repeat=3)))
def test_boundary_fill_bitwise(bc):
    patches = [white_patch(n, seed=40 + i, mach=2.0) for i, n in enumerate([(7, 5, 3), (3, 9, 4), (12, 3, 6)])]
    ref = [[f.copy() for f in U] for U in patches]
    for U in ref:
        oracle.fill_boundary(U, bc)
    b = batch_from_patches(patches, [0.1] * 3)
    ez.ghost_fill_boundary(b, bc)
    for g, o in zip(gpu_patches(b), ref):
        for a, c in zip(g, o):
            assert np.array_equal(a, c)


@pytest.mark.parametrize("bc", [(ez.BC_REFLECT, ez.BC_OUTFLOW, ez.BC_PERIODIC),
                                (ez.BC_OUTFLOW, ez.BC_REFLECT, ez.BC_REFLECT)])
def test_boundary_fill_carries_the_gas_energy(bc):
    """With a gas-energy field the boundary fill gives it the oracle's scalar
    fill (mirrored, never negated), bit for bit."""
    import torch
    patches = [white_patch(n, seed=60 + i, mach=2.0) for i, n in enumerate([(7, 5, 3), (3, 9, 4)])]
    ges = [synth.embed(np.random.default_rng(70 + i).uniform(0.5, 2.0, active(U[0]).shape))
           for i, U in enumerate(patches)]
    ref = [[f.copy() for f in U] + [g.copy()] for U, g in zip(patches, ges)]
    for U in ref:
        oracle.fill_boundary(U, bc)
    b = batch_from_patches(patches, [0.1] * 3)
    b.ge = torch.from_numpy(np.concatenate([g.ravel() for g in ges])).to(b.device)
    ez.ghost_fill_boundary(b, bc)
    for i, o in enumerate(ref):
        got = [f.cpu().numpy() for f in b.patch_fields(i)] + [b.patch_ge(i).cpu().numpy()]
        for a, c in zip(got, o):
            assert np.array_equal(a, c)


def _box(nx=24, ny=10, nz=6, seed=11):
    rng = np.random.default_rng(seed)
    shape = (nz, ny, nx)
    rho = np.exp(rng.normal(0, 0.3, shape))
    v = [rng.normal(0, 0.5, shape) for _ in range(3)]
    p = np.exp(rng.normal(0, 0.3, shape))
    return [synth.embed(f) for f in synth.prims_to_conserved(rho, *v, p, G)]


def test_closed_box_fp64_matches_oracle_and_fp32_conserves():
    U = _box()
    n = (24, 10, 6)
    dx = [1.0 / 24] * 3
    bc = (ez.BC_REFLECT,) * 3
    P = oracle.Params(gamma=G)
    ora = [f.copy() for f in U]
    dts = []
    for s in range(10):
        oracle.fill_boundary(ora, bc)
        dt = 0.4 / oracle.cfl_rate(ora, dx, P)
        oracle.step_boundary(ora, dx, dt, s, bc, P)
        dts.append(dt)
    b = batch_from_patches([U], dx)
    b32 = batch_from_patches([U], dx)
    for s, dt in enumerate(dts):
        b.dt_dev.fill_(dt)
        ez.step_boundary(b, ez.Params(gamma=G, precision=ez.FP64), s, b.dt_dev, bc)
        b32.dt_dev.fill_(dt)
        ez.step_boundary(b32, ez.Params(gamma=G, precision=ez.FP32), s, b32.dt_dev, bc)
    for a, c in zip(gpu_patches(b)[0], ora):
        assert np.array_equal(active(a), active(c))
    g32 = gpu_patches(b32)[0]
    for f in (0, 4):
        t0, t1 = float(np.sum(active(U[f]))), float(np.sum(active(g32[f])))
        assert abs(t1 - t0) <= 1e-6 * abs(t0)
    for e in l1_rel(g32, ora):
        assert e <= 1e-4


def test_outflow_tube_fp64_matches_oracle():
    nx = 64
    x = (np.arange(nx) + 0.5) / nx
    bump = 0.05 * np.exp(-((x - 0.7) / 0.08) ** 2)
    shape = (3, 4, nx)
    rho = np.broadcast_to(1.0 + bump, shape).copy()
    p = np.broadcast_to(1.0 + G * bump, shape).copy()
    vx = np.broadcast_to(np.sqrt(G) * bump, shape).copy()
    z = np.zeros(shape)
    U = [synth.embed(f) for f in synth.prims_to_conserved(rho, vx, z, z, p, G)]
    dx = [1.0 / nx, 0.1, 0.1]
    bc = (ez.BC_OUTFLOW, ez.BC_PERIODIC, ez.BC_REFLECT)
    P = oracle.Params(gamma=G)
    ora = [f.copy() for f in U]
    b = batch_from_patches([U], dx)
    for s in range(25):
        oracle.fill_boundary(ora, bc)
        dt = 0.4 / oracle.cfl_rate(ora, dx, P)
        oracle.step_boundary(ora, dx, dt, s, bc, P)
        b.dt_dev.fill_(dt)
        ez.step_boundary(b, ez.Params(gamma=G, precision=ez.FP64), s, b.dt_dev, bc)
    for a, c in zip(gpu_patches(b)[0], ora):
        assert np.array_equal(active(a), active(c))
