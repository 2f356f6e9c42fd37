"""GPU test of enzo_ppm_sweep_noalloc, the sweep entry point for callers that
cannot allocate device memory (for instance a host code that owns every device
buffer through its own pool, or one whose memory budget is fixed once time
stepping starts).  It keeps the sweep's scratch in a library-owned device array
instead of a caller workspace.

It must give the same result as enzo_ppm_sweep, the entry point that uses a
caller workspace.  Both run the same kernel, so the FP64 and FP32 outputs must
be bit-identical: the fields, the status words, and where the batch carries
them the flux registers and the gas energy; an FP32 tile size is honoured.
The checks cover several calls in a row, so later calls start from the scratch
contents an earlier call left behind.  This file is
collected last, so a run that stops at the first failure has run every other
test first.  It also passes on its own in a fresh process, because the first
call sets the scratch up.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_1307_2265_gb300 as ez
from gpu_helpers import batch_from_patches, gpu_patches, white_patch, with_registers

pytestmark = pytest.mark.gpu

SIZES = [(1, 1, 1), (3, 2, 5), (17, 5, 33), (40, 8, 8), (9, 9, 9)]


def _pair(flags, seed):
    patches = [white_patch(n, seed=seed + i) for i, n in enumerate(SIZES)]
    dx = [0.05, 0.04, 0.06]
    with_ws = batch_from_patches([[f.copy() for f in U] for U in patches], dx, flags=flags)
    no_ws = batch_from_patches([[f.copy() for f in U] for U in patches], dx, flags=flags)
    return with_ws, no_ws


@pytest.mark.parametrize("precision", [ez.FP64, ez.FP32])
@pytest.mark.parametrize("flags", [0, ez.PATCH_PERIODIC])
def test_noalloc_sweep_matches_workspace_sweep_two_calls(precision, flags):
    with_ws, no_ws = _pair(flags, seed=900 + 10 * precision + flags)
    params = ez.Params(precision=precision)
    ez.ghost_fill_periodic(with_ws)
    ez.ghost_fill_periodic(no_ws)
    dt = 0.4 * ez.timestep_cfl(with_ws, ez.Params(precision=ez.FP64, cfl=1.0))
    # two calls in a row: x sweep covering both transverse axes, then y covering z
    for direction, cover in ((0, 6), (1, 4)):
        ez.ppm_sweep(with_ws, direction, dt, cover, params)
        ez.ppm_sweep_noalloc(no_ws, direction, dt, cover, params)
        for a, b in zip(gpu_patches(with_ws), gpu_patches(no_ws)):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
    assert with_ws.read_status() == no_ws.read_status()


@pytest.mark.parametrize("precision", [ez.FP64, ez.FP32])
def test_noalloc_writes_the_same_flux_registers(precision):
    with_ws, no_ws = (with_registers(b) for b in _pair(0, seed=950 + precision))
    params = ez.Params(precision=precision)
    ez.ghost_fill_periodic(with_ws)
    ez.ghost_fill_periodic(no_ws)
    dt = 0.4 * ez.timestep_cfl(with_ws, ez.Params(precision=ez.FP64, cfl=1.0))
    for direction, cover in ((0, 6), (1, 4), (2, 0)):
        ez.ppm_sweep(with_ws, direction, dt, cover, params)
        ez.ppm_sweep_noalloc(no_ws, direction, dt, cover, params)
    assert torch.count_nonzero(with_ws.freg) > 0
    assert torch.equal(with_ws.freg, no_ws.freg)
    for a, b in zip(gpu_patches(with_ws), gpu_patches(no_ws)):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_noalloc_dual_energy_and_fp32_tile():
    """The gas energy of the dual-energy option, and an FP32 tile of 64 pencils."""
    pairs = []
    for opt in ("dual", "tile"):
        w, n = _pair(ez.PATCH_PERIODIC, seed=970 if opt == "dual" else 980)
        if opt == "dual":
            for b in (w, n):
                rho = torch.where(b.U[0] > 0, b.U[0], torch.ones_like(b.U[0]))   # ghost cells may be empty
                rho_e = b.U[4] - 0.5 * (b.U[1] ** 2 + b.U[2] ** 2 + b.U[3] ** 2) / rho
                b.ge = (rho_e * 1.01).contiguous()
            params = ez.Params(precision=ez.FP32, options=ez.OPT_DUAL)
        else:
            params = ez.Params(precision=ez.FP32, tile=(64, 64, 64))
        pairs.append((w, n, params))
    for w, n, params in pairs:
        dt = 0.4 * ez.timestep_cfl(w, ez.Params(precision=ez.FP64, cfl=1.0))
        for direction in (2, 1, 0):
            ez.ppm_sweep(w, direction, dt, 0, params)
            ez.ppm_sweep_noalloc(n, direction, dt, 0, params)
        for a, b in zip(gpu_patches(w), gpu_patches(n)):
            for x, y in zip(a, b):
                assert np.array_equal(x, y)
        if w.ge is not None:
            assert torch.equal(w.ge, n.ge)
        assert w.read_status() == n.read_status()


def test_noalloc_rejects_batches_above_the_limit():
    b = ez._Batch()
    b.npatch = 32001
    p = ez.Params().c()
    assert ez.lib().enzo_ppm_sweep_noalloc(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(p)) == -3
    assert b"fixed limit" in ez.lib().enzo_strerror(-3)


def test_noalloc_rejects_a_bad_tile_like_the_workspace_sweep():
    b = ez._Batch()
    b.npatch = 0
    p = ez.Params(precision=ez.FP32, tile=(48, 64, 64)).c()
    assert ez.lib().enzo_ppm_sweep_noalloc(ctypes.byref(b), 0, 0.1, 0, ctypes.byref(p)) == -1
