"""Fallback mode 2 (HLL re-flux of cells whose update leaves rho <= 0 or a
non-positive internal energy, Sec. 4.1.2) on the GPU against the oracle:
FP64 bit-identical on a near-vacuum rarefaction (two-shock and HLLC), with and
without the periodic flag, with the oracle's fallback cell count and no
pressure floors; bit-identical to mode 1 on ordinary flow; FP32 on the same
rarefaction floors no pressure, stays finite and conserves."""
import numpy as np
import pytest

import oracle
import paper_1307_2265_gb300 as ez
from gpu_helpers import active, batch_from_patches, gpu_patches, oracle_evolve_batch, white_patch
from paper_1307_2265_gb300 import synth

pytestmark = pytest.mark.gpu
G = 1.4


def _rarefaction(U0=6.0, N=100):
    x = (np.arange(N) + 0.5) / N
    sh = (2, 3, N)
    u = np.broadcast_to(np.where(x < 0.5, -U0, U0), sh).copy()
    z = np.zeros(sh)
    return [synth.embed(f) for f in synth.prims_to_conserved(np.ones(sh), u, z, z, np.full(sh, 0.4), G)]


@pytest.mark.parametrize("solver", [ez.SOLVER_TWOSHOCK, ez.SOLVER_HLLC])
@pytest.mark.parametrize("flags", [0, ez.PATCH_PERIODIC])
def test_mode2_fp64_bitwise_on_a_near_vacuum_rarefaction(solver, flags):
    U = _rarefaction()
    dx = [1.0 / 100, 1e30, 1e30]
    P = oracle.Params(gamma=G, p_floor=1e-10, rho_floor=1e-10, fallback=2, solver=solver)
    ref = [f.copy() for f in U]
    tot = {}
    dts = []
    for s in range(30):
        dt = 0.4 / oracle.cfl_rate(ref, dx, P)
        st = oracle.step_periodic(ref, dx, dt, s, P)
        for k, v in st.items():
            tot[k] = tot.get(k, 0) + v
        dts.append(dt)
    b = batch_from_patches([U], dx, flags=flags)
    params = ez.Params(precision=ez.FP64, gamma=G, p_floor=1e-10, rho_floor=1e-10, fallback=2, solver=solver)
    for s, dt in enumerate(dts):
        b.dt_dev.fill_(dt)
        ez.step(b, params, s, b.dt_dev)
    for a, c in zip(gpu_patches(b)[0], ref):
        assert np.array_equal(active(a), active(c))
    st = b.read_status()
    assert st["hll_cells"] == tot["hll_cells"] and st["p_floor_hits"] == 0 and st["neg_after"] == 0
    if solver == ez.SOLVER_TWOSHOCK:
        assert tot["hll_cells"] > 0


def test_mode2_equals_mode1_on_ordinary_flow():
    patches = [white_patch(n, seed=900 + i) for i, n in enumerate([(24, 16, 12), (9, 30, 5)])]
    dx = [1.0 / 24] * 3
    runs = []
    for mode in (1, 2):
        b = batch_from_patches(patches, dx, flags=ez.PATCH_PERIODIC)
        params = ez.Params(precision=ez.FP64, fallback=mode)
        for s in range(5):
            ez.timestep_cfl(b, params, out=b.dt_dev)
            ez.step(b, params, s, b.dt_dev)
        runs.append(gpu_patches(b))
        assert b.read_status()["hll_cells"] == 0
    for p1, p2 in zip(*runs):
        for a, c in zip(p1, p2):
            assert np.array_equal(active(a), active(c))


@pytest.mark.parametrize("solver", [ez.SOLVER_TWOSHOCK, ez.SOLVER_HLLC])
def test_mode2_fp32_keeps_the_rarefaction_finite(solver):
    U = _rarefaction()
    dx = [1.0 / 100, 1e30, 1e30]
    b = batch_from_patches([U], dx, flags=ez.PATCH_PERIODIC)
    tot0 = [float(active(f).sum()) for f in U]
    params = ez.Params(precision=ez.FP32, gamma=G, p_floor=1e-10, rho_floor=1e-10, fallback=2, solver=solver)
    for s in range(30):
        ez.timestep_cfl(b, params, out=b.dt_dev)
        ez.step(b, params, s, b.dt_dev)
    st = b.read_status()
    assert st["nan"] == 0 and st["p_floor_hits"] == 0 and st["neg_after"] == 0
    g = gpu_patches(b)[0]
    assert float(active(g[0]).min()) > 0.0
    for f, t0 in zip(g, tot0):
        assert abs(float(active(f).sum()) - t0) <= 1e-12 * max(1.0, float(np.abs(active(f)).sum()))


def test_mode2_noalloc_sweep_matches_the_batch_sweep():
    U = _rarefaction()
    dx = [1.0 / 100, 1e30, 1e30]
    a = batch_from_patches([U], dx, flags=ez.PATCH_PERIODIC)
    c = batch_from_patches([U], dx, flags=ez.PATCH_PERIODIC)
    p = ez.Params(precision=ez.FP32, gamma=G, p_floor=1e-10, rho_floor=1e-10, fallback=2,
                  options=ez.OPT_STEEPEN | ez.OPT_FLATTEN)
    dt = 0.4 / oracle.cfl_rate(U, dx, oracle.Params(gamma=G))
    for d in (0, 1, 2):
        ez.ppm_sweep(a, d, dt, 0, p)
        ez.ppm_sweep_noalloc(c, d, dt, 0, p)
    for x, y in zip(a.U, c.U):
        assert bool((x == y).all())
    assert a.read_status() == c.read_status()
