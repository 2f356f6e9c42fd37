"""The dual-energy option (Sec. 4.1.1) on the GPU against the oracle.

FP64 is bit-identical to the oracle, fields and gas energy, on:
- ordinary Mach-1 flow, where the pressure never comes from the gas energy and
  the gas energy is resynchronised almost everywhere;
- a cold hypersonic compression, where the pressure always comes from it;
- cold gas at rms Mach 1e4, with thousands of gas-energy pressures;
- violent data where the HLL fallback re-fluxes faces;
- a bulk flow over a density step, where the neighbourhood rule of the
  resynchronisation keeps the advected gas energy beside the dense gas.
The cold flows also run with the reconstruction options on.  FP32 stays within
the FP32 bound on ordinary flow and keeps the entropy of the cold compression
to the oracle's bound.  The ghost fills carry the gas energy."""
import math

import numpy as np
import pytest

import oracle
import paper_1307_2265_gb300 as ez
from gpu_helpers import NG, active, gpu_patches, l1_rel, white_patch
from paper_1307_2265_gb300 import synth

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0
ALL = ez.OPT_STEEPEN | ez.OPT_FLATTEN | ez.OPT_DIFFUSE


def _ge_of(U):
    rho, m1, m2, m3, E = U
    return E - 0.5 * ((m1 * m1 + m2 * m2) + m3 * m3) / rho


def _batch(patches, ges, dx, flags=0):
    sizes, offs, flat = [], [], [[] for _ in range(6)]
    off = 0
    for U, ge in zip(patches, ges):
        nz, ny, nx = U[0].shape
        sizes.append((nx - 2 * NG, ny - 2 * NG, nz - 2 * NG))
        offs.append(off)
        off += U[0].size
        for f in range(5):
            flat[f].append(U[f].ravel())
        flat[5].append(ge.ravel())
    fields = [np.concatenate(f) for f in flat]
    table = ez.patch_table(sizes, offs, dx, flags=flags)
    return ez.PatchBatch(table, fields[:5], ge=fields[5])


def _gpu_ge(b):
    return [b.patch_ge(i).cpu().numpy() for i in range(len(b.table))]


def _run_both(patches, ges, dx, dts, options, precision=ez.FP64, flags=0, p_floor=1e-30, rho_floor=1e-30):
    """Oracle and GPU over the same dt sequence; returns (oracle fields, oracle
    ge, oracle stats summed, batch)."""
    P = oracle.Params(gamma=G, options=oracle.OPT_DUAL | options, p_floor=p_floor, rho_floor=rho_floor)
    ora = [[f.copy() for f in U] for U in patches]
    oge = [g.copy() for g in ges]
    tot = {}
    for s, dt in enumerate(dts):
        for U, ge in zip(ora, oge):
            st = oracle.step_periodic_dual(U, ge, dx, dt, s, P)
            for k, v in st.items():
                tot[k] = tot.get(k, 0) + v
    b = _batch(patches, ges, dx, flags=flags)
    params = ez.Params(precision=precision, gamma=G, options=ez.OPT_DUAL | options, p_floor=p_floor,
                       rho_floor=rho_floor)
    for s, dt in enumerate(dts):
        b.dt_dev.fill_(dt)
        ez.step(b, params, s, b.dt_dev)
    return ora, oge, tot, b


def _ordinary():
    patches = [white_patch(n, seed=700 + i) for i, n in enumerate([(12, 10, 8), (9, 14, 6)])]
    ges = [synth.embed(_ge_of([active(f) for f in U])) for U in patches]
    dx = [1.0 / 12] * 3
    P0 = oracle.Params(gamma=G)
    W = [[f.copy() for f in U] for U in patches]
    dts = []
    for s in range(6):
        dt = 0.4 / max(oracle.cfl_rate(U, dx, P0) for U in W)
        for U in W:
            oracle.step_periodic(U, dx, dt, s, P0)
        dts.append(dt)
    return patches, ges, dx, dts, W


def _cold_compression(N=64):
    x = (np.arange(N) + 0.5) / N
    rho = np.ones((1, 1, N))
    u = (1.0 + 0.01 * np.sin(2 * math.pi * x)).reshape(1, 1, N)
    p = np.full((1, 1, N), 1e-6)
    z = np.zeros_like(rho)
    U = [synth.embed(f) for f in synth.prims_to_conserved(rho, u, z, z, p, G)]
    ge = synth.embed(p / (G - 1.0))
    dx = [1.0 / N, 1e30, 1e30]
    P = oracle.Params(gamma=G, options=oracle.OPT_DUAL)
    V, gv = [f.copy() for f in U], ge.copy()
    t, s, dts = 0.0, 0, []
    while t < 0.3:
        dt = 0.4 / oracle.cfl_rate(V, dx, P)
        oracle.step_periodic_dual(V, gv, dx, dt, s, P)
        dts.append(dt)
        t += dt
        s += 1
    return [U], [ge], dx, dts


def _cold_hypersonic():
    rng = np.random.default_rng(4)
    shape = (1, 2, 48)
    vx = rng.normal(0, 1, shape)
    rho = np.exp(rng.normal(0, 1, shape))
    z = np.zeros(shape)
    U = [synth.embed(f) for f in synth.prims_to_conserved(rho, vx, z, z, np.full(shape, 1e-8), G)]
    ge = synth.embed(np.full(shape, 1e-8) / (G - 1.0))
    dx = [1.0 / 48, 1e30, 1e30]
    P0 = oracle.Params(gamma=G, p_floor=1e-10, rho_floor=1e-10)
    V = [f.copy() for f in U]
    dts = []
    for s in range(12):
        dt = 0.4 / oracle.cfl_rate(V, dx, P0)
        oracle.step_periodic(V, dx, dt, s, P0)
        dts.append(dt)
    return [U], [ge], dx, dts


def _density_step(N=32, nsteps=4):
    """Left-moving bulk flow over a density step 1 | 2 (and its periodic image):
    the light cells beside the dense gas keep their advected gas energy under
    the neighbourhood rule of the resynchronisation, one of them at the
    pencil's end."""
    x = (np.arange(N) + 0.5) / N
    rho = np.where(x < 0.5, 1.0, 2.0).reshape(1, 1, N)
    u = np.full((1, 1, N), -math.sqrt(17.0))
    p = (1.0 + 0.05 * np.sin(2 * math.pi * x)).reshape(1, 1, N)
    z = np.zeros_like(rho)
    U = [synth.embed(f) for f in synth.prims_to_conserved(rho, u, z, z, p, G)]
    ge = synth.embed(p / (G - 1.0))
    dx = [1.0 / N, 1e30, 1e30]
    P = oracle.Params(gamma=G, options=oracle.OPT_DUAL)
    V, gv = [f.copy() for f in U], ge.copy()
    dts = []
    for s in range(nsteps):
        dt = 0.4 / oracle.cfl_rate(V, dx, P)
        oracle.step_periodic_dual(V, gv, dx, dt, s, P)
        dts.append(dt)
    return [U], [ge], dx, dts


def _assert_bitwise(b, ora, oge):
    for g, o in zip(gpu_patches(b), ora):
        for a, c in zip(g, o):
            assert np.array_equal(active(a), active(c))
    for g, o in zip(_gpu_ge(b), oge):
        assert np.array_equal(active(g), active(o))


@pytest.mark.parametrize("flags", [0, ez.PATCH_PERIODIC])
def test_dual_ordinary_flow_fp64_bitwise(flags):
    patches, ges, dx, dts, W = _ordinary()
    ora, oge, tot, b = _run_both(patches, ges, dx, dts, 0, flags=flags)
    _assert_bitwise(b, ora, oge)
    st = b.read_status()
    assert st["ge_pressure"] == tot["ge_pressure"] == 0 and st["nan"] == 0
    # the conserved state is the one the scheme without the option gives
    for g, w in zip(gpu_patches(b), W):
        for a, c in zip(g, w):
            assert np.array_equal(active(a), active(c))


@pytest.mark.parametrize("options", [0, ALL])
@pytest.mark.parametrize("flags", [0, ez.PATCH_PERIODIC])
def test_dual_cold_compression_fp64_bitwise(options, flags):
    patches, ges, dx, dts = _cold_compression()
    ora, oge, tot, b = _run_both(patches, ges, dx, dts, options, flags=flags)
    _assert_bitwise(b, ora, oge)
    st = b.read_status()
    assert st["ge_pressure"] > 0 and tot["ge_pressure"] > 0 and st["nan"] == 0


@pytest.mark.parametrize("flags", [0, ez.PATCH_PERIODIC])
def test_dual_neighbourhood_resync_fp64_bitwise(flags):
    patches, ges, dx, dts = _density_step()
    ora, oge, _, b = _run_both(patches, ges, dx, dts, 0, flags=flags)
    _assert_bitwise(b, ora, oge)
    e = _ge_of([active(f)[0, 0] for f in ora[0]])
    assert np.sum(active(oge[0])[0, 0] != e) >= 1       # some cells kept the advected value


@pytest.mark.parametrize("options", [0, ALL])
def test_dual_cold_hypersonic_fp64_bitwise(options):
    patches, ges, dx, dts = _cold_hypersonic()
    ora, oge, tot, b = _run_both(patches, ges, dx, dts, options, p_floor=1e-10, rho_floor=1e-10)
    _assert_bitwise(b, ora, oge)
    st = b.read_status()
    assert st["ge_pressure"] > 0 and st["nan"] == 0
    assert st["hll_cells"] == tot["hll_cells"]


def test_dual_fallback_fp64_bitwise():
    """Violent 1-D data (log-normal density and pressure with sigma 3, rms
    velocity 30, CFL 0.8): with dual energy on, the fallback is rare, and seed 48
    is the one of seeds 0-59 whose 20 steps take it (50 cells in the oracle).
    The re-fluxed faces carry the HLL gas-energy flux and the mean zone
    velocity; the result is bit-identical to the oracle's, with the same cells."""
    rng = np.random.default_rng(48)
    shape = (1, 1, 32)
    rho = np.exp(rng.normal(0, 3, shape))
    vx = rng.normal(0, 30, shape)
    p = np.exp(rng.normal(0, 3, shape))
    z = np.zeros(shape)
    U = [synth.embed(f) for f in synth.prims_to_conserved(rho, vx, z, z, p, G)]
    ge = synth.embed(p / (G - 1.0))
    dx = [1.0, 1e30, 1e30]
    P = oracle.Params(gamma=G, options=oracle.OPT_DUAL)
    V, gv, dts = [f.copy() for f in U], ge.copy(), []
    for s in range(20):
        dt = 0.8 / oracle.cfl_rate(V, dx, P)
        oracle.step_periodic_dual(V, gv, dx, dt, s, P)
        dts.append(dt)
    ora, oge, tot, b = _run_both([U], [ge], dx, dts, 0)
    _assert_bitwise(b, ora, oge)
    st = b.read_status()
    assert tot["hll_cells"] > 0 and st["hll_cells"] == tot["hll_cells"]
    assert st["ge_pressure"] > 0 and st["nan"] == 0


def test_dual_fp32_ordinary_flow_within_bound():
    patches, ges, dx, dts, _ = _ordinary()
    ora, oge, _, b = _run_both(patches, ges, dx, dts, 0, precision=ez.FP32, flags=ez.PATCH_PERIODIC)
    for g, o, gg, og in zip(gpu_patches(b), ora, _gpu_ge(b), oge):
        errs = l1_rel(g, o) + l1_rel([gg], [og])
        assert max(errs) <= 1e-4, errs


def test_dual_fp32_keeps_the_entropy_of_the_cold_compression():
    """FP32 takes the gas-energy pressure in the same zones' regime (decided in
    FP64) and holds p / rho^gamma to the oracle's 3e-3 bound."""
    patches, ges, dx, dts = _cold_compression()
    ora, oge, _, b = _run_both(patches, ges, dx, dts, 0, precision=ez.FP32, flags=ez.PATCH_PERIODIC)
    rho = active(gpu_patches(b)[0][0])[0, 0]
    ge = active(_gpu_ge(b)[0])[0, 0]
    s = (G - 1.0) * ge / rho ** G
    err = float(np.max(np.abs(s / 1e-6 - 1.0)))
    assert err < 3e-3, err
    assert np.max(np.abs(rho - 1.0)) > 0.01
    assert b.read_status()["ge_pressure"] > 0
    for e in l1_rel([b.patch_ge(0).cpu().numpy()], [oge[0]]):
        assert e <= 1e-4, e


def test_dual_noalloc_sweep_matches_the_batch_sweep():
    patches, ges, dx, dts = _cold_compression()
    a = _batch(patches, ges, dx)
    c = _batch(patches, ges, dx)
    p = ez.Params(precision=ez.FP64, gamma=G, options=ez.OPT_DUAL)
    ez.ghost_fill_periodic(a)
    ez.ghost_fill_periodic(c)
    ez.ppm_sweep(a, 0, dts[0], 0, p)
    ez.ppm_sweep_noalloc(c, 0, dts[0], 0, p)
    for x, y in zip(a.U + [a.ge], c.U + [c.ge]):
        assert bool((x == y).all())
    assert a.read_status() == c.read_status()


def test_ghost_fills_carry_the_gas_energy():
    """ge = rho before the fill: afterwards every ghost of ge equals rho's."""
    rng = np.random.default_rng(9)
    U = [rng.uniform(0.5, 2.0, (8, 9, 11)) for _ in range(5)]
    b = _batch([U], [U[0].copy()], [0.1] * 3)
    ez.ghost_fill_periodic(b)
    assert bool((b.ge == b.U[0]).all())
    b = _batch([U], [U[0].copy()], [0.1] * 3)
    ez.ghost_fill_boundary(b, (ez.BC_REFLECT, ez.BC_OUTFLOW, ez.BC_PERIODIC))
    assert bool((b.ge == b.U[0]).all())
    assert not np.array_equal(b.ge.cpu().numpy(), U[0].ravel())    # ghosts were written
