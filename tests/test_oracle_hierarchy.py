"""Pins of the hierarchy reference (oracle/hierarchy.py): SecondOrderA against
the properties Appendix A states for it (conservative, exact for linear
fields, monotone), projection, and conservation of the composite grid over a
full root step with subcycling, flux correction and projection."""
import numpy as np
import pytest

import oracle
from oracle import hierarchy as H
from paper_1307_2265_gb300 import synth


def test_second_order_a_exact_for_linear_fields_and_conservative():
    rng = np.random.default_rng(0)
    n = 200
    a, b, c, d = (rng.normal(0, 1, n) for _ in range(4))
    z, y, x = np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij")
    Q = d[:, None, None, None] + a[:, None, None, None] * x + b[:, None, None, None] * y + c[:, None, None, None] * z
    kids = H.second_order_a(Q)
    off = np.array([-0.25, 0.25])
    exact = (d[:, None, None, None] + a[:, None, None, None] * off[None, None, None, :]
             + b[:, None, None, None] * off[None, None, :, None] + c[:, None, None, None] * off[None, :, None, None])
    assert np.allclose(kids, exact, atol=1e-13)
    # conservation for arbitrary data: children average to the parent
    Q = rng.normal(0, 1, (n, 3, 3, 3))
    kids = H.second_order_a(Q)
    assert np.allclose(kids.mean(axis=(1, 2, 3)), Q[:, 1, 1, 1], atol=1e-14)


def test_second_order_a_adds_no_new_extrema_on_smooth_data():
    rng = np.random.default_rng(1)
    n = 2000
    base = rng.normal(0, 1, (n, 4))
    z, y, x = np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1], indexing="ij")
    Q = (base[:, 0, None, None, None] + base[:, 1, None, None, None] * x + base[:, 2, None, None, None] * y
         + base[:, 3, None, None, None] * z + 0.3 * rng.normal(0, 1, (n, 3, 3, 3)))
    kids = H.second_order_a(Q)
    lo = Q.reshape(n, -1).min(axis=1)
    hi = Q.reshape(n, -1).max(axis=1)
    assert np.all(kids.reshape(n, -1).min(axis=1) >= lo - 1e-12)
    assert np.all(kids.reshape(n, -1).max(axis=1) <= hi + 1e-12)


def test_minmod_definition():
    a = np.array([1.0, -2.0, 3.0, 0.0, -1.0])
    b = np.array([2.0, -1.0, -1.0, 5.0, -3.0])
    assert np.array_equal(H.minmod(a, b), np.array([1.0, -1.0, 0.0, 0.0, -1.0]))


def _small(seed=0):
    layout = synth.hierarchy_layout(16, [(4, 12), (6, 10)], [4, 8], seed=seed)
    fields = synth.hierarchy_fields(layout, config=5)
    return layout, H.make_levels(layout, fields, 1.0 / 16)


def test_projection_of_piecewise_constant_children_is_identity():
    layout, levels = _small()
    before = [f.copy() for f in levels[0]["patches"][0]["U"]]
    H.project(levels, 0)
    for a, b in zip(levels[0]["patches"][0]["U"], before):
        # the sum of 8 equal values rounds at each of its additions
        assert np.allclose(a, b, rtol=4e-16, atol=0)
        assert not np.array_equal(a, np.zeros_like(a))


@pytest.mark.slow
def test_composite_conservation_over_a_root_step():
    layout, levels = _small(seed=3)
    P = oracle.Params()
    t0 = H.composite_totals(levels)
    log = []
    H.root_step(levels, P, log=log)
    t1 = H.composite_totals(levels)
    scale = H.composite_totals([{"patches": [{"n": p["n"], "origin": p["origin"], "parent": p["parent"],
                                              "U": [np.abs(f) for f in p["U"]]} for p in L["patches"]],
                                 "dx": L["dx"]} for L in levels])
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale
    # the finer levels subcycled to catch up with their parents
    assert sum(1 for l, _ in log if l == 2) >= 2 * sum(1 for l, _ in log if l == 1) >= 2


def test_uniform_state_preserved_through_the_hierarchy():
    """Preserved to round-off: corner averages and projections sum eight equal
    values, which rounds, so the interpolated ghosts differ from the state by
    an ulp."""
    layout = synth.hierarchy_layout(16, [(4, 12), (6, 10)], [4, 8], seed=0)
    uni = []
    for l, L in enumerate(layout):
        per = []
        for i in range(len(L["n"])):
            nx, ny, nz = (int(v) for v in L["n"][i])
            sh = (nz, ny, nx)
            prims = [np.full(sh, 1.3), np.full(sh, 0.4), np.full(sh, -0.7), np.full(sh, 0.2), np.full(sh, 0.9)]
            per.append([synth.embed(f) for f in synth.prims_to_conserved(*prims, 5.0 / 3.0)])
        uni.append(per)
    levels = H.make_levels(layout, uni, 1.0 / 16)
    H.root_step(levels, oracle.Params())
    for L, ref in zip(levels, uni):
        for p, r in zip(L["patches"], ref):
            for a, b in zip(p["U"], r):
                assert np.allclose(H._active(a), H._active(b), rtol=1e-14, atol=1e-14)


# Dual energy through the hierarchy (Sec. 4.1.1 with Sec. 3): the gas energy is
# a sixth field that every hierarchy operation carries like the conserved ones.
G_COLD = 1.4
EPS_COLD = 2.0


def _ge_deviation(levels):
    worst = 0.0
    for L in levels:
        for p in L["patches"]:
            worst = max(worst, float(np.max(np.abs(H._active(p["U"][5]) / H._active(p["U"][0]) - EPS_COLD))))
    return worst


def test_dual_cold_contact_window():
    """The cold contact keeps every cell's internal energy between the two
    thresholds: above 1e-3 E (the pressure comes from E - KE) and below 0.1 E
    (no resynchronisation), so the gas energy is a passive density."""
    layout = synth.hierarchy_layout(16, [(4, 12), (6, 10)], [4, 8], seed=1)
    for lev in synth.cold_contact_fields(layout, 16, gamma=G_COLD, eps=EPS_COLD):
        for U in lev:
            A = [H._active(f) for f in U]
            frac = (A[4] - 0.5 * ((A[1] ** 2 + A[2] ** 2) + A[3] ** 2) / A[0]) / A[4]
            assert 2e-2 < frac.min() and frac.max() < 8e-2


@pytest.mark.slow
def test_dual_gas_energy_follows_the_density_in_a_cold_contact():
    """With uniform pressure and velocity the Riemann problems are contacts
    (p* = p, u* = u), the -p div v source vanishes and eps is uniform, so the
    traced eps is eps and the gas-energy flux is eps times the mass flux; with
    eps a power of two every hierarchy operation (time and SecondOrderA
    interpolation, sibling copies, flux registers and correction, projection)
    maps rho to eps rho exactly.  So ge = eps rho stays bit-exact in every cell
    of three levels over a root step with subcycling."""
    layout = synth.hierarchy_layout(16, [(4, 12), (6, 10)], [4, 8], seed=1)
    levels = H.make_levels(layout, synth.cold_contact_fields(layout, 16, gamma=G_COLD, eps=EPS_COLD), 1.0 / 16)
    log = []
    H.root_step(levels, oracle.Params(gamma=G_COLD, options=8), log=log)
    assert sum(1 for l, _ in log if l == 2) >= 2
    assert _ge_deviation(levels) == 0.0


def _keep_ge(fn, patches_of):
    """`fn` with the gas energy of the patches it touches restored afterwards
    (a planted mistake: the operation skips the sixth field)."""
    def wrapped(*args, **kw):
        keep = [p["U"][5].copy() for p in patches_of(*args)]
        fn(*args, **kw)
        for p, k in zip(patches_of(*args), keep):
            p["U"][5][...] = k
    return wrapped


@pytest.mark.parametrize("op", ["flux_correct", "project", "copy_from_siblings"])
def test_dual_pin_catches_a_skipped_gas_energy_operation(op, monkeypatch):
    """The cold-contact pin fails (by more than 1e-3) when the flux correction,
    the projection or the sibling copies leave the gas energy out (mistakes
    planted in the oracle; two levels, one root step)."""
    layout = synth.hierarchy_layout(16, [(4, 12)], [4, 8], seed=1)
    levels = H.make_levels(layout, synth.cold_contact_fields(layout, 16, gamma=G_COLD, eps=EPS_COLD), 1.0 / 16)
    target = {"flux_correct": lambda levels, l, *a: levels[l]["patches"],
              "project": lambda levels, l, *a: levels[l]["patches"],
              "copy_from_siblings": lambda level: level}[op]
    monkeypatch.setattr(H, op, _keep_ge(getattr(H, op), target))
    H.root_step(levels, oracle.Params(gamma=G_COLD, options=8))
    assert _ge_deviation(levels) > 1e-3


@pytest.mark.slow
def test_dual_hierarchy_at_low_mach_leaves_the_five_fields_as_without_it():
    """Where no cell is cold enough to take its pressure from the gas energy,
    the dual-energy hierarchy steps the five conserved fields bit-identically
    to the run without the option (the sixth field feeds nothing else)."""
    layout, plain = _small(seed=3)
    fields = synth.hierarchy_fields(layout, config=5)
    six = []
    for lev in fields:
        per = []
        for U in lev:
            A = [H._active(f) for f in U]
            per.append([f.copy() for f in U] +
                       [synth.embed(A[4] - 0.5 * ((A[1] ** 2 + A[2] ** 2) + A[3] ** 2) / A[0])])
        six.append(per)
    dual = H.make_levels(layout, six, 1.0 / 16)
    H.root_step(plain, oracle.Params())
    H.root_step(dual, oracle.Params(options=8))
    for La, Lb in zip(plain, dual):
        for pa, pb in zip(La["patches"], Lb["patches"]):
            for f in range(5):
                assert np.array_equal(pa["U"][f], pb["U"][f])


@pytest.mark.slow
def test_dual_gas_energy_follows_the_density_through_rebuilds():
    """The cold-contact pin with the hierarchy rebuilt after every root step
    (new grids interpolated by SecondOrderA, then copied from the old ones):
    ge = eps rho stays bit-exact and the grids change."""
    layout = synth.hierarchy_layout(16, [(4, 12)], [4, 8], seed=1)
    levels = H.make_levels(layout, synth.cold_contact_fields(layout, 16, gamma=G_COLD, eps=EPS_COLD), 1.0 / 16)
    rb = {"gamma": G_COLD, "crit": {"slope": 0.05, "shock_dp": 0.33, "shock_e": 0.1},
          "clus": {"efficiency": 0.3, "small_cells": 8, "buffer": 1}}
    before = [p["origin"] for p in levels[1]["patches"]]
    for _ in range(2):
        H.root_step(levels, oracle.Params(gamma=G_COLD, options=8), rebuild=rb)
    assert [p["origin"] for p in levels[1]["patches"]] != before and levels[1]["patches"]
    assert _ge_deviation(levels) == 0.0


def test_gas_energy_fills_as_a_scalar():
    """The oracle's ghost fills treat a sixth field (the gas energy) as a
    scalar: periodic wrap like the density, and under a reflecting boundary
    the mirror image without the sign change the normal momentum gets."""
    rng = np.random.default_rng(5)
    U = [synth.embed(rng.uniform(0.5, 2.0, (4, 5, 6))) for _ in range(6)]
    V = [f.copy() for f in U]
    oracle.fill_periodic(V)
    ref = U[5].copy()                  # the density's fill applied to the gas energy
    oracle.fill_periodic([ref, U[1].copy(), U[2].copy(), U[3].copy(), U[4].copy()])
    assert np.array_equal(V[5], ref)
    B = [f.copy() for f in U]
    oracle.fill_boundary(B, (oracle.BC_REFLECT, oracle.BC_OUTFLOW, oracle.BC_PERIODIC))
    ge, mx = B[5], B[1]
    # x faces: ghost layer g mirrors active cell g - 1 (storage: ghost 2 - k <-> active 3 + k)
    for k in range(3):
        assert np.array_equal(ge[3:-3, 3:-3, 2 - k], ge[3:-3, 3:-3, 3 + k])
        assert np.array_equal(mx[3:-3, 3:-3, 2 - k], -mx[3:-3, 3:-3, 3 + k])
    assert np.all(ge[3:-3, 3:-3, :3] > 0)


@pytest.mark.slow
def test_dual_hierarchy_conserves_the_five_fields():
    """With the dual-energy option (cold cells taking their pressure from the
    gas energy) a subcycled root step still conserves the composite totals of
    mass, momentum and energy to round-off: the sixth field changes the
    fluxes, not their conservative use."""
    layout, _ = _small(seed=3)
    fields = synth.hierarchy_fields(layout, config=5)
    six = []
    for lev in fields:
        per = []
        for U in lev:
            A = [H._active(f) for f in U]
            ke = 0.5 * ((A[1] ** 2 + A[2] ** 2) + A[3] ** 2) / A[0]
            V = [f.copy() for f in U]
            H._active(V[4])[...] = ke + 1e-4 * (A[4] - ke)      # cold: E - KE < 1e-3 E
            per.append(V + [synth.embed(2e-4 * (A[4] - ke))])   # ge: twice E - KE
        six.append(per)
    levels = H.make_levels(layout, six, 1.0 / 16)
    t0 = H.composite_totals(levels)
    scale = H.composite_totals([{"patches": [{"n": p["n"], "origin": p["origin"], "parent": p["parent"],
                                              "U": [np.abs(f) for f in p["U"][:5]]} for p in L["patches"]],
                                 "dx": L["dx"]} for L in levels])
    H.root_step(levels, oracle.Params(options=8), log=[])
    t1 = H.composite_totals(levels)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale
