"""Pins of the oracle's hierarchy rebuild (Sec. 3.5 clustering, Sec. 3.6
flagging), checked against the exact Riemann solution, closed forms and the
properties the paper states: shocks are flagged and contacts and rarefactions
are not, whichever way the shock runs; the clusters cover every flagged cell
with disjoint boxes that are efficient or small; a rebuild conserves the
composite totals; a dynamic W-cycle keeps a moving shock refined."""
import math

import numpy as np
import pytest

import oracle
from oracle import amr
from oracle import hierarchy as H
from paper_1307_2265_gb300 import synth

import exact_riemann as ER

NG = 3


def _tube(N=200, gamma=1.4):
    """Periodic Sod tube along x: the high state on [0, 0.5), so a shock runs
    right from x = 0.5 and its mirror runs left from x = 1."""
    x = (np.arange(N) + 0.5) / N
    shape = (1, 1, N)
    rho = np.broadcast_to(np.where(x < 0.5, 1.0, 0.125), shape).copy()
    p = np.broadcast_to(np.where(x < 0.5, 1.0, 0.1), shape).copy()
    z = np.zeros(shape)
    return [synth.embed(f) for f in synth.prims_to_conserved(rho, z, z, z, p, gamma)]


def test_shock_flags_mark_shocks_not_contacts_or_rarefactions():
    g = 1.4
    N = 200
    U = _tube(N, g)
    dx = [1.0 / N, 1e30, 1e30]
    P = oracle.Params(gamma=g)
    t = 0.0
    while t < 0.1:
        dt = min(0.4 / oracle.cfl_rate(U, dx, P), 0.1 - t)
        oracle.step_periodic(U, dx, dt, 0, P)
        t += dt
    oracle.fill_periodic(U)
    fl = amr.flag_patch(U, 1.0 / N, g, slope=0.0)[0, 0]
    ps, us = ER.star(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, g)
    # shock speed from the Rankine-Hugoniot mass balance across the right shock
    rho_s = 0.125 * ((ps / 0.1) + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * (ps / 0.1) + 1)
    S = rho_s * us / (rho_s - 0.125)
    x = (np.arange(N) + 0.5) / N
    shocks = [0.5 + S * t, 1.0 - S * t]
    contacts = [0.5 + us * t, 1.0 - us * t]
    c_l = math.sqrt(g)
    c_star = c_l * (ps / 1.0) ** ((g - 1) / (2 * g))
    fans = [(0.5 - c_l * t, 0.5 + (us - c_star) * t), (0.0 - (us - c_star) * t, 0.0 + c_l * t)]
    hit = x[(fl & amr.SHOCK) != 0]
    assert len(hit) > 0
    for xs in shocks:
        assert np.any(np.abs(hit - xs) < 3.0 / N), xs            # each shock flagged
    for xh in hit:
        assert min(abs(xh - xs) for xs in shocks) < 4.0 / N, xh    # nothing else
    for xc in contacts:
        assert np.all(np.abs(hit - xc) > 6.0 / N)
    for a, b in fans:
        assert not np.any((hit > a) & (hit < b))


def test_slope_and_mass_flags_closed_form():
    """rho_i = 1.2 + 0.5 i along x: |rho_{i+1} - rho_{i-1}| / (2 rho_i) =
    0.5 / (1.2 + 0.5 i) exceeds 0.3 for i <= 0 only (E is uniform, so only the
    density flags).  Mass flags where rho dx^3 > m."""
    n = 8
    i = np.arange(-NG, n + NG)
    rho = np.broadcast_to(1.2 + 0.5 * i, (1 + 2 * NG, 1 + 2 * NG, n + 2 * NG)).copy()
    z = np.zeros_like(rho)
    E = np.full_like(rho, 10.0)
    fl = amr.flag_patch([rho, z, z, z, E], 0.5, 1.4, slope=0.3, shock_dp=0.0)[0, 0]
    assert list((fl & amr.SLOPE) != 0) == [True] + [False] * (n - 1)
    fm = amr.flag_patch([rho, z, z, z, E], 0.5, 1.4, slope=0.0, shock_dp=0.0, mass=2.0 * 0.125)[0, 0]
    assert list((fm & amr.MASS) != 0) == list((1.2 + 0.5 * np.arange(n)) > 2.0)
    assert not amr.flag_patch([np.ones_like(rho), z, z, z, E], 0.5, 1.4).any()   # uniform: nothing


def test_shock_flags_closed_form():
    """p_i = 1 + 0.2 i, u_i = -0.5 i, rho = 1 along x (gamma 1.4): the pressure
    ratio |p_{i+1} - p_{i-1}| / min(p_{i+1}, p_{i-1}) = 0.4 / (0.8 + 0.2 i)
    exceeds 0.33 for i <= 2 (with max instead of min only i = 0 would), the
    flow converges everywhere, and e / E = (1 + 0.2 i) / (1 + 0.2 i + 0.05 i^2)
    is 1, 0.96, 0.875 for i = 0, 1, 2, so shock_e = 0.9 keeps i <= 1.  The
    same profile with the velocity reversed (diverging flow) flags nothing."""
    n, g = 8, 1.4
    i = np.arange(-NG, n + NG, dtype=np.float64)
    shape = (1 + 2 * NG, 1 + 2 * NG, n + 2 * NG)
    rho = np.ones(shape)
    p = np.broadcast_to(1.0 + 0.2 * i, shape).copy()
    u = np.broadcast_to(-0.5 * i, shape).copy()
    z = np.zeros(shape)
    E = p / (g - 1.0) + 0.5 * rho * u * u
    U = [rho, rho * u, z, z, E]
    fl = amr.flag_patch(U, 0.5, g, slope=0.0, shock_dp=0.33, shock_e=0.1)[0, 0]
    assert list((fl & amr.SHOCK) != 0) == [True] * 3 + [False] * (n - 3)
    fl = amr.flag_patch(U, 0.5, g, slope=0.0, shock_dp=0.33, shock_e=0.9)[0, 0]
    assert list((fl & amr.SHOCK) != 0) == [True] * 2 + [False] * (n - 2)
    U[1] = -U[1]
    assert not amr.flag_patch(U, 0.5, g, slope=0.0, shock_dp=0.33, shock_e=0.1).any()


def test_cluster_exact_rectangles_and_l_shape():
    F = np.zeros((1, 12, 20), np.uint8)
    F[0, 3:7, 4:15] = 1
    assert amr.cluster(F, buffer=0) == [((4, 3, 0), (15, 7, 1))]
    F = np.zeros((1, 12, 20), np.uint8)
    F[0, 2:4, 1:5] = 1
    F[0, 7:10, 12:18] = 1
    assert amr.cluster(F, buffer=0) == [((1, 2, 0), (5, 4, 1)), ((12, 7, 0), (18, 10, 1))]
    # an L: its bounding box is 44% flagged; the corner is the strongest
    # inflection of the signature, so two exact rectangles result
    F = np.zeros((1, 12, 20), np.uint8)
    F[0, 2:10, 2:5] = 1
    F[0, 7:10, 5:16] = 1
    assert amr.cluster(F, buffer=0, efficiency=0.9, small_cells=1) == [((2, 2, 0), (5, 10, 1)),
                                                                          ((5, 7, 0), (16, 10, 1))]


@pytest.mark.parametrize("seed", range(6))
def test_cluster_covers_flags_with_disjoint_efficient_boxes(seed):
    rng = np.random.default_rng(seed)
    shape = (int(rng.integers(4, 12)), int(rng.integers(6, 20)), int(rng.integers(6, 24)))
    F = np.zeros(shape, np.uint8)
    for _ in range(int(rng.integers(1, 5))):       # a few random blobs
        c = [int(rng.integers(0, s)) for s in shape]
        r = [int(rng.integers(1, 4)) for _ in shape]
        F[max(0, c[0] - r[0]):c[0] + r[0], max(0, c[1] - r[1]):c[1] + r[1], max(0, c[2] - r[2]):c[2] + r[2]] = 1
    F |= (rng.random(shape) < 0.01).astype(np.uint8)
    for buffer in (0, 1):
        boxes = amr.cluster(F, efficiency=0.5, small_cells=8, buffer=buffer)
        G = amr.grow(F, buffer) if buffer else F != 0
        cover = np.zeros(shape, np.int32)
        for lo, hi in boxes:
            assert all(0 <= lo[a] < hi[a] <= shape[2 - a] for a in range(3))
            cover[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] += 1
            vol = np.prod([hi[a] - lo[a] for a in range(3)])
            inside = int(G[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]].sum())
            assert inside >= 0.5 * vol or vol <= 8
        assert cover.max() <= 1                       # disjoint
        assert np.all(cover[G] == 1)                  # every (grown) flag covered


def _two_level(root_n=(48, 8, 8), box=((16, 3, 3), (28, 5, 5)), seed=3):
    """Root patch plus one level-1 patch over the root box `box`, fields from
    a seeded Mach-1 white-noise state on each level."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = root_n
    prims = synth.white_noise_prims(rng, (nz, ny, nx), sigma=0.3, mach=1.0, gamma=1.4)
    root = [synth.embed(f) for f in synth.prims_to_conserved(*prims, 1.4)]
    lo, hi = box
    n1 = tuple(2 * (hi[a] - lo[a]) for a in range(3))
    prims1 = synth.white_noise_prims(rng, (n1[2], n1[1], n1[0]), sigma=0.3, mach=1.0, gamma=1.4)
    fine = [synth.embed(f) for f in synth.prims_to_conserved(*prims1, 1.4)]
    layout = [{"n": np.array([root_n]), "origin": np.zeros((1, 3), int), "parent": np.array([-1])},
              {"n": np.array([n1]), "origin": np.array([[2 * lo[a] for a in range(3)]]), "parent": np.array([0])}]
    return H.make_levels(layout, [[root], [fine]], 1.0 / root_n[0])


def test_rebuild_conserves_the_composite_totals():
    """After a projection the parent equals the mean of the old fine cells, and
    SecondOrderA keeps the parent mean, so interpolating the new grids and
    copying the old ones where they overlap leaves the composite totals
    unchanged up to rounding."""
    levels = _two_level()
    H.project(levels, 0)
    before = H.composite_totals(levels)
    oracle.fill_periodic(levels[0]["patches"][0]["U"])
    boxes = amr.rebuild_level(levels, 0, 1.4, {"slope": 0.1, "shock_dp": 0.2}, {"efficiency": 0.3, "small_cells": 8})
    assert len(boxes) >= 1
    after = H.composite_totals(levels)
    assert np.all(np.abs(after - before) <= 1e-13 * np.abs(before).max()), (before, after)


def _shock_hierarchy(N=48):
    """Root N x 8 x 8 with a Mach-2 shock (gamma 1.4) running right from x =
    0.3, plus one level-1 patch around it."""
    g = 1.4
    M = 2.0
    rho1, p1 = 1.0, 1.0
    c1 = math.sqrt(g * p1 / rho1)
    rho2 = rho1 * (g + 1) * M * M / ((g - 1) * M * M + 2)
    p2 = p1 * (2 * g * M * M - (g - 1)) / (g + 1)
    u2 = M * c1 * (1 - rho1 / rho2)
    shape = (8, 8, N)
    x = (np.arange(N) + 0.5) / N
    post = np.broadcast_to(x < 0.3, shape)
    rho = np.where(post, rho2, rho1)
    u = np.where(post, u2, 0.0)
    p = np.where(post, p2, p1)
    z = np.zeros(shape)
    root = [synth.embed(f) for f in synth.prims_to_conserved(rho, u, z, z, p, g)]
    lo, hi = (10, 3, 3), (20, 5, 5)
    layout = [{"n": np.array([(N, 8, 8)]), "origin": np.zeros((1, 3), int), "parent": np.array([-1])},
              {"n": np.array([(20, 4, 4)]), "origin": np.array([[20, 6, 6]]), "parent": np.array([0])}]
    levels = H.make_levels(layout, [[root], [[np.zeros((4 + 6, 4 + 6, 20 + 6)) for _ in range(5)]]], 1.0 / N)
    amr.fill_patch_from_parent(levels[1]["patches"][0], levels[0]["patches"][0])
    return levels, g


def test_dynamic_w_cycle_keeps_the_shock_refined_and_conserves():
    levels, g = _shock_hierarchy()
    P = oracle.Params(gamma=g)
    rb = {"gamma": g, "crit": {"slope": 0.3, "shock_dp": 0.33}, "clus": {"efficiency": 0.3, "small_cells": 8}}
    tot0 = H.composite_totals(levels)
    x_prev = None
    for s in range(6):
        H.root_step(levels, P, rebuild=rb)
        root = levels[0]["patches"][0]
        oracle.fill_periodic(root["U"])
        fl = amr.flag_patch(root["U"], levels[0]["dx"], g, slope=0.0)
        xs = np.flatnonzero(((fl & amr.SHOCK) != 0)[4, 4])
        xs = xs[(xs >= 3) & (xs < 30)]                 # the main shock (the wrap at x = 1 makes its own waves)
        assert len(xs) > 0
        # every shock-flagged root cell away from the domain edge lies in level 1
        for xi in xs:
            cell = np.array([xi, 4, 4])
            assert any(np.all((np.array(p["origin"]) // 2 <= cell) & (cell < (np.array(p["origin"]) + np.array(p["n"])) // 2))
                       for p in levels[1]["patches"]), xi
        if x_prev is not None:
            assert xs.max() >= x_prev                 # the shock moves right, and the grids with it
        x_prev = xs.max()
    tot = H.composite_totals(levels)
    assert np.all(np.abs(tot - tot0) <= 1e-12 * np.abs(tot0).max()), (tot0, tot)


def test_a_level_can_empty_and_refill():
    """A uniform moving state flags nothing, so the first rebuild empties level
    1; the W-cycle then steps the root alone (the empty level just keeps pace).
    A density bump added afterwards is flagged and refined again, and the
    composite totals hold throughout."""
    g = 1.4
    N = 32
    shape = (8, 8, N)
    one = np.ones(shape)
    z = np.zeros(shape)
    root = [synth.embed(f) for f in synth.prims_to_conserved(one, 0.3 * one, z, z, one, g)]
    fine = [synth.embed(f) for f in synth.prims_to_conserved(np.ones((4, 4, 16)), 0.3 * np.ones((4, 4, 16)),
                                                             np.zeros((4, 4, 16)), np.zeros((4, 4, 16)),
                                                             np.ones((4, 4, 16)), g)]
    layout = [{"n": np.array([(N, 8, 8)]), "origin": np.zeros((1, 3), int), "parent": np.array([-1])},
              {"n": np.array([(16, 4, 4)]), "origin": np.array([(24, 6, 6)]), "parent": np.array([0])}]
    levels = H.make_levels(layout, [[root], [fine]], 1.0 / N)
    P = oracle.Params(gamma=g)
    rb = {"gamma": g, "crit": {"slope": 0.3, "shock_dp": 0.33}, "clus": {"efficiency": 0.3, "small_cells": 8}}
    tot0 = H.composite_totals(levels)
    H.root_step(levels, P, rebuild=rb)
    assert levels[1]["patches"] == []
    H.root_step(levels, P, rebuild=rb)
    assert levels[1]["t"] == levels[0]["t"]
    totA = H.composite_totals(levels)
    assert np.all(np.abs(totA - tot0) <= 1e-13 * np.abs(tot0).max())
    r = levels[0]["patches"][0]["U"]
    bump = 3.0 * np.exp(-((np.arange(N) - 16.0) / 1.5) ** 2)
    for f in range(5):
        r[f][3:-3, 3:-3, 3:-3] *= (1.0 + bump)         # rho, m, E scale together: u and p/rho kept
    tot1 = H.composite_totals(levels)
    H.root_step(levels, P, rebuild=rb)
    assert len(levels[1]["patches"]) >= 1
    tot2 = H.composite_totals(levels)
    assert np.all(np.abs(tot2 - tot1) <= 1e-13 * np.abs(tot1).max())
