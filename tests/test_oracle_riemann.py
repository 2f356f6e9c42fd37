"""Pins of the oracle's Riemann solvers (Sec. 4.1.2) against closed forms and
invariances that do not come from the oracle itself."""
import math

import numpy as np
import pytest

import exact_riemann as ex
import oracle
from paper_1307_2265_gb300 import synth


def _golden(name):
    import os
    vals = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_exact_solver_matches_textbook_sod():
    """The independent exact solver reproduces the textbook Sod star state."""
    g = _golden("sod_star.txt")
    p, u = ex.star(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    assert abs(p - g["pstar"]) < 1e-5 and abs(u - g["ustar"]) < 1e-5
    rl = ex.sample(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4, u - 1e-9)[0]
    rr = ex.sample(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4, u + 1e-9)[0]
    assert abs(rl - g["rho_star_left"]) < 1e-5 and abs(rr - g["rho_star_right"]) < 1e-5


@pytest.mark.parametrize("gamma", [1.4, 5.0 / 3.0])
def test_twoshock_equals_exact_when_both_waves_are_shocks(gamma):
    """Two-shock is exact when both waves are shocks: colliding flows of any
    strength, with asymmetric densities and pressures, in moving frames."""
    rng = np.random.default_rng(11)
    P = oracle.Params(gamma=gamma)
    cases = [(1, 1, 1, 1, -1, 1), (1, 10, 1, 1, -10, 1), (2.0, 3.0, 0.5, 0.3, -2.0, 4.0)]
    for _ in range(40):
        rl, rr = np.exp(rng.normal(0, 1, 2))
        pl, pr = np.exp(rng.normal(0, 1, 2))
        du = rng.uniform(0.5, 20.0) * math.sqrt(gamma * max(pl / rl, pr / rr))
        shift = rng.normal(0, 3)
        cases.append((rl, shift + du / 2, pl, rr, shift - du / 2, pr))
    for (rl, ul, pl, rr, ur, pr) in cases:
        ps_ex, us_ex = ex.star(rl, ul, pl, rr, ur, pr, gamma)
        if not (ps_ex > pl and ps_ex > pr):
            continue
        o = oracle.riemann([rl], [ul], [pl], [rr], [ur], [pr], P)
        assert o["iters"][0] > 0, "Newton did not converge"
        assert abs(o["pstar"][0] - ps_ex) <= 1e-12 * ps_ex
        scale = abs(us_ex) + math.sqrt(gamma * ps_ex / min(rl, rr))
        assert abs(o["ustar"][0] - us_ex) <= 1e-12 * scale
        rho_ex, u_ex, p_ex = ex.sample(rl, ul, pl, rr, ur, pr, gamma, 0.0)
        assert abs(o["rho"][0] - rho_ex) <= 1e-11 * rho_ex
        assert abs(o["p"][0] - p_ex) <= 1e-11 * p_ex
        assert abs(o["u"][0] - u_ex) <= 1e-11 * scale


def test_twoshock_close_to_exact_for_weak_rarefactions():
    """The shock and rarefaction curves agree to second order in wave strength,
    so for weak waves the two-shock p* approaches the exact one as eps^3."""
    P = oracle.Params(gamma=5.0 / 3.0)
    errs = []
    for eps in (1e-1, 1e-2):
        o = oracle.riemann([1.0], [0.0], [1.0 + eps], [1.0], [0.0], [1.0], P)
        ps, us = ex.star(1.0, 0.0, 1.0 + eps, 1.0, 0.0, 1.0, 5.0 / 3.0)
        errs.append(abs(o["pstar"][0] - ps))
    assert errs[1] < errs[0] * 2e-2           # at least ~cubic reduction for 10x weaker
    assert errs[1] < 1e-6


def test_newton_root_independent_of_guess():
    rng = np.random.default_rng(5)
    P = oracle.Params()
    st = synth.riemann_states(rng, 200, mach=2.0)
    base = oracle.riemann(*st, P)
    assert np.all(base["iters"] >= 0)
    for scale in (1e-6, 1e-2, 0.5, 3.0, 1e3):
        g = base["pstar"] * scale
        o = oracle.riemann(*st, P, pguess=g)
        assert np.all(np.abs(o["pstar"] - base["pstar"]) <= 1e-12 * base["pstar"])


def test_twoshock_root_solves_hugoniot_equation():
    """The converged p* zeroes u*_R - u*_L for the shock Hugoniot written in the
    Rankine-Hugoniot form (mass flux sqrt((p*+B)/A)), evaluated in long double."""
    rng = np.random.default_rng(7)
    gamma = 5.0 / 3.0
    P = oracle.Params(gamma=gamma)
    st = synth.riemann_states(rng, 100, mach=3.0)
    o = oracle.riemann(*st, P)
    ld = np.longdouble
    g = ld(gamma)
    for i in range(100):
        rl, ul, pl, rr, ur, pr = (ld(a[i]) for a in st)
        ps = ld(o["pstar"][i])
        if o["pstar"][i] <= P.p_floor:      # separating flows with no positive root (vacuum)
            continue
        # mass flux through a shock of pressure jump ps (either sign, as the two-shock curve)
        ml = np.sqrt(rl * ((g + 1) / 2 * ps + (g - 1) / 2 * pl))
        mr = np.sqrt(rr * ((g + 1) / 2 * ps + (g - 1) / 2 * pr))
        res = (ur + (ps - pr) / mr) - (ul - (ps - pl) / ml)
        scale = abs(ul) + abs(ur) + np.sqrt(g * pl / rl) + np.sqrt(g * pr / rr)
        assert abs(float(res)) <= 1e-12 * float(scale)


def test_galilean_boost_of_riemann_solution():
    rng = np.random.default_rng(9)
    P = oracle.Params()
    st = list(synth.riemann_states(rng, 100))
    a = oracle.riemann(*st, P)
    for boost in (-2.5, 0.7, 4.0):
        b = oracle.riemann(st[0], st[1] + boost, st[2], st[3], st[4] + boost, st[5], P)
        assert np.allclose(b["pstar"], a["pstar"], rtol=1e-12, atol=0)
        assert np.allclose(b["ustar"], a["ustar"] + boost, rtol=0, atol=1e-11 * (1 + abs(boost)))


def test_hll_is_consistent_and_upwind():
    P = oracle.Params(gamma=1.4)
    rng = np.random.default_rng(3)
    n = 50
    s = [np.exp(rng.normal(0, 1, n)), rng.normal(0, 1, n), np.exp(rng.normal(0, 1, n)),
         rng.normal(0, 1, n), rng.normal(0, 1, n)]
    F = oracle.flux(s, s, P, solver="hll")
    rho, u, p, t1, t2 = s
    E = p / 0.4 + 0.5 * rho * (u * u + t1 * t1 + t2 * t2)
    Fex = np.stack([rho * u, rho * u * u + p, rho * u * t1, rho * u * t2, u * (E + p)], axis=1)
    assert np.allclose(F, Fex, rtol=1e-13, atol=1e-13)
    # supersonic to the right: HLL takes the left physical flux
    left = [np.ones(1), np.full(1, 5.0), np.ones(1), np.zeros(1), np.zeros(1)]
    right = [np.full(1, 0.5), np.full(1, 4.0), np.full(1, 0.8), np.zeros(1), np.zeros(1)]
    F = oracle.flux(left, right, P, solver="hll")
    Fl = oracle.flux(left, left, P, solver="hll")
    assert np.array_equal(F, Fl)


def test_twoshock_flux_of_equal_states_is_physical_flux():
    P = oracle.Params()
    rng = np.random.default_rng(4)
    n = 64
    s = [np.exp(rng.normal(0, 1, n)), rng.normal(0, 2, n), np.exp(rng.normal(0, 1, n)),
         rng.normal(0, 1, n), rng.normal(0, 1, n)]
    F = oracle.flux(s, s, P)
    G = oracle.flux(s, s, P, solver="hll")
    assert np.allclose(F, G, rtol=1e-12, atol=1e-12)


def _phys(rho, u, p, t1, t2, g):
    E = p / (g - 1.0) + 0.5 * rho * (u * u + t1 * t1 + t2 * t2)
    return np.stack([rho * u, rho * u * u + p, rho * u * t1, rho * u * t2, u * (E + p)], axis=1)


def test_hllc_is_consistent_upwind_and_exact_on_contacts():
    """HLLC: F(U, U) = F(U); supersonic flow takes the upwind physical flux;
    and, unlike HLL, an isolated contact (equal u and p, any rho and transverse
    velocities) gets the exact flux of the upwind side, F = F(U_L) for u > 0,
    F(U_R) for u < 0, and (0, p, 0, 0, 0) at rest.  A wrong sign or term in the
    contact speed S* or the star state gives a mass flux off the upwind one."""
    g = 1.4
    P = oracle.Params(gamma=g)
    rng = np.random.default_rng(5)
    n = 64
    s = [np.exp(rng.normal(0, 1, n)), rng.normal(0, 1, n), np.exp(rng.normal(0, 1, n)),
         rng.normal(0, 1, n), rng.normal(0, 1, n)]
    assert np.allclose(oracle.flux(s, s, P, solver="hllc"), _phys(*s, g), rtol=1e-13, atol=1e-13)
    left = [np.ones(1), np.full(1, 5.0), np.ones(1), np.zeros(1), np.zeros(1)]
    right = [np.full(1, 0.5), np.full(1, 4.0), np.full(1, 0.8), np.zeros(1), np.zeros(1)]
    assert np.array_equal(oracle.flux(left, right, P, solver="hllc"), oracle.flux(left, left, P, solver="hllc"))
    for u0 in (0.7, -0.4, 0.0):
        rl, rr = np.exp(rng.normal(0, 1, n)), np.exp(rng.normal(0, 1, n))
        p = np.exp(rng.normal(0, 1, n))
        u = np.full(n, u0)
        L = [rl, u, p, rng.normal(0, 1, n), rng.normal(0, 1, n)]
        R = [rr, u, p, rng.normal(0, 1, n), rng.normal(0, 1, n)]
        F = oracle.flux(L, R, P, solver="hllc")
        up = _phys(*(L if u0 >= 0 else R), g)
        assert np.allclose(F, up, rtol=1e-13, atol=1e-13), u0
        Fh = oracle.flux(L, R, P, solver="hll")
        assert np.max(np.abs(Fh[:, 0] - up[:, 0])) > 1e-3        # HLL smears the contact
