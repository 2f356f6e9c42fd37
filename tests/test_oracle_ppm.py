"""Pins of the oracle's PPM steps (Sec. 4.1; CW84 1.6-1.12, 3.6-3.7) on one pencil,
against closed forms: exactness of the reconstruction for polynomials, the
no-new-extrema property of the monotone parabola, and the exact domain-of-
dependence averages carried by entropy and acoustic waves."""
import numpy as np

import oracle

G = 5.0 / 3.0
L = 24
NG = 3


def _cell_avg(poly, lo, hi):
    """Average of polynomial (numpy poly1d) over [lo, hi]."""
    P = np.polyint(poly)
    return (P(hi) - P(lo)) / (hi - lo)


def _pencil(rho, u, p, t1=None, t2=None):
    t1 = np.zeros_like(rho) if t1 is None else t1
    t2 = np.zeros_like(rho) if t2 is None else t2
    E = p / (G - 1.0) + 0.5 * rho * (u * u + t1 * t1 + t2 * t2)
    return np.stack([rho, rho * u, rho * t1, rho * t2, E])


def test_interface_values_exact_for_cubic_cell_averages():
    """Unlimited PPM interface values are exact point values of a cubic whose cell
    averages are the data (4th-order interface formula)."""
    cub = np.poly1d([2e-4, -3e-3, 0.5, 2.0])          # gentle, monotone on [0, L]
    avg = np.array([_cell_avg(cub, s, s + 1) for s in range(L)])
    one = np.ones(L)
    for var, pen in ((0, _pencil(avg, 0 * one, one)),            # density
                     (1, _pencil(one, avg - 2.0, one)),          # normal velocity
                     (3, _pencil(one, 0 * one, one, avg, 0 * one))):
        o = oracle.pencil_debug(pen, 0.0, oracle.Params(gamma=G))
        for s in range(3, L - 3):
            assert abs(o["qL"][var, s] - (cub(s) - (2.0 if var == 1 else 0.0))) < 1e-12
            assert abs(o["qR"][var, s] - (cub(s + 1) - (2.0 if var == 1 else 0.0))) < 1e-12


def test_parabola_adds_no_new_extrema():
    rng = np.random.default_rng(0)
    xs = np.linspace(0, 1, 101)
    for trial in range(30):
        rho = np.exp(rng.normal(0, 1, L))
        if trial % 3 == 0:
            rho = np.where(np.arange(L) < L // 2, 1.0, 0.125) + 0.0
        o = oracle.pencil_debug(_pencil(rho, np.zeros(L), np.ones(L)), 0.0, oracle.Params(gamma=G))
        for s in range(2, L - 2):
            qL, qR, q6 = o["qL"][0, s], o["qR"][0, s], o["q6"][0, s]
            curve = qL + xs * ((qR - qL) + q6 * (1.0 - xs))
            lo = min(rho[s - 1], rho[s], rho[s + 1])
            hi = max(rho[s - 1], rho[s], rho[s + 1])
            assert curve.min() >= lo - 1e-12 * hi and curve.max() <= hi + 1e-12 * hi
            # the parabola keeps the zone average: mean over the zone = q_s
            assert abs((qL + 0.5 * (qR - qL) + q6 / 6.0) - rho[s]) < 1e-12 * hi
            if (rho[s + 1] - rho[s]) * (rho[s] - rho[s - 1]) <= 0.0:
                assert qL == rho[s] and qR == rho[s]          # local extremum: flat


def _run_wave(u0, kind, A=1e-6, dtdx=0.3):
    """Linear wave of quadratic profile on a uniform background rho=1, p=1.
    Returns the debug arrays and the background sound speed."""
    c0 = np.sqrt(G)
    C0 = c0                      # rho0 * c0
    f = np.poly1d([0.01, 1.0, 0.0])
    favg = np.array([_cell_avg(f, s, s + 1) for s in range(L)])
    if kind == "entropy":         # delta rho only, p and u uniform
        rho, u, p = 1.0 + A * favg, np.full(L, u0), np.ones(L)
    elif kind == "right":         # right-moving acoustic: dp = C du, drho = dp / c^2
        rho, u, p = 1.0 + A * favg / c0 ** 2, u0 + A * favg / C0, 1.0 + A * favg
    else:                         # left-moving acoustic: dp = -C du
        rho, u, p = 1.0 + A * favg / c0 ** 2, u0 - A * favg / C0, 1.0 + A * favg
    o = oracle.pencil_debug(_pencil(rho, u, p), dtdx, oracle.Params(gamma=G))
    return o, f, c0


def test_entropy_wave_left_state_is_u_domain_average():
    u0, dtdx, A = 0.5, 0.3, 1e-2
    o, f, c0 = _run_wave(u0, "entropy", A=A, dtdx=dtdx)
    sig = u0 * dtdx
    for s in range(2, L - 4):
        exact = 1.0 + A * _cell_avg(f, s + 1 - sig, s + 1)
        assert abs(o["sL"][0, s] - exact) < 1e-13
        assert abs(o["sL"][1, s] - u0) < 1e-13 and abs(o["sL"][2, s] - 1.0) < 1e-13
        # upwind mass flux of pure advection is the exact time average
        assert abs(o["F"][0, s] - u0 * exact) < 1e-12


def test_acoustic_waves_traced_along_their_characteristics():
    """Left states carry each Riemann invariant from its own domain of dependence:
    subsonic right-moving wave (reference u+c, entropy correction must vanish) and
    supersonic left-moving wave (u-c correction beta- must recover J-)."""
    A, dtdx = 1e-6, 0.2
    for u0, kind in ((0.5, "right"), (0.5 * np.sqrt(G), "right"), (2.0 * np.sqrt(G), "left")):
        o, f, c0 = _run_wave(u0, kind, A=A, dtdx=dtdx)
        lam = u0 + c0 if kind == "right" else u0 - c0
        sig = lam * dtdx
        for s in range(2, L - 4):
            dp = A * _cell_avg(f, s + 1 - sig, s + 1)
            sgn = 1.0 if kind == "right" else -1.0
            # nonlinear terms are O(A^2) ~ 1e-9 here; using a wrong domain or a wrong
            # correction sign shifts the state by O(A * dsigma) ~ 1e-7
            tol = 1e-8
            assert abs(o["sL"][2, s] - (1.0 + dp)) < tol
            assert abs(o["sL"][1, s] - (u0 + sgn * dp / c0)) < tol
            assert abs(o["sL"][0, s] - (1.0 + dp / c0 ** 2)) < tol


def test_right_states_mirror_left_states():
    rng = np.random.default_rng(2)
    P = oracle.Params(gamma=G)
    rho = np.exp(rng.normal(0, 0.5, L))
    u = rng.normal(0, 1, L)
    p = np.exp(rng.normal(0, 0.5, L))
    t1 = rng.normal(0, 1, L)
    a = oracle.pencil_debug(_pencil(rho, u, p, t1), 0.25, P)
    b = oracle.pencil_debug(_pencil(rho[::-1].copy(), -u[::-1], p[::-1].copy(), t1[::-1].copy()), 0.25, P)
    for s in range(3, L - 3):
        m = L - 1 - s
        assert a["sL"][0, s] == b["sR"][0, m] and a["sL"][2, s] == b["sR"][2, m]
        assert a["sL"][1, s] == -b["sR"][1, m] and a["sL"][3, s] == b["sR"][3, m]
