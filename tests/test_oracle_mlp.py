"""Pins of the FP64 learned-guess reference (oracle/mlp.py): finite-difference
gradients, the closed-form first Adam step, the Riemann-problem invariances of
the features, and convergence of training on a known target."""
import numpy as np

import oracle
from oracle import mlp
from paper_1307_2265_gb300 import synth


def _data(n=64, seed=0):
    rng = np.random.default_rng(seed)
    st = synth.riemann_states(rng, n, mach=1.5)
    x, pref = mlp.features(*st, 5.0 / 3.0)
    return st, x, rng.normal(0, 1, n)


def test_gradients_match_central_differences():
    _, x, t = _data()
    P = mlp.init(3)
    y, cache = mlp.forward(P, x)
    g = mlp.backward(P, cache, y, t)
    rng = np.random.default_rng(1)
    for k in P:
        flat = P[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            h = 1e-6 * max(1.0, abs(flat[idx]))
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.mse(mlp.forward(P, x)[0], t)
            flat[idx] = old - h
            lm = mlp.mse(mlp.forward(P, x)[0], t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[idx]
            # central differences carry ~eps*loss/h ~ 1e-10 of round-off
            assert abs(fd - an) <= 1e-6 * max(abs(fd), abs(an)) + 1e-9, (k, idx, fd, an)


def test_silu_derivative_closed_form():
    z = np.linspace(-8, 8, 101)
    fd = (mlp.silu(z + 1e-6) - mlp.silu(z - 1e-6)) / 2e-6
    assert np.allclose(mlp.silu_grad(z), fd, rtol=1e-7, atol=1e-9)
    assert mlp.silu(0.0) == 0.0 and abs(mlp.silu(50.0) - 50.0) < 1e-12


def test_first_adam_step_moves_each_weight_by_lr():
    """At t = 1 the bias-corrected moments give m_hat / sqrt(v_hat) = sign(g),
    so every parameter with a nonzero gradient moves by exactly lr (up to eps)."""
    _, x, t = _data()
    P = mlp.init(4)
    y, cache = mlp.forward(P, x)
    g = mlp.backward(P, cache, y, t)
    P0 = {k: v.copy() for k, v in P.items()}
    mlp.adam_step(P, g, mlp.adam_init(P), lr=1e-3, eps=1e-12)
    for k in P:
        step = P0[k] - P[k]
        nz = np.abs(g[k]) > 1e-9
        assert np.allclose(step[nz], 1e-3 * np.sign(g[k][nz]), rtol=1e-6, atol=0)


def test_features_invariant_under_scalings_and_boosts():
    st, x, _ = _data(32, seed=5)
    rl, ul, pl, rr, ur, pr = st
    a, b, s = 3.7, 0.02, -1.3
    # rho -> a rho, p -> b p: velocities scale with sqrt(b / a); then a Galilean shift
    v = np.sqrt(b / a)
    x2, _ = mlp.features(a * rl, v * ul + s, b * pl, a * rr, v * ur + s, b * pr, 5.0 / 3.0)
    assert np.allclose(x, x2, rtol=0, atol=1e-12)
    # and so is the target: two-shock p* scales with b
    P = oracle.Params()
    o1 = oracle.riemann(rl, ul, pl, rr, ur, pr, P)
    o2 = oracle.riemann(a * rl, v * ul + s, b * pl, a * rr, v * ur + s, b * pr, P)
    ok = (o1["pstar"] > 1e-20) & (o2["pstar"] > 1e-20)
    assert np.allclose(mlp.target(o1["pstar"], pl, pr)[ok], mlp.target(o2["pstar"], b * pl, b * pr)[ok],
                       atol=1e-10)


def test_training_fits_the_two_shock_root():
    """A few hundred Adam steps on converged two-shock roots cut the error of the
    plain acoustic guess by a large factor on held-out states."""
    rng = np.random.default_rng(7)
    st = synth.riemann_states(rng, 6000, mach=1.0, log_rho_sd=0.5, log_p_sd=0.5)
    P_or = oracle.Params()
    o = oracle.riemann(*st, P_or)
    x, _ = mlp.features(*st, 5.0 / 3.0)
    t = mlp.target(o["pstar"], st[2], st[5])
    tr, te = slice(0, 5000), slice(5000, 6000)
    P = mlp.init(0)
    S = mlp.adam_init(P)
    for it in range(600):
        idx = rng.integers(0, 5000, 256)
        y, cache = mlp.forward(P, x[idx])
        mlp.adam_step(P, mlp.backward(P, cache, y, t[idx]), S, lr=3e-3)
    err = np.sqrt(mlp.mse(mlp.forward(P, x[te])[0], t[te]))
    # acoustic two-shock guess of the same held-out states, in the same log units
    rl, ul, pl, rr, ur, pr = (a[te] for a in st)
    CL, CR = np.sqrt(5 / 3 * pl * rl), np.sqrt(5 / 3 * pr * rr)
    p0 = np.maximum((CR * pl + CL * pr + CL * CR * (ul - ur)) / (CL + CR), 1e-30)
    base = np.sqrt(np.mean((np.log(p0 / np.sqrt(pl * pr)) - t[te]) ** 2))
    assert err < 0.5 * base, (err, base)


def test_bf16_rounding():
    a = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 0.0])
    b = mlp.bf16(a)
    assert b[0] == 1.0 and b[1] == 1.0 and b[2] == 1.0078125 and abs(b[3] + 3.140625) < 1e-12 and b[4] == 0
