"""Sedov-Taylor point blast (the blast test of Sec. 11): the similarity
constant xi0 of r_shock = xi0 (E t^2 / rho0)^(1/(nu+2)), nu = 3 spherical,
2 cylindrical (E per unit length), from the self-similar Euler equations,
integrated here rather than quoted.

With lambda = r / r_shock(t), alpha = 2/(nu+2) and
  v = alpha (r/t) V(lambda),  rho = rho0 G(lambda),  p = rho0 alpha^2 (r/t)^2 P(lambda),
the continuity, momentum and entropy equations become, with ' = d/d ln(lambda),
  G V' + (V-1) G'                          = -nu G V
  alpha (V-1) V' + (alpha/G) P'            = V - alpha V^2 - 2 alpha P / G
  -gamma alpha (V-1)/G G' + alpha (V-1)/P P' = 2 - 2 alpha V
with the strong-shock jump conditions V = P = 2/(gamma+1), G = (gamma+1)/(gamma-1)
at lambda = 1.  Energy: E = A_nu rho0 alpha^2 r_s^(nu+2) / t^2 * I with
I = int_0^1 lambda^(nu+1) (G V^2 / 2 + P / (gamma-1)) d lambda and A_nu = 4 pi
(nu = 3) or 2 pi (nu = 2), so xi0 = (A_nu alpha^2 I)^(-1/(nu+2)).  The centre
is approached as G -> 0, where the system is stiff; fixed-step RK4 in
ln(lambda) down to lambda = e^-3 drops a part of I below 1e-6 of it.
"""
import numpy as np


def _rhs(y, gamma, nu):
    a = 2.0 / (nu + 2.0)
    V, G, P = y
    A = np.array([[G, V - 1.0, 0.0],
                  [a * (V - 1.0), 0.0, a / G],
                  [0.0, -gamma * a * (V - 1.0) / G, a * (V - 1.0) / P]])
    b = np.array([-nu * G * V, V - a * V * V - 2.0 * a * P / G, 2.0 - 2.0 * a * V])
    return np.linalg.solve(A, b)


def xi0(gamma, nu=3, h=-5e-4, s_min=-3.0):
    a = 2.0 / (nu + 2.0)
    y = np.array([2.0 / (gamma + 1.0), (gamma + 1.0) / (gamma - 1.0), 2.0 / (gamma + 1.0)])

    def f(y, s):
        lam = np.exp(s)
        V, G, P = y
        return lam ** (nu + 2) * (G * V * V / 2.0 + P / (gamma - 1.0))   # lambda^(nu+1) (...) d lambda / d s

    s, integral, fp = 0.0, 0.0, f(y, 0.0)
    while s > s_min:
        k1 = _rhs(y, gamma, nu)
        k2 = _rhs(y + 0.5 * h * k1, gamma, nu)
        k3 = _rhs(y + 0.5 * h * k2, gamma, nu)
        k4 = _rhs(y + h * k3, gamma, nu)
        y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        s += h
        fn = f(y, s)
        integral += -h * 0.5 * (fp + fn)
        fp = fn
    area = 4.0 * np.pi if nu == 3 else 2.0 * np.pi
    return (area * a * a * integral) ** (-1.0 / (nu + 2))
