"""The Sedov-Taylor similarity solution of a spherical point explosion, by direct
integration of the similarity equations (test infrastructure).

With xi = r / R(t), R = xi0 (E t^2 / rho0)^(1/5) and U = dR/dt, the flow behind the
shock is rho = rho0 G(xi), v = U F(xi), p = rho0 U^2 P(xi).  Substituting into the
Euler equations (mass, momentum, and the entropy of each fluid element, since the
flow is adiabatic behind the shock) gives three first-order ODEs in xi:

    G F' + (F - xi) G'                       = -2 F G / xi
    (F - xi) F' + P' / G                     = 3/2 F
    -gamma (F - xi) G' / G + (F - xi) P' / P = 3

(3/2 and 3 come from dU/dt = -3/2 U^2 / R, i.e. R ~ t^(2/5)).  The strong-shock
jump conditions fix the values at xi = 1: G = (gamma+1)/(gamma-1),
F = P = 2/(gamma+1).  Integrating inwards and requiring that the energy behind
the shock is E,

    E = 4 pi rho0 U^2 R^3 I,   I = int_0^1 (G F^2 / 2 + P / (gamma-1)) xi^2 dxi,

with U^2 R^3 = (4/25) xi0^5 E / rho0, gives xi0 = (25 / (16 pi I))^(1/5).
"""
import math

import numpy as np
from scipy.integrate import quad, solve_ivp


def _rhs(gamma):
    def f(x, y):
        F, G, P = y
        A = np.array([[G, F - x, 0.0],
                      [F - x, 0.0, 1.0 / G],
                      [0.0, -gamma * (F - x) / G, (F - x) / P]])
        b = np.array([-2.0 * F * G / x, 1.5 * F, 3.0])
        return np.linalg.solve(A, b)
    return f


def similarity(gamma: float, xi_min: float = 1e-6) -> dict:
    """xi0, the energy integrals and the profiles F, G, P (callables of xi)."""
    y1 = [2.0 / (gamma + 1), (gamma + 1) / (gamma - 1), 2.0 / (gamma + 1)]
    sol = solve_ivp(_rhs(gamma), (1.0, xi_min), y1, rtol=1e-11, atol=1e-14,
                    dense_output=True, method="LSODA")
    if sol.status != 0:
        raise RuntimeError(sol.message)
    kin, _ = quad(lambda x: 0.5 * sol.sol(x)[1] * sol.sol(x)[0] ** 2 * x * x, xi_min, 1.0,
                  limit=200, epsabs=1e-13)
    th, _ = quad(lambda x: sol.sol(x)[2] / (gamma - 1) * x * x, xi_min, 1.0, limit=200,
                 epsabs=1e-13)
    total = kin + th
    return dict(xi0=(25.0 / (16.0 * math.pi * total)) ** 0.2, e_kin_frac=kin / total,
                F=lambda x: sol.sol(x)[0], G=lambda x: sol.sol(x)[1], P=lambda x: sol.sol(x)[2])
