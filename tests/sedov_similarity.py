"""Sedov-Taylor point-blast similarity solution (spherical, strong shock),
integrated numerically from the self-similar Euler equations — an
independent reference for the oracle's blast-wave runs.

With xi = r/R(t), R = xi0 (E t^2/rho0)^(1/5), write u = (2/5)(r/t) V(xi),
rho = rho0 G(xi), p = (4/25) rho0 (r/t)^2 P(xi).  Mass, momentum and entropy
conservation become, with ' = d/d ln xi,
    (V-1) G'/G + V' = -3V
    (V-1) V' + P'/G = -V^2 + (5/2) V - 2 P/G
    (V-1) (P'/P - gamma G'/G) = 5 - 2V
with the strong-shock values V = P = 2/(gamma+1), G = (gamma+1)/(gamma-1) at
xi = 1.  The blast energy E = (16 pi/25) rho0 R^5 t^-2 * I with
I = int_0^1 xi^4 (G V^2/2 + P/(gamma-1)) dxi fixes xi0 = ((16 pi/25) I)^(-1/5).
"""
import numpy as np
from scipy.integrate import solve_ivp


def _rhs(s, y, gamma):
    V, G, P = y
    Z = P / G
    num = -V * V + 2.5 * V - 2.0 * Z - Z * (5.0 - 2.0 * V - 3.0 * gamma * V) / (V - 1.0)
    den = (V - 1.0) - gamma * Z / (V - 1.0)
    dV = num / den
    dlnG = (-3.0 * V - dV) / (V - 1.0)
    dlnP = (5.0 - 2.0 * V) / (V - 1.0) + gamma * dlnG
    return [dV, G * dlnG, P * dlnP]


def profile(gamma, s_min=-12.0, npts=4000):
    """(xi, V, G, P) from the shock (xi = 1) inward to xi = exp(s_min)."""
    y0 = [2.0 / (gamma + 1.0), (gamma + 1.0) / (gamma - 1.0), 2.0 / (gamma + 1.0)]
    s = np.linspace(0.0, s_min, npts)
    sol = solve_ivp(_rhs, (0.0, s_min), y0, t_eval=s, args=(gamma,), rtol=1e-11, atol=1e-14, method="LSODA")
    return np.exp(sol.t), sol.y[0], sol.y[1], sol.y[2]


def xi0(gamma):
    xi, V, G, P = profile(gamma)
    f = xi ** 4 * (0.5 * G * V * V + P / (gamma - 1.0))
    # integrate over xi in [exp(s_min), 1]; the remainder near 0 is negligible (f ~ xi^4)
    I = -np.trapezoid(f, xi)
    return ((16.0 * np.pi / 25.0) * I) ** (-0.2)
