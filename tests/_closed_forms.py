"""Closed-form solutions used to pin the oracle (textbook results, not the paper's).

* Semi-infinite solid with convective surface cooling (Carslaw & Jaeger,
  "Conduction of Heat in Solids", Sec. 2.7).
* Two-phase Neumann solution of the Stefan problem with equal properties
  (Carslaw & Jaeger Sec. 11.2).
"""
import numpy as np
from scipy.optimize import brentq
from scipy.special import erf, erfc, erfcx


def robin_semi_infinite(x, t, alpha, H, Ti, Text):
    """T(x, t) for x > 0, T(x, 0) = Ti, -k T_x = h (Text - T) at x = 0, H = h / k:
    (T - Ti)/(Text - Ti) = erfc(xi) - exp(H x + H^2 alpha t) erfc(xi + H sqrt(alpha t))."""
    s = np.sqrt(alpha * t)
    xi = x / (2.0 * s)
    theta = erfc(xi) - np.exp(-xi * xi) * erfcx(xi + H * s)
    return Ti + (Text - Ti) * theta


def neumann_lambda(St, nu):
    """Root of exp(-l^2)/erf(l) - nu exp(-l^2)/erfc(l) = l sqrt(pi) / St, where
    St = c_p (T_f - T_w)/L and nu = (T_i - T_f)/(T_f - T_w) (equal diffusivities)."""
    f = lambda l: np.exp(-l * l) / erf(l) - nu * np.exp(-l * l) / erfc(l) - l * np.sqrt(np.pi) / St
    return brentq(f, 1e-6, 5.0)


def neumann_front(t, alpha, St, nu):
    """Solid-liquid front position X(t) = 2 lambda sqrt(alpha t)."""
    return 2.0 * neumann_lambda(St, nu) * np.sqrt(alpha * t)


def linear_wall_semi_infinite(x, t, alpha, Ti, rate):
    """T(x, t) for x > 0, T(x, 0) = Ti, wall temperature Ti + rate * t
    (Carslaw & Jaeger Sec. 2.5): T - Ti = rate t 4 i^2erfc(xi), with
    4 i^2erfc(z) = (1 + 2 z^2) erfc(z) - 2 z exp(-z^2)/sqrt(pi), xi = x/(2 sqrt(alpha t))."""
    xi = x / (2.0 * np.sqrt(alpha * t))
    return Ti + rate * t * ((1.0 + 2.0 * xi * xi) * erfc(xi) - 2.0 * xi * np.exp(-xi * xi) / np.sqrt(np.pi))
