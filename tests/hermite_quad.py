"""Velocity-space quadrature used to pin the oracle (tests only).

Independent of the oracle: basis functions are evaluated straight from the definition of
Sec. 2.2 (eq. dis-expansion) with numpy's probabilists' Hermite routines, and integrals
over R^3 use tensor Gauss-Hermite rules (exact for polynomial x Gaussian integrands of
the degrees used here) or Gauss-Legendre rules on truncated half-lines.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import hermite_e as He
from numpy.polynomial.legendre import leggauss


def H_values(al: np.ndarray, w, t, xi: np.ndarray) -> np.ndarray:
    """H_alpha^[w,t](xi) for every multi-index row of al; xi has shape (P,3). Returns (P, n)."""
    w = np.asarray(w, dtype=float)
    v = (xi - w[None, :]) / math.sqrt(t)
    M = int(al.sum(1).max())
    vals = [He.hermevander(v[:, d], M) for d in range(3)]  # (P, M+1)
    gauss = np.exp(-0.5 * (v ** 2).sum(1)) / (2 * math.pi * t) ** 1.5
    out = np.empty((xi.shape[0], al.shape[0]))
    for o, (a1, a2, a3) in enumerate(al):
        out[:, o] = vals[0][:, a1] * vals[1][:, a2] * vals[2][:, a3] * t ** (-(a1 + a2 + a3) / 2)
    return out * gauss[:, None]


def He_products(al: np.ndarray, w, t, xi: np.ndarray) -> np.ndarray:
    """prod_d He_{alpha_d}(v_d), v = (xi-w)/sqrt(t). Returns (P, n)."""
    w = np.asarray(w, dtype=float)
    v = (xi - w[None, :]) / math.sqrt(t)
    M = int(al.sum(1).max())
    vals = [He.hermevander(v[:, d], M) for d in range(3)]
    out = np.empty((xi.shape[0], al.shape[0]))
    for o, (a1, a2, a3) in enumerate(al):
        out[:, o] = vals[0][:, a1] * vals[1][:, a2] * vals[2][:, a3]
    return out


def gauss_rule(w, t, nq: int):
    """Nodes xi (P,3) and weights for int g(xi) d xi where g = Gaussian[w,t] * polynomial.

    Returns weights that already divide out exp(-|v|^2/2), so sum(W * g(xi)) approximates
    the integral of g."""
    x, wx = He.hermegauss(nq)
    X = np.stack(np.meshgrid(x, x, x, indexing="ij"), -1).reshape(-1, 3)
    W = (wx[:, None, None] * wx[None, :, None] * wx[None, None, :]).reshape(-1)
    w = np.asarray(w, dtype=float)
    xi = w[None, :] + math.sqrt(t) * X
    W = W * np.exp(0.5 * (X ** 2).sum(1)) * t ** 1.5
    return xi, W


def project(al: np.ndarray, w, t, g_vals: np.ndarray, xi: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Coefficients of g in F_M^[w,t]: g_alpha = t^{|alpha|/2}/alpha! int g He_alpha(v) dxi."""
    P = He_products(al, w, t, xi)
    deg = al.sum(1)
    fact = np.array([math.factorial(a) * math.factorial(b) * math.factorial(c) for a, b, c in al], dtype=float)
    integ = (W[:, None] * g_vals[:, None] * P).sum(0)
    return integ * t ** (deg / 2.0) / fact


def half_line_rule(sign: int, n: int = 400, L: float = 16.0):
    """Gauss-Legendre nodes/weights on [0, L] (sign=+1) or [-L, 0] (sign=-1)."""
    x, wx = leggauss(n)
    x = 0.5 * L * (x + 1.0)
    wx = 0.5 * L * wx
    return sign * x, wx
