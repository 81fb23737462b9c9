"""Chebyshev polynomials and the scaled Chebyshev filter (oracle; test-only).

Sec. 2.2 defines C_m(t) = cos(m arccos t) on [-1, 1] with the three-term
recurrence C_{m+1} = 2 t C_m - C_{m-1}; Alg. 1 applies the scaled form to a
block. Reading of Alg. 1's recurrence (its printed last term uses Y_i): the
update is

    Y_{i+1} = 2 sigma_{i+1} Abar Y_i - sigma_{i+1} sigma_i Y_{i-1},
    Abar = (A - c I)/e,  sigma_1 = e/(lambda - c),  sigma_{i+1} = 1/(2/sigma_1 - sigma_i),

which is the only form consistent with the sigma update: it yields
Y_m = C_m(Abar) Y_0 / C_m(t_lambda), t_lambda = (lambda - c)/e. All columns use
the same degree m.
"""
from __future__ import annotations

import numpy as np


def chebyshev_T(m: int, t: float) -> float:
    """C_m(t): cos(m arccos t) for |t| <= 1, (+/-)cosh(m arccosh |t|) outside."""
    if abs(t) <= 1.0:
        return float(np.cos(m * np.arccos(t)))
    v = float(np.cosh(m * np.arccosh(abs(t))))
    return v if (t > 0 or m % 2 == 0) else -v


def chebyshev_filter(A, Y0: np.ndarray, m: int, lam: float, c: float, e: float) -> np.ndarray:
    """Alg. 1: Y_m = C_m(Abar) Y0 / C_m(t_lambda) by the scaled three-term recurrence."""
    assert m >= 1 and e > 0

    def abar(Y):
        return (A @ Y - c * Y) / e

    sigma1 = e / (lam - c)
    Y_prev = Y0
    Y = sigma1 * abar(Y0)
    sigma = sigma1
    for _ in range(1, m):
        sigma_next = 1.0 / (2.0 / sigma1 - sigma)
        Y_next = 2.0 * sigma_next * abar(Y) - sigma_next * sigma * Y_prev
        Y_prev, Y, sigma = Y, Y_next, sigma_next
    return Y
