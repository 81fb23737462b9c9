"""Pins for oracle.chebyshev (Sec. 2.2, Alg. 1) against closed forms and a library routine."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

import scsf_inputs as si
from oracle import chebyshev, operators, sturm


def lib_T(m, t):
    """C_m(t) by numpy's Chebyshev-series evaluation (an independent library routine)."""
    coef = np.zeros(m + 1)
    coef[m] = 1.0
    return float(npcheb.chebval(t, coef))


@pytest.mark.parametrize("t", [-2.5, -1.0, -0.7, 0.0, 0.3, 0.99, 1.0, 1.4, 3.0])
def test_chebyshev_T_explicit_polynomials(t):
    explicit = [1.0, t, 2 * t**2 - 1, 4 * t**3 - 3 * t, 8 * t**4 - 8 * t**2 + 1,
                16 * t**5 - 20 * t**3 + 5 * t]
    for m, val in enumerate(explicit):
        assert chebyshev.chebyshev_T(m, t) == pytest.approx(val, rel=1e-12, abs=1e-12)
    for m in [7, 12, 20]:
        assert chebyshev.chebyshev_T(m, t) == pytest.approx(lib_T(m, t), rel=1e-10, abs=1e-12)


def test_filter_on_exact_eigenvector():
    """For an exact eigenvector v: filter(v) = C_m(t_v)/C_m(t_lambda) v, t = (x - c)/e."""
    n = 10
    A = operators.assemble(si.constant_div_a_grad(n))
    h = 1.0 / (n + 1)
    lam_min = 8.0 / h**2 * np.sin(np.pi * h / 2) ** 2
    alpha, beta = 300.0, 8.0 / h**2
    c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
    for (p, q) in [(1, 1), (2, 3), (6, 6), (10, 9)]:
        v = sturm.laplacian_2d_mode(n, p, q)
        lv = 4.0 / h**2 * (np.sin(p * np.pi * h / 2) ** 2 + np.sin(q * np.pi * h / 2) ** 2)
        for m in [1, 2, 7, 16]:
            y = chebyshev.chebyshev_filter(A, v[:, None], m, lam_min, c, e)[:, 0]
            expect = lib_T(m, (lv - c) / e) / lib_T(m, (lam_min - c) / e)
            np.testing.assert_allclose(y, expect * v, rtol=1e-12, atol=1e-13)


def test_filter_block_matches_spectral_definition():
    """Y_m = V diag(C_m(t_i)/C_m(t_lambda)) V^T Y0 on a random-coefficient operator (brute force)."""
    n = 6
    op = si.div_a_grad_chain(n, 1, seed=4)[0]
    A = operators.assemble(op)
    w, V = np.linalg.eigh(A.toarray())
    lam, alpha, beta = w[0], w[8], w[-1] * 1.01
    c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
    Y0 = np.random.default_rng(0).standard_normal((n * n, 5))
    for m in [3, 10, 20]:
        scale = np.array([lib_T(m, (x - c) / e) for x in w]) / lib_T(m, (lam - c) / e)
        ref = V @ (scale[:, None] * (V.T @ Y0))
        got = chebyshev.chebyshev_filter(A, Y0, m, lam, c, e)
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-10 * np.max(np.abs(ref)))
