"""Pins of the correctly rounded block products (oracle/products.py).

Exact rational arithmetic (fractions.Fraction) is the independent reference: every FP64
input is a rational number, so the exact sum is known and rounds to one FP64 value.
"""
from fractions import Fraction

import numpy as np

from oracle import products


def _rational_tn(A, B):
    m, n = A.shape[1], B.shape[1]
    C = np.empty((m, n))
    for i in range(m):
        for j in range(n):
            s = sum((Fraction(float(a)) * Fraction(float(b)) for a, b in zip(A[:, i], B[:, j])),
                    Fraction(0))
            C[i, j] = float(s)  # Fraction -> float rounds to nearest
    return C


def test_two_product_is_error_free():
    rng = np.random.default_rng(0)
    a = rng.standard_normal(200) * 10.0 ** rng.integers(-30, 30, 200)
    b = rng.standard_normal(200) * 10.0 ** rng.integers(-30, 30, 200)
    p, e = products.two_product(a, b)
    for x, y, pp, ee in zip(a, b, p, e):
        assert Fraction(float(pp)) + Fraction(float(ee)) == Fraction(float(x)) * Fraction(float(y))


def test_exact_tn_matches_rational_arithmetic():
    rng = np.random.default_rng(1)
    K, m, n = 37, 4, 3
    A = rng.standard_normal((K, m)) * np.logspace(-30, 3, m)
    B = rng.standard_normal((K, n)) * np.logspace(3, -12, n)
    assert np.array_equal(products.exact_tn(A, B), _rational_tn(A, B))


def test_cancellation_that_plain_summation_loses():
    A = np.array([[1e16], [1.0], [-1e16], [2.0 ** -60]])
    B = np.ones((4, 1))
    left_to_right = 0.0
    for v in A[:, 0]:
        left_to_right += v  # 1e16 + 1 rounds back to 1e16: the 1 is lost
    assert left_to_right == 2.0 ** -60
    assert products.exact_tn(A, B)[0, 0] == float(Fraction(1) + Fraction(2) ** -60)


def test_integer_matrices_and_nn_form():
    rng = np.random.default_rng(2)
    X = rng.integers(-1000, 1000, (50, 7)).astype(np.float64)
    M = rng.integers(-1000, 1000, (7, 5)).astype(np.float64)
    assert np.array_equal(products.exact_nn(X, M), X @ M)  # small integers: exact in FP64
    assert np.array_equal(products.exact_tn(X, X), X.T @ X)
