"""Correctly rounded block products (oracle; test-only).

The block products of Alg. 3 (Gram matrices X^T X of the orthonormalisation step, the
Rayleigh-Ritz matrix Q^T (A Q), the rotation X = Q Z) are plain sums of products. The
oracle computes each entry as the FP64 number nearest to the exact real sum: every
product a b is split without error into p + e (Dekker's TwoProduct with Veltkamp's
splitting, valid while no product overflows or underflows), and math.fsum returns the
correctly rounded sum of all 2 K terms. No blocking, no reordering that could matter:
the result does not depend on the order of the terms at all.
"""
from __future__ import annotations

import math

import numpy as np

_SPLIT = 134217729.0  # 2^27 + 1 (Veltkamp)


def _split(a):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def two_product(a, b):
    """p, e with p = fl(a b) and p + e = a b exactly (elementwise)."""
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def exact_tn(A, B):
    """C[i, j] = round(sum_k A[k, i] B[k, j]) for A [K, m], B [K, n] (FP64)."""
    A = np.asarray(A, dtype=np.float64)
    B = np.asarray(B, dtype=np.float64)
    m, n = A.shape[1], B.shape[1]
    C = np.empty((m, n))
    for i in range(m):
        p, e = two_product(A[:, i:i + 1], B)  # [K, n]
        for j in range(n):
            C[i, j] = math.fsum(np.concatenate([p[:, j], e[:, j]]))
    return C


def exact_nn(X, M):
    """Y[r, j] = round(sum_k X[r, k] M[k, j]) for X [rows, K], M [K, n] (FP64)."""
    return exact_tn(np.asarray(X, dtype=np.float64).T, M)
