"""Dense eigensolvers (oracle; test-only).

``smallest_eigenpairs`` is the plain definition of what the method returns
(Eq. (eq:eq_basic) with the k algebraically smallest pairs): the full dense
symmetric eigendecomposition (LAPACK through numpy) truncated to k.

``cyclic_jacobi`` is the textbook cyclic-by-row Jacobi method for tiny
symmetric matrices; it pins the library routine on small inputs and serves as
an independent check of the reduced eigensolve.
"""
from __future__ import annotations

import numpy as np


def smallest_eigenpairs(A, k: int):
    """The k algebraically smallest eigenpairs of symmetric A (dense, N <= a few thousand)."""
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A, dtype=np.float64)
    w, V = np.linalg.eigh(Ad)
    return w[:k], V[:, :k]


def cyclic_jacobi(S: np.ndarray, tol: float = 1e-15, max_sweeps: int = 50):
    """All eigenpairs of a small symmetric matrix by cyclic Jacobi rotations.

    Each rotation zeroes S[p, q] using the classical angle choice
    (t = sign(theta)/(|theta| + sqrt(theta^2 + 1)), theta = (S_qq - S_pp)/(2 S_pq)).
    Returns ascending eigenvalues and the matching eigenvectors as columns.
    """
    S = np.array(S, dtype=np.float64, copy=True)
    n = S.shape[0]
    V = np.eye(n)
    for _ in range(max_sweeps):
        off = np.sqrt(np.sum(np.tril(S, -1) ** 2))
        if off <= tol * np.sqrt(np.sum(S * S)):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if S[p, q] == 0.0:
                    continue
                theta = (S[q, q] - S[p, p]) / (2.0 * S[p, q])
                t = np.sign(theta) / (abs(theta) + np.sqrt(theta * theta + 1.0)) if theta != 0 else 1.0
                c = 1.0 / np.sqrt(t * t + 1.0)
                s = t * c
                J = np.eye(n)
                J[p, p] = c
                J[q, q] = c
                J[p, q] = s
                J[q, p] = -s
                S = J.T @ S @ J
                V = V @ J
    w = np.diag(S).copy()
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]
