"""Comparisons between two eigen-solutions (oracle side; test-only).

Eigenvalues are compared as sorted lists. Eigenvectors are compared per
cluster of (near-)equal eigenvalues by the largest principal angle between the
spanned subspaces, since any orthonormal basis of a degenerate eigenspace is
an equally valid answer.
"""
from __future__ import annotations

import numpy as np


def max_rel_eig_error(ref: np.ndarray, got: np.ndarray) -> float:
    ref = np.sort(np.asarray(ref, dtype=np.float64))
    got = np.sort(np.asarray(got, dtype=np.float64))
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), np.finfo(float).tiny)))


def clusters(evals: np.ndarray, rel_gap: float = 1e-6):
    """Split ascending eigenvalues into runs whose consecutive relative gap is < rel_gap."""
    groups = [[0]]
    for i in range(1, len(evals)):
        scale = max(abs(evals[i]), abs(evals[i - 1]), np.finfo(float).tiny)
        if (evals[i] - evals[i - 1]) / scale < rel_gap:
            groups[-1].append(i)
        else:
            groups.append([i])
    return groups


def max_subspace_angle(U: np.ndarray, V: np.ndarray) -> float:
    """Largest principal angle (radians) between span(U) and span(V), U, V orthonormal-ish."""
    Qu, _ = np.linalg.qr(U)
    Qv, _ = np.linalg.qr(V)
    s = np.linalg.svd(Qu.T @ Qv, compute_uv=False)
    return float(np.arccos(np.clip(np.min(s), -1.0, 1.0)))


def max_cluster_angle(ref_vals, ref_vecs, got_vecs, rel_gap: float = 1e-6, skip_last: bool = True) -> float:
    """Max principal angle over eigenvalue clusters of ref (both in ascending order).

    A cluster that touches the end of the list may continue past it, so it is
    skipped when ``skip_last`` is set.
    """
    worst = 0.0
    groups = clusters(np.asarray(ref_vals), rel_gap)
    for g in groups:
        if skip_last and g[-1] == len(ref_vals) - 1 and len(groups) > 1:
            continue
        worst = max(worst, max_subspace_angle(ref_vecs[:, g], got_vecs[:, g]))
    return worst


def orthonormality_error(X: np.ndarray) -> float:
    return float(np.max(np.abs(X.T @ X - np.eye(X.shape[1]))))
