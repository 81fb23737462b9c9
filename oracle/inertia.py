"""Sylvester inertia count of a banded symmetric matrix (oracle; test-only).

The number of eigenvalues of A below sigma equals the number of negative
pivots of the LDL^T factorisation of A - sigma I (Sylvester's law of inertia).
For the 5-point operators in row-major order A is banded with half-bandwidth
n, so elimination only touches an (n+1) x (n+1) window that slides down the
diagonal: O(N n^2) work and O(n^2) memory. A count of exactly k below
sigma = (lambda_k + lambda_{k+1})/2 certifies that no eigenvalue was missed.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def count_below(A: sp.spmatrix, sigma: float, bandwidth: int) -> int:
    """Number of eigenvalues of symmetric banded A that are < sigma."""
    A = sp.csr_matrix(A, dtype=np.float64)
    N = A.shape[0]
    w = bandwidth
    size = w + 1

    def band_row(r):
        """Row r of A - sigma I restricted to columns r..r+w, as a dense vector."""
        out = np.zeros(size)
        start, end = A.indptr[r], A.indptr[r + 1]
        cols = A.indices[start:end]
        vals = A.data[start:end]
        m = (cols >= r) & (cols <= r + w)
        out[cols[m] - r] = vals[m]
        out[0] -= sigma
        return out

    # window W holds rows/cols r..r+w of the partially eliminated matrix
    W = np.zeros((size, size))
    for t in range(min(size, N)):
        row = band_row(t)
        W[t, t:] = row[: size - t]
        W[t:, t] = row[: size - t]
    negatives = 0
    for r in range(N):
        piv = W[0, 0]
        if piv == 0.0:
            piv = -np.finfo(float).tiny
        if piv < 0:
            negatives += 1
        l = W[1:, 0] / piv
        W[1:, 1:] -= piv * np.outer(l, l)
        # slide the window by one
        W[:-1, :-1] = W[1:, 1:]
        W[-1, :] = 0.0
        W[:, -1] = 0.0
        nr = r + size
        if nr < N:
            row = band_row(nr)          # columns nr..nr+w; only nr itself is in the window
            W[-1, -1] = row[0]
            # couplings of row nr to rows r+1..r+w (columns < nr): original entries
            start, end = A.indptr[nr], A.indptr[nr + 1]
            cols = A.indices[start:end]
            vals = A.data[start:end]
            m = (cols > r) & (cols < nr)
            W[-1, cols[m] - (r + 1)] = vals[m]
            W[cols[m] - (r + 1), -1] = vals[m]
    return negatives
