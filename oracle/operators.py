"""FDM operators, spectral bounds and the residual metric (oracle; test-only).

Sec. 2.1 (Eq. (eq_p)) turns an operator on an n x n grid into a sparse matrix
with row-major node order; App. D.2 item 1 states the generalized Poisson
operator -div(K grad h) discretised by central differences with Dirichlet
boundaries. We assemble the symmetric (conservative) 5-point form

  (A u)_ij = [ a_{i+1/2,j}(u_ij - u_{i+1,j}) + a_{i-1/2,j}(u_ij - u_{i-1,j})
             + a_{i,j+1/2}(u_ij - u_{i,j+1}) + a_{i,j-1/2}(u_ij - u_{i,j-1}) ] / h^2

with u = 0 outside the grid, node index I = i*n + j and h = 1/(n+1).
The -Lap u + V u operator is the same with a == 1 plus diag(V).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def assemble_div_a_grad(n: int, ax: np.ndarray, ay: np.ndarray) -> sp.csr_matrix:
    """Sparse A for -div(a grad u) (App. D.2 item 1; Sec. 2.1 node order).

    ax[f, j] is a on the x-face between nodes (f-1, j) and (f, j), f = 0..n;
    ay[i, g] is a on the y-face between nodes (i, g-1) and (i, g), g = 0..n.
    """
    h = 1.0 / (n + 1)
    inv_h2 = 1.0 / (h * h)
    rows, cols, vals = [], [], []
    for i in range(n):
        for j in range(n):
            I = i * n + j
            a_w = ax[i, j]          # face between (i-1, j) and (i, j)
            a_e = ax[i + 1, j]      # face between (i, j) and (i+1, j)
            a_s = ay[i, j]          # face between (i, j-1) and (i, j)
            a_n = ay[i, j + 1]      # face between (i, j) and (i, j+1)
            rows.append(I); cols.append(I); vals.append((a_w + a_e + a_s + a_n) * inv_h2)
            if i > 0:
                rows.append(I); cols.append(I - n); vals.append(-a_w * inv_h2)
            if i < n - 1:
                rows.append(I); cols.append(I + n); vals.append(-a_e * inv_h2)
            if j > 0:
                rows.append(I); cols.append(I - 1); vals.append(-a_s * inv_h2)
            if j < n - 1:
                rows.append(I); cols.append(I + 1); vals.append(-a_n * inv_h2)
    N = n * n
    return sp.csr_matrix((np.array(vals), (np.array(rows), np.array(cols))), shape=(N, N))


def assemble_lap_plus_v(n: int, V: np.ndarray) -> sp.csr_matrix:
    """Sparse A for -Lap u + V u: 5-point Laplacian plus diag(V) (App. D.2 item 3 stand-in)."""
    ones_x = np.ones((n + 1, n))
    ones_y = np.ones((n, n + 1))
    A = assemble_div_a_grad(n, ones_x, ones_y)
    return (A + sp.diags(V.reshape(-1))).tocsr()


def laplacian(n: int) -> sp.csr_matrix:
    """-Lap_h: the 5-point Dirichlet Laplacian (a == 1 in the conservative form)."""
    return assemble_div_a_grad(n, np.ones((n + 1, n)), np.ones((n, n + 1)))


def assemble_plate_stiffness(n: int, D: np.ndarray) -> sp.csr_matrix:
    """K for div(grad(D lap u)) (App. D.2 item 4): K = L diag(D) L with L = -Lap_h.

    Reading of the boundary condition: the paper states only "Dirichlet"; a fourth-order
    operator needs two conditions, taken as u = 0 and D lap u = 0 on the boundary (the
    simply supported plate). Both come from composing two Dirichlet Laplacians: the inner
    one sees u = 0 outside, the outer one sees D lap u = 0 outside. K is symmetric
    positive definite with a 13-point stencil."""
    L = laplacian(n)
    return (L @ sp.diags(D.reshape(-1)) @ L).tocsr()


def assemble_plate(n: int, D: np.ndarray, rho: np.ndarray) -> sp.csr_matrix:
    """The generalized problem K u = lambda M u, M = diag(rho), in symmetric standard form
    C = M^{-1/2} K M^{-1/2}: C v = lambda v with u = M^{-1/2} v."""
    s = sp.diags(1.0 / np.sqrt(rho.reshape(-1)))
    return (s @ assemble_plate_stiffness(n, D) @ s).tocsr()


def assemble(op) -> sp.csr_matrix:
    """Dispatch on the workload type (duck-typed: .ax/.ay, .V, .D/.rho (standard form of the
    plate problem), or CSR arrays taken as given)."""
    if hasattr(op, "rho"):
        return assemble_plate(op.n, op.D, op.rho)
    if hasattr(op, "row_ptr"):
        return sp.csr_matrix((op.val, op.col, op.row_ptr), shape=(op.rows, op.rows))
    if hasattr(op, "ax"):
        return assemble_div_a_grad(op.n, op.ax, op.ay)
    return assemble_lap_plus_v(op.n, op.V)


def gershgorin_bounds(A: sp.csr_matrix):
    """[lo, hi] containing the spectrum of symmetric A (Gershgorin disc theorem).

    hi is the upper end beta of the unwanted interval [alpha, beta] in the
    filter parameters of Sec. 2.2.
    """
    A = A.tocsr()
    d = A.diagonal()
    absrow = np.asarray(abs(A).sum(axis=1)).ravel()
    radius = absrow - np.abs(d)
    return float(np.min(d - radius)), float(np.max(d + radius))


def relative_residuals(A, X: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """App. D.5: ||A v - lambda v||_2 / ||A v||_2 for each column v of X."""
    AX = A @ X
    return np.linalg.norm(AX - X * lam[None, :], axis=0) / np.linalg.norm(AX, axis=0)
