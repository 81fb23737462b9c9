"""Closed forms and 1-D Sturm bisection (oracle; test-only).

* App. C: the 1-D Dirichlet second difference on N-1 interior nodes,
  (1/dx^2) tridiag(1, -2, 1), whose negation has eigenvalues
  (4/dx^2) sin^2(j pi dx / 2), j = 1..N-1 (dx = 1/N on the unit interval).
* The 2-D Dirichlet 5-point Laplacian on the n x n interior grid (h = 1/(n+1))
  has eigenvalues (4/h^2)(sin^2(i pi h/2) + sin^2(j pi h/2)) with eigenvectors
  sin(i pi x) sin(j pi y).
* Separable coefficients a = a(x): -div(a grad u) block-diagonalises over the
  discrete sine modes in y into n symmetric tridiagonals
  L_x^a + mu_q diag(a(x_i)), mu_q = (4/h^2) sin^2(q pi h / 2); their union is
  the spectrum. Each tridiagonal is solved by bisection on the Sturm count.
* Separable potential V = V1(x) + V2(y): -Lap + V is T1 (x) I + I (x) T2 with the 1-D
  operators T = (1/h^2) tridiag(-1, 2, -1) + diag(V_r), so its eigenvalues are the sums
  mu_i + nu_j of theirs.
"""
from __future__ import annotations

import numpy as np


def laplacian_1d_eigenvalues(n_interior: int) -> np.ndarray:
    """Eigenvalues of -(1/dx^2) tridiag(1,-2,1) on n_interior nodes of [0, 1], ascending."""
    dx = 1.0 / (n_interior + 1)
    j = np.arange(1, n_interior + 1)
    return 4.0 / dx**2 * np.sin(j * np.pi * dx / 2.0) ** 2


def laplacian_2d_eigenvalues(n: int) -> np.ndarray:
    """All n^2 eigenvalues of the 2-D Dirichlet 5-point Laplacian, ascending."""
    mu = laplacian_1d_eigenvalues(n)
    return np.sort((mu[:, None] + mu[None, :]).ravel())


def laplacian_2d_mode(n: int, p: int, q: int) -> np.ndarray:
    """Unit-norm eigenvector sin(p pi x_i) sin(q pi y_j) in row-major node order (p, q >= 1)."""
    h = 1.0 / (n + 1)
    x = (np.arange(n) + 1.0) * h
    v = np.outer(np.sin(p * np.pi * x), np.sin(q * np.pi * x)).ravel()
    return v / np.linalg.norm(v)


def sturm_count(d: np.ndarray, e: np.ndarray, x: float) -> int:
    """Number of eigenvalues < x of the symmetric tridiagonal (diag d, off-diag e).

    Counts negative pivots of the LDL^T factorisation of T - x I (Sylvester's
    law of inertia). A pivot of magnitude <= pivmin is replaced by -pivmin
    before its sign is taken, with pivmin = tiny * max(1, max e_i^2) so that
    e_i^2 / pivot cannot overflow.
    """
    e2 = e * e
    pivmin = np.finfo(float).tiny * max(1.0, float(np.max(e2)) if len(e2) else 1.0)
    count = 0
    q = d[0] - x
    if abs(q) <= pivmin:
        q = -pivmin
    if q < 0:
        count += 1
    for i in range(1, len(d)):
        q = d[i] - x - e2[i - 1] / q
        if abs(q) <= pivmin:
            q = -pivmin
        if q < 0:
            count += 1
    return count


def tridiagonal_eigenvalues_bisection(d: np.ndarray, e: np.ndarray, k: int) -> np.ndarray:
    """The k smallest eigenvalues of a symmetric tridiagonal by bisection."""
    n = len(d)
    r = np.zeros(n)
    r[:-1] += np.abs(e)
    r[1:] += np.abs(e)
    lo, hi = float(np.min(d - r)), float(np.max(d + r))
    out = np.empty(k)
    for idx in range(k):
        a, b = lo, hi
        for _ in range(200):
            mid = 0.5 * (a + b)
            if mid <= a or mid >= b:
                break
            if sturm_count(d, e, mid) > idx:
                b = mid
            else:
                a = mid
        out[idx] = 0.5 * (a + b)
    return out


def separable_tridiagonals(n: int, ax_col: np.ndarray, a_nodes: np.ndarray):
    """The n tridiagonals (d_q, e) of the separable a = a(x) case.

    ax_col[f] = a at x-face f (f = 0..n), a_nodes[i] = a(x_i).
    """
    h = 1.0 / (n + 1)
    inv_h2 = 1.0 / h**2
    d0 = (ax_col[:-1] + ax_col[1:]) * inv_h2
    e = -ax_col[1:-1] * inv_h2
    mu = laplacian_1d_eigenvalues(n)
    return [(d0 + mu[q] * a_nodes, e) for q in range(n)]


def separable_smallest(n: int, ax_col: np.ndarray, a_nodes: np.ndarray, k: int) -> np.ndarray:
    """The k smallest eigenvalues of -div(a(x) grad u) on the n x n grid (ascending)."""
    vals = []
    for d, e in separable_tridiagonals(n, ax_col, a_nodes):
        vals.append(tridiagonal_eigenvalues_bisection(d, e, min(k, n)))
    return np.sort(np.concatenate(vals))[:k]


def sturm_counts(d: np.ndarray, e: np.ndarray, xs: np.ndarray) -> np.ndarray:
    """sturm_count for every shift in xs at once (the same recurrence, vectorised over xs)."""
    e2 = e * e
    pivmin = np.finfo(float).tiny * max(1.0, float(np.max(e2)) if len(e2) else 1.0)
    xs = np.asarray(xs, dtype=float)
    q = d[0] - xs
    q = np.where(np.abs(q) <= pivmin, -pivmin, q)
    count = (q < 0).astype(np.int64)
    for i in range(1, len(d)):
        q = d[i] - xs - e2[i - 1] / q
        q = np.where(np.abs(q) <= pivmin, -pivmin, q)
        count += q < 0
    return count


def tridiagonal_smallest(d: np.ndarray, e: np.ndarray, k: int) -> np.ndarray:
    """The k smallest eigenvalues of a symmetric tridiagonal: bisection on the Sturm count,
    all k brackets advanced together (the same steps as tridiagonal_eigenvalues_bisection)."""
    r = np.zeros(len(d))
    r[:-1] += np.abs(e)
    r[1:] += np.abs(e)
    lo, hi = float(np.min(d - r)), float(np.max(d + r))
    idx = np.arange(k)
    a = np.full(k, lo)
    b = np.full(k, hi)
    for _ in range(200):
        mid = 0.5 * (a + b)
        above = sturm_counts(d, e, mid) > idx
        b = np.where(above, mid, b)
        a = np.where(above, a, mid)
    return 0.5 * (a + b)


def separable_smallest_fast(n: int, ax_col: np.ndarray, a_nodes: np.ndarray, k: int) -> np.ndarray:
    """separable_smallest with the vectorised bisection."""
    vals = [tridiagonal_smallest(d, e, min(k, n)) for d, e in separable_tridiagonals(n, ax_col, a_nodes)]
    return np.sort(np.concatenate(vals))[:k]


def separable_lap_plus_v_smallest(n: int, V: np.ndarray, k: int, m: int) -> np.ndarray:
    """The k smallest eigenvalues of -Lap + V on the n x n grid for separable V[i, j] =
    V1[i] + V2[j], from the m + 1 smallest eigenvalues of each 1-D operator. Raises if the
    k-th sum is not provably below every sum that uses an eigenvalue beyond the m-th."""
    v1 = V[:, 0].copy()
    v2 = V[0, :] - V[0, 0]
    if np.max(np.abs(V - (v1[:, None] + v2[None, :]))) > 1e-9 * max(1.0, np.max(np.abs(V))):
        raise ValueError("V is not separable")
    h = 1.0 / (n + 1)
    e = np.full(n - 1, -1.0 / h**2)
    mu = tridiagonal_smallest(2.0 / h**2 + v1, e, m + 1)
    nu = tridiagonal_smallest(2.0 / h**2 + v2, e, m + 1)
    sums = np.sort((mu[:m, None] + nu[None, :m]).ravel())[:k]
    if not sums[-1] < min(mu[0] + nu[m], mu[m] + nu[0]):
        raise ValueError("m too small for k")
    return sums
