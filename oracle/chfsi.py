"""Chebyshev filtered subspace iteration and the warm-started chain (oracle; test-only).

Follows Alg. 3 (Sec. 3.2) step by step, with Householder QR for the
orthonormalisation as the paper states (numpy.linalg.qr is LAPACK's
Householder QR) and a dense symmetric eigensolve for the reduced problem.

Readings taken where the paper is silent or garbled:
* Block width k_b = k + nex with nex = ceil(0.2 k) (App. D.4's inherited
  subspace of 20% of L); the warm start is the whole final k_b block of the
  previous problem with its Ritz values (Alg. 3 input, Sec. 3.2).
* Filter parameters (Sec. 2.2): [alpha, beta] is the unwanted interval with
  alpha = the largest Ritz value of the current block and beta = the
  Gershgorin upper bound of A; lambda = the smallest active Ritz value;
  c = (alpha+beta)/2, e = (beta-alpha)/2; updated after every Rayleigh-Ritz.
* Head of a chain (random start, Sec. 3.2): lambda = Gershgorin lower bound,
  alpha = lo + 2 (k_b/N)(hi - lo).
* Alg. 3's Rayleigh-quotient step with its garbled G = Q_0^T A Q is read as G = Q_a^T A Q_a over the
  active (unlocked) columns of Q = qr([locked | filtered active]).
* Locking (Alg. 3, lock step): the leading contiguous run of active Ritz pairs (ascending
  Ritz value) whose relative residual (App. D.5) is <= tol is locked; the loop
  ends once at least k pairs are locked; the k smallest locked pairs are
  returned.
* At most ``max_iter`` (default 100) outer iterations; otherwise the result is
  flagged not converged.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import numpy as np

from .chebyshev import chebyshev_filter
from .operators import assemble, gershgorin_bounds, relative_residuals


def block_width(k: int) -> int:
    """k_b = k + ceil(0.2 k) (App. D.4)."""
    return k + int(math.ceil(0.2 * k))


@dataclass
class SolveResult:
    evals: np.ndarray        # [k] ascending
    evecs: np.ndarray        # [N, k]
    resid: np.ndarray        # [k] relative residuals (App. D.5)
    block: np.ndarray        # [N, k_b] final block (warm start for the next problem)
    block_ritz: np.ndarray   # [k_b] its Ritz values
    iters: int
    converged: bool


def head_bounds(lo: float, hi: float, kb: int, N: int):
    """Filter bounds for a random start: lambda = lo, alpha = lo + 2 (k_b/N)(hi - lo)."""
    return lo, lo + 2.0 * (kb / N) * (hi - lo)


def chfsi_solve(A, k: int, degree: int, tol: float, V0: np.ndarray, lam: float, alpha: float,
                max_iter: int = 100) -> SolveResult:
    """Alg. 3 for one problem A, from block V0 [N, k_b] and filter bounds (lam, alpha)."""
    N, kb = V0.shape
    _, beta = gershgorin_bounds(A)
    X = np.array(V0, dtype=np.float64, copy=True)  # active block
    locked_V = np.zeros((N, 0))
    locked_w = np.zeros(0)
    w_act = np.zeros(0)
    it = 0
    while True:
        it += 1
        c = 0.5 * (alpha + beta)
        e = 0.5 * (beta - alpha)
        Y = chebyshev_filter(A, X, degree, lam, c, e)
        nl = locked_V.shape[1]
        Q, _ = np.linalg.qr(np.hstack([locked_V, Y]))
        Qa = Q[:, nl:]
        G = Qa.T @ (A @ Qa)
        G = 0.5 * (G + G.T)
        w, Z = np.linalg.eigh(G)
        X = Qa @ Z
        r = relative_residuals(A, X, w)
        nconv = 0
        while nconv < X.shape[1] and r[nconv] <= tol:
            nconv += 1
        locked_V = np.hstack([locked_V, X[:, :nconv]])
        locked_w = np.concatenate([locked_w, w[:nconv]])
        X = X[:, nconv:]
        w_act = w[nconv:]
        r_act = r[nconv:]
        if locked_V.shape[1] >= k or it >= max_iter or X.shape[1] == 0:
            break
        lam = float(w_act[0])
        alpha = float(w_act[-1])
    converged = locked_V.shape[1] >= k
    block = np.hstack([locked_V, X])
    block_ritz = np.concatenate([locked_w, w_act])
    order = np.argsort(block_ritz[: locked_V.shape[1]], kind="stable")
    if converged:
        sel = order[:k]
        evals = locked_w[sel]
        evecs = locked_V[:, sel]
    else:
        evals = np.full(k, np.nan)
        evecs = np.full((N, k), np.nan)
        nl = locked_V.shape[1]
        evals[:nl] = locked_w[order]
        evecs[:, :nl] = locked_V[:, order]
    resid = relative_residuals(A, evecs, evals) if converged else np.full(k, np.nan)
    return SolveResult(evals, evecs, resid, block, block_ritz, it, converged)


def solve_chain(ops, k: int, degree: int, tol: float, head_seed: int = 0,
                max_iter: int = 100, V0: Optional[np.ndarray] = None, keep_vectors: bool = True):
    """Sequential SCSF solve over an already sorted list of operators (Sec. 3.2).

    The first problem starts from a seeded Gaussian block; every later one is
    warm-started from the previous final block and Ritz values.
    """
    results = []
    prev = None
    for i, op in enumerate(ops):
        A = assemble(op)
        N = A.shape[0]
        kb = block_width(k)
        if prev is None:
            lo, hi = gershgorin_bounds(A)
            block = V0 if V0 is not None else np.random.default_rng(head_seed).standard_normal((N, kb))
            lam, alpha = head_bounds(lo, hi, kb, N)
        else:
            block = prev.block
            lam, alpha = float(np.min(prev.block_ritz)), float(np.max(prev.block_ritz))
        res = chfsi_solve(A, k, degree, tol, block, lam, alpha, max_iter=max_iter)
        prev = res
        if not keep_vectors:
            res = SolveResult(res.evals, None, res.resid, None, None, res.iters, res.converged)
        results.append(res)
    return results
