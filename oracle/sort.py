"""Truncated-FFT greedy sort, Alg. 2 (oracle; test-only).

Readings of Alg. 2 taken here:
* Trunc_{p0}(FFT(P)) keeps the unshifted DFT indices [0, p0)^2 and uses the
  unitary 1/p normalisation for a p x p matrix, the one App. F needs for
  Parseval's identity to hold. It is evaluated as a direct (not fast) DFT of
  the kept block, which is the definition written out.
* The distance compared is the squared Frobenius norm of the difference of
  the kept blocks (same argmin as the norm itself, without a square root).
* The running minimum starts at +infinity (Alg. 2 starts it at 1000, which
  fails when every distance exceeds 1000).
* Candidates are visited in ascending original index with a strict '<', so the
  smallest index wins ties. Indices are 0-based: problem 1 of the paper is 0.
"""
from __future__ import annotations

import numpy as np


def truncated_dft(P: np.ndarray, p0: int) -> np.ndarray:
    """Alg. 2, feature step: F[k1, k2] = (1/p) sum_{x,y} P[x,y] exp(-2 pi i (k1 x + k2 y)/p)."""
    p = P.shape[0]
    assert P.shape == (p, p) and 0 < p0 <= p
    k = np.arange(p0)
    x = np.arange(p)
    W = np.exp(-2j * np.pi * np.outer(k, x) / p)  # [p0, p]
    return (W @ P.astype(np.complex128) @ W.T) / p


def features(fields: np.ndarray, p0: int) -> np.ndarray:
    """[n_ops, p, p] real -> [n_ops, p0, p0] complex truncated DFT blocks."""
    return np.stack([truncated_dft(P, p0) for P in fields])


def squared_distance(Fa: np.ndarray, Fb: np.ndarray) -> float:
    """Squared Frobenius norm of Fa - Fb over real and imaginary parts."""
    d = Fa - Fb
    return float(np.sum(d.real * d.real + d.imag * d.imag))


def greedy_chain(F: np.ndarray, start: int = 0):
    """Alg. 2, greedy step: nearest-neighbour chain from ``start``.

    Returns (perm, rel_gaps) where perm is the visiting order (int32) and
    rel_gaps[s] = (second best - best) / scale at step s, with scale the
    largest squared feature norm (used by tests to flag near-ties, where the
    two sides' roundings could legitimately pick different problems).
    """
    n_ops = F.shape[0]
    flat = np.concatenate([F.real.reshape(n_ops, -1), F.imag.reshape(n_ops, -1)], axis=1)
    scale = float(np.max(np.sum(flat * flat, axis=1))) if n_ops else 1.0
    remaining = [j for j in range(n_ops) if j != start]
    perm = [start]
    gaps = []
    i0 = start
    while remaining:
        best, second, j_min = np.inf, np.inf, -1
        for j in remaining:                      # ascending original index
            d = squared_distance(F[i0], F[j])
            if d < best:
                second, best, j_min = best, d, j
            elif d < second:
                second = d
        gaps.append((second - best) / max(scale, np.finfo(float).tiny) if np.isfinite(second) else np.inf)
        remaining.remove(j_min)
        perm.append(j_min)
        i0 = j_min
    return np.array(perm, dtype=np.int32), np.array(gaps)


def scsf_sort(fields: np.ndarray, p0: int, start: int = 0):
    """Alg. 2 end to end: features then greedy chain. Returns (perm, rel_gaps)."""
    return greedy_chain(features(fields, p0), start)
