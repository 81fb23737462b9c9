"""Pins for oracle.sort (Alg. 2, App. F) against the library FFT, Parseval and brute force."""
import itertools

import numpy as np
import pytest

import scsf_inputs as si
from oracle import sort


@pytest.mark.parametrize("p,p0", [(8, 3), (16, 8), (7, 7)])
def test_truncated_dft_matches_library_fft(p, p0):
    """Alg. 2, truncation reading: unshifted [0, p0)^2 block of the DFT, unitary 1/p scaling."""
    P = np.random.default_rng(p).standard_normal((p, p))
    ref = np.fft.fft2(P)[:p0, :p0] / p
    np.testing.assert_allclose(sort.truncated_dft(P, p0), ref, rtol=1e-12, atol=1e-12)


def test_parseval_full_block_equals_spatial_distance():
    """App. F: with p0 = p the frequency distance equals the spatial Frobenius distance."""
    rng = np.random.default_rng(1)
    A, B = rng.standard_normal((2, 12, 12))
    d_freq = sort.squared_distance(sort.truncated_dft(A, 12), sort.truncated_dft(B, 12))
    assert d_freq == pytest.approx(np.sum((A - B) ** 2), rel=1e-12)


def _brute_force_chain(fields, p0, start):
    """Independent greedy chain: library FFT features, full distance matrix, np.argmin."""
    p = fields.shape[1]
    F = np.stack([np.fft.fft2(P)[:p0, :p0] / p for P in fields]).reshape(len(fields), -1)
    D = np.abs(F[:, None, :] - F[None, :, :]) ** 2
    D = D.sum(axis=2)
    order = [start]
    left = set(range(len(fields))) - {start}
    while left:
        cand = sorted(left)
        j = cand[int(np.argmin(D[order[-1], cand]))]
        order.append(j)
        left.remove(j)
    return order


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_greedy_chain_brute_force(seed):
    rng = np.random.default_rng(seed)
    n_ops = int(rng.integers(3, 9))
    fields = np.stack([op.P for op in si.div_a_grad_chain(16, n_ops, seed=seed)])
    start = int(rng.integers(0, n_ops))
    perm, gaps = sort.scsf_sort(fields, 8, start)
    assert perm.tolist() == _brute_force_chain(fields, 8, start)
    assert sorted(perm.tolist()) == list(range(n_ops))
    assert perm[0] == start and len(gaps) == n_ops - 1


def test_one_parameter_family_sorts_ascending():
    """P_t = t B visited from the smallest t must come out in ascending t (distance |t - s| |B|)."""
    B = np.random.default_rng(7).standard_normal((10, 10))
    t = np.array([0.7, 0.1, 2.5, 1.3, 0.4, 1.9])
    fields = np.stack([ti * B for ti in t])
    perm, _ = sort.scsf_sort(fields, 4, start=int(np.argmin(t)))
    assert t[perm].tolist() == sorted(t.tolist())


def test_ties_go_to_smallest_index():
    B = np.random.default_rng(8).standard_normal((6, 6))
    fields = np.stack([B, 2 * B, 2 * B, 2 * B])
    perm, gaps = sort.scsf_sort(fields, 3, start=0)
    assert perm.tolist() == [0, 1, 2, 3]
    assert gaps[0] == 0.0


def test_exhaustive_small_permutation_property():
    """Every greedy step picks a global minimiser among the remaining (checked exhaustively)."""
    fields = np.stack([op.P for op in si.div_a_grad_chain(8, 5, seed=9)])
    F = sort.features(fields, 4)
    perm, _ = sort.greedy_chain(F, 2)
    for s in range(1, len(perm)):
        prev, chosen = perm[s - 1], perm[s]
        rest = [j for j in range(len(perm)) if j not in perm[:s]]
        dists = {j: sort.squared_distance(F[prev], F[j]) for j in rest}
        assert all(dists[chosen] <= dists[j] for j in rest)
    assert len(set(itertools.chain(perm.tolist()))) == 5
