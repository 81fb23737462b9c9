"""Pins for the comparison helpers every parity test relies on (oracle.compare): a helper
that returned 0, ignored order or swallowed a NaN would make those tests vacuous."""
import numpy as np
import pytest

from oracle import compare


def test_max_rel_eig_error_values_order_and_nan():
    assert compare.max_rel_eig_error([1.0, 2.0, 4.0], [1.0, 2.002, 4.0]) == pytest.approx(1e-3)
    # compared as sorted lists
    assert compare.max_rel_eig_error([4.0, 1.0, 2.0], [2.0, 4.0, 1.0]) == 0.0
    # relative to |ref|, also for negative eigenvalues
    assert compare.max_rel_eig_error([-10.0, 5.0], [-10.5, 5.0]) == pytest.approx(0.05)
    # a NaN never passes a "<= tol" check
    assert not compare.max_rel_eig_error([1.0, 2.0], [1.0, np.nan]) <= 1.0


def test_clusters_split_on_relative_gap():
    ev = np.array([1.0, 1.0 + 1e-9, 2.0, 3.0, 3.0 * (1 + 1e-8), 3.5])
    assert compare.clusters(ev, rel_gap=1e-6) == [[0, 1], [2], [3, 4], [5]]
    assert compare.clusters(ev, rel_gap=1e-12) == [[0], [1], [2], [3], [4], [5]]


def test_subspace_angle_closed_form():
    t = 0.3
    U = np.array([[1.0], [0.0], [0.0]])
    V = np.array([[np.cos(t)], [np.sin(t)], [0.0]])
    assert compare.max_subspace_angle(U, V) == pytest.approx(t, abs=1e-12)
    # scaling and sign of a basis do not matter; a rotated basis of the same plane gives 0
    P = np.eye(4)[:, :2]
    R = np.array([[np.cos(1.1), -np.sin(1.1)], [np.sin(1.1), np.cos(1.1)]])
    assert compare.max_subspace_angle(P, -3.0 * P @ R) == pytest.approx(0.0, abs=1e-7)


def test_cluster_angle_accepts_any_basis_of_a_degenerate_pair_and_flags_a_wrong_vector():
    vals = np.array([1.0, 2.0, 2.0, 3.0, 4.0])
    Q, _ = np.linalg.qr(np.random.default_rng(0).standard_normal((8, 5)))
    got = Q.copy()
    c, s = np.cos(0.7), np.sin(0.7)
    got[:, 1], got[:, 2] = c * Q[:, 1] + s * Q[:, 2], -s * Q[:, 1] + c * Q[:, 2]
    assert compare.max_cluster_angle(vals, Q, got) == pytest.approx(0.0, abs=1e-7)
    bad = got.copy()
    bad[:, 0] = np.cos(0.2) * Q[:, 0] + np.sin(0.2) * Q[:, 3]
    assert compare.max_cluster_angle(vals, Q, bad) == pytest.approx(0.2, abs=1e-9)


def test_orthonormality_error_values():
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((10, 4)))
    assert compare.orthonormality_error(Q) <= 1e-15
    Q[:, 2] *= 1.01
    assert compare.orthonormality_error(Q) == pytest.approx(1.01**2 - 1.0, rel=1e-9)
