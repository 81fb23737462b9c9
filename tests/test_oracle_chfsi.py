"""Pins for oracle.chfsi (Alg. 3 + warm-started chain, Sec. 3.2)."""
import numpy as np
import pytest

import scsf_inputs as si
from oracle import chfsi, compare, dense, inertia, operators, sturm


def test_block_width_rule():
    """App. D.4: 20 -> 4 extra, 100 -> 20, 400 -> 80."""
    assert [chfsi.block_width(k) for k in (20, 100, 200, 300, 400)] == [24, 120, 240, 360, 480]


def test_chain_matches_dense_definition():
    ops = si.div_a_grad_chain(16, 4, seed=0)
    res = chfsi.solve_chain(ops, k=12, degree=16, tol=1e-8, head_seed=3)
    for op, r in zip(ops, res):
        A = operators.assemble(op)
        w, V = dense.smallest_eigenpairs(A, 12)
        assert r.converged
        assert compare.max_rel_eig_error(w, r.evals) < 1e-10
        assert np.max(r.resid) <= 1e-8
        assert compare.orthonormality_error(r.evecs) < 1e-12
        assert compare.max_cluster_angle(w, V, r.evecs) < 1e-6
        assert r.block.shape == (256, chfsi.block_width(12))


def test_laplacian_closed_form():
    n = 20
    res = chfsi.solve_chain([si.constant_div_a_grad(n)], k=10, degree=16, tol=1e-10, head_seed=1)[0]
    assert res.converged
    ref = sturm.laplacian_2d_eigenvalues(n)[:10]
    assert compare.max_rel_eig_error(ref, res.evals) < 1e-12


def test_separable_large_grid_and_inertia():
    """a = a(x): compare to 1-D Sturm bisection; certify no missed eigenvalue by inertia."""
    n, k = 40, 16
    op = si.separable_div_a_grad(n, seed=2)
    r = chfsi.solve_chain([op], k=k, degree=20, tol=1e-9, head_seed=5)[0]
    assert r.converged
    ref = sturm.separable_smallest(n, op.ax[:, 0], op.P[:, 0], k + 1)
    assert compare.max_rel_eig_error(ref[:k], r.evals) < 1e-10
    A = operators.assemble(op)
    nxt = np.sort(r.block_ritz)[k]
    sigma = 0.5 * (r.evals[-1] + min(nxt, ref[k]))
    assert inertia.count_below(A, sigma, n) == k


def test_warm_start_from_identical_problem_converges_fast():
    """Sec. 3.2 / App. E similarity study: the same problem again converges in 1-2 iterations."""
    op = si.div_a_grad_chain(16, 1, seed=6)[0]
    res = chfsi.solve_chain([op, op], k=10, degree=16, tol=1e-8, head_seed=0)
    assert res[0].iters > 3
    assert res[1].iters <= 2
    np.testing.assert_allclose(res[1].evals, res[0].evals, rtol=1e-10)


def test_not_converged_flag():
    op = si.div_a_grad_chain(16, 1, seed=6)[0]
    r = chfsi.solve_chain([op], k=10, degree=2, tol=1e-14, head_seed=0, max_iter=2)[0]
    assert not r.converged and r.iters == 2


def test_chain_on_general_csr_matches_dense_definition():
    """Alg. 3 takes any symmetric matrix: on an irregular graph Laplacian plus potential
    (no grid) the oracle chain reaches the dense eigenpairs."""
    ops = si.knn_graph_chain(403, 3, seed=3)
    res = chfsi.solve_chain(ops, k=10, degree=12, tol=1e-9, head_seed=2)
    for op, r in zip(ops, res):
        A = operators.assemble(op)
        w, V = dense.smallest_eigenpairs(A, 10)
        assert r.converged
        assert compare.max_rel_eig_error(w, r.evals) < 1e-10
        assert np.max(r.resid) <= 1e-9
        assert compare.orthonormality_error(r.evecs) < 1e-12
