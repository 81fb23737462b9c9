"""Pins for oracle.operators / oracle.sturm / oracle.inertia / oracle.dense (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp

import scsf_inputs as si
from oracle import dense, inertia, operators, sturm


def test_assembly_matches_worked_example_eq_p(golden):
    """Sec. 2.1 Eq. (eq_p): a == 1 on a 2x2 grid gives -(1/h^2) x the printed stencil matrix."""
    M = golden("eq_p_2x2.txt")
    A = operators.assemble(si.constant_div_a_grad(2)).toarray()
    h = 1.0 / 3.0
    np.testing.assert_allclose(A * h * h, -M, rtol=0, atol=1e-14)


def test_1d_closed_form_matches_app_c_matrix(golden):
    """App. C: eigenvalues of -(1/dx^2) tridiag(1,-2,1) are (4/dx^2) sin^2(j pi dx/2)."""
    T = golden("app_c_tridiag5.txt")
    dx = 1.0 / 6.0
    w = np.linalg.eigvalsh(-T / dx**2)
    np.testing.assert_allclose(sturm.laplacian_1d_eigenvalues(5), w, rtol=1e-13)


@pytest.mark.parametrize("n", [3, 6, 7])
def test_2d_laplacian_spectrum_closed_form(n):
    """a == 1: lambda_ij = 4/h^2 (sin^2(i pi h/2) + sin^2(j pi h/2)) (independent closed form)."""
    h = 1.0 / (n + 1)
    i = np.arange(1, n + 1)
    mu = 4.0 / h**2 * np.sin(i * np.pi * h / 2) ** 2
    ref = np.sort((mu[:, None] + mu[None, :]).ravel())
    A = operators.assemble(si.constant_div_a_grad(n))
    w = np.linalg.eigvalsh(A.toarray())
    np.testing.assert_allclose(w, ref, rtol=1e-12)
    np.testing.assert_allclose(sturm.laplacian_2d_eigenvalues(n), ref, rtol=1e-13)


def test_laplacian_sine_modes_are_eigenvectors():
    n = 9
    A = operators.assemble(si.constant_div_a_grad(n))
    h = 1.0 / (n + 1)
    for p, q in [(1, 1), (2, 5), (9, 3)]:
        v = sturm.laplacian_2d_mode(n, p, q)
        lam = 4.0 / h**2 * (np.sin(p * np.pi * h / 2) ** 2 + np.sin(q * np.pi * h / 2) ** 2)
        assert np.linalg.norm(A @ v - lam * v) <= 1e-12 * lam


def test_constant_coefficient_scales_spectrum():
    n = 5
    A1 = operators.assemble(si.constant_div_a_grad(n, 1.0)).toarray()
    A3 = operators.assemble(si.constant_div_a_grad(n, 3.0)).toarray()
    np.testing.assert_allclose(np.linalg.eigvalsh(A3), 3 * np.linalg.eigvalsh(A1), rtol=1e-13)


def test_variable_coefficient_structure():
    """Symmetric, 5-point pattern, and u = const gives only boundary flux terms."""
    n = 6
    op = si.div_a_grad_chain(n, 1, seed=11)[0]
    A = operators.assemble(op).toarray()
    np.testing.assert_array_equal(A, A.T)
    h = 1.0 / (n + 1)
    rowsum = (A @ np.ones(n * n)).reshape(n, n) * h * h
    # interior rows sum to zero; boundary rows keep the boundary face coefficients
    expect = np.zeros((n, n))
    expect[0, :] += op.ax[0, :]
    expect[-1, :] += op.ax[n, :]
    expect[:, 0] += op.ay[:, 0]
    expect[:, -1] += op.ay[:, n]
    np.testing.assert_allclose(rowsum, expect, rtol=1e-12, atol=1e-12)
    # coupling between (i, j) and (i+1, j) is -a at the face between them
    i, j = 2, 3
    assert A[i * n + j, (i + 1) * n + j] == pytest.approx(-op.ax[i + 1, j] / h**2, rel=1e-14)
    assert A[i * n + j, i * n + j + 1] == pytest.approx(-op.ay[i, j + 1] / h**2, rel=1e-14)


def test_lap_plus_v_constant_shift():
    n = 5
    V = np.full((n, n), 7.5)
    A = operators.assemble(si.LapPlusVOp(n, V)).toarray()
    np.testing.assert_allclose(np.linalg.eigvalsh(A), sturm.laplacian_2d_eigenvalues(n) + 7.5, rtol=1e-12)


def test_gershgorin_contains_spectrum_and_is_tight_for_laplacian():
    n = 8
    op = si.div_a_grad_chain(n, 1, seed=3)[0]
    A = operators.assemble(op)
    lo, hi = operators.gershgorin_bounds(A)
    w = np.linalg.eigvalsh(A.toarray())
    assert lo <= w[0] and w[-1] <= hi
    lo1, hi1 = operators.gershgorin_bounds(operators.assemble(si.constant_div_a_grad(n)))
    h = 1.0 / (n + 1)
    assert hi1 == pytest.approx(8.0 / h**2, rel=1e-14)
    assert lo1 == pytest.approx(0.0, abs=1e-9)


def test_relative_residual_definition():
    """App. D.5: exact pair -> 0; eigenvalue off by a factor (1+eps) -> eps."""
    n = 7
    A = operators.assemble(si.constant_div_a_grad(n))
    h = 1.0 / (n + 1)
    v = sturm.laplacian_2d_mode(n, 2, 3)
    lam = 4.0 / h**2 * (np.sin(2 * np.pi * h / 2) ** 2 + np.sin(3 * np.pi * h / 2) ** 2)
    X = np.stack([v, v], axis=1)
    r = operators.relative_residuals(A, X, np.array([lam, lam * (1 + 1e-6)]))
    assert r[0] < 1e-14
    assert r[1] == pytest.approx(1e-6, rel=1e-6)


def test_separable_case_matches_dense():
    n = 12
    op = si.separable_div_a_grad(n, seed=5)
    A = operators.assemble(op)
    w = np.linalg.eigvalsh(A.toarray())[:25]
    ws = sturm.separable_smallest(n, op.ax[:, 0], op.P[:, 0], 25)
    np.testing.assert_allclose(ws, w, rtol=1e-12)


def test_sturm_bisection_closed_form():
    n = 40
    dx = 1.0 / (n + 1)
    d = np.full(n, 2.0 / dx**2)
    e = np.full(n - 1, -1.0 / dx**2)
    w = sturm.tridiagonal_eigenvalues_bisection(d, e, 10)
    np.testing.assert_allclose(w, sturm.laplacian_1d_eigenvalues(n)[:10], rtol=1e-13)


def test_vectorised_bisection_matches_scalar_and_library():
    rng = np.random.default_rng(3)
    d = rng.standard_normal(30) * 5
    e = rng.standard_normal(29)
    w = np.linalg.eigvalsh(np.diag(d) + np.diag(e, 1) + np.diag(e, -1))[:12]
    v = sturm.tridiagonal_smallest(d, e, 12)
    np.testing.assert_allclose(v, w, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(v, sturm.tridiagonal_eigenvalues_bisection(d, e, 12), rtol=1e-14,
                               atol=1e-14)
    xs = np.array([-3.0, 0.0, 2.5])
    assert list(sturm.sturm_counts(d, e, xs)) == [sturm.sturm_count(d, e, x) for x in xs]


def test_separable_fast_matches_dense():
    n = 12
    op = si.separable_div_a_grad(n, seed=6)
    w = np.linalg.eigvalsh(operators.assemble(op).toarray())[:30]
    np.testing.assert_allclose(sturm.separable_smallest_fast(n, op.ax[:, 0], op.P[:, 0], 30), w,
                               rtol=1e-12)


def test_separable_potential_matches_dense_and_rejects_short_lists():
    n = 12
    op = si.separable_lap_plus_v(n, seed=4)
    w = np.linalg.eigvalsh(operators.assemble(op).toarray())[:40]
    np.testing.assert_allclose(sturm.separable_lap_plus_v_smallest(n, op.V, 40, m=11), w,
                               rtol=1e-11, atol=1e-9)
    with pytest.raises(ValueError):
        sturm.separable_lap_plus_v_smallest(n, op.V, 40, m=3)
    with pytest.raises(ValueError):
        sturm.separable_lap_plus_v_smallest(n, op.V + np.eye(n), 10, m=11)


@pytest.mark.parametrize("seed", [0, 1])
def test_inertia_count_matches_dense(seed):
    n = 9
    op = si.div_a_grad_chain(n, 1, seed=seed)[0]
    A = operators.assemble(op)
    w = np.linalg.eigvalsh(A.toarray())
    for k in [1, 5, 17, 40]:
        sigma = 0.5 * (w[k - 1] + w[k])
        assert inertia.count_below(A, sigma, n) == k


def test_cyclic_jacobi_matches_closed_form_and_library():
    n = 4
    A = operators.assemble(si.constant_div_a_grad(n)).toarray()
    w, V = dense.cyclic_jacobi(A)
    np.testing.assert_allclose(w, sturm.laplacian_2d_eigenvalues(n), rtol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(n * n), atol=1e-13)
    np.testing.assert_allclose(A @ V, V * w[None, :], atol=1e-11 * np.max(np.abs(w)))
    S = np.random.default_rng(2).standard_normal((9, 9))
    S = S + S.T
    wj, _ = dense.cyclic_jacobi(S)
    np.testing.assert_allclose(wj, np.linalg.eigvalsh(S), rtol=1e-12, atol=1e-13)


def test_knn_graph_csr_is_laplacian_plus_potential():
    """The CSR input family: symmetric, sorted CSR; the Laplacian part annihilates constants
    (A 1 = V exactly, up to rounding), so the smallest eigenvalue lies in [min V, max V]
    (Rayleigh quotient of the constant vector and L >= 0); Gershgorin encloses the spectrum."""
    ops = si.knn_graph_chain(301, 2, seed=7)
    for op in ops:
        A = operators.assemble(op)
        assert A.shape == (301, 301) and op.row_ptr[0] == 0 and op.row_ptr[-1] == len(op.val)
        assert abs(A - A.T).max() == 0.0
        for r in range(op.rows):  # columns ascending within each row
            seg = op.col[op.row_ptr[r]:op.row_ptr[r + 1]]
            assert np.all(np.diff(seg) > 0)
        lens = np.diff(op.row_ptr)
        assert lens.min() >= 7 and lens.max() > lens.min()  # irregular rows
        off = A - sp.diags(A.diagonal())
        assert np.all(off.data <= 0)  # nonpositive off-diagonal weights
        V = A @ np.ones(op.rows)
        assert np.all(V >= 0)
        w = np.linalg.eigvalsh(A.toarray())
        assert V.min() - 1e-12 <= w[0] <= V.max() + 1e-12
        assert w[0] <= V.mean() + 1e-12  # Rayleigh quotient of the constant vector
        lo, hi = operators.gershgorin_bounds(A)
        assert lo <= w[0] + 1e-12 and w[-1] <= hi + 1e-12
    # the potential's centre moves along the chain: the two problems differ only on the diagonal
    A0, A1 = (operators.assemble(o) for o in ops)
    D = (A0 - A1).tocoo()
    assert np.all(D.row[D.data != 0] == D.col[D.data != 0])


def test_plate_stencil_is_the_textbook_biharmonic_stencil():
    """D == 1: an interior row of K is the 13-point biharmonic stencil (20, -8, 2, 1) / h^4;
    next to a simply supported edge the centre is 19 (ghost value -u_1), at a corner 18.
    Variable D: K_II = (16 D_I + sum of D over the interior neighbours) / h^4."""
    n = 9
    h = 1.0 / (n + 1)
    K = operators.assemble_plate_stiffness(n, np.ones((n, n))).toarray() * h**4
    I = lambda i, j: i * n + j
    c = I(4, 4)
    assert K[c, c] == pytest.approx(20.0)
    for di, dj, v in [(1, 0, -8), (0, 1, -8), (-1, 0, -8), (0, -1, -8), (1, 1, 2), (1, -1, 2),
                      (-1, 1, 2), (-1, -1, 2), (2, 0, 1), (0, 2, 1), (-2, 0, 1), (0, -2, 1)]:
        assert K[c, I(4 + di, 4 + dj)] == pytest.approx(v)
    assert np.count_nonzero(np.abs(K[c]) > 1e-12) == 13
    assert K[I(0, 4), I(0, 4)] == pytest.approx(19.0) and K[I(0, 0), I(0, 0)] == pytest.approx(18.0)
    assert np.max(np.count_nonzero(np.abs(K) > 1e-12, axis=1)) == 13
    D = np.random.default_rng(3).uniform(0.5, 2.0, (n, n))
    Kd = operators.assemble_plate_stiffness(n, D).toarray() * h**4
    for (i, j) in [(4, 4), (0, 3), (0, 0), (8, 8)]:
        nb = sum(D[i + di, j + dj] for di, dj in [(1, 0), (-1, 0), (0, 1), (0, -1)]
                 if 0 <= i + di < n and 0 <= j + dj < n)
        assert Kd[I(i, j), I(i, j)] == pytest.approx(16 * D[i, j] + nb)


def test_uniform_plate_spectrum_closed_form():
    """D, rho constant: the modes are the Laplacian's sine modes and
    lambda_ij = (D / rho) (4/h^2 (sin^2(i pi h/2) + sin^2(j pi h/2)))^2."""
    n, d0, r0 = 14, 2.5, 0.8
    h = 1.0 / (n + 1)
    op = si.constant_plate(n, d0, r0)
    C = operators.assemble(op)
    i = np.arange(1, n + 1)
    lam1 = 4.0 / h**2 * np.sin(i * np.pi * h / 2) ** 2
    ref = np.sort((d0 / r0 * (lam1[:, None] + lam1[None, :]) ** 2).ravel())
    w = np.linalg.eigvalsh(C.toarray())
    assert np.max(np.abs(w - ref)) <= 1e-11 * ref[-1]
    phi = sturm.laplacian_2d_mode(n, 2, 3)
    lam = d0 / r0 * (lam1[1] + lam1[2]) ** 2
    assert np.linalg.norm(C @ phi - lam * phi) <= 1e-12 * lam * np.linalg.norm(phi)


def test_plate_standard_form_matches_generalized_problem():
    """The symmetric standard form C = M^{-1/2} K M^{-1/2} has the generalized eigenvalues
    of (K, M = diag(rho)) (LAPACK's generalized symmetric-definite solver), and
    u = M^{-1/2} v solves K u = lambda M u with u^T M u = 1."""
    import scipy.linalg as sla
    op = si.plate_chain(11, 1, seed=5)[0]
    K = operators.assemble_plate_stiffness(op.n, op.D).toarray()
    M = np.diag(op.rho.reshape(-1))
    wg = sla.eigh(K, M, eigvals_only=True)
    C = operators.assemble(op).toarray()
    assert np.max(np.abs(C - C.T)) <= 1e-15 * np.max(np.abs(C))  # symmetric up to rounding
    w, V = np.linalg.eigh(C)
    assert np.max(np.abs(w - wg)) <= 1e-12 * wg[-1]
    assert w[0] > 0  # symmetric positive definite
    U = V / np.sqrt(op.rho.reshape(-1))[:, None]
    assert np.max(np.abs(K @ U - (M @ U) * w)) <= 1e-11 * wg[-1]
    assert np.max(np.abs(U.T @ M @ U - np.eye(len(w)))) <= 1e-12
