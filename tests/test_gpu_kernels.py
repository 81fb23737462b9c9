"""Kernel-level parity: assembly bounds, Chebyshev filter, reduced eigensolve (GPU vs oracle)."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

import scsf_inputs as si
from oracle import chebyshev, operators, sturm
from tests.gpu_util import host, need_gpu, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["div", "lapv"])
def test_gershgorin_bounds(kind):
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op = si.div_a_grad_chain(33, 1, seed=2)[0] if kind == "div" else si.lap_plus_v_chain(33, 1, seed=2)[0]
    lo, hi = scsf.assemble_bounds(to_dev([op], dev)[0])
    rlo, rhi = operators.gershgorin_bounds(operators.assemble(op))
    assert lo == pytest.approx(rlo, rel=1e-13, abs=1e-9 * abs(rhi))
    assert hi == pytest.approx(rhi, rel=1e-13)


@pytest.mark.parametrize("n,ncols,degree", [(20, 37, 1), (20, 37, 2), (33, 24, 7), (17, 120, 16),
                                            (40, 5, 20)])
def test_filter_matches_oracle(n, ncols, degree):
    """Alg. 1 on a random block: GPU recurrence vs oracle recurrence (FP64)."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op = si.div_a_grad_chain(n, 1, seed=n)[0]
    A = operators.assemble(op)
    lo, hi = operators.gershgorin_bounds(A)
    lam, alpha = lo + 0.001 * (hi - lo), lo + 0.05 * (hi - lo)
    c, e = 0.5 * (alpha + hi), 0.5 * (hi - alpha)
    X = si.gaussian_block(n * n, ncols, seed=3)
    ref = chebyshev.chebyshev_filter(A, X, degree, lam, c, e)
    Y = scsf.cheb_filter(to_dev([op], dev)[0], torch.as_tensor(X, device=dev), degree, lam, c, e)
    got = host(Y)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(got - ref)) <= 1e-12 * scale


def test_filter_exact_eigenvector_closed_form():
    """Laplacian sine mode v: filter(v) = C_m(t_v)/C_m(t_lambda) v (library Chebyshev values)."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    n, m = 24, 16
    op = si.constant_div_a_grad(n)
    h = 1.0 / (n + 1)
    lam_min = 8.0 / h**2 * np.sin(np.pi * h / 2) ** 2
    alpha, beta = 400.0, 8.0 / h**2
    c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
    modes = [(1, 1), (2, 3), (7, 7)]
    X = np.stack([sturm.laplacian_2d_mode(n, p, q) for p, q in modes], axis=1)
    Y = host(scsf.cheb_filter(to_dev([op], dev)[0], torch.as_tensor(X.copy(), device=dev), m,
                              lam_min, c, e))
    coef = np.zeros(m + 1)
    coef[m] = 1.0
    for col, (p, q) in enumerate(modes):
        lv = 4.0 / h**2 * (np.sin(p * np.pi * h / 2) ** 2 + np.sin(q * np.pi * h / 2) ** 2)
        expect = npcheb.chebval((lv - c) / e, coef) / npcheb.chebval((lam_min - c) / e, coef)
        np.testing.assert_allclose(Y[:, col], expect * X[:, col], rtol=1e-11, atol=1e-13)


def _random_sym(k, seed, spread=1.0):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    w = np.sort(rng.uniform(-spread, spread, k)) * 100.0
    return (Q * w) @ Q.T


@pytest.mark.parametrize("k", [1, 2, 3, 24, 37, 120, 160])
def test_small_eigh_random(k):
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    S = _random_sym(k, seed=k)
    S = 0.5 * (S + S.T)
    w, Z = scsf.small_eigh(torch.as_tensor(S, device=dev))
    w, Z = host(w), host(Z)
    ref = np.linalg.eigvalsh(S)
    nrm = np.max(np.abs(ref))
    assert np.max(np.abs(w - ref)) <= 1e-13 * nrm * max(1, k) ** 0.5
    assert np.max(np.abs(Z.T @ Z - np.eye(k))) <= 1e-13
    assert np.max(np.abs(S @ Z - Z * w[None, :])) <= 1e-12 * nrm
    assert np.all(np.diff(w) >= 0)


def test_small_eigh_degenerate_and_near_diagonal():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    rng = np.random.default_rng(0)
    k = 48
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    w0 = np.repeat(np.arange(1.0, 13.0), 4)  # exact 4-fold clusters
    S = (Q * w0) @ Q.T
    S = 0.5 * (S + S.T)
    w, Z = scsf.small_eigh(torch.as_tensor(S, device=dev))
    w, Z = host(w), host(Z)
    np.testing.assert_allclose(w, w0, rtol=0, atol=1e-12 * 12)
    assert np.max(np.abs(Z.T @ Z - np.eye(k))) <= 1e-13
    assert np.max(np.abs(S @ Z - Z * w[None, :])) <= 1e-12 * 12
    D = np.diag(np.linspace(1.0, 50.0, 120)) + 1e-7 * _random_sym(120, 5)
    D = 0.5 * (D + D.T)
    w, Z = scsf.small_eigh(torch.as_tensor(D, device=dev))
    np.testing.assert_allclose(host(w), np.linalg.eigvalsh(D), rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("rows,k,n", [(1000, 120, 120), (257, 37, 5), (64, 480, 480)])
def test_block_rotate_matches_numpy(rows, k, n):
    """Y = X M (the rotation of Alg. 3) against the library product, FP64."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    rng = np.random.default_rng(rows + k)
    X = rng.standard_normal((rows, k))
    M = rng.standard_normal((k, n))
    Y = host(scsf.block_rotate_fp64(torch.as_tensor(X, device=dev), torch.as_tensor(M, device=dev)))
    ref = X @ M
    assert np.max(np.abs(Y - ref)) <= 1e-13 * k * np.max(np.abs(ref))


@pytest.mark.parametrize("rows,k,lo_exp", [(5000, 120, -30), (3001, 200, -30), (700, 7, 0),
                                           (600, 1, 0), (2000, 127, -10), (2000, 128, -10),
                                           (3000, 160, -30), (900, 33, -3)])
def test_cholqr2_orthonormal_and_reproduces_x(rows, k, lo_exp):
    """Cholesky QR2 (Alg. 3, orthonormalisation) on X = Z diag(s) with Z Gaussian and column
    scales s down to 1e-30 (a Gram entry of 1e-60 is below FP32's range, so the FP32 first
    factor must work on the scaled Gram matrix): Q^T Q = I, Q R = X with R = Q^T X upper
    triangular, and Q equal to the library's Householder Q (its columns signed so that R has
    a positive diagonal; the column scales leave Q unchanged). k = 200 takes the wide path."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    rng = np.random.default_rng(rows + k)
    Z = rng.standard_normal((rows, k))
    s = 10.0 ** rng.uniform(lo_exp, 0.0, k)
    X = Z * s[None, :]
    Q, shifts = scsf.cholqr2(torch.as_tensor(X, device=dev))
    Q = host(Q)
    assert shifts == (0, 0)
    assert np.max(np.abs(Q.T @ Q - np.eye(k))) <= 1e-13
    R = Q.T @ X
    assert np.max(np.abs(np.tril(R, -1)) / s[None, :]) <= 1e-12
    assert np.max(np.abs(Q @ np.triu(R) - X) / s[None, :]) <= 1e-12
    Qr, Rr = np.linalg.qr(Z)
    Qr = Qr * np.sign(np.diag(Rr))[None, :]
    assert np.max(np.abs(Q - Qr)) <= 1e-11


@pytest.mark.parametrize("k", [24, 120, 150])
def test_cholqr2_shifted_restart_on_dependent_columns(k):
    """Nine columns within 1e-7 of each other: the FP32 first factor's pivots for eight of them
    are rounding noise, one of which is not positive, so it restarts on S + s I (shifted
    Cholesky QR); the FP64 second pass then needs no shift, Q spans X (Q R = X with
    R = Q^T X upper triangular) and is orthonormal to the level that one FP64 pass reaches on
    the shifted first factor's condition number."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    rng = np.random.default_rng(k)
    X = rng.standard_normal((4000, k))
    X[:, 1:9] = X[:, [0]] + 1e-7 * rng.standard_normal((4000, 8))
    Q, shifts = scsf.cholqr2(torch.as_tensor(X, device=dev))
    Q = host(Q)
    assert shifts[0] >= 1 and shifts[1] == 0
    assert np.max(np.abs(Q.T @ Q - np.eye(k))) <= 1e-4
    R = Q.T @ X
    assert np.max(np.abs(Q @ np.triu(R) - X)) <= 1e-8 * np.max(np.abs(X))
