"""Tensor-core block products (digit split on tcgen05, FP64 accuracy) against the oracle's
correctly rounded products: the Gram matrix X^T X and Q^T (A Q) of Alg. 3's
orthonormalisation and Rayleigh-Ritz steps, and the rotation X = Q Z."""
import numpy as np
import pytest

from oracle import products
from tests.gpu_util import host, need_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _block(rows, cols, seed, scales=None):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((rows, cols))
    if scales is not None:
        X *= scales[None, :]
    return X


def _check_tn(C, A, B, tol_norm, tol_abs):
    ref = products.exact_tn(A, B)
    norms = np.outer(np.linalg.norm(A, axis=0), np.linalg.norm(B, axis=0))
    absprod = np.abs(A).T @ np.abs(B)
    err = np.abs(C - ref)
    nz = norms > 0
    worst_norm = np.max(err[nz] / norms[nz]) if nz.any() else 0.0
    worst_abs = np.max(err[nz] / absprod[nz]) if nz.any() else 0.0
    print(f"normwise {worst_norm:.2e}  componentwise {worst_abs:.2e}")
    assert np.all(err[~nz] == 0.0)
    assert worst_norm <= tol_norm
    assert worst_abs <= tol_abs


@pytest.mark.parametrize("rows,m,n", [(3001, 70, 45), (640, 120, 120), (64, 1, 33), (130, 200, 9)])
def test_gram_general_matches_exact_product(rows, m, n):
    """C = A^T B, ragged sizes (K not a multiple of 64, widths across tile edges), column
    scales from 1e-30 to 1e3, one all-zero column."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    A = _block(rows, m, 1, np.logspace(-30, 3, m))
    B = _block(rows, n, 2, np.logspace(3, -30, n))
    B[:, n // 2] = 0.0
    C = host(scsf.block_gram(torch.as_tensor(A, device=dev), torch.as_tensor(B, device=dev)))
    _check_tn(C, A, B, 1e-14, 1e-13)


def test_gram_symmetric_forms():
    """X^T X (B = A, shared digit planes) and Q^T (L Q) with L a symmetric tridiagonal
    operator (B != A, symmetric result): upper tiles only, mirrored."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    rows, k = 2500, 150
    X = _block(rows, k, 3, np.logspace(-10, 2, k))
    C = host(scsf.block_gram(torch.as_tensor(X, device=dev), symmetric=True))
    assert np.array_equal(C, C.T)
    _check_tn(C, X, X, 1e-14, 1e-13)
    LX = 2.0 * X
    LX[1:] -= X[:-1]
    LX[:-1] -= X[1:]
    C2 = host(scsf.block_gram(torch.as_tensor(X, device=dev), torch.as_tensor(LX, device=dev),
                              symmetric=True))
    assert np.array_equal(C2, C2.T)
    ref = products.exact_tn(X, LX)
    norms = np.outer(np.linalg.norm(X, axis=0), np.linalg.norm(LX, axis=0))
    assert np.max(np.abs(C2 - ref) / norms) <= 1e-14


def test_gram_deterministic_and_fp64_method_agrees():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    X = torch.as_tensor(_block(16384, 120, 4), device=dev)
    c1 = host(scsf.block_gram(X, symmetric=True))
    c2 = host(scsf.block_gram(X, symmetric=True))
    assert np.array_equal(c1, c2)  # integer level sums: no order dependence
    c64 = host(scsf.block_gram(X, symmetric=True, method=scsf.PRODUCT_FP64))
    assert np.max(np.abs(c1 - c64)) <= 1e-12 * np.max(np.abs(c64))


def test_gram_large_k400_shape():
    """The 256 x 256, k = 400 block (N = 65536, k_b = 480): split over K and many tiles."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    rng = np.random.default_rng(5)
    X = rng.standard_normal((65536, 480))
    C = host(scsf.block_gram(torch.as_tensor(X, device=dev), symmetric=True))
    ref = X.T @ X  # library product; its own error is ~sqrt(K) eps
    d = np.sqrt(np.diag(ref))
    assert np.max(np.abs(C - ref) / np.outer(d, d)) <= 2e-14


@pytest.mark.parametrize("rows,k,n", [(3001, 70, 45), (257, 120, 120), (4096, 480, 40)])
def test_rotation_matches_exact_product(rows, k, n):
    """Y = X M with row scales 1e-20..1e5 and a triangular M (Cholesky QR's X R^-1)."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    rng = np.random.default_rng(rows + k)
    X = rng.standard_normal((rows, k)) * np.logspace(-20, 5, rows)[:, None]
    M = np.triu(rng.standard_normal((k, n)))
    Y = host(scsf.block_rotate(torch.as_tensor(X, device=dev), torch.as_tensor(M, device=dev)))
    ref = products.exact_nn(X, M)
    norms = np.outer(np.linalg.norm(X, axis=1), np.linalg.norm(M, axis=0))
    nz = norms > 0
    assert np.max(np.abs(Y - ref)[nz] / norms[nz]) <= 1e-14


@pytest.mark.parametrize("rows,m,n,sym", [(5000, 120, 120, True), (3001, 40, 72, False)])
def test_four_digit_gram_is_fp32_class(rows, m, n, sym):
    """The FP32 phase's products keep 4 base-128 digits per operand (28 bits against a
    row or column maximum): against the exactly rounded product the error stays at the
    FP32 level, normwise below 1e-7 of |a_i| |b_j| (Gaussian columns scaled over 1e-6..1e3);
    a wrong digit, level or tile would show as an error of order one."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    A = _block(rows, m, 11, np.logspace(-6, 3, m))
    B = A if sym else _block(rows, n, 12, np.logspace(2, -4, n))
    C = host(scsf.block_gram(torch.as_tensor(A, device=dev),
                             None if sym else torch.as_tensor(B, device=dev),
                             symmetric=sym, slices=4))
    ref = products.exact_tn(A, B)
    norms = np.outer(np.linalg.norm(A, axis=0), np.linalg.norm(B, axis=0))
    err = np.max(np.abs(C - ref) / norms)
    print(f"4 digits: normwise {err:.2e}")
    assert err <= 1e-7
    assert err >= 1e-12  # really the short split, not the 8-digit one


def test_four_digit_rotation_is_fp32_class():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    rng = np.random.default_rng(13)
    X = rng.standard_normal((4099, 120)) * np.logspace(-3, 3, 4099)[:, None]
    M = rng.standard_normal((120, 120))
    Y = host(scsf.block_rotate(torch.as_tensor(X, device=dev), torch.as_tensor(M, device=dev),
                               slices=4))
    ref = products.exact_nn(X, M)
    norms = np.outer(np.linalg.norm(X, axis=1), np.linalg.norm(M, axis=0))
    assert np.max(np.abs(Y - ref) / norms) <= 1e-7


def test_rotation_alpha_beta_update():
    """Y <- Y - V C (deflation against locked columns)."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    rng = np.random.default_rng(9)
    V = rng.standard_normal((5000, 30))
    Cm = rng.standard_normal((30, 90))
    Y0 = rng.standard_normal((5000, 90))
    Y = torch.as_tensor(Y0.copy(), device=dev)
    scsf.block_rotate(torch.as_tensor(V, device=dev), torch.as_tensor(Cm, device=dev), Y,
                      alpha=-1.0, beta=1.0)
    ref = Y0 - products.exact_nn(V, Cm)
    assert np.max(np.abs(host(Y) - ref)) <= 1e-14 * np.max(np.abs(ref))


def test_nonfinite_input_gives_nan_not_garbage():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    A = _block(300, 40, 7)
    A[17, 5] = np.nan
    C = host(scsf.block_gram(torch.as_tensor(A, device=dev), symmetric=True))
    assert np.all(np.isnan(C[5, :])) and np.all(np.isnan(C[:, 5]))
    rest = np.delete(np.delete(C, 5, 0), 5, 1)
    assert np.all(np.isfinite(rest))
