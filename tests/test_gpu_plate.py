"""The thin-plate vibration operator (App. D.2 item 4): device assembly of its 13-point
standard form, the filter and bounds on it, and chain solves of the generalized problem
against the oracle (dense generalized eigensolver, and the uniform plate's closed form)."""
import numpy as np
import pytest

import scsf_inputs as si
from oracle import chebyshev, operators
from tests.gpu_util import host, need_gpu, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RES_TOL = 1e-8
EIG_RTOL = 1e-10
EPS = np.finfo(np.float64).eps


def _eig_close(ref, got, C):
    """Eigenvalues agree to 1e-10 relative, or to the FP64 representation limit of C: the
    stored matrix and every product with it carry errors of a few eps ||C||, which move an
    eigenvalue by as much (Weyl); the biharmonic's ||C|| / lambda_1 reaches 10^7 at n = 100,
    so its lowest eigenvalues are fixed only to ~1e-9 relative in FP64."""
    beta = operators.gershgorin_bounds(C)[1]
    return bool(np.all(np.abs(np.asarray(got) - ref) <= EIG_RTOL * np.abs(ref) + 2 * EPS * beta))


def _uniform_plate_spectrum(n, d0, r0, k):
    """(D / rho) (lambda_i + lambda_j)^2 over the 1-D Dirichlet Laplacian eigenvalues."""
    h = 1.0 / (n + 1)
    lam1 = 4.0 / h**2 * np.sin(np.arange(1, n + 1) * np.pi * h / 2) ** 2
    return np.sort((d0 / r0 * (lam1[:, None] + lam1[None, :]) ** 2).ravel())[:k]


@pytest.mark.parametrize("n,ncols", [(23, 33), (40, 120)])
def test_plate_apply_and_filter_match_oracle(n, ncols):
    """Degree 1 with lambda = 1, c = 0, e = 1 applies C itself: C X element by element against
    the oracle's assembled standard form (ragged N = 529 and N = 1600); then a degree-9 filter
    against the oracle's recurrence."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op = si.plate_chain(n, 1, seed=21)[0]
    C = operators.assemble(op)
    X = np.random.default_rng(n).standard_normal((n * n, ncols))
    dop = to_dev([op], dev)[0]
    CX = host(scsf.cheb_filter(dop, torch.as_tensor(X, device=dev), 1, 1.0, 0.0, 1.0))
    ref = C @ X
    assert np.max(np.abs(CX - ref)) <= 1e-13 * np.max(np.abs(ref))
    lo, hi = operators.gershgorin_bounds(C)
    lam, alpha = lo, lo + 1e-3 * (hi - lo)
    c, e = 0.5 * (alpha + hi), 0.5 * (hi - alpha)
    ref9 = chebyshev.chebyshev_filter(C, X, 9, lam, c, e)
    got9 = host(scsf.cheb_filter(dop, torch.as_tensor(X, device=dev), 9, lam, c, e))
    assert np.max(np.abs(got9 - ref9)) <= 1e-12 * np.max(np.abs(ref9))


def test_plate_bounds_match_oracle():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op = si.plate_chain(37, 1, seed=22)[0]
    lo, hi = scsf.assemble_bounds(to_dev([op], dev)[0])
    rlo, rhi = operators.gershgorin_bounds(operators.assemble(op))
    assert abs(lo - rlo) <= 1e-13 * rhi and abs(hi - rhi) <= 1e-13 * rhi


@pytest.mark.parametrize("n,k", [(32, 40), (100, 100)])
def test_uniform_plate_closed_form(n, k):
    """D = 2, rho = 0.5: every eigenvalue against (D / rho)(lambda_i + lambda_j)^2 (n = 100 is
    the paper's matrix dimension, N = 10^4); the modes are M-orthonormal (u^T M u = I)."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    d0, r0 = 2.0, 0.5
    op = si.constant_plate(n, d0, r0)
    params = scsf.Params(k=k, degree=40, tol=RES_TOL, max_iter=400, precision=scsf.FP64, seed=9)
    ev, rs, vec, stats = scsf.solve(to_dev([op], dev), params, want_vectors=True)
    ref = _uniform_plate_spectrum(n, d0, r0, k)
    assert stats[0]["converged"]
    assert np.max(host(rs)) <= RES_TOL
    assert _eig_close(ref, host(ev)[0], operators.assemble(op))
    U = host(vec)[0]
    assert np.max(np.abs(r0 * U.T @ U - np.eye(k))) <= 1e-12


def test_plate_chain_matches_generalized_dense_definition():
    """A warm-started chain of three variable plates (24 x 24, k = 20): eigenvalues against
    LAPACK's generalized symmetric-definite solver on (K, M), modes u with K u = lambda M u
    and u^T M u = I, largest-magnitude entry positive."""
    dev = need_gpu()
    import scipy.linalg as sla
    import paper_2510_23215_gb300 as scsf
    ops = si.plate_chain(24, 3, seed=23)
    params = scsf.Params(k=20, degree=30, tol=RES_TOL, max_iter=400, precision=scsf.FP64, seed=2)
    ev, rs, vec, stats = scsf.solve(to_dev(ops, dev), params, want_vectors=True)
    ev, rs, vec = host(ev), host(rs), host(vec)
    for j, op in enumerate(ops):
        K = operators.assemble_plate_stiffness(op.n, op.D).toarray()
        m = op.rho.reshape(-1)
        w = sla.eigh(K, np.diag(m), eigvals_only=True)[:20]
        assert _eig_close(w, ev[j], operators.assemble(op))
        assert np.max(rs[j]) <= RES_TOL
        U = vec[j]
        KU = K @ U
        r = np.linalg.norm(KU - (m[:, None] * U) * ev[j], axis=0) / np.linalg.norm(KU, axis=0)
        assert np.max(r) <= 1e-6  # the M-weighted form of a 1e-8 standard-form residual
        assert np.max(np.abs(U.T @ (m[:, None] * U) - np.eye(20))) <= 1e-12
        idx = np.argmax(np.abs(U), axis=0)
        assert np.all(U[idx, np.arange(20)] > 0)
    assert all(s["converged"] for s in stats)


def test_plate_rejected_where_unsupported():
    """The mixed form and the FP32 / defect-corrected filters take 5-point stencils only."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op = to_dev([si.plate_chain(24, 1, seed=24)[0]], dev)[0]
    with pytest.raises(scsf.ScsfError):
        scsf.solve([op], scsf.Params(k=8, nex=4, degree=8, precision=scsf.MIXED))
    X32 = torch.zeros((24 * 24, 8), dtype=torch.float32, device=dev)
    with pytest.raises(scsf.ScsfError):
        scsf.cheb_filter_f32(op, X32, 4, 0.0, 5.0, 2.0)
