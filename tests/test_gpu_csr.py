"""The CSR operator kind: general symmetric sparse matrices through the FP64 path (filter,
Gershgorin bounds, chain solve, batched solve) against the oracle on the same matrices."""
import numpy as np
import pytest
import scipy.sparse as sp

import scsf_inputs as si
from oracle import chebyshev, compare, dense, operators, sturm
from tests.gpu_util import host, need_gpu, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RES_TOL = 1e-8
EIG_RTOL = 1e-10


def _csr_of(A):
    """The CSR arrays of a scipy matrix as a device operator (int32 indices)."""
    import paper_2510_23215_gb300 as scsf
    A = A.tocsr()
    A.sort_indices()
    return scsf.Operator.csr(A.indptr.astype(np.int32), A.indices.astype(np.int32),
                             A.data.astype(np.float64), torch.device("cuda", 0))


def _with_empty_rows(A, rows):
    """A with every entry of the given rows and columns removed (empty CSR rows)."""
    keep = np.ones(A.shape[0])
    keep[rows] = 0.0
    D = sp.diags(keep)
    B = (D @ A @ D).tocsr()
    B.eliminate_zeros()
    return B


@pytest.mark.parametrize("ncols", [1, 33, 120])
def test_csr_filter_matches_oracle_with_empty_rows(ncols):
    """Alg. 1 on an irregular CSR matrix with a ragged row count (2999) and five empty rows,
    element by element against the oracle's recurrence."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    A = _with_empty_rows(operators.assemble(si.knn_graph_chain(2999, 1, seed=11)[0]),
                         [0, 17, 1500, 2997, 2998])
    assert np.all(np.diff(A.indptr)[[0, 17, 1500, 2997, 2998]] == 0)
    lo, hi = operators.gershgorin_bounds(A)
    lam, alpha = lo, lo + 0.05 * (hi - lo)
    c, e = 0.5 * (alpha + hi), 0.5 * (hi - alpha)
    X = np.random.default_rng(ncols).standard_normal((A.shape[0], ncols))
    degree = 9
    ref = chebyshev.chebyshev_filter(A, X, degree, lam, c, e)
    got = host(scsf.cheb_filter(_csr_of(A), torch.as_tensor(X, device=dev), degree, lam, c, e))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_csr_bounds_match_oracle_and_stencil():
    """Gershgorin bounds of a CSR matrix against the oracle's; the CSR form of a stencil
    operator gives the stencil path's bounds."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    A = operators.assemble(si.knn_graph_chain(1001, 1, seed=12)[0])
    lo, hi = scsf.assemble_bounds(_csr_of(A))
    rlo, rhi = operators.gershgorin_bounds(A)
    assert abs(lo - rlo) <= 1e-13 * abs(rhi) and abs(hi - rhi) <= 1e-13 * abs(rhi)
    op = si.div_a_grad_chain(37, 1, seed=13)[0]
    s_lo, s_hi = scsf.assemble_bounds(to_dev([op], dev)[0])
    c_lo, c_hi = scsf.assemble_bounds(_csr_of(operators.assemble(op)))
    assert abs(s_lo - c_lo) <= 1e-12 * s_hi and abs(s_hi - c_hi) <= 1e-12 * s_hi


def test_csr_chain_matches_dense_definition():
    """A warm-started chain of three kNN-graph operators (2999 rows, k = 20): eigenvalues
    against the dense definition, residuals recomputed by the oracle, orthonormal vectors."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    ops = si.knn_graph_chain(2999, 3, seed=14)
    params = scsf.Params(k=20, degree=16, tol=RES_TOL, precision=scsf.FP64, seed=3)
    ev, rs, vec, stats = scsf.solve(to_dev(ops, dev), params, want_vectors=True)
    ev, rs, vec = host(ev), host(rs), host(vec)
    for j, op in enumerate(ops):
        A = operators.assemble(op)
        w, _ = dense.smallest_eigenpairs(A, 20)
        assert compare.max_rel_eig_error(w, ev[j]) <= EIG_RTOL
        assert np.max(rs[j]) <= RES_TOL
        assert np.max(operators.relative_residuals(A, vec[j], ev[j])) <= 1.05 * RES_TOL
        assert compare.orthonormality_error(vec[j]) <= 1e-12
    assert all(s["converged"] for s in stats)


@pytest.mark.parametrize("n,k", [(40, 24), (128, 100)])
def test_csr_form_of_stencil_matches_exact_spectrum(n, k):
    """The CSR form of a separable stencil operator (128 x 128 at k = 100: the headline
    shape) solved through the CSR kernels: every eigenvalue against Sturm bisection, and
    the stencil path on the same operator within the same tolerance."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op = si.separable_div_a_grad(n, seed=15)
    ref = sturm.separable_smallest_fast(n, op.ax[:, 0], op.P[:, 0], k)
    params = scsf.Params(k=k, degree=20, tol=RES_TOL, precision=scsf.FP64, seed=4)
    ev_c, rs_c, _, st_c = scsf.solve([_csr_of(operators.assemble(op))], params)
    ev_s, rs_s, _, _ = scsf.solve(to_dev([op], dev), params)
    assert st_c[0]["converged"]
    assert np.max(host(rs_c)) <= RES_TOL
    assert compare.max_rel_eig_error(ref, host(ev_c)[0]) <= EIG_RTOL
    assert compare.max_rel_eig_error(ref, host(ev_s)[0]) <= EIG_RTOL


def test_csr_batched_with_stencil_chains_matches_sequential():
    """CSR and stencil chains in flight together give the same bits as each chain alone."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    chains = [
        (to_dev(si.knn_graph_chain(2001, 2, seed=16), dev),
         scsf.Params(k=12, degree=16, tol=RES_TOL, precision=scsf.FP64, seed=5)),
        (to_dev(si.div_a_grad_chain(32, 2, seed=17), dev),
         scsf.Params(k=16, degree=16, tol=RES_TOL, precision=scsf.FP64, seed=6)),
        (to_dev(si.knn_graph_chain(1500, 3, seed=18), dev),
         scsf.Params(k=30, degree=16, tol=RES_TOL, precision=scsf.FP64, seed=7)),
    ]
    res = scsf.solve_batched(chains, concurrency=3)
    for (ops, params), (ev, rs, _, _, status) in zip(chains, res):
        assert status == 0 and float(rs.max()) <= RES_TOL
        ev1, rs1, _, _ = scsf.solve(ops, params)
        assert torch.equal(ev, ev1) and torch.equal(rs, rs1)


def test_csr_rejected_where_unsupported():
    """The mixed form, the FP32 and defect-corrected filters take stencils only; a chain
    takes only the operator kind and size it was made for."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    csr = to_dev(si.knn_graph_chain(500, 1, seed=19), dev)[0]
    with pytest.raises(ValueError):
        scsf.solve([csr], scsf.Params(k=8, degree=8, precision=scsf.MIXED))
    with pytest.raises(ValueError):
        scsf.Chain(scsf.Params(k=8, degree=8, precision=scsf.MIXED), 0, dev, rows=500)
    p64 = scsf.Params(k=8, degree=8, precision=scsf.FP64)
    grid_chain = scsf.Chain(p64, 24, dev)
    with pytest.raises(scsf.ScsfError):
        grid_chain.step(csr)
    row_chain = scsf.Chain(p64, 0, dev, rows=499)
    with pytest.raises(scsf.ScsfError):
        row_chain.step(csr)  # 500 rows on a 499-row chain
    with pytest.raises(scsf.ScsfError):
        row_chain.step(to_dev([si.constant_div_a_grad(24)], dev)[0])
    X32 = torch.zeros((500, 8), dtype=torch.float32, device=dev)
    with pytest.raises(scsf.ScsfError):
        scsf.cheb_filter_f32(csr, X32, 4, 0.0, 5.0, 2.0)
    X = torch.zeros((500, 8), dtype=torch.float64, device=dev)
    theta = torch.zeros(8, dtype=torch.float64, device=dev)
    with pytest.raises((ValueError, scsf.ScsfError)):
        scsf.cheb_filter_dc(csr, X, theta, 4, 0.0, 5.0, 2.0)
