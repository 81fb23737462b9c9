"""Mixed-precision form (FP32 phase + FP64 finish) against the oracle and the FP64 form."""
import numpy as np
import pytest

import scsf_inputs as si
from oracle import chebyshev, compare, dense, operators
from tests.gpu_util import host, need_gpu, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EIG_RTOL = 1e-10
RES_TOL = 1e-8


@pytest.mark.parametrize("n,ncols,degree", [(20, 36, 1), (33, 24, 7), (17, 120, 20), (40, 4, 16)])
def test_filter_f32_matches_oracle(n, ncols, degree):
    """FP32 recurrence vs the FP64 oracle: error at FP32 level, relative to the block size."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op = si.div_a_grad_chain(n, 1, seed=n + 1)[0]
    A = operators.assemble(op)
    lo, hi = operators.gershgorin_bounds(A)
    lam, alpha = lo + 0.001 * (hi - lo), lo + 0.05 * (hi - lo)
    c, e = 0.5 * (alpha + hi), 0.5 * (hi - alpha)
    X = si.gaussian_block(n * n, ncols, seed=4)
    ref = chebyshev.chebyshev_filter(A, X.astype(np.float32).astype(np.float64), degree, lam, c, e)
    Y = scsf.cheb_filter_f32(to_dev([op], dev)[0], torch.as_tensor(X, dtype=torch.float32, device=dev),
                             degree, lam, c, e)
    got = host(Y).astype(np.float64)
    scale = np.max(np.abs(ref))
    # each step rounds to FP32 and the recurrence amplifies at most like the filter itself
    assert np.max(np.abs(got - ref)) <= 2e-5 * degree * scale


def _filter_setup(n, seed):
    op = si.div_a_grad_chain(n, 1, seed=seed)[0]
    A = operators.assemble(op)
    lo, hi = operators.gershgorin_bounds(A)
    lam, alpha = lo + 0.001 * (hi - lo), lo + 0.05 * (hi - lo)
    return op, A, lam, 0.5 * (alpha + hi), 0.5 * (hi - alpha)


@pytest.mark.parametrize("n,ncols,degree", [(20, 37, 1), (24, 13, 13), (17, 120, 20)])
def test_filter_dc_any_theta_matches_oracle(n, ncols, degree):
    """The split Y = X diag(y(theta)) + Z is exact for any theta: with random X and theta
    the remainder is as large as Y, so the error is at the FP32 filter's level."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op, A, lam, c, e = _filter_setup(n, n + 3)
    X = si.gaussian_block(n * n, ncols, seed=5)
    theta = np.random.default_rng(6).uniform(lam, 2 * c, ncols)
    ref = chebyshev.chebyshev_filter(A, X, degree, lam, c, e)
    Y = scsf.cheb_filter_dc(to_dev([op], dev)[0], torch.as_tensor(X, device=dev),
                            torch.as_tensor(theta, device=dev), degree, lam, c, e)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(host(Y) - ref)) <= 2e-5 * degree * scale


@pytest.mark.parametrize("n,ncols,degree,noise", [(24, 37, 20, 1e-6), (20, 50, 60, 1e-9)])
def test_filter_dc_near_eigenvectors_reaches_fp64_accuracy(n, ncols, degree, noise):
    """Near Ritz pairs the residual block is small, so the FP32 remainder carries an
    error of eps32 times its own size: the result agrees with the FP64 filter far
    below the FP32 level (1e-9 relative, against 2e-5 per step for the FP32 filter)."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op, A, lam, c, e = _filter_setup(n, n + 7)
    w, V = np.linalg.eigh(A.toarray())
    rng = np.random.default_rng(8)
    X = V[:, :ncols] + noise * rng.standard_normal((n * n, ncols))
    theta = np.einsum("ij,ij->j", X, A @ X) / np.einsum("ij,ij->j", X, X)
    ref = chebyshev.chebyshev_filter(A, X, degree, lam, c, e)
    Y = scsf.cheb_filter_dc(to_dev([op], dev)[0], torch.as_tensor(X, device=dev),
                            torch.as_tensor(theta, device=dev), degree, lam, c, e)
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(host(Y) - ref)) <= 1e-9 * scale


@pytest.mark.parametrize("n,ncols,degree,noise,tol", [(24, 37, 20, 1e-6, 1e-9),
                                                       (20, 50, 60, 1e-9, 1e-9),
                                                       (17, 13, 13, None, 2e-5)])
def test_filter_dc_grouped_matches_oracle_per_group(n, ncols, degree, noise, tol):
    """Per-group degrees: columns [4g, 4g+4) come out as the degree-m_g filter of those
    columns (the oracle's Alg. 1 run per group), ragged last group included; near Ritz pairs
    at FP64 accuracy, from random blocks (noise None) at the FP32 filter's level."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op, A, lam, c, e = _filter_setup(n, n + 11)
    rng = np.random.default_rng(12)
    if noise is None:
        X = si.gaussian_block(n * n, ncols, seed=13)
        theta = rng.uniform(lam, 2 * c, ncols)
    else:
        w, V = np.linalg.eigh(A.toarray())
        X = V[:, :ncols] + noise * rng.standard_normal((n * n, ncols))
        theta = np.einsum("ij,ij->j", X, A @ X) / np.einsum("ij,ij->j", X, X)
    groups = (ncols + 3) // 4
    gdeg = rng.integers(1, degree + 1, groups)
    gdeg[0], gdeg[-1] = 1, degree
    Y = host(scsf.cheb_filter_dc(to_dev([op], dev)[0], torch.as_tensor(X, device=dev),
                                 torch.as_tensor(theta, device=dev), degree, lam, c, e,
                                 group_degrees=gdeg.tolist()))
    refs = [chebyshev.chebyshev_filter(A, X[:, 4 * g:4 * g + 4], int(gdeg[g]), lam, c, e)
            for g in range(groups)]
    # the block's scale, as for the uniform degree (damped groups are far below it)
    scale = max(np.max(np.abs(r)) for r in refs)
    for g in range(groups):
        bound = tol * scale if noise is not None else tol * int(gdeg[g]) * scale
        assert np.max(np.abs(Y[:, 4 * g:4 * g + 4] - refs[g])) <= bound, g


def test_filter_dc_grouped_rejects_bad_degrees():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op, A, lam, c, e = _filter_setup(12, 5)
    X = torch.as_tensor(si.gaussian_block(144, 8, seed=1), device=dev)
    th = torch.zeros(8, dtype=torch.float64, device=dev)
    for bad in ([0, 4], [4, 5], [4]):
        with pytest.raises((scsf.ScsfError, ValueError)):
            scsf.cheb_filter_dc(to_dev([op], dev)[0], X, th, 4, lam, c, e, group_degrees=bad)


@pytest.mark.parametrize("n", [128, 180])
def test_resident_filter_variants_match_oracle(n):
    """The cluster-resident filters at a grid where the register-strip kernel applies (128) and
    one where a band needs more than 1024 threads, so only the shared-memory kernels apply
    (180): both the FP32 filter and the defect-corrected one against the oracle's Alg. 1, twice
    (the second call runs the shape tuner's cached choice)."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op, A, lam, c, e = _filter_setup(n, n + 21)
    ncols, degree = 8, 6
    X = si.gaussian_block(n * n, ncols, seed=n)
    ref = chebyshev.chebyshev_filter(A, X.astype(np.float32).astype(np.float64), degree, lam, c, e)
    dop = to_dev([op], dev)[0]
    for _ in range(2):
        Y = host(scsf.cheb_filter_f32(dop, torch.as_tensor(X, dtype=torch.float32, device=dev),
                                      degree, lam, c, e)).astype(np.float64)
        assert np.max(np.abs(Y - ref)) <= 2e-5 * degree * np.max(np.abs(ref))
    theta = np.random.default_rng(n).uniform(lam, 2 * c, ncols)
    ref_dc = chebyshev.chebyshev_filter(A, X, degree, lam, c, e)
    for _ in range(2):
        Y = host(scsf.cheb_filter_dc(dop, torch.as_tensor(X, device=dev),
                                     torch.as_tensor(theta, device=dev), degree, lam, c, e))
        assert np.max(np.abs(Y - ref_dc)) <= 2e-5 * degree * np.max(np.abs(ref_dc))


def _check(op, evals, resid, evecs, k, ref_vals, ref_vecs=None):
    A = operators.assemble(op)
    assert np.max(resid) <= RES_TOL
    assert np.max(operators.relative_residuals(A, evecs, evals)) <= 1.05 * RES_TOL
    assert compare.orthonormality_error(evecs) <= 1e-12
    assert compare.max_rel_eig_error(ref_vals, evals) <= EIG_RTOL
    if ref_vecs is not None:
        assert compare.max_cluster_angle(ref_vals, ref_vecs, evecs) <= 1e-5


def test_mixed_poisson32_chain_matches_dense_definition():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    ops = si.div_a_grad_chain(32, 16, seed=0)
    perm = host(scsf.sort(torch.as_tensor(np.stack([o.P for o in ops]), device=dev), p0=8))
    ordered = [ops[i] for i in perm]
    p = scsf.Params(k=20, degree=16, tol=1e-8, precision=scsf.MIXED)
    ev, rs, vec, stats = scsf.solve(to_dev(ordered, dev), p, want_vectors=True)
    ev, rs, vec = host(ev), host(rs), host(vec)
    for j, op in enumerate(ordered):
        w, V = dense.smallest_eigenpairs(operators.assemble(op), 20)
        _check(op, ev[j], rs[j], vec[j], 20, w, V)
    assert all(s["converged"] for s in stats)
    assert all(s["iters_fp32"] >= 1 for s in stats)


def test_mixed_matches_fp64_form_on_poisson128_prefix():
    """The first 12 problems of the 128 x 128, k = 100 chain: both forms give the same pairs."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    n, k = 128, 100
    ops = si.div_a_grad_chain(n, 200, seed=1)
    perm = host(scsf.sort(torch.as_tensor(np.stack([o.P for o in ops]), device=dev), p0=8))
    ordered = to_dev([ops[i] for i in perm[:12]], dev)
    ev64, rs64, _, st64 = scsf.solve(ordered, scsf.Params(k=k, degree=20, tol=1e-8))
    evm, rsm, vecm, stm = scsf.solve(ordered, scsf.Params(k=k, degree=20, tol=1e-8,
                                                          precision=scsf.MIXED), want_vectors=True)
    ev64, evm = host(ev64), host(evm)
    for j in range(12):
        assert compare.max_rel_eig_error(ev64[j], evm[j]) <= EIG_RTOL
        assert float(rsm[j].max()) <= RES_TOL
    op0 = ops[perm[0]]
    A = operators.assemble(op0)
    assert np.max(operators.relative_residuals(A, host(vecm)[0], evm[0])) <= 1.05 * RES_TOL
    assert compare.orthonormality_error(host(vecm)[0]) <= 1e-12
    assert all(s["iters_fp32"] >= 1 for s in stm)


def test_mixed_high_degree_matches_dense_definition():
    """The chosen form's tuning (degree 60 in both phases) gives the same pairs."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    ops = si.div_a_grad_chain(48, 4, seed=21)
    p = scsf.Params(k=40, degree=60, degree_fp32=60, tol=1e-8, precision=scsf.MIXED)
    ev, rs, vec, stats = scsf.solve(to_dev(ops, dev), p, want_vectors=True)
    for j, op in enumerate(ops):
        w, V = dense.smallest_eigenpairs(operators.assemble(op), 40)
        _check(op, host(ev)[j], host(rs)[j], host(vec)[j], 40, w, V)
    assert all(s["converged"] for s in stats)


def test_mixed_rejects_block_width_not_multiple_of_four():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    with pytest.raises(scsf.ScsfError):
        scsf.Chain(scsf.Params(k=10, nex=3, precision=scsf.MIXED), 16, device=dev)


def test_mixed_column_degree_filters_fewer_elements_same_pairs():
    """Per-column degrees in the FP64 phase (scsf_params.column_degree): the same eigenpairs
    to the tolerance as the uniform degree, with fewer defect-corrected filter elements."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    ops = si.div_a_grad_chain(48, 6, seed=21)
    res = {}
    for coldeg in (False, True):
        p = scsf.Params(k=40, degree=40, degree_fp32=24, tol=1e-10, precision=scsf.MIXED,
                        column_degree=coldeg)
        ev, rs, vec, stats = scsf.solve(to_dev(ops, dev), p, want_vectors=True)
        res[coldeg] = (host(ev), host(rs), host(vec), stats)
    ev, rs, vec, stats = res[True]
    for j, op in enumerate(ops):
        A = operators.assemble(op)
        w, V = dense.smallest_eigenpairs(A, 40)
        assert np.max(rs[j]) <= 1e-10
        assert np.max(operators.relative_residuals(A, vec[j], ev[j])) <= 1.05e-10
        assert compare.orthonormality_error(vec[j]) <= 1e-12
        assert compare.max_rel_eig_error(w, ev[j]) <= EIG_RTOL
    e_uni = sum(s["filter_dc_elems"] for s in res[False][3])
    e_col = sum(s["filter_dc_elems"] for s in res[True][3])
    assert e_col < e_uni
