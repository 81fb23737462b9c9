"""End-to-end parity of the warm-started chain solve (Alg. 3 along a sorted chain)."""
import numpy as np
import pytest
import scipy.linalg as sla

import scsf_inputs as si
from oracle import chfsi, compare, dense, inertia, operators, sturm
from oracle import sort as osort
from tests.gpu_util import host, need_gpu, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EIG_RTOL = 1e-10   # eigenvalue relative error at residual <= 1e-8
RES_TOL = 1e-8


def _check_result(op, evals, resid, evecs, k, ref_vals=None, ref_vecs=None):
    A = operators.assemble(op)
    assert np.all(np.isfinite(evals)) and np.all(np.diff(evals) >= 0)
    assert np.max(resid) <= RES_TOL
    r_cpu = operators.relative_residuals(A, evecs, evals)
    assert np.max(r_cpu) <= 1.05 * RES_TOL
    assert compare.orthonormality_error(evecs) <= 1e-12
    if ref_vals is not None:
        assert compare.max_rel_eig_error(ref_vals, evals) <= EIG_RTOL
    if ref_vecs is not None:
        assert compare.max_cluster_angle(ref_vals, ref_vecs, evecs) <= 1e-5


def test_poisson32_chain_matches_dense_definition():
    """16 problems, 32 x 32, k = 20, degree 16, sorted with p0 = 8, vs dense eigh of each."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    ops = si.div_a_grad_chain(32, 16, seed=0)
    perm = host(scsf.sort(torch.as_tensor(np.stack([o.P for o in ops]), device=dev), p0=8))
    ordered = [ops[i] for i in perm]
    ev, rs, vec, stats = scsf.solve(to_dev(ordered, dev), scsf.Params(k=20, degree=16, tol=1e-8),
                                    want_vectors=True)
    ev, rs, vec = host(ev), host(rs), host(vec)
    for j, op in enumerate(ordered):
        w, V = dense.smallest_eigenpairs(operators.assemble(op), 20)
        _check_result(op, ev[j], rs[j], vec[j], 20, w, V)
    assert all(s["converged"] for s in stats)


def test_laplacian_closed_form_with_degenerate_pairs():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    n, k = 24, 12
    ev, rs, vec, _ = scsf.solve(to_dev([si.constant_div_a_grad(n)], dev),
                                scsf.Params(k=k, degree=16, tol=1e-9), want_vectors=True)
    ref = sturm.laplacian_2d_eigenvalues(n)[:k]
    assert compare.max_rel_eig_error(ref, host(ev)[0]) <= 1e-11
    assert compare.orthonormality_error(host(vec)[0]) <= 1e-12


def test_separable_grid128_k100():
    """a = a(x): the spectrum is the union of n tridiagonal spectra (library tridiagonal solver)."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    n, k = 128, 100
    op = si.separable_div_a_grad(n, seed=4)
    ev, rs, vec, stats = scsf.solve(to_dev([op], dev), scsf.Params(k=k, degree=20, tol=1e-8),
                                    want_vectors=True)
    vals = []
    for d, e in sturm.separable_tridiagonals(n, op.ax[:, 0], op.P[:, 0]):
        vals.append(sla.eigh_tridiagonal(d, e, eigvals_only=True, select="i", select_range=(0, k - 1)))
    ref = np.sort(np.concatenate(vals))[:k]
    assert compare.max_rel_eig_error(ref, host(ev)[0]) <= EIG_RTOL
    assert np.max(host(rs)) <= RES_TOL


def test_lap_plus_v_operator():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    ops = si.lap_plus_v_chain(24, 3, seed=2)
    ev, rs, vec, _ = scsf.solve(to_dev(ops, dev), scsf.Params(k=16, degree=16, tol=1e-8),
                                want_vectors=True)
    for j, op in enumerate(ops):
        w, V = dense.smallest_eigenpairs(operators.assemble(op), 16)
        _check_result(op, host(ev)[j], host(rs)[j], host(vec)[j], 16, w, V)


def test_poisson128_full_chain_sampled():
    """The full 200-problem, 128 x 128, k = 100, degree 20 chain as the benchmark runs it;
    sampled problems are checked on the CPU (residuals, orthonormality, inertia, oracle ChFSI)."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    n, k, n_ops = 128, 100, 200
    ops = si.div_a_grad_chain(n, n_ops, seed=1)
    perm = host(scsf.sort(torch.as_tensor(np.stack([o.P for o in ops]), device=dev), p0=8))
    ordered = [ops[i] for i in perm]
    chain = scsf.Chain(scsf.Params(k=k, degree=20, tol=1e-8), n, device=dev)
    sample = {0, 1, 57, 199}
    kept = {}
    iters = []
    for j, op in enumerate(ordered):
        ev, rs, vec, st = chain.step(to_dev([op], dev)[0], want_vectors=j in sample)
        iters.append(st["iters"])
        assert st["converged"]
        assert float(rs.max()) <= RES_TOL
        if j in sample:
            kept[j] = (host(ev), host(rs), host(vec))
    for j, (ev, rs, vec) in kept.items():
        op = ordered[j]
        _check_result(op, ev, rs, vec, k)
        A = operators.assemble(op)
        sigma = ev[-1] * (1 + 1e-9)
        assert inertia.count_below(A, sigma, n) == k
    # the oracle's own ChFSI on the head problem
    ref = chfsi.solve_chain([ordered[0]], k=k, degree=20, tol=1e-8, head_seed=11)[0]
    assert ref.converged
    assert compare.max_rel_eig_error(ref.evals, kept[0][0]) <= EIG_RTOL


def test_similar_operators_warm_start_cuts_iterations():
    """Sec. 3.2 / the paper's perturbation study: along a chain of similar operators the
    warm start needs far fewer outer iterations than the random head, with the same answers."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    n, k = 48, 24
    ops = si.perturbed_div_a_grad_chain(n, 8, seed=3, eps=1e-3)
    ev, rs, vec, stats = scsf.solve(to_dev(ops, dev), scsf.Params(k=k, degree=16, tol=1e-8),
                                    want_vectors=True)
    iters = [s["iters"] for s in stats]
    # the oracle's Alg. 3 takes 25 iterations for the head and 15 for each warm-started one
    assert max(iters[1:]) + 5 <= iters[0], iters
    for j in (0, 7):
        w, V = dense.smallest_eigenpairs(operators.assemble(ops[j]), k)
        _check_result(ops[j], host(ev)[j], host(rs)[j], host(vec)[j], k, w, V)


def test_identical_problem_warm_start_converges_in_two():
    """Seeding the chain with an exact solution: the same problem converges in <= 2 iterations."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    n, k = 32, 20
    op = si.div_a_grad_chain(n, 1, seed=9)[0]
    dop = to_dev([op], dev)[0]
    p = scsf.Params(k=k, degree=16, tol=1e-8)
    chain = scsf.Chain(p, n, device=dev)
    ev0, _, _, st0 = chain.step(dop)
    ev1, _, _, st1 = chain.step(dop)
    assert st0["iters"] > 2 and st1["iters"] <= 2
    np.testing.assert_allclose(host(ev1), host(ev0), rtol=1e-10)
    # explicit seed path: eigenvectors plus extra dense columns
    w, V = dense.smallest_eigenpairs(operators.assemble(op), p.kb)
    fresh = scsf.Chain(p, n, device=dev)
    fresh.seed(torch.as_tensor(np.ascontiguousarray(V), device=dev), w.tolist())
    ev2, _, _, st2 = fresh.step(dop)
    assert st2["iters"] <= 2
    assert compare.max_rel_eig_error(w[:k], host(ev2)) <= EIG_RTOL


def test_not_converged_and_invalid_arguments():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    op = to_dev(si.div_a_grad_chain(16, 1, seed=1), dev)[0]
    chain = scsf.Chain(scsf.Params(k=10, degree=2, tol=1e-14, max_iter=1), 16, device=dev)
    ev, rs, _, st = chain.step(op, raise_on_nonconvergence=False)
    assert not st["converged"] and st["iters"] == 1
    assert np.isnan(host(ev)).any()
    with pytest.raises(scsf.ScsfError) as ei:
        chain.step(op)
    assert ei.value.status == scsf.ERR_NOT_CONVERGED
    with pytest.raises(ValueError):
        scsf.Chain(scsf.Params(k=430), 32, device=dev)  # k_b = 516 > 512
    other = to_dev(si.div_a_grad_chain(20, 1, seed=1), dev)[0]
    with pytest.raises(scsf.ScsfError):
        chain.step(other)
    with pytest.raises(ValueError):
        scsf.solve([scsf.Operator(scsf.DIV_A_GRAD, 16, ax=op.ax.cpu(), ay=op.ay.cpu())],
                   scsf.Params(k=4))


def test_eigenvector_sign_convention():
    """Returned eigenvectors: the largest-magnitude entry (lowest row on ties) is positive,
    and the sign flip leaves residuals and orthonormality intact."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    ops = si.div_a_grad_chain(24, 3, seed=12)
    ev, rs, vec, _ = scsf.solve(to_dev(ops, dev), scsf.Params(k=10, degree=16, tol=1e-8),
                                want_vectors=True)
    ev, rs, vec = host(ev), host(rs), host(vec)
    for j, op in enumerate(ops):
        V = vec[j]
        idx = np.argmax(np.abs(V), axis=0)  # first maximum: lowest row on ties
        assert np.all(V[idx, np.arange(V.shape[1])] > 0)
        _check_result(op, ev[j], rs[j], V, 10)


def test_non_finite_operator_coefficients_are_rejected():
    """A NaN or Inf coefficient (or a plate density <= 0) reaches the Gershgorin bounds, and
    the chain rejects the operator before iterating: SCSF_ERR_INVALID_ARG, in both forms."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    div = si.div_a_grad_chain(24, 1, seed=41)[0]
    div.ax[3, 4] = np.nan
    lapv = si.lap_plus_v_chain(24, 1, seed=42)[0]
    lapv.V[0, 0] = np.inf
    plate = si.plate_chain(24, 1, seed=43)[0]
    plate.rho[2, 2] = -1.0
    csr = si.knn_graph_chain(500, 1, seed=44)[0]
    csr.val[5] = np.nan
    cases = [(div, scsf.MIXED), (div, scsf.FP64), (lapv, scsf.FP64), (plate, scsf.FP64),
             (csr, scsf.FP64)]
    for op, prec in cases:
        with pytest.raises(scsf.ScsfError) as err:
            scsf.solve(to_dev([op], dev), scsf.Params(k=8, nex=4, degree=8, precision=prec))
        assert err.value.status == scsf.ERR_INVALID_ARG
    lo, hi = scsf.assemble_bounds(to_dev([div], dev)[0])
    assert np.isnan(lo) or np.isnan(hi)


@pytest.mark.parametrize("kind", ["div", "lapv", "plate"])
def test_lanczos_upper_bound_encloses_spectrum_and_keeps_results(kind):
    """Sec. 3.2's Lanczos estimate of the spectrum's upper end (16 steps, largest Ritz value
    plus the last residual norm): it lies above lambda_max (dense definition) and below the
    Gershgorin bound, and the solve returns the same pairs with no more outer iterations."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    if kind == "div":
        ops = si.div_a_grad_chain(40, 3, seed=12)
    elif kind == "lapv":
        ops = si.lap_plus_v_chain(40, 3, seed=13)
    else:
        ops = si.plate_chain(30, 2, seed=14)
    tol = 1e-7 if kind == "plate" else 1e-8
    out = {}
    for bound in (scsf.BOUND_GERSHGORIN, scsf.BOUND_LANCZOS):
        p = scsf.Params(k=16, degree=20, tol=tol, max_iter=300, seed=3, bound=bound)
        out[bound] = scsf.solve(to_dev(ops, dev), p)
    ev_g, rs_g, _, st_g = out[scsf.BOUND_GERSHGORIN]
    ev_l, rs_l, _, st_l = out[scsf.BOUND_LANCZOS]
    for j, op in enumerate(ops):
        A = operators.assemble(op)
        lmax = float(np.linalg.eigvalsh(A.toarray() if hasattr(A, "toarray") else A)[-1])
        assert st_l[j]["beta"] >= lmax
        assert st_l[j]["beta"] <= st_l[j]["beta_gershgorin"]
        assert st_g[j]["beta"] == st_g[j]["beta_gershgorin"]
        assert compare.max_rel_eig_error(host(ev_g)[j], host(ev_l)[j]) <= 1e-10
    assert float(rs_l.max()) <= tol
    iters_g = sum(s["iters"] for s in st_g)
    iters_l = sum(s["iters"] for s in st_l)
    print(f"{kind}: outer iterations Gershgorin {iters_g}, Lanczos {iters_l}; "
          f"beta / lambda_max {[round(s['beta'] / s['beta_gershgorin'], 3) for s in st_l]}")
    assert iters_l <= iters_g
