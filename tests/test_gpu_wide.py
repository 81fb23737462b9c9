"""Wide blocks (k_b > 160): the global-memory reduced eigensolve and blocked Cholesky, and
solves at k = 200, 256 and 400 (the 256 x 256, k_b = 480 shape) against exact spectra of
separable operators."""
import numpy as np
import pytest

import scsf_inputs as si
from oracle import compare, operators, sturm
from tests.gpu_util import host, need_gpu, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RES_TOL = 1e-8
EIG_RTOL = 1e-10


@pytest.mark.parametrize("k", [161, 240, 480])
def test_small_eigh_wide_random(k):
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    rng = np.random.default_rng(k)
    S = rng.standard_normal((k, k))
    S = S + S.T
    w, Z = scsf.small_eigh(torch.as_tensor(S, device=dev))
    w, Z = host(w), host(Z)
    ref = np.linalg.eigvalsh(S)
    nrm = np.max(np.abs(ref))
    assert np.max(np.abs(w - ref)) <= 1e-12 * nrm
    assert np.max(np.abs(S @ Z - Z * w)) <= 1e-11 * nrm
    assert np.max(np.abs(Z.T @ Z - np.eye(k))) <= 1e-12


def test_small_eigh_wide_near_diagonal_with_cluster():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    k = 300
    rng = np.random.default_rng(1)
    d = np.sort(rng.uniform(1, 1000, k))
    d[10] = d[11] * (1 + 1e-9)  # a near-degenerate pair
    E = 1e-3 * rng.standard_normal((k, k))
    S = np.diag(d) + E + E.T
    w, Z = scsf.small_eigh(torch.as_tensor(S, device=dev))
    w, Z = host(w), host(Z)
    ref = np.linalg.eigvalsh(S)
    assert np.max(np.abs(w - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(Z.T @ Z - np.eye(k))) <= 1e-12


def _check(op, ev, rs, vec, ref):
    A = operators.assemble(op)
    assert np.max(rs) <= RES_TOL
    assert np.max(operators.relative_residuals(A, vec, ev)) <= 1.05 * RES_TOL
    assert compare.orthonormality_error(vec) <= 1e-12
    assert compare.max_rel_eig_error(ref, ev) <= EIG_RTOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_separable_k200(precision):
    """a = a(x) on 64 x 64, k = 200 (k_b = 240): every eigenvalue against Sturm bisection."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    n, k = 64, 200
    ops = [si.separable_div_a_grad(n, seed=s) for s in (21, 22)]
    prec = scsf.FP64 if precision == "fp64" else scsf.MIXED
    params = scsf.Params(k=k, degree=20, degree_fp32=40, tol=RES_TOL, precision=prec)
    ev, rs, vec, stats = scsf.solve(to_dev(ops, dev), params, want_vectors=True)
    ev, rs, vec = host(ev), host(rs), host(vec)
    for j, op in enumerate(ops):
        ref = sturm.separable_smallest_fast(n, op.ax[:, 0], op.P[:, 0], k)
        _check(op, ev[j], rs[j], vec[j], ref)
    assert all(s["converged"] for s in stats)


def test_separable_potential_256_k400_mixed():
    """The 256 x 256, k = 400 shape (k_b = 480) in the mixed form, on a separable potential
    V = 10 (g1(x) + g2(y)) whose spectrum is the sums of two 1-D spectra."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    n, k = 256, 400
    op = si.separable_lap_plus_v(n, seed=2)
    params = scsf.Params(k=k, degree=60, degree_fp32=60, tol=RES_TOL, precision=scsf.MIXED)
    ev, rs, _, stats = scsf.solve(to_dev([op], dev), params, want_vectors=False)
    ref = sturm.separable_lap_plus_v_smallest(n, op.V, k, m=60)
    assert np.max(host(rs)) <= RES_TOL
    assert compare.max_rel_eig_error(ref, host(ev)[0]) <= EIG_RTOL
    assert stats[0]["converged"]


def test_batched_uneven_wide_chains_match_sequential():
    """Chains of uneven grids and k up to 256 (k_b up to 308) in flight together give the same
    bits as each chain alone, and every pair meets the tolerance."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    specs = [(48, 150, 2, 31), (40, 20, 3, 32), (56, 256, 1, 33), (64, 60, 2, 34)]
    chains = []
    for n, k, n_ops, seed in specs:
        ops = to_dev(si.div_a_grad_chain(n, n_ops, seed=seed), dev)
        chains.append((ops, scsf.Params(k=k, degree=40, degree_fp32=40, tol=RES_TOL,
                                        precision=scsf.MIXED, seed=seed)))
    res = scsf.solve_batched(chains, concurrency=4)
    for (ops, params), (ev, rs, _, _, status) in zip(chains, res):
        assert status == 0
        assert float(rs.max()) <= RES_TOL
        ev1, rs1, _, _ = scsf.solve(ops, params)
        assert torch.equal(ev, ev1) and torch.equal(rs, rs1)
