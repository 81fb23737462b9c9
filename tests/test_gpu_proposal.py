"""Learned head proposal: forward/gradient parity with the CPU FP64 oracle, training,
target preparation, prolongation."""
import numpy as np
import pytest

import scsf_inputs as si
from oracle import proposal as oprop
from tests.gpu_util import host, need_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fields(B, n=64, seed=0):
    return np.stack([o.P for o in si.div_a_grad_chain(n, B, seed=seed)])


def _targets(B, seed=0):
    rng = np.random.default_rng(seed)
    Q = np.stack([np.linalg.qr(rng.standard_normal((1024, 64)))[0] for _ in range(B)])
    t = rng.standard_normal((B, 2)) + np.array([3.0, 6.0])
    return t, Q


def _oracle_params(prop):
    """GPU master parameters with the matrices rounded to BF16, as the GPU uses them."""
    p = host(prop.params).astype(np.float64)
    mask = oprop.matrix_mask()
    p[mask] = oprop.bf16_round(p[mask])
    return p


def test_param_layout_matches_oracle():
    need_gpu()
    import paper_2510_23215_gb300 as scsf
    assert scsf.library().scsf_proposal_param_count() == oprop.COUNT


def test_forward_matches_oracle():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    prop = scsf.Proposal(seed=3, device=dev)
    F = _fields(3, n=64, seed=1)
    bounds, block = prop.forward(torch.as_tensor(F, device=dev))
    s_ref, Y_ref = oprop.forward(_oracle_params(prop), F)
    np.testing.assert_allclose(host(bounds), s_ref, rtol=2e-4, atol=2e-4 * np.abs(s_ref).max())
    err = np.abs(host(block) - Y_ref).max() / np.abs(Y_ref).max()
    assert err < 2e-4


def test_gradient_matches_oracle_finite_differences():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    prop = scsf.Proposal(seed=5, device=dev)
    B = 2
    F = _fields(B, n=64, seed=2)
    t, Q = _targets(B, seed=2)
    (l1, l2, l3), grad = prop.gradient(torch.as_tensor(F, device=dev),
                                       torch.as_tensor(t, dtype=torch.float32, device=dev),
                                       torch.as_tensor(Q, dtype=torch.float32, device=dev))
    p0 = _oracle_params(prop)
    ref = oprop.loss(p0, F, t, Q)
    np.testing.assert_allclose([l1, l2, l3], ref, rtol=1e-3)
    g = host(grad).astype(np.float64)
    rng = np.random.default_rng(0)
    # the largest gradient entries of every parameter block, plus random ones
    picks = []
    for name, (a, n) in oprop.OFFSETS.items():
        blk = np.abs(g[a:a + n])
        picks.append(a + int(np.argmax(blk)))
        picks.append(a + int(rng.integers(0, n)))
    total = lambda p: oprop.objective(p, F, t, Q)  # noqa: E731
    checked = 0
    for idx in picks:
        if abs(g[idx]) < 1e-3 * np.abs(g).max():
            continue
        h = 1e-3 * max(abs(p0[idx]), 1e-2)
        pp, pm = p0.copy(), p0.copy()
        pp[idx] += h
        pm[idx] -= h
        fd = (total(pp) - total(pm)) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-2 * abs(fd) + 1e-6 * np.abs(g).max(), (idx, fd, g[idx])
        checked += 1
    assert checked >= 10


def test_training_reduces_loss():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    prop = scsf.Proposal(seed=7, device=dev)
    B = 8
    F = torch.as_tensor(_fields(B, n=64, seed=4), device=dev)
    t, Q = _targets(B, seed=4)
    t = torch.as_tensor(t, dtype=torch.float32, device=dev)
    Q = torch.as_tensor(Q, dtype=torch.float32, device=dev)
    obj = lambda ls: ls[0] + oprop.MU * ls[1] + ls[2]  # noqa: E731
    first = obj(prop.train_step(F, t, Q, lr=1e-3))
    for _ in range(150):
        last = obj(prop.train_step(F, t, Q, lr=1e-3))
    assert last < 0.5 * first


def test_targets_are_orthonormal_pooled_eigenvectors():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    prop = scsf.Proposal(seed=1, device=dev)
    n = 64
    rng = np.random.default_rng(3)
    ev = rng.standard_normal((2, n * n, 70))
    Q = host(prop.targets(torch.as_tensor(ev, device=dev), n)).astype(np.float64)
    for b in range(2):
        pooled = ev[b, :, :64].reshape(32, 2, 32, 2, 64).sum(axis=(1, 3)).reshape(1024, 64)
        np.testing.assert_allclose(Q[b].T @ Q[b], np.eye(64), atol=1e-5)
        # same span: projecting the pooled vectors onto Q loses nothing
        resid = pooled - Q[b] @ (Q[b].T @ pooled)
        assert np.abs(resid).max() <= 1e-5 * np.abs(pooled).max()


def test_prolongation_reproduces_bilinear_functions_inside():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    ctx = scsf.Context(0)
    n, f = 128, 4
    I, J = np.meshgrid(np.arange(32), np.arange(32), indexing="ij")
    # coarse node (I, J) sits at fine index f I + (f - 1)/2
    xi, xj = f * I + 1.5, f * J + 1.5
    coarse = np.stack([0.3 * xi + 0.7 * xj + 0.01 * xi * xj + c for c in range(64)], axis=-1)
    block = torch.as_tensor(coarse.reshape(1, 1024, 64), dtype=torch.float32, device=dev)
    fine = torch.zeros((n * n, 64), dtype=torch.float64, device=dev)
    ctx.check(scsf.library().scsf_proposal_prolong(ctx.handle, block.data_ptr(), 1, n,
                                                   fine.data_ptr(), 64))
    got = host(fine).reshape(n, n, 64)
    fi, fj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    inside = (fi >= 2) & (fi <= n - 3) & (fj >= 2) & (fj <= n - 3)
    for c in (0, 17, 63):
        ref = 0.3 * fi + 0.7 * fj + 0.01 * fi * fj + c
        np.testing.assert_allclose(got[..., c][inside], ref[inside], rtol=2e-6, atol=2e-5)


def test_trained_proposal_gain_on_heldout_heads():
    """Train on 320 plain solves (64 x 64 grids, labels: the 64 lowest eigenpairs), then solve
    16 held-out operators as chain heads for k = 53 (block width 64, every column from the
    proposal; the library composes the head block) from the Gaussian block and from the
    proposal. The network must have learned the subspace (held-out sum of squared
    principal-angle sines far below the 64 of an unrelated block) and the bounds, both starts
    must reach the tolerance, and the proposal must take fewer filter iterations."""
    dev = need_gpu()
    from paper_2510_23215_gb300 import proposal_train
    r = proposal_train.run(n=64, n_train=320, n_test=16, steps=800, degree=20, lr=1e-3, seed=77,
                           device=dev, k_eval=53)
    print("proposal gain:", {k: r[k] for k in ("heldout_loss", "mean_iters_random", "mean_iters_proposal")})
    sub, _, bounds = r["heldout_loss"]
    assert sub < 6.4
    assert bounds < 0.02
    assert r["resid_random"] <= 1e-8 and r["resid_proposal"] <= 1e-8
    assert r["mean_iters_proposal"] < r["mean_iters_random"]


def test_chain_seeds_head_and_far_steps_from_the_proposal():
    """The far-step rule: the head and the steps whose sort distance is above the 90th
    percentile start from the proposal block; every problem still meets the tolerance."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    from paper_2510_23215_gb300 import proposal_train
    ops = si.div_a_grad_chain(64, 21, seed=9)
    prop = scsf.Proposal(seed=2, device=dev)
    params = scsf.Params(k=64, degree=20, tol=1e-8, max_iter=200)
    perm, seeded, out = proposal_train.solve_chain_with_proposal(ops, prop, params, dev)
    assert sorted(perm) == list(range(21))
    # 20 step distances, 90th percentile: the two largest are above it
    assert seeded[0] == 0 and len(seeded) == 3
    _, dist = scsf.sort(torch.as_tensor(np.stack([o.P for o in ops]), device=dev), p0=8,
                        return_distances=True)
    d = host(dist)
    assert d[0] == 0.0
    assert set(seeded[1:]) == set(int(i) + 1 for i in np.argsort(d[1:])[-2:])
    for ev, rs, st in out:
        assert float(rs.max()) <= 1e-8 and st["converged"]
