"""Batched solve (many chains in flight) against sequential solves and the oracle."""
import numpy as np
import pytest

import scsf_inputs as si
from oracle import compare, dense, operators
from tests.gpu_util import host, need_gpu, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _chains(dev, precision, specs):
    import paper_2510_23215_gb300 as scsf
    chains, raw = [], []
    for n, k, n_ops, seed in specs:
        ops = si.div_a_grad_chain(n, n_ops, seed=seed)
        raw.append(ops)
        chains.append((to_dev(ops, dev), scsf.Params(k=k, degree=16, tol=1e-8, seed=seed,
                                                     precision=precision)))
    return chains, raw


# uneven grids and block widths (k + ceil(0.2 k) divisible by 4 for the mixed form)
SPECS = [(40, 20, 3, 11), (24, 10, 4, 12), (32, 30, 2, 13), (28, 16, 3, 14), (36, 40, 2, 15)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_equals_sequential_exactly(precision):
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    prec = scsf.FP64 if precision == "fp64" else scsf.MIXED
    chains, raw = _chains(dev, prec, SPECS)
    batched = scsf.solve_batched(chains, concurrency=4, want_vectors=True)
    for (ops, params), (ev, rs, vec, stats, status) in zip(chains, batched):
        assert status == scsf.OK
        ev_s, rs_s, vec_s, _ = scsf.solve(ops, params, want_vectors=True)
        # same kernels on another stream: bit-identical
        assert torch.equal(ev, ev_s) and torch.equal(rs, rs_s) and torch.equal(vec, vec_s)
    # the oracle's definition on one problem of each chain
    for (ops, params), (ev, rs, vec, _, _), r in zip(chains, batched, raw):
        w, V = dense.smallest_eigenpairs(operators.assemble(r[-1]), params.k)
        assert compare.max_rel_eig_error(w, host(ev)[-1]) <= 1e-10
        assert float(rs.max()) <= 1e-8
        assert compare.max_cluster_angle(w, V, host(vec)[-1]) <= 1e-5


def test_batched_concurrency_does_not_change_results():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    chains, _ = _chains(dev, scsf.FP64, SPECS[:3])
    a = scsf.solve_batched(chains, concurrency=1)
    b = scsf.solve_batched(chains, concurrency=3)
    for x, y in zip(a, b):
        assert torch.equal(x[0], y[0]) and torch.equal(x[1], y[1])


def test_batched_rejects_unsupported_chain():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    chains, _ = _chains(dev, scsf.FP64, SPECS[:2])
    chains.append((chains[0][0], scsf.Params(k=430)))  # block width 516 over the limit
    with pytest.raises(ValueError):
        scsf.solve_batched(chains, concurrency=2)
