"""scsf_sort (Alg. 2) vs the oracle: permutation bit-exact away from oracle-flagged near-ties."""
import numpy as np
import pytest

import scsf_inputs as si
from oracle import sort as osort
from tests.gpu_util import host, need_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NEAR_TIE = 1e-10  # relative gap (second - best)/max ||F||^2 below which a step is a near-tie


def _check_perm(fields, p0, start, dev):
    import paper_2510_23215_gb300 as scsf
    perm = host(scsf.sort(torch.as_tensor(fields, device=dev), p0=p0, start=start))
    ref, gaps = osort.scsf_sort(fields, p0, start)
    ties = np.nonzero(gaps < NEAR_TIE)[0]
    upto = len(ref) if len(ties) == 0 else int(ties[0]) + 1
    assert perm[:upto].tolist() == ref[:upto].tolist()
    assert sorted(perm.tolist()) == list(range(len(ref)))
    return len(ties)


def test_sort_poisson128_full_size():
    """The 200-problem, 128 x 128, p0 = 8 workload."""
    dev = need_gpu()
    fields = np.stack([o.P for o in si.div_a_grad_chain(128, 200, seed=1)])
    assert _check_perm(fields, 8, 0, dev) == 0


def test_sort_lapv256_full_size():
    """The 1000-problem, 256 x 256, p0 = 8 potential workload."""
    dev = need_gpu()
    fields = np.stack([o.V for o in si.lap_plus_v_chain(256, 1000, seed=2)])
    assert _check_perm(fields, 8, 0, dev) == 0


@pytest.mark.parametrize("seed", range(6))
def test_sort_small_random_starts(seed):
    dev = need_gpu()
    rng = np.random.default_rng(seed)
    n_ops = int(rng.integers(1, 9))
    p = int(rng.integers(3, 40))
    p0 = int(rng.integers(1, p + 1))
    fields = rng.standard_normal((n_ops, p, p))
    _check_perm(fields, p0, int(rng.integers(0, n_ops)), dev)


def test_sort_ties_smallest_index_and_family():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    B = np.random.default_rng(8).standard_normal((6, 6))
    fields = np.stack([B, 2 * B, 2 * B, 2 * B, 2 * B])
    perm = host(scsf.sort(torch.as_tensor(fields, device=dev), p0=3, start=0))
    assert perm.tolist() == [0, 1, 2, 3, 4]
    t = np.array([0.7, 0.1, 2.5, 1.3, 0.4, 1.9, 3.3, 0.05])
    fam = np.stack([ti * B for ti in t])
    perm = host(scsf.sort(torch.as_tensor(fam, device=dev), p0=6, start=int(np.argmin(t))))
    assert t[perm].tolist() == sorted(t.tolist())


def test_sort_rejects_bad_arguments():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    f = torch.zeros((4, 8, 8), dtype=torch.float64, device=dev)
    with pytest.raises(scsf.ScsfError):
        scsf.sort(f, p0=9)
    with pytest.raises(scsf.ScsfError):
        scsf.sort(f, p0=2, start=4)
    with pytest.raises(ValueError):
        scsf.sort(f.cpu().cuda().transpose(1, 2), p0=2)


def test_sort_distances_match_oracle_features():
    """scsf_sort_dist: the permutation of scsf_sort and, per step, the squared distance of
    the oracle's truncated-DFT features between consecutive problems."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    ops = si.div_a_grad_chain(32, 40, seed=3)
    F = np.stack([o.P for o in ops])
    perm, dist = scsf.sort(torch.as_tensor(F, device=dev), p0=8, return_distances=True)
    perm, dist = host(perm), host(dist)
    assert np.array_equal(perm, host(scsf.sort(torch.as_tensor(F, device=dev), p0=8)))
    feats = osort.features(F, 8)
    ref = [0.0] + [osort.squared_distance(feats[perm[i - 1]], feats[perm[i]]) for i in range(1, 40)]
    np.testing.assert_allclose(dist, ref, rtol=1e-12, atol=0)
