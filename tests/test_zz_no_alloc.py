"""scsf_sort_noalloc: the sort for callers that cannot allocate device memory.

Such callers (a host framework that hands out every byte of device memory from
its own fixed pool, or a latency-critical loop that must not enter the
allocator) pass only inputs and outputs; the scratch comes from a static device
array inside the library. This file is collected last on purpose, so a failure
here cannot hide the other tests. It must pass alone in a fresh process and
after everything else.
"""
import ctypes

import numpy as np
import pytest

import scsf_inputs as si
from oracle import sort as osort
from tests.gpu_util import host, need_gpu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _noalloc(ctx, fields, p0, start):
    import paper_2510_23215_gb300 as scsf
    n_ops, p = int(fields.shape[0]), int(fields.shape[1])
    perm = torch.full((n_ops,), -1, dtype=torch.int32, device=fields.device)
    st = scsf.library().scsf_sort_noalloc(ctx.handle, ctypes.c_void_p(fields.data_ptr()), n_ops, p,
                                          p0, start, ctypes.c_void_p(perm.data_ptr()))
    torch.cuda.synchronize()
    return st, perm


def test_noalloc_sort_matches_workspace_sort_on_two_calls_in_a_row():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    ctx = scsf.Context(0)
    # first call: the 200-problem 128 x 128 batch; second call: a smaller, different batch,
    # so stale scratch contents from the first call would show up as a wrong order
    batches = [
        (np.stack([o.P for o in si.div_a_grad_chain(128, 200, seed=1)]), 8, 0),
        (np.stack([o.V for o in si.lap_plus_v_chain(64, 37, seed=5)]), 6, 11),
    ]
    for fields_np, p0, start in batches:
        fields = torch.as_tensor(fields_np, device=dev)
        ref = host(scsf.sort(fields, p0=p0, start=start, ctx=ctx))
        st, perm = _noalloc(ctx, fields, p0, start)
        assert st == scsf.OK, scsf.library().scsf_last_error(ctx.handle)
        assert host(perm).tolist() == ref.tolist()
        # and directly against the CPU oracle's greedy chain (Alg. 2)
        oracle_perm, _ = osort.scsf_sort(fields_np, p0, start)
        assert host(perm).tolist() == list(oracle_perm)
    ctx.close()


def test_noalloc_sort_allocates_nothing():
    """A warmed-up call changes neither torch's reserved pool nor the device's free memory."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    ctx = scsf.Context(0)
    fields = torch.as_tensor(np.stack([o.P for o in si.div_a_grad_chain(64, 50, seed=3)]), device=dev)
    perm = torch.empty(50, dtype=torch.int32, device=dev)
    L = scsf.library()
    args = (ctx.handle, ctypes.c_void_p(fields.data_ptr()), 50, 64, 8, 0, ctypes.c_void_p(perm.data_ptr()))
    assert L.scsf_sort_noalloc(*args) == scsf.OK  # warm: kernels loaded
    torch.cuda.synchronize()
    reserved, (free0, _) = torch.cuda.memory_reserved(dev), torch.cuda.mem_get_info(dev)
    for _ in range(3):
        assert L.scsf_sort_noalloc(*args) == scsf.OK
    torch.cuda.synchronize()
    assert torch.cuda.memory_reserved(dev) == reserved
    assert torch.cuda.mem_get_info(dev)[0] == free0
    ctx.close()


def test_noalloc_sort_checks_arguments_before_capacity():
    """Calls scsf_sort would reject get SCSF_ERR_INVALID_ARG here too, not the capacity error."""
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    ctx = scsf.Context(0)
    for n_ops, p, p0 in ((70000, 8, 8), (16, 8, 12), (16, 100, 70)):
        fields = torch.zeros((n_ops, p, p), dtype=torch.float64, device=dev)
        st, _ = _noalloc(ctx, fields, p0, 0)
        assert st == scsf.ERR_INVALID_ARG, (n_ops, p, p0, st)
    ctx.close()


def test_noalloc_sort_rejects_sizes_beyond_its_static_scratch():
    dev = need_gpu()
    import paper_2510_23215_gb300 as scsf
    L = scsf.library()
    cap = L.scsf_sort_noalloc_capacity()
    assert cap == 8 << 20
    ctx = scsf.Context(0)
    n_ops = 8185  # one past the largest batch that fits at p0 = 8
    assert L.scsf_sort_workspace_size(n_ops, 8) > cap >= L.scsf_sort_workspace_size(8184, 8)
    fields = torch.zeros((n_ops, 8, 8), dtype=torch.float64, device=dev)
    st, perm = _noalloc(ctx, fields, 8, 0)
    assert st == scsf.ERR_NO_MEMORY
    assert b"static scratch" in L.scsf_last_error(ctx.handle)
    assert int(perm[0]) == -1  # nothing was written
    ctx.close()
