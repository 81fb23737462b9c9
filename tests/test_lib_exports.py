"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every declared symbol."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    with open(os.path.join(ROOT, "include", "scsf.h")) as f:
        text = f.read()
    for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(scsf_\w+)\s*\(", text, re.M):
        names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("scsf_sort", "scsf_solve", "scsf_chain_step", "scsf_create"):
        assert required in names


def test_library_loads_and_exports_every_symbol():
    import __graft_entry__
    __graft_entry__.build()
    import ctypes
    import paper_2510_23215_gb300 as scsf
    lib = ctypes.CDLL(scsf.lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(scsf.EXPORTED_SYMBOLS) <= declared_functions()
    L = scsf.library()
    assert L.scsf_version() >= 100
    assert L.scsf_max_block_width() == 512


def test_workspace_queries_without_gpu():
    import ctypes
    import paper_2510_23215_gb300 as scsf
    L = scsf.library()
    p = scsf.Params(k=100, degree=20)._c()
    ws = L.scsf_solve_workspace_size(ctypes.byref(p), 128)
    assert ws >= 4 * 128 * 128 * 120 * 8
    wide = scsf.Params(k=400)._c()  # k_b = 480: the wide-block path
    assert L.scsf_solve_workspace_size(ctypes.byref(wide), 256) >= 4 * 256 * 256 * 480 * 8
    too_big = scsf.Params(k=430)._c()  # k_b = 516 > 512
    assert L.scsf_solve_workspace_size(ctypes.byref(too_big), 128) == 0
    assert L.scsf_sort_workspace_size(200, 8) >= 200 * 8 * 8 * 16
    # FP64 stencil chains also hold the thin plate's 13-slot CSR form (4 N + 156 N bytes)
    ws_f64 = L.scsf_solve_workspace_size(ctypes.byref(p), 128)
    mixed = scsf.Params(k=100, degree=20, precision=scsf.MIXED)._c()
    assert ws_f64 >= 4 * 128 * 128 * 120 * 8 + 160 * 128 * 128
    assert L.scsf_solve_workspace_size(ctypes.byref(mixed), 128) > 0
    # CSR chains: FP64 only, sized by rows, no stencil-side plate buffers
    rows = L.scsf_solve_workspace_size_rows(ctypes.byref(p), 128 * 128)
    assert 4 * 128 * 128 * 120 * 8 <= rows < ws_f64
    assert L.scsf_solve_workspace_size_rows(ctypes.byref(mixed), 128 * 128) == 0
    assert L.scsf_solve_workspace_size_rows(ctypes.byref(p), 0) == 0
    assert L.scsf_solve_workspace_size_rows(ctypes.byref(p), 1 << 31) == 0
    # Cholesky QR2 building block: 1 <= ncols <= min(rows, 512)
    assert L.scsf_cholqr2_scratch(5000, 120) >= 5000 * 120 * 8 + 3 * 120 * 120 * 8
    assert L.scsf_cholqr2_scratch(3001, 200) > L.scsf_cholqr2_scratch(3001, 160)
    assert L.scsf_cholqr2_scratch(100, 101) == 0
    assert L.scsf_cholqr2_scratch(1000, 513) == 0


def test_context_creation_fails_loudly_without_gpu():
    import torch
    import paper_2510_23215_gb300 as scsf
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        scsf.Context(0)


def test_operator_descriptors_refuse_host_tensors_and_bad_shapes():
    """Every operator kind's descriptor is built from CUDA tensors only (no CPU path), and
    the binding checks shapes and dtypes before any call."""
    import torch
    import paper_2510_23215_gb300 as scsf
    import scsf_inputs as si
    csr = scsf.Operator.csr([0, 1, 2], [0, 1], [1.0, 2.0], device="cpu")
    assert csr.N == 2 and csr.row_ptr.dtype == torch.int32
    with pytest.raises(ValueError, match="CUDA"):
        csr._c()
    plate = scsf.Operator.from_workload(si.constant_plate(4), "cpu")
    assert plate.kind == scsf.PLATE and plate.N == 16
    with pytest.raises(ValueError, match="CUDA"):
        plate._c()
    stencil = scsf.Operator.from_workload(si.constant_div_a_grad(4), "cpu")
    with pytest.raises(ValueError, match="CUDA"):
        stencil._c()
    bad = scsf.Operator(scsf.PLATE, 4, D=torch.zeros((4, 4), dtype=torch.float32),
                        rho=torch.ones((4, 4), dtype=torch.float64))
    with pytest.raises(TypeError):
        bad._c()
    with pytest.raises(ValueError):
        scsf.Operator(99, 4)._c()


def test_far_steps_rule_matches_numpy_quantile():
    """scsf_far_steps (host code): the head and the steps above the quantile of the step
    distances (numpy's default linear interpolation) restart from the proposal."""
    import numpy as np
    import paper_2510_23215_gb300 as scsf
    rng = np.random.default_rng(4)
    for n, q in ((21, 0.9), (2, 0.9), (57, 0.5), (10, 1.0), (10, 0.0)):
        d = np.concatenate([[0.0], rng.exponential(size=n - 1)])
        far = scsf.far_steps(d, q)
        thr = np.quantile(d[1:], q)
        assert far[0] and far[1:] == [bool(x > thr) for x in d[1:]]
    assert scsf.far_steps([0.0], 0.9) == [True]
    with pytest.raises(scsf.ScsfError):
        scsf.far_steps([0.0, 1.0], 1.5)
