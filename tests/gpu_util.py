"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2510_23215_gb300 as scsf
    scsf.library()
    return torch.device("cuda", 0)


def to_dev(ops, dev):
    import paper_2510_23215_gb300 as scsf
    return [scsf.Operator.from_workload(o, dev) for o in ops]


def host(t):
    return t.detach().cpu().numpy()
