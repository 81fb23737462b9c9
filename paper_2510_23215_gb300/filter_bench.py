"""Time the Chebyshev filter kernels alone (CUDA events on the launching stream).

A filter of degree m launches m stencil steps; the per-step device time is taken as
(t(m + 100) - t(m)) / 100, so operator assembly and the end passes cancel. Shapes:

* ``128x120``: one chain of the 128 x 128, k = 100 workload (N = 16384, k_b = 120);
  its three blocks fit in L2, so the rate is an effective one;
* ``256x480``: the 256 x 256, k = 400 block (N = 65536, k_b = 480, 3 x 126 MB in FP32),
  which streams every step through DRAM;
* ``--kernel plate``: the FP64 step on the thin-plate operator's 13-slot CSR form
  (e.g. ``100x120``: N = 10^4, k_b = 120; 24 B per node and column plus 156 B per node).

    python -m paper_2510_23215_gb300.filter_bench --kernel f32 --shape 256x480
    python -m paper_2510_23215_gb300.filter_bench --kernel dc --shape 128x120 --degree 3 --once
    python -m paper_2510_23215_gb300.filter_bench --kernel rot --shape 128x120
    python -m paper_2510_23215_gb300.filter_bench --kernel plate --shape 100x120 --once
    python -m paper_2510_23215_gb300.filter_bench --kernel gram --shape 128x120 --once

``--once`` runs one filter of the given degree (``gram``: one tensor-core Gram product X^T X,
8 digits, N = n^2 rows) and exits (a short command for profilers).
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import Context, Operator, assemble_bounds, cheb_filter, cheb_filter_dc, cheb_filter_f32

# algorithmic bytes per (node, column) per step: read Y_i and Y_{i-1}, write Y_{i+1}
# (FP32: 12 B); the defect-corrected step also reads the residual block (16 B)
BYTES_PER_ELEM = {"f32": 12.0, "dc": 16.0, "plate": 24.0}
# FP64 ALU rate of GB300 from unit counts and clocks: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def measure_rotation(shape: str, device, reps: int = 20) -> dict:
    """Y = X M with X FP64 [N, k_b] and M [k_b, k_b] (the rotation X = Q Z of Alg. 3), timed
    alone: CUDA events around `reps` launches."""
    from . import block_rotate_fp64 as block_rotate
    n, kb = (int(v) for v in shape.split("x"))
    g = torch.Generator(device="cpu").manual_seed(1)
    X = torch.randn((n * n, kb), generator=g, dtype=torch.float64).to(device)
    M = torch.randn((kb, kb), generator=g, dtype=torch.float64).to(device)
    ctx = Context(device.index or 0, torch.cuda.current_stream(device))
    st = torch.cuda.current_stream(device)
    block_rotate(X, M, ctx=ctx)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        block_rotate(X, M, ctx=ctx)
    e1.record(st)
    torch.cuda.synchronize(device)
    us = e0.elapsed_time(e1) / reps * 1e3
    flops = 2.0 * n * n * kb * kb
    return {"kernel": "rot", "shape": shape, "avg_us": us, "flops_per_launch": flops,
            "tflops": flops / (us * 1e-6) / 1e12, "peak_tflops": FP64_PEAK_TFLOPS}


def setup(kernel: str, shape: str, device, seed: int = 0):
    """(runner(degree), elements per step) for the kernel at the shape."""
    import scsf_inputs as si  # seeded operator generators (no method arithmetic)
    n, kb = (int(v) for v in shape.split("x"))
    if kernel == "plate":
        op = Operator.from_workload(si.plate_chain(n, 1, seed=6)[0], device)
        ctx = Context(device.index or 0, torch.cuda.current_stream(device))
        lo, hi = assemble_bounds(op, ctx)
        alpha = lo + 0.01 * (hi - lo)
        c, e = 0.5 * (alpha + hi), 0.5 * (hi - alpha)
        g = torch.Generator(device="cpu").manual_seed(seed)
        X = torch.randn((n * n, kb), generator=g, dtype=torch.float64).to(device)
        return (lambda d: cheb_filter(op, X, d, lo, c, e, ctx=ctx)), n * n * kb
    if n == 256:
        op = Operator.from_workload(si.lap_plus_v_chain(n, 1, seed=2)[0], device)
    else:
        op = Operator.from_workload(si.div_a_grad_chain(n, 1, seed=5)[0], device)
    ctx = Context(device.index or 0, torch.cuda.current_stream(device))
    lo, hi = assemble_bounds(op, ctx)
    lam, alpha = lo + 1e-3 * (hi - lo), lo + 2.0 * kb / (n * n) * (hi - lo)
    c, e = 0.5 * (alpha + hi), 0.5 * (hi - alpha)
    g = torch.Generator(device="cpu").manual_seed(seed)
    if kernel == "f32":
        X = torch.randn((n * n, kb), generator=g, dtype=torch.float32).to(device)
        return (lambda d: cheb_filter_f32(op, X, d, lam, c, e, ctx=ctx)), n * n * kb
    X = torch.randn((n * n, kb), generator=g, dtype=torch.float64).to(device)
    theta = torch.linspace(lam, alpha, kb, dtype=torch.float64, device=device)
    return (lambda d: cheb_filter_dc(op, X, theta, d, lam, c, e, ctx=ctx)), n * n * kb


def per_step_us(run, degree: int, device, reps: int = 3) -> float:
    st = torch.cuda.current_stream(device)
    times = []
    for deg in (degree, degree + 100):
        run(deg)
        torch.cuda.synchronize(device)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(reps):
            run(deg)
        e1.record(st)
        torch.cuda.synchronize(device)
        times.append(e0.elapsed_time(e1) / reps)
    return (times[1] - times[0]) / 100 * 1e3


def measure(kernel: str, shape: str, device, degree: int = 20) -> dict:
    run, elems = setup(kernel, shape, device)
    us = per_step_us(run, degree, device)
    kb = int(shape.split("x")[1])
    nbytes = BYTES_PER_ELEM[kernel] * elems + (156.0 * elems / kb if kernel == "plate" else 0.0)
    return {"kernel": kernel, "shape": shape, "avg_us": us, "bytes_per_launch": nbytes,
            "gbs": nbytes / (us * 1e-6) / 1e9}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--kernel", choices=["f32", "dc", "rot", "plate", "gram"], default="f32")
    ap.add_argument("--shape", default="128x120")
    ap.add_argument("--degree", type=int, default=20)
    ap.add_argument("--once", action="store_true")
    a = ap.parse_args()
    dev = torch.device("cuda", 0)
    if a.kernel == "rot":
        print(json.dumps(measure_rotation(a.shape, dev)))
        return
    if a.kernel == "gram":
        from . import block_gram, block_gram_kernel_time
        n, kb = (int(v) for v in a.shape.split("x"))
        g = torch.Generator(device="cpu").manual_seed(2)
        X = torch.randn((n * n, kb), generator=g, dtype=torch.float64).to(dev)
        if a.once:
            block_gram(X, symmetric=True)
            torch.cuda.synchronize(dev)
            print("ok")
            return
        ms = block_gram_kernel_time(X, reps=20)
        flops = 36 * 2.0 * n * n * kb * kb
        print(json.dumps({"kernel": "gram", "shape": a.shape, "avg_us": ms * 1e3,
                          "bf16_tflops": flops / (ms * 1e-3) / 1e12}))
        return
    if a.once:
        run, _ = setup(a.kernel, a.shape, dev)
        run(a.degree)
        torch.cuda.synchronize(dev)
        print("ok")
        return
    r = measure(a.kernel, a.shape, dev, a.degree)
    print(json.dumps(r))


if __name__ == "__main__":
    np.set_printoptions(precision=4)
    main()
