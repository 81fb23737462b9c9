"""Benchmark: eigenpairs/s of the SCSF hot path (truncated-FFT sort + warm-started
Chebyshev filtered subspace iteration) on GB300, at relative residual <= 1e-8.

One step = the whole path over one batch: sort 200 synthetic -div(a grad u)
operators on a 128 x 128 grid (p0 = 8), then solve them in sorted order, each problem
warm-started from its predecessor, for the k = 100 smallest eigenpairs (tol 1e-8). The timed
form is the mixed one (FP32 phase, then FP64 phase with the defect-corrected filter; block
products on the tensor cores), with the sorted sequence cut into 8 chains solved
concurrently, each chain head started from the learned proposal (trained before timing). Beside it: the plain FP64 form at its own best degree and the same 8 chains
(the tuned comparison), and the paper's form as written (degree 20, one sequential chain).
Each rank runs its own batch (weak scaling, no data-path collective).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

BOUNDS = {"gershgorin": 0, "lanczos": 1}  # scsf_bound values
ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import scsf_inputs as si  # noqa: E402

METRIC = "eigenpairs/s at rel. residual <=1e-8 (SCSF sort + warm-started ChFSI chain)"
UNIT = "eigenpairs/s"
WORKLOAD = dict(name="poisson128_k100", n=128, n_ops=200, k=100, degree=20, p0=8, tol=1e-8, seed=1)
L2_FLUSH_BYTES = 512 << 20
# algorithmic bytes per (node, column) per filter step: read Y_i and Y_{i-1}, write Y_{i+1}
# (FP64: 24 B, FP32: 12 B); the defect-corrected step also reads the residual block (16 B)
BYTES_PER_ELEM = {"cheb_step_f64": 24.0, "cheb_step_f32": 12.0, "cheb_step_dc": 16.0}
# dram__bytes_read.sum + dram__bytes_write.sum per launch from one earlier ncu capture of each
# kernel at the named shape (copied, not measured in this run); absent where not captured
TRAFFIC_SOURCE = "one ncu capture of the kernel (dram__bytes_read.sum + dram__bytes_write.sum)"
TRAFFIC_PER_LAUNCH = {"cheb_step_f32_256x256_kb480": 353.1e6, "strip_filter_f32_128x120": 8.08e6,
                      "oz_gemm_gram_16384x120": 33.66e6}
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz


def isolated_filter_rates(degree: int, dev):
    """Per-step device time of each filter kernel launched alone on the launching stream
    (paper_2510_23215_gb300.filter_bench): at one chain of the workload (N = 16384,
    kb = 120) and, for the FP32 step, at N = 65536, kb = 480, whose blocks exceed L2."""
    from paper_2510_23215_gb300 import filter_bench as fb
    out = {}
    for name, kern in (("cheb_step_f32", "f32"), ("cheb_step_dc", "dc")):
        r = fb.measure(kern, "128x120", dev, max(degree, 20))
        out[name] = {"avg_us_alone": r["avg_us"], "shape_alone": "N = 16384, kb = 120"}
    r = fb.measure("f32", "256x480", dev, 20)
    out["cheb_step_f32_256x256_kb480"] = {"avg_us_alone": r["avg_us"],
                                           "bytes_per_launch": r["bytes_per_launch"]}
    return out


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_time_pairs(ms: float, pairs: float, world_size: int, device):
    """Whole-job figures over the ranks: the slowest rank's time and the sum of the pairs."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    p = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    if world_size > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t[0]), float(p[0])


def _workload_ops(rank: int):
    w = WORKLOAD
    return si.div_a_grad_chain(w["n"], w["n_ops"], seed=w["seed"] + 1000 * rank)


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while active."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# --------------------------------------------------------------------------- ours
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2510_23215_gb300 as scsf

    ws, rank, local = _dist()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the SCSF library has no CPU path)")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    scsf.library()  # fails loudly when the extension is missing
    w = WORKLOAD
    n, k, n_ops = w["n"], w["k"], w["n_ops"]
    forms = {"mixed": scsf.MIXED, "fp64": scsf.FP64}
    chosen = args.form
    ops = _workload_ops(rank)
    prop, proposal_leg = None, None
    if not args.no_proposal:
        prop, proposal_leg = leg_learned_proposal(args, rank, dev)
    # host copies (pinned) for the end-to-end leg; device copies resident for the kernel leg
    h_fields = torch.from_numpy(np.stack([o.P for o in ops])).pin_memory()
    h_ax = torch.from_numpy(np.stack([o.ax for o in ops])).pin_memory()
    h_ay = torch.from_numpy(np.stack([o.ay for o in ops])).pin_memory()
    d_fields, d_ax, d_ay = h_fields.to(dev), h_ax.to(dev), h_ay.to(dev)
    ctx = scsf.Context(local, torch.cuda.current_stream(dev))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    h_evals = torch.empty((n_ops, k), dtype=torch.float64).pin_memory()
    h_resid = torch.empty((n_ops, k), dtype=torch.float64).pin_memory()
    st = torch.cuda.current_stream(dev)

    def step(fields, ax, ay, precision, chunks=1, degree=None):
        if precision == scsf.MIXED:  # the chosen form: tuned degrees, proposal at chain heads
            params = scsf.Params(k=k, degree=args.degree_fp64, degree_fp32=args.degree_fp32,
                                 tol=w["tol"], seed=7 + rank, precision=precision,
                                 switch_tol=args.switch_tol, proposal=prop,
                                 column_degree=bool(args.column_degree), bound=BOUNDS[args.bound])
        else:                        # the plain form: its own degree (default: the workload's)
            params = scsf.Params(k=k, degree=degree or w["degree"], tol=w["tol"], seed=7 + rank,
                                 precision=precision)
        perm = scsf.sort(fields, p0=w["p0"], start=0, ctx=ctx).cpu().tolist()
        dops = [scsf.Operator(scsf.DIV_A_GRAD, n, ax=ax[i], ay=ay[i], field=fields[i]) for i in perm]
        if chunks <= 1:
            ev, rs, _, stats = scsf.solve(dops, params, ctx=ctx)
            return ev, rs, stats
        # App. D.6: contiguous chunks of the sorted sequence, one chain each, all in flight
        bounds = np.linspace(0, len(dops), chunks + 1).round().astype(int)
        chains = [(dops[a:b], params) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        res = scsf.solve_batched(chains, concurrency=args.concurrency or len(chains), ctx=ctx)
        ev = torch.cat([r[0] for r in res])
        rs = torch.cat([r[1] for r in res])
        stats = [s for r in res for s in r[3]]
        return ev, rs, stats

    def barrier():
        torch.cuda.synchronize(dev)
        if ws > 1:
            dist.barrier()

    def timed(precision, steps, warmup, sample_clocks=False, chunks=1, phase_timing=False,
              degree=None):
        for _ in range(warmup):
            step(d_fields, d_ax, d_ay, precision, chunks, degree)
        barrier()
        ctx.set_timing(phase_timing)
        times, all_stats, good = [], [], 0
        last_ev, max_res = None, 0.0
        launches0 = scsf.launch_count()
        clk = ClockSampler(local) if sample_clocks else None
        if clk:
            clk.__enter__()
        for _ in range(steps):
            flush.zero_()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ev, rs, stats = step(d_fields, d_ax, d_ay, precision, chunks, degree)
            e1.record(st)
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1))
            all_stats.extend(stats)
            good += int((rs <= w["tol"]).sum().item())
            max_res = max(max_res, float(rs.max().item()))
            last_ev = ev
        if clk:
            clk.__exit__(None, None, None)
        ctx.set_timing(False)
        return {"ms": sum(times), "stats": all_stats, "pairs": good, "max_resid": max_res,
                "last_ev": last_ev, "launches": scsf.launch_count() - launches0,
                "clocks": clk.summary() if clk else None}

    def reduce_max_sum(ms, pairs):
        return reduce_time_pairs(ms, pairs, ws, dev)

    main = timed(forms[chosen], args.steps, args.warmup, sample_clocks=True, chunks=args.chunks)
    total_ms, pairs = reduce_max_sum(main["ms"], main["pairs"])
    value = pairs / (total_ms * 1e-3)
    # one more step with per-phase CUDA events (they add host syncs, so the timed steps above
    # run without them): the phase split and the in-step kernel times come from this step
    instrumented = timed(forms[chosen], 1, 0, chunks=args.chunks, phase_timing=True)

    # end to end through the public API with host buffers (chosen form)
    e2e_ms = 0.0
    h2d = (h_fields.numel() + h_ax.numel() + h_ay.numel()) * 8
    d2h = 2 * n_ops * k * 8
    e2e_pairs = 0
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        f = h_fields.to(dev, non_blocking=True)
        a = h_ax.to(dev, non_blocking=True)
        b = h_ay.to(dev, non_blocking=True)
        ev, rs, _ = step(f, a, b, forms[chosen], args.chunks)
        h_evals.copy_(ev, non_blocking=True)
        h_resid.copy_(rs, non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize(dev)
        e2e_ms += e0.elapsed_time(e1)
        e2e_pairs += int((h_resid <= w["tol"]).sum().item())
    e2e_ms, e2e_pairs = reduce_max_sum(e2e_ms, e2e_pairs)
    e2e_value = e2e_pairs / (e2e_ms * 1e-3)

    other, paper_form = None, None
    if not args.no_plain and chosen != "fp64":
        # the tuned comparison: plain FP64 at its best degree, same chains in flight
        plain = timed(forms["fp64"], args.plain_steps, 1, chunks=args.plain_chunks,
                      degree=args.plain_degree)
        p_ms, p_pairs = reduce_max_sum(plain["ms"], plain["pairs"])
        other = {"form": f"plain FP64 (Alg. 3 in FP64), degree {args.plain_degree}, "
                         f"{args.plain_chunks} concurrent chains",
                 "value": p_pairs / (p_ms * 1e-3), "ms_per_step": p_ms / args.plain_steps,
                 "steps": args.plain_steps, "warmup": 1, "degree": args.plain_degree,
                 "chunks": args.plain_chunks,
                 "iters_per_op_mean": float(np.mean([s["iters"] for s in plain["stats"]]))}
        if not args.no_paper_form:
            # the paper's form as written: workload degree, one sequential chain (context)
            pf = timed(forms["fp64"], 1, 0, chunks=1)
            f_ms, f_pairs = reduce_max_sum(pf["ms"], pf["pairs"])
            paper_form = {"form": f"plain FP64, degree {w['degree']}, one sequential chain",
                          "value": f_pairs / (f_ms * 1e-3), "ms_per_step": f_ms, "steps": 1,
                          "iters_per_op_mean": float(np.mean([s["iters"] for s in pf["stats"]]))}

    all_stats = instrumented["stats"]
    # per-phase device time of the instrumented step: CUDA events on each chain's own stream,
    # summed over chains (chains run concurrently, so these add up to more than the wall)
    phase_ms = {p: sum(s[f"t_{p}_ms"] for s in all_stats) for p in
                ("filter", "filter32", "filter_dc", "orth", "rr", "eig", "rot", "resid")}
    launches = {"cheb_step_f64": sum(s["filter_steps"] for s in all_stats),
                "cheb_step_f32": sum(s["filter32_steps"] for s in all_stats),
                "cheb_step_dc": sum(s["filter_dc_steps"] for s in all_stats)}
    elems = {"cheb_step_f64": sum(s["filter_elems"] for s in all_stats),
             "cheb_step_f32": sum(s["filter32_elems"] for s in all_stats),
             "cheb_step_dc": sum(s["filter_dc_elems"] for s in all_stats)}
    phase_of = {"cheb_step_f64": "filter", "cheb_step_f32": "filter32", "cheb_step_dc": "filter_dc"}
    peaks, peak_kind = _measured_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    kernels = {}
    for name, nl in launches.items():
        if not nl:
            continue
        avg = phase_ms[phase_of[name]] * 1e-3 / nl
        kernels[name] = {"launches": nl, "avg_us_in_step": avg * 1e6,
                         "bytes_per_launch": BYTES_PER_ELEM[name] * elems[name] / nl,
                         "elems_per_launch": elems[name] / nl}
    iso = isolated_filter_rates(args.degree_fp32, dev)
    for name, r in iso.items():
        if name in kernels:
            kernels[name].update(r)
    # the roofline line reports the kernel that takes the largest share of the GPU's resources
    # in the step: the tensor-core block product (Gram, Rayleigh-Ritz, rotation, triangular
    # solve, deflation), which runs on every SM; the longest kernels of a serialised launch
    # list (Cholesky, tridiagonal reduction, cluster filters) occupy one SM or a few clusters.
    # It is timed alone on the launching stream at the step's shape: the FP64-accurate Gram
    # X^T X of one chain's block (N = 16384, k_b = 120, 8 base-128 digits: 36 BF16 digit-plane
    # products of 2 N k_b^2 flop each).
    kb = scsf.block_width(k)

    def gram_roofline(rows, cols, peak):
        g = torch.Generator(device="cpu").manual_seed(2)
        X = torch.randn((rows, cols), generator=g, dtype=torch.float64).to(dev)
        ms = scsf.block_gram_kernel_time(X, reps=20, ctx=ctx)
        flops = 36 * 2.0 * rows * cols * cols
        ach = flops / (ms * 1e-3) / 1e12
        return {"bound": "tensor", "kernel": "oz_gemm_kernel<8> (FP64-accurate Gram, BF16 digit planes)",
                "shape": f"N = {rows}, k_b = {cols}", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak, "avg_us_alone": ms * 1e3,
                "flops_per_launch": flops,
                "fp64_equivalent_tflops": 2.0 * rows * cols * cols / (ms * 1e-3) / 1e12}

    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    roofline = gram_roofline(n * n, kb, bf16_peak)
    roofline.update({
        "traffic": TRAFFIC_PER_LAUNCH.get("oz_gemm_gram_16384x120"), "traffic_source": TRAFFIC_SOURCE,
        "peak_source": f"MEASURED_PEAKS.json bf16_tflops (burst; the kernel is timed alone) ({peak_kind})",
        "note": ("algorithmic flops = 36 digit-plane products x 2 N k_b^2; the kernel also pays the "
                 "readout of exact integer level sums every 4 chunks of 64 rows and pads k_b to its "
                 "128 x 32 tiles")})
    roofline_k400 = gram_roofline(65536, 480, bf16_peak)
    # the filters, resident in cluster shared memory: per step they move no DRAM data (ncu:
    # 8 MB per 100-step launch), so their bound is on-chip; reported per step
    res = kernels.get("cheb_step_f32", {})
    roofline_filter = None
    if res.get("avg_us_alone"):
        fl = 14.0 * res["elems_per_launch"]  # flop per (node, column) per step
        roofline_filter = {"bound": "alu", "kernel": "strip_filter_cluster_kernel<4, FP32> (per step)",
                           "achieved": fl / (res["avg_us_alone"] * 1e-6) / 1e12,
                           "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                           "frac": fl / (res["avg_us_alone"] * 1e-6) / 1e12 / FP32_PEAK_TFLOPS,
                           "traffic": TRAFFIC_PER_LAUNCH.get("strip_filter_f32_128x120"),
                           "note": ("14 flop per (node, column) per step; traffic is per launch of "
                                    "100 steps; limited by shared-memory issue and cluster "
                                    "barriers, not by DRAM")}
    big = iso.get("cheb_step_f32_256x256_kb480")
    roofline_dram = None
    if big:
        ach_b = big["bytes_per_launch"] / (big["avg_us_alone"] * 1e-6) / 1e9
        roofline_dram = {"bound": "hbm", "kernel": "cheb_step_f32_kernel", "shape": "N = 65536, kb = 480",
                         "achieved": ach_b, "peak": hbm_peak, "unit": "GB/s", "frac": ach_b / hbm_peak,
                         "traffic": TRAFFIC_PER_LAUNCH.get("cheb_step_f32_256x256_kb480"),
                         "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})",
                         "note": ("per-step kernel (the grid is too large for cluster residency): "
                                  "3 x 126 MB FP32 blocks, every step streams through DRAM")}
    dom_phase = max(("filter", "filter32", "filter_dc", "orth", "rr", "eig", "rot", "resid"),
                    key=lambda p: phase_ms[p])
    roofline["dominant_phase"] = dom_phase

    other_configs = {}
    if not args.no_k400:
        other_configs["lapv256_k400"] = leg_lapv256_k400(args, rank, dev, ctx, st, hbm_peak)
    if not args.no_batched:
        other_configs["batched_uneven_64x32"] = leg_batched_uneven(args, rank, dev, ctx, st)
    cpu, err_vs_oracle = None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(ops, args.cpu_sample_ops)
        # the oracle's eigenvalues of the sampled problems (the first problems of the sorted
        # sequence, i.e. of the first chain) against the GPU's from the last timed step
        got = main["last_ev"].detach().cpu().numpy()
        errs = [float(np.max(np.abs(got[i] - ref) / np.abs(ref)))
                for i, ref in enumerate(cpu.pop("evals"))]
        err_vs_oracle = {"problems": len(errs), "max_rel_eig_err": max(errs),
                         "oracle": "CPU FP64 ChFSI (Householder QR) of the same problems",
                         "max_resid_all_pairs": main["max_resid"]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if chosen == "fp64" else "f32+f64",
        "data": "synthetic",
        "config": {"workload": w["name"], "grid": f"{n}x{n}", "N": n * n, "n_ops_per_gpu": n_ops,
                   "k": k, "block_width": scsf.block_width(k), "degree": w["degree"], "p0": w["p0"],
                   "tol": w["tol"],
                   "form": {"mixed": "mixed: FP32 phase + FP64 finish" + (
                                "; chain heads from the learned proposal" if prop else ""),
                            "fp64": "plain FP64"}[chosen] + (
                       f"; sorted sequence cut into {args.chunks} chains solved concurrently"
                       if args.chunks > 1 else "; one sequential chain"),
                   "chunks": args.chunks,
                   "concurrency": args.concurrency or args.chunks,
                   "degrees": ({"fp32_phase": args.degree_fp32, "fp64_phase": args.degree_fp64}
                               if chosen == "mixed" else {"fp64": w["degree"]}),
                   "switch_tol": args.switch_tol if chosen == "mixed" else None,
                   "column_degree": bool(args.column_degree) if chosen == "mixed" else None,
                   "bound": args.bound,
                   "field_law": "a = exp(0.5 f/8), f = sum of 8x8 cosine modes, N(0,1) coefficients",
                   "l2": "flushed (512 MiB write) before every timed step",
                   "parallelism": f"replicas over chains x{ws}"},
        "eigenpairs_per_step": pairs / args.steps / ws,
        "iters_per_op_mean": float(np.mean([s["iters"] for s in all_stats])),
        "iters_fp32_per_op_mean": float(np.mean([s["iters_fp32"] for s in all_stats])),
        "chol_shifts_per_op_mean": {"fp32": float(np.mean([s["chol_shifts_fp32"] for s in all_stats])),
                                    "fp64": float(np.mean([s["chol_shifts"] for s in all_stats]))},
        "filter_dc_elems_per_op_mean": float(np.mean([s["filter_dc_elems"] for s in all_stats])),
        "phase_ms_per_step": phase_ms,
        "phase_note": ("per-phase CUDA-event time of one extra instrumented step, summed over "
                       "the concurrent chains' streams"),
        "ms_instrumented_step": instrumented["ms"],
        "plain_fp64": other,
        "speedup_vs_plain_fp64": (value / other["value"]) if other else None,
        "plain_fp64_paper_form": paper_form,
        "speedup_vs_paper_form": (value / paper_form["value"]) if paper_form else None,
        "err_vs_oracle": err_vs_oracle,
        "other_configs": other_configs,
        "learned_proposal": proposal_leg,
        "roofline": roofline,
        "roofline_tensor_k400_shape": roofline_k400,
        "roofline_filter": roofline_filter,
        "roofline_filter_dram": roofline_dram,
        "kernels": kernels,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(main["launches"]),
        "clocks": main["clocks"],
        "cpu_baseline": cpu,
        "peaks_source": peak_kind,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- other configurations
def _nex_mult4(k: int) -> int:
    """nex >= ceil(0.2 k) with k + nex a multiple of 4 (the mixed form's float4 block rows)."""
    nex = -(-k // 5)
    while (k + nex) % 4:
        nex += 1
    return nex


def _timed_call(fn, dev, st):
    import torch
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    out = fn()
    e1.record(st)
    torch.cuda.synchronize(dev)
    return out, e0.elapsed_time(e1)


def leg_lapv256_k400(args, rank, dev, ctx, st, hbm_peak):
    """The k = 400 workload: 1000 operators -Lap u + V u on 256 x 256 (V = 10 f, 12 x 12
    modes), sorted on the GPU; a prefix of the sorted sequence solved in the mixed form as
    concurrent chains. Every returned pair is checked at the FP64 residual 1e-8."""
    import torch
    import paper_2510_23215_gb300 as scsf
    n, k, n_ops, prefix, chains = 256, 400, 1000, args.k400_prefix, args.k400_chains
    ops = si.lap_plus_v_chain(n, n_ops, seed=2 + 1000 * rank)
    fields = torch.as_tensor(np.stack([o.P for o in ops]), device=dev)
    vs = torch.as_tensor(np.stack([o.V for o in ops]), device=dev)
    params = scsf.Params(k=k, degree=args.k400_degree_fp64, degree_fp32=args.k400_degree_fp32,
                         tol=1e-8, seed=5 + rank, precision=scsf.MIXED,
                         column_degree=bool(args.column_degree), bound=BOUNDS[args.bound])

    def step(count, n_chains):
        perm = scsf.sort(fields, p0=8, ctx=ctx).cpu().tolist()[:count]
        dops = [scsf.Operator(scsf.LAP_PLUS_V, n, v=vs[i]) for i in perm]
        b = np.linspace(0, count, n_chains + 1).round().astype(int)
        res = scsf.solve_batched([(dops[x:y], params) for x, y in zip(b[:-1], b[1:]) if y > x],
                                 concurrency=n_chains, ctx=ctx)
        rs = torch.cat([r[1] for r in res])
        return rs, [s_ for r in res for s_ in r[3]], perm

    step(8, 2)  # warm-up: kernels, graphs, tuned launch widths
    (rs, stats, perm), ms = _timed_call(lambda: step(prefix, chains), dev, st)
    pairs = int((rs <= 1e-8).sum().item())
    # in-run FP32 filter rate: one chain over the first problems with per-phase events
    ctx.set_timing(True)
    dops = [scsf.Operator(scsf.LAP_PLUS_V, n, v=vs[i]) for i in perm[:3]]
    _, _, _, st3 = scsf.solve(dops, params, ctx=ctx)
    ctx.set_timing(False)
    t32 = sum(x["t_filter32_ms"] for x in st3) * 1e-3
    by32 = 12.0 * sum(x["filter32_elems"] for x in st3)
    gbs = by32 / t32 / 1e9 if t32 > 0 else None
    return {
        "workload": "lapv256_k400", "metric": METRIC, "unit": UNIT,
        "value": pairs / (ms * 1e-3), "ms_per_step": ms, "steps": 1, "warmup": 1,
        "pairs": pairs, "max_resid": float(rs.max().item()),
        "config": {"grid": f"{n}x{n}", "N": n * n, "k": k, "block_width": scsf.block_width(k),
                   "n_ops_sorted": n_ops, "solved_prefix": prefix, "chains": chains,
                   "law": "V = 10 f, f = sum of 12 x 12 cosine modes, N(0,1) coefficients",
                   "form": "mixed (FP32 phase + FP64 finish), block products on tensor cores",
                   "degrees": {"fp32_phase": args.k400_degree_fp32,
                               "fp64_phase": args.k400_degree_fp64}},
        "iters_per_op_mean": float(np.mean([x["iters"] for x in stats])),
        "roofline_filter_in_run": {
            "bound": "hbm", "kernel": "cheb_step_f32_kernel (per-step FP32 filter, blocks > L2)",
            "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
            "frac": (gbs / hbm_peak) if gbs else None,
            "note": "12 B per (node, column) per step over the FP32 filter's CUDA-event time "
                    "inside one chain's solve of 3 problems"},
    }


def leg_batched_uneven(args, rank, dev, ctx, st):
    """64 sorted chains of 32 operators each, grid side and k drawn per chain (n in 64..192,
    k in 32..256), -div(a grad u) law; each chain sorted on the GPU and all chains solved by
    one batched call (mixed form), every pair checked at 1e-8."""
    import torch
    import paper_2510_23215_gb300 as scsf
    specs = si.batched_chain_specs(args.batched_chains, 32, seed=3 + 1000 * rank)
    data = []
    for sp in specs:
        ops = si.div_a_grad_chain(sp.n, sp.n_ops, sp.seed)
        data.append((sp, torch.as_tensor(np.stack([o.P for o in ops]), device=dev),
                     torch.as_tensor(np.stack([o.ax for o in ops]), device=dev),
                     torch.as_tensor(np.stack([o.ay for o in ops]), device=dev)))

    def step(items):
        chains = []
        for sp, f, ax, ay in items:
            perm = scsf.sort(f, p0=8, ctx=ctx).cpu().tolist()
            dops = [scsf.Operator(scsf.DIV_A_GRAD, sp.n, ax=ax[i], ay=ay[i]) for i in perm]
            chains.append((dops, scsf.Params(k=sp.k, nex=_nex_mult4(sp.k),
                                             degree=args.batched_degree_fp64,
                                             degree_fp32=args.batched_degree_fp32, tol=1e-8, seed=sp.seed,
                                             precision=scsf.MIXED,
                                             column_degree=bool(args.column_degree),
                                             bound=BOUNDS[args.bound])))
        res = scsf.solve_batched(chains, concurrency=args.batched_concurrency, ctx=ctx)
        return res

    step(data[:8])  # warm-up
    res, ms = _timed_call(lambda: step(data), dev, st)
    pairs = sum(int((r[1] <= 1e-8).sum().item()) for r in res)
    want = sum(sp.k * sp.n_ops for sp, *_ in data)
    return {
        "workload": "batched_uneven_64x32", "metric": METRIC, "unit": UNIT,
        "value": pairs / (ms * 1e-3), "ms_per_step": ms, "steps": 1, "warmup": 1,
        "pairs": pairs, "pairs_wanted": want,
        "max_resid": max(float(r[1].max().item()) for r in res),
        "statuses": sorted({int(r[4]) for r in res}),
        "config": {"chains": len(data), "ops_per_chain": 32, "n_range": [64, 192],
                   "k_range": [32, 256], "concurrency": args.batched_concurrency,
                   "form": "mixed, one batched call (worker threads, one stream each)",
                   "degrees": {"fp32_phase": args.batched_degree_fp32,
                               "fp64_phase": args.batched_degree_fp64}},
    }


def leg_learned_proposal(args, rank, dev):
    """The learned head proposal on the 128 x 128 -div(a grad u) law: labels from the plain
    method (the 64 lowest eigenpairs of each training operator), Adam training of the
    library's network, then held-out operators solved as chain heads (k = 53, block width
    64, every column from the proposal) from the Gaussian block and from the proposal.
    Returns the trained proposal (used at every chain head of the chosen form) and the
    held-out comparison."""
    import dataclasses
    import torch
    import paper_2510_23215_gb300 as scsf
    from paper_2510_23215_gb300 import proposal_train as pt
    n, n_train, n_test = 128, args.proposal_train, args.proposal_test
    t0 = time.perf_counter()
    train_ops = si.div_a_grad_chain(n, n_train, seed=4 + 1000 * rank)
    test_ops = si.div_a_grad_chain(n, n_test, seed=5 + 1000 * rank)
    params = scsf.Params(k=scsf.Proposal.KY, degree=20, tol=1e-8, max_iter=400)
    prop = scsf.Proposal(seed=11 + rank, device=dev)
    fields = torch.as_tensor(np.stack([o.P for o in train_ops]), device=dev)
    Q, tb = pt.label(train_ops, n, params, dev, proposal=prop)
    t_label = time.perf_counter() - t0
    t0 = time.perf_counter()
    pt.train(prop, fields, Q, tb, args.proposal_steps, lr=1e-3)
    t_train = time.perf_counter() - t0
    tf = torch.as_tensor(np.stack([o.P for o in test_ops[:64]]), device=dev)
    tQ, ttb = pt.label(test_ops[:64], n, params, dev, proposal=prop)
    held, _ = prop.gradient(tf.contiguous(), ttb.contiguous(), tQ.contiguous())
    p_eval = dataclasses.replace(params, k=53)
    its = pt.head_iterations(prop, test_ops, p_eval, dev)
    r, q = np.mean(its["random"]), np.mean(its["proposal"])
    return prop, {
        "workload": "learned_proposal_128", "n": n, "train": n_train, "test": n_test,
        "adam_steps": args.proposal_steps, "k_eval": 53, "block_width": p_eval.kb,
        "heldout_loss": {"subspace_sin2_sum_of_64": held[0], "bounds_sq_err": held[2]},
        "mean_iters_random_head": float(r), "mean_iters_proposal_head": float(q),
        "iteration_gain": float(1.0 - q / r),
        "max_resid": max(its["resid_random"], its["resid_proposal"]),
        "label_s": round(t_label, 1), "train_s": round(t_train, 1),
        "note": ("bounded instance of the 5000 / 500 protocol; labels from plain solves; "
                 "both heads reach residual 1e-8"),
    }


# --------------------------------------------------------------------------- CPU oracle
def cpu_baseline(ops, sample_ops: int):
    """The CPU oracle as it stands (numpy FP64, Householder-QR ChFSI) on a bounded sample:
    the sort of the whole batch plus the chain solve of its first `sample_ops` problems."""
    from oracle import chfsi
    from oracle import sort as osort
    w = WORKLOAD
    t0 = time.perf_counter()
    perm, _ = osort.scsf_sort(np.stack([o.P for o in ops]), w["p0"], 0)
    t_sort = time.perf_counter() - t0
    t0 = time.perf_counter()
    res = chfsi.solve_chain([ops[i] for i in perm[:sample_ops]], k=w["k"], degree=w["degree"],
                            tol=w["tol"], head_seed=3, keep_vectors=False)
    t_solve = time.perf_counter() - t0
    pairs = sum(int(np.sum(r.resid <= w["tol"])) for r in res)
    t = t_solve + t_sort * sample_ops / len(ops)
    return {"value": pairs / t, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"sort of all {len(ops)} problems (prorated) + chain solve of the first "
                      f"{sample_ops} sorted problem(s); numpy/LAPACK default thread pool",
            "seconds": t_sort + t_solve, "iters": [r.iters for r in res],
            "evals": [r.evals for r in res]}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    ops = _workload_ops(0)
    vals, secs = [], []
    cb = None
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(ops, args.cpu_sample_ops)
        cb.pop("evals")
        vals.append(cb["value"])
        secs.append(cb["seconds"])
    value = float(np.mean(vals))
    w = WORKLOAD
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w["name"], "grid": f"{w['n']}x{w['n']}", "k": w["k"],
                   "degree": w["degree"], "p0": w["p0"], "tol": w["tol"],
                   "form": "CPU FP64 oracle (Householder-QR ChFSI)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": cb["cores"],
                         "sample": cb["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-sample-ops", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", choices=["mixed", "fp64"], default="mixed",
                    help="headline form (default: the mixed form; plain FP64 is timed beside it)")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison leg")
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--plain-degree", type=int, default=100,
                    help="plain FP64 comparison: filter degree (its best on this workload)")
    ap.add_argument("--plain-chunks", type=int, default=8,
                    help="plain FP64 comparison: concurrent chains")
    ap.add_argument("--no-paper-form", action="store_true",
                    help="skip the paper's form (degree 20, one sequential chain)")
    ap.add_argument("--degree-fp32", type=int, default=80, help="mixed form: FP32-phase degree")
    ap.add_argument("--degree-fp64", type=int, default=110,
                    help="mixed form: FP64-phase degree (130 measured faster but let the FP32 first "
                         "Cholesky factor lose FP64 orthonormality: 1e-11; 110 keeps 2e-15)")
    ap.add_argument("--batched-degree-fp32", type=int, default=60,
                    help="64-chain leg: FP32-phase degree (its grids and k are smaller)")
    ap.add_argument("--batched-degree-fp64", type=int, default=100, help="64-chain leg: FP64-phase degree")
    ap.add_argument("--k400-degree-fp32", type=int, default=60,
                    help="k = 400 leg: FP32-phase degree (its filter streams through DRAM)")
    ap.add_argument("--k400-degree-fp64", type=int, default=100, help="k = 400 leg: FP64-phase degree")
    ap.add_argument("--column-degree", type=int, choices=[0, 1], default=1,
                    help="mixed form: per-column-group degrees in the FP64 phase")
    ap.add_argument("--bound", choices=sorted(BOUNDS), default="gershgorin",
                    help="upper end of the filter interval: Gershgorin or Lanczos estimate")
    ap.add_argument("--switch-tol", type=float, default=0.0,
                    help="mixed form: wanted residual at which the FP32 phase hands over (0: off)")
    ap.add_argument("--chunks", type=int, default=8,
                    help="contiguous chunks of the sorted sequence solved as concurrent chains")
    ap.add_argument("--concurrency", type=int, default=0,
                    help="chains in flight at once (0: all chunks; more chunks than slots "
                         "balance uneven chains)")
    ap.add_argument("--no-k400", action="store_true", help="skip the 256 x 256, k = 400 leg")
    ap.add_argument("--k400-prefix", type=int, default=64,
                    help="k = 400 leg: solved prefix of the 1000 sorted problems")
    ap.add_argument("--k400-chains", type=int, default=4, help="k = 400 leg: concurrent chains")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-chain uneven leg")
    ap.add_argument("--no-proposal", action="store_true",
                    help="no learned proposal (not trained, not used at chain heads)")
    ap.add_argument("--proposal-train", type=int, default=320)
    ap.add_argument("--proposal-test", type=int, default=32)
    ap.add_argument("--proposal-steps", type=int, default=800)
    ap.add_argument("--batched-chains", type=int, default=64)
    ap.add_argument("--batched-concurrency", type=int, default=8)
    ap.add_argument("--n-ops", type=int, default=None,
                    help="problems per batch (default 200; smaller only for profiler captures)")
    args = ap.parse_args()
    if args.n_ops is not None:
        WORKLOAD["n_ops"] = args.n_ops
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
