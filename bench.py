#!/usr/bin/env python
"""Benchmark of the GoFD stiffness product and PCG on one GB300 per rank.

Workload (the 2D L-shaped domain [-1,1]^2 minus [0,1]^2): a seeded jittered
Delaunay mesh of ~6.0e4 vertices, overlay grid 1024^2 on [-1,1]^2 embedded in a
2048^2 circulant.  A step is one FP32 stiffness product y = I^T A_FD I x
(gather, FFT convolution, scatter) on device-resident interior vectors; L2 is
flushed (256 MB write) before every timed step.  The headline value is the
algorithmic bytes of one product divided by its time (GB/s), and the roofline
is that product against the measured HBM copy bandwidth.  Beside it: per-kernel
times (the slowest stage in its own key), the same product end to end through
the host-buffer C-ABI call, and these extras:
  * time to relative residual 1e-8, mixed-precision refinement vs plain FP64
    PCG, on the L-shape at alpha in {0.5, 1, 1.5}, on the 2048^2 graded disk
    (alpha = 1.2, vertex data) and on the 256^3 ball (alpha = 1.5, with the
    error against the closed form);
  * the graded-disk gradient: forward solve and adjoint (dL/df, dL/dX) times;
  * the 48-instance x 8 right-hand-side batch through grid groups, with one
    right-hand side at a time in FP64 beside it (sampled, scaled);
  * the FP64 CPU oracle's product timed on the host cores.

Multi-GPU runs (torchrun) execute independent replicas (the product does not
shard): no data-path collective; the aggregate value sums all ranks' bytes
over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import meshgen as mg  # noqa: E402

METRIC = "A_h matvec GB/s + PCG time to rel-res 1e-8: mixed vs FP64, 1 GB300"
N_GRID = 1024
ALPHAS = (0.5, 1.0, 1.5)


def b_alg(d, n_loc, n_v, n_grid, P, b):
    """Algorithmic bytes of one stiffness product (precision b bytes):
    ELL read, I^T CSR read, u and y, grid vector written and read, FFT output
    written and read at the located nodes, real even symbol."""
    return ((d + 1) * (4 + b) * n_loc                  # ELL of I_h^FD
            + (d + 1) * (4 + b) * n_loc + 4 * (n_v + 1)  # CSR of I^T
            + 2 * b * n_v                              # u, y
            + 2 * b * n_grid                           # v = I u written, read by the FFT
            + b * n_grid + b * n_loc                   # A_FD v written, read at located nodes
            + b * (P // 2 + 1) ** d)                   # symbol


WORKLOADS = {
    "lshape1024": "2D L-shape [-1,1]^2\\[0,1]^2, 6.05e4 vertices, 1024^2 grid in a 2048^2 circulant, alpha=1",
    "graded2048": "2D graded unit disk, 2.1e5 vertices, 2048^2 grid in a 4096^2 circulant, alpha=1.2",
    "ball256": "3D unit ball, 1.3e5 vertices, 256^3 grid in a 512^3 circulant, alpha=1.5",
    "batch48": "48 instances (16 ring disks + 16 L-shapes, 5e3-1.5e5 vertices log-uniform, alpha cycling "
               "0.5/1/1.5, grids 256^2-2048^2) x 8 right-hand sides (f=1 + 7 Gaussian bumps, width 0.1)",
}
# DRAM bytes of one FP32 L-shape product: dram__bytes_read.sum +
# dram__bytes_write.sum of each of its five kernels, averaged over five
# products of an ncu launch list of these kernels that keeps L2 as the program
# leaves it (--cache-control none) after the same 256 MB L2 flush the timed
# loop does, summed over the kernels; the writes are mostly the flush
# buffer's dirty lines written back.  (total, reads)
NCU_PRODUCT_DRAM_BYTES = {"lshape1024": (80510464, 45347072)}
BATCH_METRIC = "batched block-PCG: right-hand sides solved to rel-res 1e-8 per second (mixed), 1 GB300"
BATCH_RHS = 8


def workload(name="lshape1024", alpha=None, grid=0):
    """Mesh, alpha and overlay grid of a workload; grid > 0 replaces its grid
    size (a smaller case of the same kernels, for profiling captures)."""
    if name == "graded2048":
        lo, hi, h = mg.grid_box(2, grid or 2048)
        v, s = mg.graded_disk_mesh(mg.grid_box(2, 2048)[2], seed=mg.seed_for(4))
        return v, s, 1.2 if alpha is None else alpha, h, lo, hi
    if name == "ball256":
        v, s = mg.ball_shell_mesh(seed=mg.seed_for(3))
        lo, hi, h = mg.grid_box(3, grid or 256)
        return v, s, 1.5 if alpha is None else alpha, h, lo, hi
    v, s = mg.lshape_mesh(seed=mg.seed_for(2))
    lo, hi, h = mg.grid_box(2, grid or N_GRID)
    return v, s, 1.0 if alpha is None else alpha, h, lo, hi


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons (200 ms)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for nm, val in zip(names, r[5:9]):
                    if val.strip() == "Active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def shard(items, rank, world):
    """This rank's share of independent work items (round robin; no collective)."""
    return items[rank::world]


def max_over_ranks(value, world, device):
    """The largest value over the ranks (the slowest rank's time); one all-reduce."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(steps_cap=None, budget_s=20.0):
    """The FP64 oracle's stiffness product on the host cores, at full size."""
    import scipy.fft
    from oracle import gofd as oracle
    v, s, alpha, h, lo, hi = workload()
    t0 = time.perf_counter()
    ref = oracle.build(2, v, s, alpha, h, lo, hi, exact_weights=False, pruned=True)
    t_setup = time.perf_counter() - t0
    u = mg.random_vector(len(v), 3)
    cores = os.cpu_count() or 1
    times = []
    with scipy.fft.set_workers(cores):
        oracle.stiffness_apply(ref, u)       # warm
        t_start = time.perf_counter()
        while True:
            t1 = time.perf_counter()
            oracle.stiffness_apply(ref, u)
            times.append(time.perf_counter() - t1)
            if (steps_cap and len(times) >= steps_cap) or time.perf_counter() - t_start > budget_s:
                break
    P = ref.P
    B = b_alg(2, len(ref.nodes), len(v), ref.n_grid, P, 8)
    t = statistics.mean(times)
    return ref, {"value": B / t / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle", "ms_per_step": t * 1e3,
                 "sample": f"{len(times)} FP64 stiffness products (scipy.fft workers={cores}) on the full "
                           f"L-shape workload, mean {t * 1e3:.1f} ms each; oracle set-up {t_setup:.1f} s untimed"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    steps = args.steps
    _, cb = cpu_baseline(steps_cap=steps + args.warmup, budget_s=120.0)
    cb["value"] = round(cb["value"], 4)   # the line's value
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "GB/s",
            "n_gpus": args.gpus, "steps": steps, "warmup": args.warmup,
            "ms_per_step": round(cb["ms_per_step"], 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded jittered L-shape Delaunay mesh)",
            "config": {"workload": "2D L-shape, 6.0e4 vertices, 1024^2 grid, 2048^2 circulant, alpha=1",
                       "l2": "inputs larger than L2 (CPU)"},
            "cpu_baseline": cb,
            "e2e": {"value": round(cb["value"], 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def ball_solves(dev, prob=None):
    """The 3D ball configuration: mixed vs FP64 PCG to 1e-8, f = 1, and the
    error against the closed form u = C (1 - |x|^2)^(3/4), C = 0.300901
    (alpha = 1.5, d = 3)."""
    import torch
    from paper_2307_14437_gb300 import Problem
    v, s, alpha, h, lo, hi = workload("ball256")
    own = prob is None
    row = {}
    if own:
        t1 = time.perf_counter()
        prob = Problem(v, s, alpha, h, lo, hi)
        row["setup_s"] = round(time.perf_counter() - t1, 3)
        prob.autotune(nb=1)
    f3 = torch.ones(prob.n_grid, dtype=torch.float64, device=dev)
    for mode in ("mixed", "fp64"):
        prob.solve(f3, mode=mode, tol=1e-8)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        u3, info3 = prob.solve(f3, mode=mode, tol=1e-8)
        torch.cuda.synchronize()
        row[mode] = {"s": round(time.perf_counter() - t1, 5), "inner_iters": info3["inner_iters"],
                     "outer_iters": info3["outer_iters"], "rel_res_fp64": info3["rel_res_fp64"]}
        ex = 0.300901 * np.maximum(0.0, 1.0 - np.sum(v ** 2, axis=1)) ** 0.75
        row[mode]["rel_l2_err_vs_closed_form"] = float(np.linalg.norm(u3.cpu().numpy() - ex) / np.linalg.norm(ex))
    row["speedup_mixed_vs_fp64"] = round(row["fp64"]["s"] / row["mixed"]["s"], 3)
    row["vertices"] = len(v)
    if own:
        prob.close()
    return row


def gradient_times(dev, pg, vg, ft):
    """The differentiation configuration: L = 1/2 ||u - u_target||^2 with
    u = S^{-1} h^{2s} D_h f (vertex data f = 1), u_target the solve of
    f_target; time of the forward solve and of the adjoint (its solve and
    dL/df, dL/dX), both mixed precision to 1e-10."""
    import torch
    u_t, _ = pg.solve(ft, rhs="vertex", mode="mixed", tol=1e-10)
    f = torch.ones(len(vg), dtype=torch.float64, device=dev)
    for _ in range(2):                                   # the first round warms
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        u, fi = pg.solve(f, rhs="vertex", mode="mixed", tol=1e-10)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        gf, gx, ai = pg.adjoint(f, u, u - u_t, mode="mixed", tol=1e-10)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
    return {"forward_s": round(t2 - t1, 5), "adjoint_s": round(t3 - t2, 5), "total_s": round(t3 - t1, 5),
            "forward_inner_iters": fi["inner_iters"], "adjoint_inner_iters": ai["inner_iters"],
            "grad_f_entries": int(gf.numel()), "grad_X_entries": int(gx.numel()),
            "finite": bool(torch.isfinite(gf).all() and torch.isfinite(gx).all())}


def run_gofd(args):
    import torch
    from paper_2307_14437_gb300 import Problem
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    v, s, alpha, h, lo, hi = workload(args.workload, grid=args.grid)
    t0 = time.perf_counter()
    prob = Problem(v, s, alpha, h, lo, hi)
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    if args.shapes:                          # launch shapes given: no tuning (profiling captures)
        prob.set_launch_shapes(*[int(a) for a in args.shapes.split(",")])
    else:
        prob.autotune(nb=1)                  # launch shapes of the product (part of the set-up)
    t_tune = time.perf_counter() - t0
    inf = prob.info()
    d, n_loc, n_v, nint, P = inf["d"], inf["n_loc"], inf["n_v"], inf["n_interior"], inf["P"]
    B32 = b_alg(d, n_loc, n_v, inf["n_grid"], P, 4)

    gen = torch.Generator(device="cpu").manual_seed(5)
    x = torch.zeros(nint + 1, dtype=torch.float32)
    x[:nint] = torch.rand(nint, generator=gen) * 2 - 1
    x = x.to(dev)
    y = torch.empty(nint + 1, dtype=torch.float32, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        prob.apply_interior(x, y)
    clocks = Clocks(local)
    barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        evs[i][0].record(stream)
        prob.apply_interior(x, y)
        evs[i][1].record(stream)
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = statistics.mean(step_ms)
    ms_max = max_over_ranks(ms, world, dev)
    value = world * B32 / (ms_max * 1e-3) / 1e9

    # per-kernel times (events after each launch), same L2 flush
    stages = {}
    for i in range(max(10, min(args.steps, 100))):
        flush.fill_(float(i))
        prof = prob.apply_interior_profiled(x, y)
        kernels_per_product = len(prof)          # one event pair per kernel launch
        for name, t in prof:
            stages.setdefault(name, []).append(t)
    stage_ms = {k: statistics.mean(vv) for k, vv in stages.items()}
    dom = max(stage_ms, key=stage_ms.get)   # slowest stage (events between kernels)
    H = P // 2 + 1
    n = inf["n"][0]
    # algorithmic bytes per launch of each kernel (FP32)
    nl = n ** (d - 1)
    # algorithmic bytes of each stage: the terms of b_alg() it accounts for
    # (FFT-internal spectrum passes excluded): ELL, x, v; v, FFT output; the
    # symbol; FFT output read at the located nodes, I^T, y
    kbytes = {
        "gather": (d + 1) * 8 * n_loc + 4 * nint + 4 * n ** d,
        "gather_row_fft": (d + 1) * 8 * n_loc + 4 * nint + 4 * n ** d,
        "row_fft": 4 * n ** d,
        "col_fft_conv": 4 * H ** d,
        "axis12_conv": 4 * H ** d,
        "symbol_mul": 4 * H ** d,
        "row_ifft": 4 * n ** d,
        "scatter": 4 * n_loc + (d + 1) * 8 * n_loc + 4 * (n_v + 1) + 4 * nint,
    }
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    achieved = B32 / (ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": "stiffness product (%d kernels: %s)" % (len(stage_ms), ", ".join(stage_ms)),
                "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s", "frac": round(achieved / hbm, 4),
                "traffic": NCU_PRODUCT_DRAM_BYTES[args.workload][0] if args.workload in NCU_PRODUCT_DRAM_BYTES
                and not args.grid else None,
                "traffic_read": NCU_PRODUCT_DRAM_BYTES[args.workload][1] if args.workload in NCU_PRODUCT_DRAM_BYTES
                and not args.grid else None,
                "bytes_alg": B32, "ms_per_product": round(ms, 5),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy), of measured" if "hbm_gbs" in pk
                else "fallback 6.8 TB/s",
                "stage_ms": {k: round(vv, 5) for k, vv in stage_ms.items()},
                "stage_note": "events after every kernel (no launch overlap between stages); 2 us timer steps"}
    dominant = {"kernel": dom, "ms": round(stage_ms[dom], 5), "bytes_alg": kbytes.get(dom),
                "achieved": round(kbytes[dom] / (stage_ms[dom] * 1e-3) / 1e9, 1) if dom in kbytes else None,
                "unit": "GB/s", "frac": round(kbytes[dom] / (stage_ms[dom] * 1e-3) / 1e9 / hbm, 4)
                if dom in kbytes else None}

    # end to end through the host-buffer C-ABI call (pinned host memory)
    u_h = torch.empty(n_v, dtype=torch.float32, pin_memory=True)
    u_h.copy_(torch.rand(n_v, generator=gen) * 2 - 1)
    y_h = torch.empty(n_v, dtype=torch.float32, pin_memory=True)
    u_np, y_np = u_h.numpy(), y_h.numpy()
    for _ in range(3):
        prob.apply_host(u_np, out=y_np)
    e2e_ms = []
    for i in range(max(5, min(args.steps, 50))):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        prob.apply_host(u_np, out=y_np)
        e2e_ms.append((time.perf_counter() - t1) * 1e3)
    e2e_t = statistics.mean(e2e_ms)
    e2e = {"value": round(world * B32 / (e2e_t * 1e-3) / 1e9, 2), "unit": "GB/s",
           "h2d_bytes_per_step": 4 * n_v, "d2h_bytes_per_step": 4 * n_v, "ms_per_step": round(e2e_t, 4),
           "note": "pinned host buffers, read and written in place by the kernels over the CPU-GPU link"}

    # the FP64 product: bound by FP64 arithmetic (its FFT passes); roofline
    # against the measured FP64 FMA rate, with the unpruned FFT flop count
    # 2 x 2.5 P^d log2(P^d) per product as the algorithmic work
    from paper_2307_14437_gb300.gofd import fma_rates
    fp64_peak, fp32_peak = fma_rates()
    x64 = x.double()
    y64 = torch.empty_like(x64)
    for _ in range(3):
        prob.apply_interior(x64, y64)
    ev64 = []
    for i in range(20):
        flush.fill_(float(i))
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        prob.apply_interior(x64, y64)
        b_.record(stream)
        ev64.append((a_, b_))
    torch.cuda.synchronize()
    ms64 = statistics.mean(a_.elapsed_time(b_) for a_, b_ in ev64)
    fft_flops = 2 * 2.5 * P ** d * math.log2(P ** d)
    # the mixed solver's residual product: FP64 gather and scatter, the FFT
    # convolution in double-float arithmetic (2D)
    df = None
    if d == 2:
        ydf = torch.empty_like(x64)
        for _ in range(3):
            prob.apply_interior(x64, ydf, prec="fp64_df")
        evdf = []
        for i in range(20):
            flush.fill_(float(i))
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            prob.apply_interior(x64, ydf, prec="fp64_df")
            b_.record(stream)
            evdf.append((a_, b_))
        torch.cuda.synchronize()
        msdf = statistics.mean(a_.elapsed_time(b_) for a_, b_ in evdf)
        dif = float(torch.linalg.norm(ydf[:nint] - y64[:nint]) / torch.linalg.norm(y64[:nint]))
        df = {"ms_per_product": round(msdf, 4), "speedup_vs_fp64": round(ms64 / msdf, 2),
              "rel_diff_vs_fp64_product": dif,
              "note": "FP64 inputs and outputs, FP64 gather and scatter, FFT convolution in double-float"}
    roofline_fp64 = {"bound": "fp64_alu", "ms_per_product": round(ms64, 4),
                     "achieved": round(fft_flops / (ms64 * 1e-3) / 1e9, 1), "peak": round(fp64_peak, 1),
                     "unit": "GFLOP/s", "frac": round(fft_flops / (ms64 * 1e-3) / 1e9 / fp64_peak, 4),
                     "work": "2 x 2.5 P^d log2 P^d flops per product (unpruned FFTs)",
                     "peak_source": "measured FP64 FMA rate (gofd_fma_rates), this run",
                     "fp32_fma_gflops": round(fp32_peak, 1), "double_float_residual_product": df}

    # time to relative residual 1e-8: mixed refinement vs plain FP64 PCG
    pcg = {}
    if not args.no_pcg and args.workload == "lshape1024":
        for a in ALPHAS:
            pa = prob if a == alpha else Problem(v, s, a, h, lo, hi)
            if pa is not prob:
                pa.autotune(nb=1)
            f = torch.ones(pa.n_grid, dtype=torch.float64, device=dev)
            row = {"setup_s": round(t_setup, 3) if a == alpha else None}
            for mode in ("mixed", "fp64"):
                pa.solve(f, mode=mode, tol=1e-8)          # warm
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                _, info = pa.solve(f, mode=mode, tol=1e-8)
                torch.cuda.synchronize()
                row[mode] = {"s": round(time.perf_counter() - t1, 5), "inner_iters": info["inner_iters"],
                             "outer_iters": info["outer_iters"], "rel_res_fp64": info["rel_res_fp64"]}
            row["speedup_mixed_vs_fp64"] = round(row["fp64"]["s"] / row["mixed"]["s"], 3)
            # the same mixed solve with a plain FP64 residual convolution
            pr = Problem(v, s, a, h, lo, hi, fp64_residual=1)
            pr.autotune(nb=1)
            pr.solve(f, mode="mixed", tol=1e-8)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, info = pr.solve(f, mode="mixed", tol=1e-8)
            torch.cuda.synchronize()
            row["mixed, plain FP64 residual"] = {"s": round(time.perf_counter() - t1, 5),
                                                 "inner_iters": info["inner_iters"],
                                                 "outer_iters": info["outer_iters"],
                                                 "rel_res_fp64": info["rel_res_fp64"]}
            pr.close()
            pcg[f"alpha={a}"] = row
            if pa is not prob:
                pa.close()
        # the paper's IC(1) preconditioner (9-point pattern), both unknown orders,
        # triangular solves as one persistent launch each (ic_solve 0) and, in
        # multicolour order, as one launch per level (ic_solve 1)
        for ordering, ic_solve in ((1, 0), (0, 0), (1, 1)):
            t1 = time.perf_counter()
            pp = Problem(v, s, alpha, h, lo, hi, precond=9, ordering=ordering, ic_solve=ic_solve)
            t_pc = time.perf_counter() - t1
            f = torch.ones(pp.n_grid, dtype=torch.float64, device=dev)
            pp.solve(f, mode="mixed", tol=1e-8)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, info = pp.solve(f, mode="mixed", tol=1e-8)
            torch.cuda.synchronize()
            pi = pp.info()
            key = f"alpha={alpha} ic1 ordering={'multicolour' if ordering else 'natural'}"
            pcg[key + (", one launch per level" if ic_solve else "")] = {
                "mixed_s": round(time.perf_counter() - t1, 5), "inner_iters": info["inner_iters"],
                "outer_iters": info["outer_iters"], "rel_res_fp64": info["rel_res_fp64"],
                "levels": pi["precond_levels"], "factor_nnz": pi["precond_nnz"], "build_s": round(t_pc, 3)}
            pp.close()
    if not args.no_pcg and args.workload == "lshape1024":
        # the circulant alternative of Section 3.3 (precond = 2) at each alpha
        for a in ALPHAS:
            pc = Problem(v, s, a, h, lo, hi, precond=2)
            pc.autotune(nb=1)
            f = torch.ones(pc.n_grid, dtype=torch.float64, device=dev)
            pc.solve(f, mode="mixed", tol=1e-8)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, info = pc.solve(f, mode="mixed", tol=1e-8)
            torch.cuda.synchronize()
            pcg[f"alpha={a} circulant precond (Section 3.3 alternative)"] = {
                "mixed_s": round(time.perf_counter() - t1, 5), "inner_iters": info["inner_iters"],
                "outer_iters": info["outer_iters"], "rel_res_fp64": info["rel_res_fp64"]}
            pc.close()
    if not args.no_pcg and args.workload in ("lshape1024", "graded2048"):
        # the 2048^2 configuration: graded disk, alpha = 1.2, vertex data f_target (GoFD-3)
        if args.workload == "graded2048":
            pg, vg = prob, v
        else:
            vg_, sg_, ag_, hg_, log_, hig_ = workload("graded2048")
            pg, vg = Problem(vg_, sg_, ag_, hg_, log_, hig_), vg_
            pg.autotune(nb=1)
        ft = torch.tensor(mg.target_bump(vg), device=dev)
        row = {}
        for mode in ("mixed", "fp64"):
            pg.solve(ft, rhs="vertex", mode=mode, tol=1e-8)   # warm
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, info = pg.solve(ft, rhs="vertex", mode=mode, tol=1e-8)
            torch.cuda.synchronize()
            row[mode] = {"s": round(time.perf_counter() - t1, 5), "inner_iters": info["inner_iters"],
                         "outer_iters": info["outer_iters"], "rel_res_fp64": info["rel_res_fp64"]}
        row["speedup_mixed_vs_fp64"] = round(row["fp64"]["s"] / row["mixed"]["s"], 3)
        # the diagonal of S as preconditioner (its set-up timed apart)
        g_args = (v, s, alpha, h, lo, hi) if pg is prob else (vg_, sg_, ag_, hg_, log_, hig_)
        t1 = time.perf_counter()
        pj = Problem(*g_args, precond=1)
        row["diagonal_precond_build_s"] = round(time.perf_counter() - t1, 3)
        pj.autotune(nb=1)
        for mode in ("mixed", "fp64"):
            pj.solve(ft, rhs="vertex", mode=mode, tol=1e-8)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, info = pj.solve(ft, rhs="vertex", mode=mode, tol=1e-8)
            torch.cuda.synchronize()
            row[mode + " + diagonal precond"] = {"s": round(time.perf_counter() - t1, 5),
                                                 "inner_iters": info["inner_iters"],
                                                 "outer_iters": info["outer_iters"],
                                                 "rel_res_fp64": info["rel_res_fp64"]}
        row["gradients dL/df, dL/dX"] = gradient_times(dev, pg, vg, ft)
        row["gradients dL/df, dL/dX, diagonal precond"] = gradient_times(dev, pj, vg, ft)
        pj.close()
        pcg["graded disk 2048^2 alpha=1.2, f_target vertex data"] = row
        if pg is not prob:
            pg.close()
    if not args.no_pcg and args.workload == "lshape1024":
        # the paper's preconditioner in its own setting, h_FD about a_h (Section
        # 3.3, Remark 3.5): the same L-shape mesh on the grid with h just below
        # a_h, alpha 1 and 1.8 (s = 0.9), plain CG against IC(1) of the 5- and
        # 9-point stencil matrices (multicolour order) and against the
        # circulant alternative the section names, mixed precision to 1e-8
        n_c = int(math.ceil(2.0 / inf["a_h"])) + 1
        lo_c, hi_c, h_c = mg.grid_box(2, n_c)
        ic = {}
        for a in (1.0, 1.8):
            for pat in (0, 5, 9, 2):
                pp = Problem(v, s, a, h_c, lo_c, hi_c, precond=pat, ordering=1 if pat in (5, 9) else 0)
                f = torch.ones(pp.n_grid, dtype=torch.float64, device=dev)
                pp.solve(f, mode="mixed", tol=1e-8)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                _, info = pp.solve(f, mode="mixed", tol=1e-8)
                torch.cuda.synchronize()
                label = {0: "plain CG", 2: "circulant (Section 3.3 alternative)"}.get(pat, f"IC(1) {pat}-point")
                ic[f"alpha={a} {label}"] = {
                    "s": round(time.perf_counter() - t1, 5), "inner_iters": info["inner_iters"],
                    "rel_res_fp64": info["rel_res_fp64"], "h_over_a_h": round(h_c / info["a_h"], 3)}
                pp.close()
        pcg[f"L-shape {n_c}^2 (h about a_h): preconditioners"] = ic
    if not args.no_pcg and args.workload == "lshape1024":
        # the small unit-disk configuration: FP64 PCG to 1e-10, f = 1, against
        # the closed form u = (2/pi) (1 - |x|^2)^(1/2) (alpha = 1, Section 5)
        v1, s1 = mg.disk_ring_mesh(rings=25, seed=mg.seed_for(1))
        lo1, hi1, h1 = mg.grid_box(2, 128)
        p1 = Problem(v1, s1, 1.0, h1, lo1, hi1)
        f1 = torch.ones(p1.n_grid, dtype=torch.float64, device=dev)
        p1.solve(f1, mode="fp64", tol=1e-10)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        u1, info1 = p1.solve(f1, mode="fp64", tol=1e-10)
        torch.cuda.synchronize()
        ex = (2.0 / math.pi) * np.sqrt(np.maximum(0.0, 1.0 - np.sum(v1 ** 2, axis=1)))
        err = np.abs(u1.cpu().numpy() - ex)
        pcg["unit disk 128^2 alpha=1 FP64 to 1e-10"] = {
            "s": round(time.perf_counter() - t1, 5), "inner_iters": info1["inner_iters"],
            "rel_res_fp64": info1["rel_res_fp64"], "max_abs_err_vs_closed_form": float(err.max()),
            "rel_l2_err_vs_closed_form": float(np.linalg.norm(err) / np.linalg.norm(ex))}
        p1.close()
    if not args.no_pcg and args.workload == "ball256":
        pcg["ball 256^3 alpha=1.5 f=1"] = ball_solves(dev, prob)
    if not args.no_pcg and args.workload == "lshape1024":
        # the 3D ball configuration and the batched configuration beside the L-shape line
        t1 = time.perf_counter()
        pcg["ball 256^3 alpha=1.5 f=1"] = ball_solves(dev)
        pcg["ball 256^3 alpha=1.5 f=1"]["wall_s"] = round(time.perf_counter() - t1, 2)
        t1 = time.perf_counter()
        batch = batch_workload(dev, rank, world, warm=1, steps=1, single="sampled")
        batch["wall_s"] = round(time.perf_counter() - t1, 2)
    else:
        batch = None
    clk = clocks.stop()

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_max, 5), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded jittered L-shape Delaunay mesh, uniform random x)",
                "config": {"workload": WORKLOADS[args.workload] + ", FP32 stiffness product (%d vertices, %d interior)"
                                       % (n_v, nint) + (", grid replaced by %d^%d" % (args.grid, d) if args.grid else ""),
                           "l2": "flushed (256 MB write) before every timed step",
                           "n_loc": n_loc, "setup_s": round(t_setup, 3), "autotune_s": round(t_tune, 3),
                           "launch_shapes": {"lines_per_cta": inf["tune_lines_per_cta"],
                                             "cols_per_cta": inf["tune_cols_per_cta"],
                                             "scatter_lanes": inf["tune_scatter_lanes"],
                                             "col_elems": inf["tune_col_elems"],
                                             "row_elems": inf["tune_row_elems"]}},
                "roofline": roofline, "dominant_kernel": dominant, "roofline_fp64_product": roofline_fp64,
                "e2e": e2e, "pcg": pcg, "batch": batch,
                "gpu_launches": kernels_per_product * args.steps, "clocks": clk}
        if world == 1 and not args.no_cpu and args.workload == "lshape1024":
            try:
                line["cpu_baseline"] = cpu_baseline()[1]
            except Exception as exc:  # the baseline is reported, never required
                line["cpu_baseline"] = {"value": None, "unit": "GB/s", "cores": os.cpu_count(), "kind": "oracle",
                                        "sample": f"failed: {exc}"}
        print(json.dumps(line), flush=True)
    prob.close()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _min_height(v, s):
    """Smallest triangle height: twice the area over the longest edge (2D)."""
    p = v[s]
    e0, e1, e2 = p[:, 1] - p[:, 0], p[:, 2] - p[:, 1], p[:, 0] - p[:, 2]
    area2 = np.abs(e0[:, 0] * e2[:, 1] - e0[:, 1] * e2[:, 0])
    longest = np.maximum(np.maximum(np.linalg.norm(e0, axis=1), np.linalg.norm(e1, axis=1)),
                         np.linalg.norm(e2, axis=1))
    return float(np.min(area2 / longest))


def batch_grid_nodes(a_h):
    """Smallest n in {256, 512, 1024, 2048} with 2/(n-1) <= a_h/2 (else 2048)."""
    for n in (256, 512, 1024, 2048):
        if 2.0 / (n - 1) <= 0.5 * a_h:
            return n
    return 2048


def batch_workload(dev, rank, world, warm=1, steps=1, single="sampled"):
    """The batched workload: 48 instances x 8 right-hand sides.  Instances on
    one overlay grid at one alpha form a Group (all their columns in one
    lock-step block PCG, FP32 inner, FP64 refinement, converged columns
    skipped by the product kernels, launch shapes from the group autotuner);
    the groups run concurrently.  A step is the whole batch.  Beside it, one
    right-hand side at a time in plain FP64 PCG: all 384 (single="all"), or
    column i mod 8 of instance i, scaled by 8 (single="sampled")."""
    import torch
    from paper_2307_14437_gb300 import Group, Problem, group_key, solve_many
    all_specs = mg.batch_instances()
    specs = shard(all_specs, rank, world)              # instances are independent: shard, no collective
    meshes, probs, Fs, rows = {}, [], [], []
    t0 = time.perf_counter()
    for sp in specs:
        key = (sp["kind"], sp["mesh"])
        if key not in meshes:
            meshes[key] = mg.batch_mesh(sp)
        v, s = meshes[key]
        n = batch_grid_nodes(_min_height(v, s))
        lo, hi, h = mg.grid_box(2, n)
        t1 = time.perf_counter()
        pr = Problem(v, s, sp["alpha"], h, lo, hi)
        t_setup = time.perf_counter() - t1
        inside = mg.in_disk if sp["kind"] == "disk" else mg.in_lshape
        F = mg.rhs_family(mg.grid_points(lo, h, n), BATCH_RHS, seed=sp["seed"] + 7, inside=inside)
        probs.append(pr)
        Fs.append(torch.tensor(F, device=dev))
        rows.append({"kind": sp["kind"], "n_v": len(v), "n": n, "alpha": sp["alpha"], "setup_s": round(t_setup, 3)})
    t_build = time.perf_counter() - t0
    t1 = time.perf_counter()
    members = {}
    for i, pr in enumerate(probs):
        members.setdefault(group_key(pr), []).append(i)
    groups, gtune = {}, {}
    for key, idx in members.items():
        groups[key] = Group([probs[i] for i in idx], BATCH_RHS)
        gtune[f"{key[1][0]}^2 alpha={key[4]} ({len(idx)} instances)"] = round(groups[key].autotune(), 4)
    for pr in probs:                                     # shapes of the one-at-a-time solves
        pr.autotune(nb=1)
    t_tune = time.perf_counter() - t1
    torch.cuda.synchronize()

    for _ in range(warm):
        solve_many(probs, Fs, mode="mixed", tol=1e-8, groups=groups)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(steps):
        out = solve_many(probs, Fs, mode="mixed", tol=1e-8, groups=groups)
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t1) / steps
    worst = max(i["rel_res_fp64"] for _, infos in out for i in infos)
    for r, (_, infos) in zip(rows, out):
        r["inner_iters"] = max(i["inner_iters"] for i in infos)

    # end to end: right-hand sides from pinned host memory, solutions back to pinned host memory
    Fh = [f.cpu().pin_memory() for f in Fs]
    Uh = [torch.empty((BATCH_RHS, pr.n_v), dtype=torch.float64, pin_memory=True) for pr in probs]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    Fd = [f.to(dev, non_blocking=True) for f in Fh]
    res = solve_many(probs, Fd, mode="mixed", tol=1e-8, groups=groups)
    for u_h, (U, _) in zip(Uh, res):
        u_h.copy_(U, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t1

    # one right-hand side at a time, plain FP64 PCG (no batching, no refinement)
    t1 = time.perf_counter()
    n_single = 0
    for i, (pr, F) in enumerate(zip(probs, Fs)):
        cols = range(BATCH_RHS) if single == "all" else ((i + rank) % BATCH_RHS,)
        for c in cols:
            pr.solve(F[c].contiguous(), mode="fp64", tol=1e-8)
            n_single += 1
    torch.cuda.synchronize()
    t_single = (time.perf_counter() - t1) * (len(probs) * BATCH_RHS / max(1, n_single))

    # the batched FP32 product of the largest instance against the HBM roofline
    big = max(range(len(probs)), key=lambda i: rows[i]["n"] * 1e9 + rows[i]["n_v"])
    pr = probs[big]
    inf = pr.info()
    ld = inf["n_interior"] + 1
    X = torch.zeros((BATCH_RHS, ld), dtype=torch.float32, device=dev)
    X[:, :ld - 1] = torch.rand((BATCH_RHS, ld - 1), device=dev) * 2 - 1
    Y = torch.empty_like(X)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    pr.autotune(nb=BATCH_RHS)
    for _ in range(3):
        pr.apply_interior_batch(X, Y)
    st = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    for a, b in ev:
        flush.fill_(1.0)
        a.record(st)
        pr.apply_interior_batch(X, Y)
        b.record(st)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    B = BATCH_RHS * b_alg(2, inf["n_loc"], inf["n_v"], inf["n_grid"], inf["P"], 4) \
        - (BATCH_RHS - 1) * 4 * (inf["P"] // 2 + 1) ** 2        # the symbol is read once per batch
    hbm = peaks().get("hbm_gbs", 6800.0)
    nsolves = len(all_specs) * BATCH_RHS                # all ranks together
    t_max = max_over_ranks(t_batch, world, dev)
    t_single = max_over_ranks(t_single, world, dev)
    t_e2e = max_over_ranks(t_e2e, world, dev)
    result = {
        "solves_per_s": round(nsolves / t_max, 3), "s_per_batch": round(t_max, 4), "steps": steps, "warmup": warm,
        "worst_rel_res_fp64": worst,
        "config": {"workload": WORKLOADS["batch48"], "instances": len(all_specs), "rhs_per_instance": BATCH_RHS,
                   "grids": {str(k): sum(r["n"] == k for r in rows) for k in (256, 512, 1024, 2048)},
                   "groups": gtune, "group_note": "Group autotune ms per product of all the group's columns",
                   "l2": "inputs larger than L2 for the large instances; no flush between solves",
                   "build_s": round(t_build, 2), "autotune_s": round(t_tune, 2)},
        "one_at_a_time_fp64": {
            "s": round(t_single, 3), "solves_per_s": round(nsolves / t_single, 3),
            "speedup_batched_mixed": round(t_single / t_max, 3),
            "sample": "all %d right-hand sides" % nsolves if single == "all" else
            "%d solves (column i mod 8 of instance i), time scaled by 8 to the %d right-hand sides"
            % (n_single, len(probs) * BATCH_RHS)},
        "e2e": {"value": round(nsolves / t_e2e, 3), "unit": "solves/s",
                "h2d_bytes_per_step": int(sum(f.numel() * 8 for f in Fh)),
                "d2h_bytes_per_step": int(sum(u.numel() * 8 for u in Uh))},
        "roofline": {"bound": "hbm", "kernel": "batched FP32 product (8 columns), largest instance",
                     "instance": rows[big], "achieved": round(B / (ms * 1e-3) / 1e9, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(B / (ms * 1e-3) / 1e9 / hbm, 4), "traffic": None,
                     "ms": round(ms, 4)},
        "instances": rows}
    for g in groups.values():
        g.close()
    for pr in probs:
        pr.close()
    return result


def run_batch(args):
    """The batched workload as its own line (all 384 one-at-a-time solves)."""
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    clocks = Clocks(local)
    r = batch_workload(dev, rank, world, warm=max(1, min(args.warmup, 1)), steps=max(1, min(args.steps, 2)),
                       single="all")
    clk = clocks.stop()
    if rank == 0:
        line = {"metric": BATCH_METRIC, "value": r["solves_per_s"], "unit": "solves/s", "n_gpus": world,
                "steps": r["steps"], "warmup": r["warmup"], "ms_per_step": round(1e3 * r["s_per_batch"], 2),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 refinement)",
                "data": "synthetic (seeded jittered Delaunay disks and L-shapes, f=1 + Gaussian bumps)",
                "config": r["config"], "worst_rel_res_fp64": r["worst_rel_res_fp64"],
                "one_at_a_time_fp64": r["one_at_a_time_fp64"], "e2e": r["e2e"], "roofline": r["roofline"],
                "instances": r["instances"], "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gofd", choices=["gofd", "reference"])
    ap.add_argument("--no-pcg", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="lshape1024", choices=sorted(WORKLOADS))
    ap.add_argument("--grid", type=int, default=0,
                    help="replace the workload's grid size (a smaller case for profiling; not a bench line)")
    ap.add_argument("--shapes", default="",
                    help="launch shapes lines,cols,lanes,col_elems,row_elems,batch_chunk instead of autotuning")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch48":
        return run_batch(args)
    return run_gofd(args)


if __name__ == "__main__":
    sys.exit(main())
