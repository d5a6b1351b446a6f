"""Benchmark: 256^2 RGB restorations/s of the i-DEQ inertial solver on GB300.

Workload (one step = one full solve of one batch): 8 RGB 256x256 synthetic
images under per-image 25x25 random-walk motion blur, noise sigma 0.02, 4-scale
residual U-Net regulariser (64/128/256/512, 17.0 M seeded random weights),
lambda 0.1, tau 0.75, beta 0.8, solved from x0 = A^T y to the relative
fixed-point residual 1e-4 (App. D.1.3).  The chosen form runs the network
convolutions with FP16 operands (FP32 accumulation) on the tcgen05 tensor
cores -- BF16 operands stall above that residual -- and the plain form is FP32
throughout.  Inputs are synthetic (seeded), weights random-init.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is device-timed (CUDA events, inputs resident in
HBM); `e2e` times the same solve through the C ABI with the observations copied
from pinned host memory and the restorations copied back, every step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "256² RGB restorations/s at matched PSNR (±0.05 dB), chosen form vs plain FP32"
WORKLOADS = {
    "C1a": "C1a: 8 x RGB 256x256, 25x25 random-walk motion blur, sigma 0.02, "
           "U-Net 64/128/256/512 (17.0M params), lambda 0.1, tau 0.75, beta 0.8, tol 1e-4",
    "C1b": "C1b: 8 x RGB 256x256 inpainting (30% of pixels kept), sigma 0.02, "
           "U-Net 64/128/256/512, lambda 0.1, tau 0.75, beta 0.8, tol 1e-4",
    "C5": "C5: 4 x complex 256x256 MRI (x4 Cartesian undersampling, 8% centre), "
          "k-space sigma 0.01, 2-channel U-Net 32/64/128/256, lambda 0.1, tau 0.75, beta 0.8, tol 1e-4",
    "C6": "C6: 4 x grey 256x256 Rician denoising, sigma 0.1, U-Net 32/64/128/256, "
          "lambda 0.1, tau 0.009, beta 0.8, tol 1e-4",
    "C4": "C4: 32 x RGB 256x256, A(x) = tanh(2 k*x)/tanh 2 with 15x15 Gaussian k (sigma 2), "
          "sigma 0.01, U-Net 64/128/256/512, lambda 0.1, tau 0.2, beta 0.8, tol 1e-4; "
          "warm start 3-48-48-48-48-48-3 ReLU CNN trained on FP16-solver equilibria",
}
WORKLOADS["C3"] = ("C3: DEQ training step on 16 x RGB 128x128 patches, 9x9 Gaussian blur "
                   "sigma U[0.5,3], noise U[0.005,0.05], U-Net 32/64/128/256 (4.25M params); "
                   "forward solve to 1e-3, implicit adjoint to 1e-3, one Adam step")
WARM_TRAIN_IMAGES = 512   # held-out equilibria the warm start is trained on
WARM_TRAIN_STEPS = 600    # Adam steps (batch 8, lr 1e-3)
WORKLOAD = WORKLOADS["C1a"]
CONV_REPS = 20  # repetitions of the conv launch sequence in the roofline timing
UPDATE_REPS = 60  # timed calls of the update pass


def make_op_and_y(B, cfg, wl, ctx, x_true, dev):
    """The forward model of the workload and y = A(x*) + n formed on the device by
    the library (inpainting: y = M(x* + n); MRI: y = M(F x* + n))."""
    import torch
    noise = torch.tensor(wl["noise"], device=dev)
    if cfg["op"] == "mask":
        op = B.make_operator(B.IDEQ_OP_MASK, None, torch.tensor(wl["mask"], device=dev))
        return op, B.ideq_apply_A(ctx, op, x_true + noise)
    if cfg["op"] == "mri":
        m = torch.tensor(wl["mask"], device=dev)
        op = B.make_operator(B.IDEQ_OP_MRI, None, m)
        return op, B.ideq_apply_A(ctx, op, x_true) + noise * m[:, None].float()
    if cfg["op"] == "rician":  # y = |x + n_re + i n_im|
        op = B.make_operator(B.IDEQ_OP_RICIAN, sigma=cfg["noise_sigma"])
        return op, torch.sqrt((x_true + noise[:, 0]) ** 2 + noise[:, 1] ** 2).contiguous()
    op = B.make_operator(B.IDEQ_OP_BLUR, torch.tensor(wl["kern"], device=dev))
    return op, B.ideq_apply_A(ctx, op, x_true) + noise


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparison solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--ncu-steps", type=int, default=0,
                    help="profiling mode: run this many inertial steps of the batch and exit "
                         "(no timing, no JSON), for ncu captures")
    ap.add_argument("--precision", default="fp16", choices=["fp16", "bf16", "fp32"],
                    help="convolution arithmetic of the profiling mode")
    ap.add_argument("--batch", type=int, default=0, help="profiling mode: batch size override")
    ap.add_argument("--workload", default="C1a", choices=sorted(WORKLOADS),
                    help="synthetic workload (default: the 8 x RGB 256^2 motion-blur batch)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(vals, device=None):
    """Element-wise max over all ranks of a list of floats; the values themselves
    on a single process.  Every rank must call it (it is a collective)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in vals]
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_rate(world, units_per_rank, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "conv_tc_c1a_fp16_traffic.md")
KERNEL_SRC = os.path.join(ROOT, "paper_2605_19705_gb300", "csrc", "conv_tc.cu")


def recorded_traffic():
    """Per-launch DRAM bytes (read + write) of the tcgen05 conv from the committed
    ncu capture, or None when the kernel source changed since it was taken."""
    import hashlib
    try:
        rec = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if ":" in line and line.split(":")[0].strip() in ("per_launch_bytes",
                                                                  "kernel_source_sha256"):
                    k, v = line.split(":", 1)
                    rec[k.strip()] = v.strip().strip("`")
        with open(KERNEL_SRC, "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()
        if rec.get("kernel_source_sha256") != h:
            return None
        return float(rec["per_launch_bytes"])
    except (OSError, KeyError, ValueError):
        return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms in the background."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def bench_config(name, cfg, world):
    """The `config` object of the JSON line (the same for both arms)."""
    return {"workload": WORKLOADS[name], "batch_per_gpu": cfg["n"],
            "image": f"{cfg['c']}x{cfg['h']}x{cfg['w']}",
            "form": "fp16 tcgen05 convolutions (fp32 accumulate), fp32 iterate and data step, "
                    "fp64 reductions, x0 = A^T y",
            "parallelism": f"replicas x{world} (independent batches)",
            "l2": "working set ~1.5 GB per solve (> 129 MB L2); no flush needed"}


def load_workload(n_override=None, name="C1a"):
    import numpy as np
    from synth import get_config, workload
    cfg = get_config(name)
    if n_override:
        cfg["n"] = n_override
    wl = workload(cfg)
    return cfg, wl, np


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2605_19705_gb300 import build as pbuild
    pbuild.build()
    from paper_2605_19705_gb300 import binding as B

    cfg, wl, _ = load_workload(name=args.workload)
    n = cfg["n"]
    dev = torch.device("cuda", local)
    weights = torch.tensor(wl["weights"], device=dev)
    desc = B.net_desc(cfg["net"], cfg["c"])
    # observations y = A(x*) + n formed on the device by the library's forward model
    x_true = torch.tensor(wl["x_true"], device=dev)
    ctx = B.Context(desc, weights, B.IDEQ_FP16)
    op, y = make_op_and_y(B, cfg, wl, ctx, x_true, dev)
    params = B.make_params(cfg["lam"], cfg["tau"], cfg["beta"], cfg["B"], cfg["tol"],
                           cfg["max_iter"])
    info = B.InfoBuffers(n, dev)
    out = torch.empty_like(y)
    st = torch.cuda.current_stream()

    def solve_once():
        B.ideq_solve(ctx, op, y, params, out=out, info=info)

    def psnr(x):
        mse = ((x.double() - x_true.double()) ** 2).mean(dim=(1, 2, 3))
        return (10 * torch.log10(1.0 / mse)).cpu().numpy()

    for _ in range(args.warmup):
        solve_once()
    torch.cuda.synchronize()
    B.ideq_launch_count(ctx)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    iters = []
    for _ in range(args.steps):
        solve_once()
        iters.append(info.iters.clone())
    e1.record(st)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    launches = B.ideq_launch_count(ctx)
    ms = reduce_max([ms], dev)[0]
    psnr_c = psnr(out)
    iters_t = torch.stack(iters).cpu()
    it_c = iters_t.float().mean().item()
    # roofline of the conv kernel: the tcgen05 conv launches of one regulariser
    # evaluation, back to back as in the solve (programmatic dependent launch kept),
    # CONV_REPS times between one pair of CUDA events on the solve's stream
    conv_ms, conv_launches, conv_flops = B.ideq_time_convs(ctx, CONV_REPS)
    B.ideq_launch_count(ctx)
    # work of one timed solve: the loop runs until the last image stops (checked
    # after every iteration) and the convolutions skip frozen images, so the conv
    # work is the method's own, sum_i iters_i x the FLOPs of one image-iteration
    it_max = int(iters_t.max())
    executed_iters = it_max
    per_image_iter_flops = B.ideq_plan_flops(ctx) / n
    image_iters_per_step = float(iters_t.sum()) / args.steps
    algo_flops_per_step = image_iters_per_step * per_image_iter_flops

    # ---- the fused update pass alone (x_new = z - tau (grad f + lambda grad g) with the
    # FP64 step norms), through the allocation-free entry point on buffers of this
    # batch's size; six buffer sets in rotation exceed L2, so every call reads HBM
    sets = [[torch.rand_like(y) for _ in range(5)] for _ in range(6)]
    nrm = torch.zeros(2, n, dtype=torch.float64, device=dev)
    for k in range(6):
        z_, f_, g_, x_, o_ = sets[k]
        B.ideq_red_update_noalloc(z_, f_, g_, x_, o_, 0.1, 0.75, nrm[0], nrm[1])
    torch.cuda.synchronize()
    # the calls are captured in one CUDA graph, so the host's per-call cost (larger
    # than the kernel's ~10 us) is not what the events time
    ug = torch.cuda.CUDAGraph()
    with torch.cuda.graph(ug):
        for k in range(UPDATE_REPS):
            z_, f_, g_, x_, o_ = sets[k % 6]
            B.ideq_red_update_noalloc(z_, f_, g_, x_, o_, 0.1, 0.75, nrm[0], nrm[1])
    ug.replay()
    torch.cuda.synchronize()
    u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    u0.record(st)
    ug.replay()
    u1.record(st)
    torch.cuda.synchronize()
    upd_ms = u0.elapsed_time(u1) / UPDATE_REPS
    del ug
    upd_bytes = 5 * y.numel() * 4
    del sets

    # ---- end to end through the C ABI: pinned host y in, x_hat out, every step
    y_host = y.cpu().pin_memory()
    x_host = torch.empty_like(y_host).pin_memory()
    y_dev = torch.empty_like(y)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        y_dev.copy_(y_host, non_blocking=True)
        B.ideq_solve(ctx, op, y_dev, params, out=out, info=info)
        x_host.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s = reduce_max([e2e_s], dev)[0]
    e2e_bytes = y_host.numel() * 4

    # ---- plain FP32 form, same inputs (one solve) for the matched-PSNR comparison
    plain = None
    if not args.no_plain and rank == 0:
        ctx32 = B.Context(desc, weights, B.IDEQ_FP32)
        info32 = B.InfoBuffers(n, dev)
        out32 = torch.empty_like(y)
        B.ideq_solve(ctx32, op, y, params, out=out32, info=info32)  # warm-up / plan build
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(st)
        B.ideq_solve(ctx32, op, y, params, out=out32, info=info32)
        a1.record(st)
        torch.cuda.synchronize()
        pms = a0.elapsed_time(a1)
        p32 = psnr(out32)
        rel = float(((out.double() - out32.double()).norm() / out32.double().norm()).item())
        fma = B.ideq_fp32_fma_peak()
        plain_flops = float(info32.iters.sum().item()) * B.ideq_plan_flops(ctx32) / n
        plain = {"value": n / (pms / 1e3), "unit": "restorations/s", "ms_per_solve": pms,
                 "mean_iters": float(info32.iters.float().mean().item()),
                 "psnr_db_mean": float(p32.mean()),
                 "max_abs_psnr_delta_db": float(np.max(np.abs(psnr_c - p32))),
                 "rel_l2_chosen_vs_plain": rel,
                 "roofline": {"bound": "alu", "achieved": plain_flops / (pms / 1e3) / 1e12,
                              "peak": fma, "unit": "TFLOP/s",
                              "frac": plain_flops / (pms / 1e3) / 1e12 / fma,
                              "peak_source": "FP32 FFMA microbenchmark (ideq_fp32_fma_peak, "
                                             "measured in this run)",
                              "work": "sum over images of iterations x conv FLOPs per image"}}
        ctx32.close()

    peaks, src = measured_peaks()
    achieved = conv_flops / (conv_ms / 1e3) / 1e12 if conv_ms > 0 else 0.0
    # the convs are timed back to back at full clocks: the burst peak
    peak = float(peaks.get("bf16_tflops", peaks.get("bf16_tflops_sustained")))
    peak_sus = float(peaks.get("bf16_tflops_sustained", peak))
    avg_launch_ms = conv_ms / max(conv_launches, 1)
    # conv time of one step: the timed full-batch evaluation scaled to the images
    # that were still running (an estimate: tile waves do not scale exactly)
    conv_ms_per_step = conv_ms / CONV_REPS * image_iters_per_step / n
    step_tflops = algo_flops_per_step / (ms / args.steps / 1e3) / 1e12
    value = job_rate(world, n * args.steps, ms / 1e3)
    res = {
        "metric": METRIC, "value": value, "unit": "restorations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16",
        "data": "synthetic (seeded images, kernels, noise; random-init U-Net weights)",
        "config": bench_config(args.workload, cfg, world),
        "mean_iters": it_c, "psnr_db_mean": float(psnr_c.mean()),
        "e2e": {"value": job_rate(world, n * args.steps, e2e_s), "unit": "restorations/s",
                "h2d_bytes_per_step": e2e_bytes, "d2h_bytes_per_step": e2e_bytes},
        "gpu_launches": launches,
        "roofline": {"bound": "tensor", "kernel": "conv_tc_kernel (all tcgen05 conv launches)",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None, "traffic": recorded_traffic(),
                     "traffic_unit": "bytes per launch (ncu dram__bytes_read+write)",
                     "peak_source": f"bf16_tflops burst ({src}); FP16 operands run at the BF16 rate",
                     "frac_of_sustained": achieved / peak_sus if peak_sus else None,
                     "launches_timed": conv_launches, "avg_launch_ms": avg_launch_ms,
                     "timing": f"CUDA events around {CONV_REPS} back-to-back repetitions of one "
                               "regulariser evaluation's tcgen05 conv launches on the solve's "
                               "stream (programmatic dependent launch kept), after the timed region",
                     "conv_ms_per_step": conv_ms_per_step,
                     "conv_ms_per_step_basis": "full-batch conv time x (sum of image "
                                               "iterations / batch)",
                     "executed_iters_per_step": executed_iters,
                     "image_iters_per_step": image_iters_per_step,
                     "step_flop_frac": step_tflops / peak if peak else None,
                     "step_tflops": step_tflops,
                     "step_work": "sum over images of their iterations x conv FLOPs per image "
                                  "iteration (frozen images' work not counted), per timed step"},
        "clocks": clk,
        "update_pass": {"bound": "hbm", "achieved": upd_bytes / (upd_ms / 1e3) / 1e9,
                        "peak": float(peaks.get("hbm_gbs", 6800.0)), "unit": "GB/s",
                        "frac": upd_bytes / (upd_ms / 1e3) / 1e9 / float(peaks.get("hbm_gbs", 6800.0)),
                        "us_per_pass": upd_ms * 1e3, "bytes_per_pass": upd_bytes,
                        "timing": f"CUDA events around one replay of a CUDA graph of "
                                  f"{UPDATE_REPS} calls of ideq_red_update_noalloc "
                                  "(red_update_kernel + per-image norm sums) rotating over 6 "
                                  "buffer sets (> L2)"},
    }
    if plain:
        res["plain_fp32"] = plain
        res["speedup_vs_plain_fp32"] = value / world / plain["value"]
    if rank == 0 and not args.no_cpu:
        res["cpu_baseline"] = cpu_baseline(it_c, args.workload)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline(iters_per_image, name="C1a"):
    """The FP64 oracle timed on the host cores on a bounded sample (one inertial
    step of one 256^2 image of the same workload), extrapolated to
    restorations/s with the iteration count per image."""
    import numpy as np
    from oracle import nets, operators, solver
    cfg, wl, _ = load_workload(name=name)
    net = nets.Net.from_config(cfg["net"], cfg["c"], wl["weights"])
    ops = operators.make_operators(cfg, wl)
    y0 = operators.observe(ops[:1], wl["x_true"][:1], wl["noise"][:1])[0]
    x0 = ops[0].AT(y0)
    t0 = time.perf_counter()
    solver.red_step(net, ops[0], y0, x0, cfg["lam"], cfg["tau"])
    dt = time.perf_counter() - t0
    return {"value": 1.0 / (dt * iters_per_image), "unit": "restorations/s",
            "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"1 inertial step of 1 image ({cfg['c']}x{cfg['h']}x{cfg['w']}) = {dt:.2f} s, extrapolated "
                      f"to {iters_per_image:.1f} iterations per restoration"}


def run_profile_steps(args):
    """Plan set-up plus args.ncu_steps inertial steps (ideq_step) of the benchmark
    batch; the target of the ncu captures summarised under profiles/."""
    import torch
    from paper_2605_19705_gb300 import build as pbuild
    pbuild.build()
    from paper_2605_19705_gb300 import binding as B
    cfg, wl, _ = load_workload(args.batch or None, name=args.workload)
    prec = {"fp16": B.IDEQ_FP16, "bf16": B.IDEQ_BF16, "fp32": B.IDEQ_FP32}[args.precision]
    ctx = B.Context(B.net_desc(cfg["net"], cfg["c"]), torch.tensor(wl["weights"], device="cuda"),
                    prec)
    xt = torch.tensor(wl["x_true"], device="cuda")
    op, y = make_op_and_y(B, cfg, wl, ctx, xt, "cuda")
    xk = B.ideq_apply_AT(ctx, op, y)
    if args.workload == "C3":  # the parameter gradient: JFB backward passes at A^T y
        v = (2.0 * (xk - xt) / xk.numel()).contiguous()
        g = torch.zeros(wl["weights"].size, device="cuda")
        dl = torch.zeros(1, device="cuda")
        p = B.make_params(cfg["lam"], cfg["tau"], cfg["beta"])
        for _ in range(args.ncu_steps):
            B.ideq_solve_backward(ctx, op, y, xk, v, p, B.make_adj(B.IDEQ_ADJ_JFB), g, dl)
        torch.cuda.synchronize()
        return
    xkm1 = xk.clone()
    params = B.make_params(cfg["lam"], cfg["tau"], cfg["beta"])
    for _ in range(args.ncu_steps):
        B.ideq_step(ctx, op, y, xk, xkm1, params)
    torch.cuda.synchronize()


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import numpy as np
    from oracle import nets, operators, solver
    cfg, wl, _ = load_workload()
    net = nets.Net.from_config(cfg["net"], cfg["c"], wl["weights"])
    ops = operators.make_operators(cfg, wl)
    y0 = operators.observe(ops[:1], wl["x_true"][:1], wl["noise"][:1])[0]
    x = ops[0].AT(y0)
    xp = x.copy()
    gold = os.path.join(ROOT, "tests", "golden", "c1a_oracle_iters.json")
    iters = None
    if os.path.exists(gold):
        with open(gold) as f:
            g = json.load(f)
        iters = float(np.mean([im["iters"] for im in g["images"]]))
    for _ in range(args.warmup):
        solver.red_step(net, ops[0], y0, x, cfg["lam"], cfg["tau"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        z = x + cfg["beta"] * (x - xp)
        xp, x = x, solver.red_step(net, ops[0], y0, z, cfg["lam"], cfg["tau"])[0]
    dt = (time.perf_counter() - t0) / args.steps
    it = iters if iters else float("nan")
    v = 1.0 / (dt * it)
    res = {"impl": "reference", "metric": METRIC, "value": v, "unit": "restorations/s",
           "n_gpus": world, "device": "host cores (FP64 oracle)", "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config("C1a", cfg, world),
           "cpu_baseline": {"kind": "oracle", "cores": os.cpu_count(), "value": v,
                            "unit": "restorations/s",
                            "sample": f"each step = 1 inertial step of 1 image (3x256x256) "
                                      f"in FP64 NumPy, extrapolated with {it} iterations per "
                                      f"restoration (oracle solve of the same workload)"},
           "e2e": {"value": v, "unit": "restorations/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(res), flush=True)


def run_warm(args):
    """C4: the learned warm start on the saturation workload.  Trains W_phi with the
    library's own kernels on equilibria that the plain FP16 solver produces for
    WARM_TRAIN_IMAGES held-out images (seeds disjoint from the benchmark batch),
    then solves the 32-image benchmark batch from A^T y (plain) and from the warm
    start, both to the same relative step 1e-4, and reports restorations/s,
    iterations and PSNR of both (and of the plain FP32 form)."""
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2605_19705_gb300 import build as pbuild
    pbuild.build()
    from paper_2605_19705_gb300 import binding as B
    from paper_2605_19705_gb300 import warmstart as W
    from synth import get_config, workload
    cfg, wl, _ = load_workload(name="C4")
    n = cfg["n"]
    dev = torch.device("cuda", local)
    desc = B.net_desc(cfg["net"], cfg["c"])
    ctx = B.Context(desc, torch.tensor(wl["weights"], device=dev), B.IDEQ_FP16)
    wdesc = B.net_desc(cfg["warm"], cfg["c"])
    W.warm_set(ctx, wdesc, torch.tensor(wl["warm_weights"], device=dev))
    params = B.make_params(cfg["lam"], cfg["tau"], cfg["beta"], cfg["B"], cfg["tol"],
                           cfg["max_iter"])
    # ---- training set: equilibria of the plain FP16 solver on held-out images
    t0 = time.perf_counter()
    atys, xbars, it_tr = [], [], []
    for b in range(WARM_TRAIN_IMAGES // n):
        tc = get_config("C4", seeds=dict(img=20000 + n * b, noise=21000 + n * b, weights=2001,
                                        kernel=0, mask=0, warm=2004))
        twl = workload(tc)
        op_b = B.make_operator(B.IDEQ_OP_SATBLUR, torch.tensor(twl["kern"], device=dev),
                               sat_gain=tc["sat_gain"])
        y_b = B.ideq_apply_A(ctx, op_b, torch.tensor(twl["x_true"], device=dev)) + \
            torch.tensor(twl["noise"], device=dev)
        info_b = B.InfoBuffers(n, dev)
        x_b, _ = B.ideq_solve(ctx, op_b, y_b, params, info=info_b)
        atys.append(B.ideq_apply_AT(ctx, op_b, y_b))
        xbars.append(x_b.clone())
        it_tr.append(info_b.iters.float().mean().item())
    atys, xbars = torch.cat(atys), torch.cat(xbars)
    torch.cuda.synchronize()
    t_eq = time.perf_counter() - t0
    t0 = time.perf_counter()
    hist = W.train(ctx, atys, xbars, steps=WARM_TRAIN_STEPS, lr=1e-3, batch=8)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del atys, xbars
    # ---- the benchmark batch: plain vs warm start at equal residual
    x_true = torch.tensor(wl["x_true"], device=dev)
    op = B.make_operator(B.IDEQ_OP_SATBLUR, torch.tensor(wl["kern"], device=dev),
                         sat_gain=cfg["sat_gain"])
    y = B.ideq_apply_A(ctx, op, x_true) + torch.tensor(wl["noise"], device=dev)
    st = torch.cuda.current_stream()

    def psnr(x):
        mse = ((x.double() - x_true.double()) ** 2).mean(dim=(1, 2, 3))
        return (10 * torch.log10(1.0 / mse)).cpu().numpy()

    res = {}
    for name, init in (("plain", B.IDEQ_INIT_ATY), ("warm", B.IDEQ_INIT_WARM)):
        p = B.make_params(cfg["lam"], cfg["tau"], cfg["beta"], cfg["B"], cfg["tol"],
                          cfg["max_iter"], init)
        info = B.InfoBuffers(n, dev)
        out = torch.empty_like(y)
        for _ in range(args.warmup):
            B.ideq_solve(ctx, op, y, p, out=out, info=info)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its = []
        e0.record(st)
        for _ in range(args.steps):
            B.ideq_solve(ctx, op, y, p, out=out, info=info)
            its.append(info.iters.clone())
        e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        it = torch.stack(its).float()
        res[name] = {"value": n / (ms / 1e3), "unit": "restorations/s", "ms_per_solve": ms,
                     "mean_iters": it.mean().item(), "max_iters": int(it.max().item()),
                     "max_rel_res": float(info.rel_res.max().item()),
                     "psnr_db_mean": float(psnr(out).mean()), "x": out.clone()}
    aty = B.ideq_apply_AT(ctx, op, y)
    x0w = W.warm_forward(ctx, aty)
    xp = res["plain"]["x"]
    e_aty = float((aty - xp).norm() / xp.norm())
    e_warm = float((x0w - xp).norm() / xp.norm())
    dpsnr = float(np.max(np.abs(psnr(res["warm"]["x"]) - psnr(xp))))
    # plain FP32 form, one solve
    ctx32 = B.Context(desc, torch.tensor(wl["weights"], device=dev), B.IDEQ_FP32)
    info32 = B.InfoBuffers(n, dev)
    out32 = torch.empty_like(y)
    B.ideq_solve(ctx32, op, y, params, out=out32, info=info32)
    torch.cuda.synchronize()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(st)
    B.ideq_solve(ctx32, op, y, params, out=out32, info=info32)
    a1.record(st)
    torch.cuda.synchronize()
    pms = a0.elapsed_time(a1)
    for r in res.values():
        r.pop("x")
    line = {
        "metric": "256² RGB restorations/s at equal residual, FP16 + learned warm start vs "
                  "FP16 from A^T y vs plain FP32",
        "value": res["warm"]["value"], "unit": "restorations/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["warm"]["ms_per_solve"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16",
        "data": "synthetic (seeded images, noise; random-init U-Net and warm-start weights)",
        "config": {"workload": WORKLOADS["C4"], "batch_per_gpu": n, "image": "3x256x256"},
        "warm_start": {"train_images": WARM_TRAIN_IMAGES, "train_steps": WARM_TRAIN_STEPS,
                       "train_loss_first_last": [hist[0], hist[-1]],
                       "train_mean_iters": float(np.mean(it_tr)),
                       "seconds_equilibria": t_eq, "seconds_training": t_train,
                       "x0_rel_err_aty": e_aty, "x0_rel_err_warm": e_warm,
                       "iterations_saved_mean": res["plain"]["mean_iters"] - res["warm"]["mean_iters"],
                       "max_abs_psnr_delta_db": dpsnr},
        "fp16_plain": res["plain"], "fp16_warm": res["warm"],
        "plain_fp32": {"value": n / (pms / 1e3), "unit": "restorations/s", "ms_per_solve": pms,
                       "mean_iters": float(info32.iters.float().mean().item()),
                       "psnr_db_mean": float(psnr(out32).mean())},
        "speedup_vs_plain_fp32": res["warm"]["value"] / (n / (pms / 1e3)),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_train(args):
    """C3: DEQ training steps of the regulariser (App. D.1.2-D.1.3) through
    ideq_train_step -- forward solve to 1e-3, MSE loss against the ground truth,
    implicit adjoint solve to 1e-3, parameter gradient (tcgen05 weight gradients),
    one Adam step -- timed with CUDA events; then the weight-gradient pass alone
    (ideq_time_wgrad) for its roofline."""
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2605_19705_gb300 import build as pbuild
    pbuild.build()
    from paper_2605_19705_gb300 import binding as B
    cfg, wl, _ = load_workload(name="C3")
    n = cfg["n"]
    dev = torch.device("cuda", local)
    ctx = B.Context(B.net_desc(cfg["net"], cfg["c"]), torch.tensor(wl["weights"], device=dev),
                    B.IDEQ_FP16)
    op = B.make_operator(B.IDEQ_OP_BLUR, torch.tensor(wl["kern"], device=dev))
    x_true = torch.tensor(wl["x_true"], device=dev)
    y = B.ideq_apply_A(ctx, op, x_true) + torch.tensor(wl["noise"], device=dev)
    params = B.make_params(cfg["lam"], cfg["tau"], cfg["beta"], cfg["B"], cfg["tol"],
                           cfg["max_iter"])
    # the adjoint iteration u <- J_R^T u + v with the forward's heavy-ball inertia
    # (its fixed point is the implicit gradient's; plain iteration crawls along the
    # directions the blur removes, where J_R's eigenvalues approach 1)
    adj = B.make_adj(B.IDEQ_ADJ_IMPLICIT, cfg["adj_tol"], 3000, cfg["beta"])
    lr = 1e-5
    info = B.InfoBuffers(n, dev)
    binfo_iters = []
    x = torch.empty_like(y)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        B.ideq_train_step(ctx, op, y, x_true, params, adj, lr, x_out=x, loss=loss, info=info)
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fw_iters, losses = [], []
    e0.record(st)
    for _ in range(args.steps):
        B.ideq_train_step(ctx, op, y, x_true, params, adj, lr, x_out=x, loss=loss, info=info)
        fw_iters.append(info.iters.clone())
        losses.append(loss.clone())
    e1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    # the backward alone (adjoint iterations per image from its info) and the
    # weight-gradient pass alone
    binfo = B.InfoBuffers(n, dev)
    v = (2.0 * (x - x_true) / x.numel()).contiguous()
    g = torch.zeros(wl["weights"].size, device=dev)
    dl = torch.zeros(1, device=dev)
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(st)
    B.ideq_solve_backward(ctx, op, y, x, v, params, adj, g, dl, binfo)
    b1.record(st)
    torch.cuda.synchronize()
    bwd_ms = b0.elapsed_time(b1)
    wg_ms, wg_flops, wg_tc = B.ideq_time_wgrad(ctx, 10)
    peaks, src = measured_peaks()
    peak = float(peaks.get("bf16_tflops", peaks.get("bf16_tflops_sustained")))
    wg_tflops = wg_flops / (wg_ms / 1e3) / 1e12
    line = {
        "metric": "DEQ training steps/s (forward solve + implicit adjoint + Adam), 16 x RGB 128^2",
        "value": 1e3 / ms, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16",
        "data": "synthetic (seeded patches, kernels, noise; random-init U-Net weights)",
        "config": {"workload": WORKLOADS["C3"], "batch_per_gpu": n, "image": "3x128x128",
                   "lr": lr, "adjoint": "implicit, u <- J_R^T u + v with heavy-ball beta "
                                        f"{cfg['beta']}, tol 1e-3"},
        "images_per_s": n * 1e3 / ms,
        "forward_mean_iters": float(torch.stack(fw_iters).float().mean().item()),
        "adjoint_mean_iters": float(binfo.iters.float().mean().item()),
        "backward_ms": bwd_ms,
        "loss_first_last": [float(losses[0].item()), float(losses[-1].item())],
        "wgrad": {"bound": "tensor", "achieved": wg_tflops, "peak": peak, "unit": "TFLOP/s",
                  "frac": wg_tflops / peak, "ms_per_pass": wg_ms / 10,
                  "tensor_core_convs": wg_tc,
                  "timing": "CUDA events around 10 weight-gradient passes of the last backward"
                            f" (both products per conv); peak: bf16_tflops burst ({src})"},
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.ncu_steps > 0:
        run_profile_steps(a)
    elif a.impl == "ours" and a.workload == "C4":
        run_warm(a)
    elif a.impl == "ours" and a.workload == "C3":
        run_train(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
