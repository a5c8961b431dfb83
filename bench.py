"""Throughput benchmark of the Legendre-coefficient path on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload NAME] [--path split_fp16|f32|bf16|f64]

One step = one forward pass of the sampled-input path over one batch with
inputs resident in HBM: input split -> tcgen05 Abel GEMM -> twisted FFT with
the (2n+1) scaling (leg_forward).  The default workload is B=4096 random
decaying Chebyshev series at K=1025 Chebyshev-Lobatto nodes, N=512
coefficients, M=2048 trapezoid points (exact tau rule), on the split-FP16 path
whose error against the FP64 oracle is measured in the same run.

Timing: W untimed warm-up steps; then, for each of K steps, L2 is flushed
(a 512 MiB write) and the step is timed with CUDA events recorded by the
library on the launch stream between its stages (leg_forward_profiled).
Barrier + synchronize bracket the timed steps; the max over ranks is taken.
Under torchrun (N > 1) every rank runs its own batch (weak scaling, no
collective on the data path).

--impl reference times the FP64 CPU oracle (the paper's method written out
directly, route 2) on the host cores, on a bounded sample of the same
workload per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "Legendre coeffs/sec (B*N/s) at <=1e-6 rel err vs FP64 oracle; % roofline vs plain FP64"
UNIT = "coeffs/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cheb_b4096_k1025_n512_m2048")
    ap.add_argument("--path", default="split_fp16", choices=["split_fp16", "f32", "bf16", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64/FP32 comparison paths")
    return ap.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str):
        self.gpu = gpu_index
        self.proc = None
        # LEG_CLOCKS_DIR keeps the raw samples; otherwise they go to the temp directory
        out = os.environ.get("LEG_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, "clocks_bench_%s_%d.csv" % (gpu_index, os.getpid()))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def wait_first(self, timeout: float = 3.0):
        """Block until the sampler has written its first sample (so that the
        samples cover the work that follows), at most `timeout` seconds."""
        t0 = time.time()
        while self.proc is not None and time.time() - t0 < timeout:
            self.fh.flush()
            if os.path.getsize(self.path) > 0:
                return
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        return parse_clocks(self.path)


def parse_clocks(path: str):
    """Median SM clock, maximum clock and the throttle reasons seen in a CSV
    of ClockSampler.FIELDS rows (None without a valid row)."""
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    with open(path) as fh:
        for line in fh:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle (CPU)
def oracle_rate(name: str, seconds: float = 12.0, max_fns: int = 256):
    """Route 2 of the FP64 oracle on a bounded sample of the workload."""
    from oracle import oracle as O
    cfg = workloads.CONFIGS[name]
    N, M, K = cfg["N"], cfg["M"], cfg["K"]
    Q = O.exact_tau_points(K)
    f = workloads.workload_inputs(name).astype(np.float64)
    n = 2
    t0 = time.time()
    O.coeffs_abel(N, M, Q, f_cl=f[:n])
    dt = time.time() - t0
    # the cost is dominated by the per-point barycentric weights (shared by the
    # functions of one call), so grow the sample while it fits the budget
    while dt < seconds / 3 and n < max_fns:
        n = min(max_fns, n * 4)
        t0 = time.time()
        O.coeffs_abel(N, M, Q, f_cl=f[:n])
        dt = time.time() - t0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": n * N / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of %d functions of %s, oracle route 2 (Abel + trapezoid, direct Fourier sum), "
                      "FP64, OpenMP, %.2f s" % (n, cfg["B"], name, dt)}, n, dt


def reference_arm(args, rank, world):
    if rank != 0:
        return
    name = args.workload
    cfg = workloads.CONFIGS[name]
    from oracle import oracle as O
    N, M, K = cfg["N"], cfg["M"], cfg["K"]
    Q = O.exact_tau_points(K)
    f = workloads.workload_inputs(name).astype(np.float64)
    # size one step to about 2 s of CPU work, and all steps to about a minute
    base, n, dt = oracle_rate(name, seconds=6.0, max_fns=64)
    per_fn = dt / n
    budget = min(2.0, 60.0 / max(1, args.steps + args.warmup))
    S = max(1, min(cfg["B"], int(budget / max(per_fn, 1e-9))))
    for _ in range(args.warmup):
        O.coeffs_abel(N, M, Q, f_cl=f[:S])
    times = []
    for i in range(args.steps):
        lo = (i * S) % max(1, cfg["B"] - S + 1)
        t0 = time.perf_counter()
        O.coeffs_abel(N, M, Q, f_cl=f[lo:lo + S])
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = S * N / (ms / 1e3)
    cores = base["cores"]
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "B": cfg["B"], "K": K, "N": N, "M": M, "Q": Q,
                   "path": "oracle route 2 (CPU)", "sample_per_step": S},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d functions per step of %s" % (S, name)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
PATHS = {"split_fp16": 3, "f32": 1, "bf16": 2, "f64": 0}
DTYPE_STR = {
    "split_fp16": "f16 split (8 tcgen05 products, f32 accum, exact leading accumulator) + df32 FFT",
    "f32": "f32", "bf16": "bf16 (f32 accum) + f32 FFT", "f64": "f64",
}


# Peak arithmetic rates of the FFT stage (ops/s in units of 1e12), from unit
# counts and clocks: 152 SMs x 128 FP32 lanes x 2.07 GHz (one FP32 add, mul or
# FMA per lane per cycle); FP64: the GB300's nominal 1.25 TFLOP/s dense.
ALU_PEAK_TOPS = {"f32": 152 * 128 * 2.07e9 / 1e12, "f64": 1.25}

# DRAM bytes (read + write) per launch measured by ncu for the current kernels
# (one ncu capture per kernel); keyed by (stage, path, workload).
TRAFFIC = {
    ("abel_gemm", "split_fp16", "cheb_b4096_k1025_n512_m2048"): 69294080,   # tc_gemm_pair_split_fp16_...
    ("fft", "split_fp16", "cheb_b4096_k1025_n512_m2048"): 34181120,         # dct16_forward_dfl_...
}


def fft_fp32_ops(M, N):
    """FP32 operations of the double-float transform of one function (the
    algorithmic operation count of the method's FFT stage at the precision it
    needs): a length-H complex FFT (H = M/4) with (H/2) log2 H radix-2
    butterflies of 4 mul + 6 add, the fold (L = M/2 values: 3.5 add + 2.5 mul
    each), the recombination (H x 8 add + 4 mul), the scan (H add) and the
    output (N x 1 add + 1 mul), each double-float add costing 8 FP32 operations
    (TwoSum + trailing add) and each multiply 4 (exact product by FMA + 2 FMA)."""
    H, L = M // 4, M // 2
    lg = int(round(np.log2(H)))
    adds = 3 * H * lg + 3.5 * L + 8 * H + H + N
    muls = 2 * H * lg + 2.5 * L + 4 * H + N
    return 8 * adds + 4 * muls


def relerr(c, ref):
    return float(np.max(np.max(np.abs(c - ref), 1) / np.max(np.abs(ref), 1)))


def run_path(leg, torch, name, path, rank, steps, warmup, flush, sample_err=0, flags=0, clocks=None):
    cfg = workloads.CONFIGS[name]
    B, K, N, M = cfg["B"], cfg["K"], cfg["N"], cfg["M"]
    dt = PATHS[path]
    t0 = time.time()
    plan = leg.Plan(N, M, K, 0, dt, flags=flags)
    torch.cuda.synchronize()
    plan_s = time.time() - t0
    f_np = workloads.workload_inputs(name, salt=rank)
    io = torch.float64 if dt == leg.F64 else torch.float32
    f = torch.from_numpy(f_np).to(device="cuda", dtype=io)
    c = torch.empty((B, N), dtype=io, device="cuda")
    plan.reserve(B)
    for _ in range(warmup):
        plan.forward(f, c)
    torch.cuda.synchronize()
    # timed steps: one event pair around the whole forward (kernels overlap
    # through programmatic dependent launch), L2 flushed before each; the
    # clock sampler runs over exactly these steps
    if clocks is not None:
        clocks.start()
        clocks.wait_first()
    step_ms = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.forward(f, c)
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    clk = clocks.stop() if clocks is not None else None
    # stage breakdown: events between the kernels (serialises them), separate passes
    stage = []
    for _ in range(min(steps, 10)):
        flush.zero_()
        stage.append(plan.forward_profiled(f, c))
    plan.status()
    out = {"plan": plan, "f": f, "c": c, "f_np": f_np, "plan_s": plan_s, "stage": stage, "step_ms": step_ms,
           "clk": clk}
    if sample_err:
        out["c_sample"] = c[:sample_err].double().cpu().numpy()
    return out


def time_steps(torch, fn, flush, steps, warmup):
    """Mean CUDA-event time (ms) of fn() over `steps` calls, L2 flushed before each."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.mean(ts)


def extra_workloads(leg, torch, flush, rank):
    """The other workloads of the method, measured on the split path."""
    out = {}
    # ragged batch: 10,000 closed-form functions, N log-uniform in [32, 8192]
    cfg = workloads.CONFIGS["ragged_10000"]
    rng = np.random.default_rng(workloads.SEED_BASE + 3 + 1000 * rank)
    fam, par, n = workloads.ragged_spec(cfg["count"], rng, cfg["Nmin"], cfg["Nmax"])
    lay = workloads.ragged_layout(fam, par, n, rng)
    t0 = time.time()
    plans = [leg.Plan(*workloads.bucket_sizes(Nb), dtype=leg.SPLIT_FP16) for Nb in lay["buckets"]]
    batch = leg.Ragged(plans, lay["bidx"], n, lay["in_off"], lay["out_off"])
    torch.cuda.synchronize()
    setup = time.time() - t0
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    f = torch.empty(lay["n_in"], dtype=torch.float32, device="cuda")
    leg.sample_cl(dev(fam, torch.int32), dev(par, torch.float64), dev(lay["K"], torch.int32),
                  dev(lay["in_off"], torch.int64), f, coef=dev(lay["coef"], torch.float64),
                  coef_off=dev(lay["coef_off"], torch.int64))
    c = torch.empty(lay["n_out"], dtype=torch.float32, device="cuda")
    ms = time_steps(torch, lambda: batch.forward(f, c), flush, 10, 3)
    batch.status()
    out["ragged_10000"] = {"value": float(np.sum(n)) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                           "functions": cfg["count"], "coefficients": int(np.sum(n)),
                           "buckets": lay["buckets"], "plan_build_s": setup,
                           "launches_per_step": 2 + len(lay["buckets"]), "cuda_graph": True}
    del batch, plans, f, c
    # differentiation workload: forward + backward on the split path
    name = "cheb_b1024_k4097_n2048_m8192"
    cf = workloads.CONFIGS[name]
    plan = leg.Plan(cf["N"], cf["M"], cf["K"], 0, leg.SPLIT_FP16)
    x = torch.from_numpy(workloads.workload_inputs(name)).cuda()
    cc = torch.empty((cf["B"], cf["N"]), dtype=torch.float32, device="cuda")
    df = torch.empty_like(x)
    plan.reserve(cf["B"])

    def fwd_bwd():
        plan.forward(x, cc)
        plan.backward(cc, df)
    ms = time_steps(torch, fwd_bwd, flush, 10, 3)
    plan.status()
    out["differentiation_b1024_k4097_n2048_m8192"] = {
        "value": cf["B"] * cf["N"] / (ms / 1e3), "unit": UNIT + " (forward + backward)", "ms_per_step": ms}
    del plan, x, cc, df
    return out


def max_over_ranks(torch, dist, x: float, device) -> float:
    """The largest value of the host float x over the ranks of the default
    process group (x itself without one): the whole job lasts as long as its
    slowest rank."""
    if dist is None:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, ms_per_step: float) -> float:
    """Units per second of the whole job: every rank processes its own
    units_per_rank per step (weak scaling, no exchange between ranks), and the
    step lasts ms_per_step (the maximum over ranks)."""
    return world * units_per_rank / (ms_per_step / 1e3)


def gpu_arm(args, rank, world, local_rank):
    import torch
    import paper_1106_0463_gb300 as leg

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    name = args.workload
    cfg = workloads.CONFIGS[name]
    B, K, N, M = cfg["B"], cfg["K"], cfg["N"], cfg["M"]
    rows = M // 2 + 1
    peaks, peak_src = load_peaks()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # ---------------- timed region: the selected path
    barrier()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    phys = vis.split(",")[local_rank].strip() if vis else str(local_rank)
    clocks = ClockSampler(phys)
    res = run_path(leg, torch, name, args.path, rank, args.steps, args.warmup, flush, sample_err=16, clocks=clocks)
    barrier()
    clk = res["clk"]
    stage = np.array(res["stage"])              # profiled passes x 3 (ms)
    total_ms = float(np.sum(res["step_ms"]))
    total_ms = max_over_ranks(torch, dist, total_ms, "cuda")
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(world, B * N, ms_per_step)
    prep_ms, gemm_ms, fft_ms = (float(v) for v in stage.mean(0))

    # ---------------- e2e through the public API with pinned host buffers:
    # leg_forward_host copies f in and c out, overlapped with the computation
    plan, f, c = res["plan"], res["f"], res["c"]
    f_host = torch.from_numpy(res["f_np"]).to(f.dtype).pin_memory()
    c_host = torch.empty(c.shape, dtype=c.dtype).pin_memory()
    st = torch.cuda.current_stream()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        plan.forward_host(f_host, c_host, sync=False)
        e1.record(st)
        e1.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    # the bare copies, for reference (not part of the e2e number)
    copy_ms = {}
    for direction, dst, src in (("h2d", f, f_host), ("d2h", c_host, c)):
        ts = []
        for i in range(args.warmup + args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            dst.copy_(src, non_blocking=True)
            e1.record(st)
            e1.synchronize()
            if i >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        copy_ms[direction] = statistics.mean(ts)
    e2e_step = max_over_ranks(torch, dist, statistics.mean(e2e_ms), "cuda")
    e2e = {"value": whole_job_rate(world, B * N, e2e_step), "unit": UNIT,
           "h2d_bytes_per_step": f_host.numel() * f_host.element_size(),
           "d2h_bytes_per_step": c_host.numel() * c_host.element_size(),
           "api": "leg_forward_host (pinned host buffers, read and written in place by the kernels)",
           "ms_per_step": e2e_step, "bare_copy_ms": copy_ms}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---------------- parity on sampled functions (oracle, CPU)
    from oracle import oracle as O
    ref = O.coeffs_abel(N, M, O.exact_tau_points(K), f_cl=res["f_np"][:16].astype(np.float64))
    err = relerr(res["c_sample"], ref)

    # ---------------- rooflines (algorithmic work per launch / CUDA-event stage time)
    Kp = (K + 31) // 32 * 32                               # K padded to the GEMM's 32-wide K blocks
    flops_useful = 2.0 * B * rows * K                      # per GEMM launch (distinct rows, eq. 2.12)
    products = {"split_fp16": 8, "bf16": 1, "f32": 1, "f64": 1}[args.path]
    gemm_rows = rows - 1 if args.path == "split_fp16" else rows   # split: row 0 is a00 e_0, done by the split
    executed = products * 2.0 * B * gemm_rows * Kp
    fft_bytes = B * rows * (8 if args.path in ("split_fp16", "f64") else 4) + B * N * (8 if args.path == "f64" else 4)
    nplanes = 7 if args.path == "split_fp16" else 1
    prep_bytes = B * K * 4 + nplanes * B * Kp * 2 + B * 4 + (B * 8 if args.path == "split_fp16" else 0)
    peak_tensor = peaks.get("bf16_tflops", 1899.1)
    gemm_roof = {"kernel": "tc_gemm_kernel (Abel GEMM)", "bound": "tensor",
                 "achieved": flops_useful / (gemm_ms / 1e3) / 1e12, "peak": peak_tensor, "unit": "TFLOP/s",
                 "flops_per_launch": flops_useful, "executed_flops_per_launch": executed,
                 "executed_tflops": executed / (gemm_ms / 1e3) / 1e12,
                 "traffic": TRAFFIC.get(("abel_gemm", args.path, name)),
                 "peak_source": "%s bf16_tflops (fp16 dense rate equals bf16)" % peak_src}
    gemm_roof["frac"] = gemm_roof["achieved"] / peak_tensor
    hbm = peaks.get("hbm_gbs", 6696.2)
    fft_hbm = fft_bytes / (fft_ms / 1e3) / 1e9
    if args.path in ("split_fp16", "f64"):
        # double-float (or FP64) transform: bound by FP32 (FP64) arithmetic, see fft_fp32_ops
        ops = fft_fp32_ops(M, N) * B
        peak_alu = ALU_PEAK_TOPS["f64" if args.path == "f64" else "f32"]
        fft_roof = {"kernel": "dct16_forward_kernel (FFT stage)", "bound": "alu",
                    "achieved": ops / (fft_ms / 1e3) / 1e12, "peak": peak_alu, "unit": "Tops/s",
                    "ops_per_launch": ops, "hbm_gbs": fft_hbm, "hbm_frac": fft_hbm / hbm,
                    "traffic": TRAFFIC.get(("fft", args.path, name)),
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz max SM clock"}
        fft_roof["frac"] = fft_roof["achieved"] / peak_alu
    else:
        fft_roof = {"kernel": "fft_forward_kernel (FFT stage)", "bound": "hbm", "achieved": fft_hbm, "peak": hbm,
                    "unit": "GB/s", "frac": fft_hbm / hbm, "bytes_per_launch": fft_bytes,
                    "traffic": TRAFFIC.get(("fft", args.path, name)), "peak_source": "%s hbm_gbs" % peak_src}
    kernels = {"abel_gemm": gemm_ms, "fft": fft_ms, "input_split": prep_ms}
    dom = max(kernels, key=kernels.get)
    if dom == "fft":
        roof = fft_roof
    elif dom == "abel_gemm" and args.path in ("split_fp16", "bf16"):
        roof = gemm_roof
    else:
        by = {"input_split": prep_bytes, "abel_gemm": B * K * 4 + rows * K * 4 + B * rows * 4}[dom]
        achieved = by / (kernels[dom] / 1e3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None, "bytes_per_launch": by, "peak_source": "%s hbm_gbs" % peak_src}
    stages = {
        "input_split": {"ms": prep_ms, "bytes": prep_bytes,
                        "gbs": prep_bytes / (prep_ms / 1e3) / 1e9 if prep_ms > 0 else None},
        "abel_gemm": dict(gemm_roof, ms=gemm_ms) if args.path in ("split_fp16", "bf16") else
                     {"ms": gemm_ms, "useful_tflops": flops_useful / (gemm_ms / 1e3) / 1e12},
        "fft": dict(fft_roof, ms=fft_ms),
    }

    extras = {}
    if not args.no_extras and args.path != "f64":
        for p_name, st_n in (("f64", 3), ("f32", 5)):
            if p_name == args.path:
                continue
            r = run_path(leg, torch, name, p_name, rank, st_n, 2, flush, sample_err=16)
            ms = float(np.mean(r["step_ms"]))
            extras[p_name + "_gpu_path"] = {"value": B * N / (ms / 1e3), "ms_per_step": ms,
                                            "max_rel_err": relerr(r["c_sample"], ref)}
            del r
    if not args.no_extras and args.path == "split_fp16":
        # the same map with L = R A multiplied out at plan time: split + one GEMM
        r = run_path(leg, torch, name, "split_fp16", rank, 10, 3, flush, sample_err=16, flags=leg.FLAG_COLLAPSED)
        st_ms = np.array(r["stage"]).mean(0)
        ms = float(np.mean(r["step_ms"]))
        cf_useful = 2.0 * B * N * K
        cf_exec = 8 * 2.0 * B * N * Kp
        extras["collapsed_split_fp16"] = {
            "value": B * N / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "max_rel_err": relerr(r["c_sample"], ref),
            "input_split_ms": float(st_ms[0]), "gemm_ms": float(st_ms[1]), "plan_build_s": r["plan_s"],
            "gemm_useful_tflops": cf_useful / (st_ms[1] / 1e3) / 1e12,
            "gemm_executed_tflops": cf_exec / (st_ms[1] / 1e3) / 1e12,
            "gemm_executed_frac": cf_exec / (st_ms[1] / 1e3) / 1e12 / peak_tensor,
            "launches_per_step": 2}
        del r
    if not args.no_extras:
        extras.update(extra_workloads(leg, torch, flush, rank))
    cpu = None
    if not args.no_cpu_baseline:
        cpu, _, _ = oracle_rate(name)
    launches_per_step = {"split_fp16": 3, "bf16": 3, "f32": 2, "f64": 2}[args.path]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_STR[args.path], "data": "synthetic",
        "config": {"workload": name, "B": B, "K": K, "N": N, "M": M, "Q": (K + 1) // 2, "path": args.path,
                   "l2": "flushed (512 MiB write) before every timed step",
                   "inputs": "random decaying Chebyshev series sampled at CL nodes, FP32, seeded"},
        "max_rel_err": err, "err_sample": "16 functions vs FP64 oracle route 2",
        "roofline": roof, "stages": stages, "plan_build_s": res["plan_s"],
        "e2e": e2e, "clocks": clk, "gpu_launches": launches_per_step * args.steps,
        "cpu_baseline": cpu,
    }
    if extras:
        line.update(extras)
        if "f64_gpu_path" in extras:
            line["speedup_vs_fp64_gpu_path"] = value / world / extras["f64_gpu_path"]["value"]
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    gpu_arm(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
