"""Throughput benchmark of the Legendre-coefficient path on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload NAME] [--path split_fp16|f32|bf16|f64] [--no-extras]

One step = one forward pass of the sampled-input path over one batch with
inputs resident in HBM: input split -> tcgen05 Abel GEMM -> transform with the
(2n+1) scaling.  The headline workload is the largest dense
single-GPU configuration: B=256 random decaying Chebyshev series at K=8193
Chebyshev-Lobatto nodes, N=4096 coefficients, M=16384 trapezoid points (exact
tau rule), on the split-FP16 path, its error against the FP64 oracle measured
in the same run on sampled functions (the first and last of every function
tile of the GEMM among them).

The same JSON line carries, under "workloads", every other configuration of
the method with its own error against the oracle, time and roofline: the
plain method (one function, c_n = 0.5^n checked to 1e-12), B=4096 at K=1025
(split-FP16, plain FP32, FP64, collapsed operator), the ragged batch of
10,000 closed-form functions, the differentiation workload (forward +
backward, with the FP64 GPU path's time beside it), the precision sweep of
the headline workload (FP64, FP32, BF16 next to split-FP16), the sine-form
transform (Eq. 2.13) on the headline workload, and Table 1's |x|^{3/2} on
the plain method at several (M, Q).

Timing of the headline value: W untimed warm-up batches, then the K steps
as K distinct batches (the workload's batch scaled per step, more bytes than
L2 in all) in one leg_forward_batches call between a pair of CUDA events:
each batch's split and GEMM on a high-priority stream, the previous batch's
transform beside it on a low-priority one.  Barrier + synchronize bracket the
timed region; the max over ranks is taken.  The same workload one batch per
step (L2 flushed by a 512 MiB write before each, CUDA events on the launch
stream) gives the single_batch figures, stage times and error; the other
workloads are timed that way too.  e2e runs the K batches from pinned host
memory through leg_forward_host_batches.  Under torchrun (N > 1) every rank
runs its own batches (weak scaling, no collective on the data path).

--impl reference times the FP64 CPU oracle on the host cores, on a bounded
sample of the same workload per step.
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
HEADLINE = "cheb_b256_k8193_n4096_m16384"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE)
    ap.add_argument("--path", default="split_fp16", choices=["split_fp16", "f32", "bf16", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-route2", action="store_true",
                    help="also time oracle route 2 with explicit operators at B=4096, K=1025 (the build takes minutes)")
    ap.add_argument("--no-extras", action="store_true", help="headline workload only")
    ap.add_argument("--tile", type=int, default=None,
                    help="GEMM tile width of the headline plan (0 = the library's model); with --transform, "
                         "skips the autotuner")
    ap.add_argument("--transform", default=None, choices=["reg", "stockham", "sine"],
                    help="transform kernel of the headline plan")
    ap.add_argument("--radix", type=int, default=0, choices=[0, 8, 16],
                    help="radix of the register-tiled transform passes (with --tile and --transform)")
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
def host_cores() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def exact_config(name: str) -> bool:
    """M > N + K - 1 with the exact tau rule: the discrete method has no
    discretisation error on these sampled inputs and the oracle's route 1
    (Eq. 2.3) and route 2 (Theorem 1) agree to rounding."""
    cfg = workloads.CONFIGS[name]
    return cfg["M"] > cfg["N"] + cfg["K"] - 1


def oracle_quadrature_points(cfg) -> int:
    """Gauss points of route 1 that integrate f P_n exactly for n < N on the
    degree-(K-1) interpolant."""
    return (cfg["K"] + cfg["N"]) // 2 + 4


def oracle_coeffs(O, name, f):
    """Oracle coefficients of the sampled functions f (rows, FP64): route 1 on
    the exact configurations, route 2 otherwise."""
    cfg = workloads.CONFIGS[name]
    if exact_config(name):
        return O.coeffs_direct(cfg["N"], oracle_quadrature_points(cfg), f_cl=f)
    return O.coeffs_abel(cfg["N"], cfg["M"], O.exact_tau_points(cfg["K"]), f_cl=f)


def oracle_route_name(name):
    return ("route 1 (Eq. 2.3, %d-point Gauss rule; the configuration is exact, so routes 1 and 2 agree to "
            "rounding)" % oracle_quadrature_points(workloads.CONFIGS[name]) if exact_config(name)
            else "route 2 (Abel + trapezoid, direct Fourier sum)")


def oracle_rate(name: str, seconds: float = 10.0, max_fns: int = 256):
    """The oracle as it stands on a bounded sample of the workload (about
    `seconds` of CPU work), in coefficients per second."""
    from oracle import oracle as O
    cfg = workloads.CONFIGS[name]
    f = workloads.workload_inputs(name).astype(np.float64)
    n = 2
    t0 = time.time()
    oracle_coeffs(O, name, f[:n])
    dt = time.time() - t0
    while dt < seconds / 3 and n < max_fns:
        n = min(max_fns, n * 4)
        t0 = time.time()
        oracle_coeffs(O, name, f[:n])
        dt = time.time() - t0
    # a sample shorter than `seconds` (the whole batch done quickly) is run
    # again until the total reaches it, so the rate rests on seconds of work
    reps = 1
    while dt < seconds and reps < 64:
        t0 = time.time()
        oracle_coeffs(O, name, f[:n])
        dt += time.time() - t0
        reps += 1
    return {"value": reps * n * cfg["N"] / dt, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": "%d of %d functions of %s%s, oracle %s, FP64, OpenMP, %.2f s"
                      % (n, cfg["B"], name, " (%d times)" % reps if reps > 1 else "", oracle_route_name(name),
                         dt)}, reps * n, dt


def oracle_route2_operator_rate(name: str):
    """Route 2 with its explicit operators built once (not timed): C = (F A^T) R^T
    for the whole batch by the BLAS behind numpy, A the M x K Abel-interpolation
    operator and R the N x M twisted Fourier sum (Eqs. 2.4, 2.5)."""
    from oracle import oracle as O
    cfg = workloads.CONFIGS[name]
    f = workloads.workload_inputs(name).astype(np.float64)
    Q = O.exact_tau_points(cfg["K"])
    t0 = time.time()
    A = O.abel_operator(cfg["M"], cfg["K"], Q)
    R = O.twisted_dft_matrix(cfg["N"], cfg["M"])
    build = time.time() - t0
    (f[:64] @ A.T) @ R.T
    t0 = time.perf_counter()
    C = (f @ A.T) @ R.T
    dt = time.perf_counter() - t0
    ref = oracle_coeffs(O, name, f[:2])
    return {"value": cfg["B"] * cfg["N"] / dt, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": "all %d functions of %s, oracle route 2 with the explicit operators A (%d x %d) and R "
                      "(%d x %d) built once in %.1f s (not timed): C = (F A^T) R^T by numpy's BLAS, %.3f s"
                      % (cfg["B"], name, cfg["M"], cfg["K"], cfg["N"], cfg["M"], build, dt),
            "max_rel_diff_vs_route1": relerr(C[:2], ref)}


def reference_arm(args, rank, world):
    if rank != 0:
        return
    name = args.workload
    cfg = workloads.CONFIGS[name]
    from oracle import oracle as O
    f = workloads.workload_inputs(name).astype(np.float64)
    # one step is a bounded sample (about 2 s of CPU work, less for many steps)
    base, n, dt = oracle_rate(name, seconds=4.0, max_fns=64)
    per_fn = dt / n
    budget = min(2.0, 60.0 / max(1, args.steps + args.warmup))
    S = max(1, min(cfg["B"], int(budget / max(per_fn, 1e-9))))
    for _ in range(args.warmup):
        oracle_coeffs(O, name, f[:S])
    times = []
    for i in range(args.steps):
        lo = (i * S) % max(1, cfg["B"] - S + 1)
        t0 = time.perf_counter()
        oracle_coeffs(O, name, f[lo:lo + S])
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = S * cfg["N"] / (ms / 1e3)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "B": cfg["B"], "K": cfg["K"], "N": cfg["N"], "M": cfg["M"],
                   "Q": O.exact_tau_points(cfg["K"]), "path": "FP64 CPU oracle, " + oracle_route_name(name),
                   "sample_per_step": S},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                         "sample": "%d functions per step of %s" % (S, name)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ rooflines
PATHS = {"split_fp16": 3, "f32": 1, "bf16": 2, "f64": 0}
DTYPE_STR = {
    "split_fp16": "f16 split (8 tcgen05 products, f32 accum, exact leading accumulator) + df32 FFT",
    "f32": "f32", "bf16": "bf16 (f32 accum) + f32 FFT", "f64": "f64",
}
PRODUCTS = {"split_fp16": 8, "bf16": 1, "f32": 1, "f64": 1}
TRANSFORM_NAMES = {0: "register-tiled real-even (Eq. 2.4 with the twist as a first difference)",
                   1: "shared-memory Stockham real-even", 2: "register-tiled sine form (Eq. 2.13)"}
LAUNCHES = {"split_fp16": 3, "bf16": 3, "f32": 2, "f64": 2}

# Peak arithmetic rates of the FFT stage (ops/s in units of 1e12), from unit
# counts and clocks: 152 SMs x 128 FP32 lanes x 2.07 GHz (one FP32 add, mul or
# FMA per lane per cycle); FP64: the GB300's nominal 1.25 TFLOP/s dense.
ALU_PEAK_TOPS = {"f32": 152 * 128 * 2.07e9 / 1e12, "f64": 1.25}

# DRAM bytes (read + write) per launch measured by ncu for the current kernels
# (one ncu capture per kernel, summaries under profiles/); keyed by
# (stage, path, workload).  A kernel changed since its capture has no entry.
TRAFFIC = {
    ("abel_gemm", "split_fp16", "cheb_b256_k8193_n4096_m16384"): 441804032,   # tc_gemm_pair_split_fp16_cheb_b256_...
    ("fft_sine", "split_fp16", "cheb_b256_k8193_n4096_m16384"): 17057024,     # dst16_forward_dfl_cheb_b256_...
    ("abel_gemm", "split_fp16", "ragged"): 628728064,                          # tc_gemm_grouped_split_fp16_ragged_10000
}


def fft_fp32_ops(M, N, fp64=False):
    """FP32 operations of the double-float real-even transform of one function
    (the algorithmic operation count of the FFT stage at the precision it
    needs): a length-H complex FFT (H = M/4) with (H/2) log2 H radix-2
    butterflies of 4 mul + 6 add, the fold (L = M/2 values: 3.5 add + 2.5 mul
    each), the recombination (H x 8 add + 4 mul), the scan (H add) and the
    output (N x 1 add + 1 mul), each double-float add costing 8 FP32 operations
    (TwoSum + trailing add) and each multiply 4 (exact product by FMA + 2 FMA);
    with fp64, one FP64 operation each."""
    H, L = M // 4, M // 2
    lg = int(round(np.log2(H)))
    adds = 3 * H * lg + 3.5 * L + 8 * H + H + N
    muls = 2 * H * lg + 2.5 * L + 4 * H + N
    return adds + muls if fp64 else 8 * adds + 4 * muls


def dst_fp32_ops(M, N, fp64=False):
    """FP32 operations of the double-float sine-form transform (Eq. 2.13) of
    one function, same conventions: the length-H FFT, the merged pre-twiddle
    (two W values per k < H: 3 add + 2 mul each; their sum and difference:
    4 add; the twiddle product: 4 mul + 2 add; 2 add) and the output (N x 2
    mul)."""
    H = M // 4
    lg = int(round(np.log2(H)))
    adds = 3 * H * lg + 14 * H
    muls = 2 * H * lg + 8 * H + 2 * N
    return adds + muls if fp64 else 8 * adds + 4 * muls


def relerr(c, ref):
    """max over functions of max_n |c - c_ref| / max_n |c_ref|."""
    c = np.atleast_2d(np.asarray(c, dtype=np.float64))
    return float(np.max(np.max(np.abs(c - ref), 1) / np.max(np.abs(ref), 1)))


def gemm_roofline(B, rows, K, Kp, path, gemm_ms, peaks, peak_src, traffic, name):
    """The Abel GEMM's roofline: useful FLOP (2 B rows K, the distinct rows of
    Eq. 2.12) over the CUDA-event stage time against the measured dense
    tensor peak; executed FLOP of the split products and the algorithmic HBM
    bytes (operator planes, input planes, G) beside it."""
    hbm = peaks.get("hbm_gbs", 6800.0)
    peak = peaks.get("bf16_tflops", 1900.0)
    useful = 2.0 * B * rows * K
    gemm_rows = rows - 1 if path == "split_fp16" else rows   # split: row 0 is a00 e_0, done by the split
    executed = PRODUCTS[path] * 2.0 * B * gemm_rows * Kp
    n_a = {"split_fp16": 3, "bf16": 1, "f32": 1, "f64": 1}[path]
    n_f = {"split_fp16": 7, "bf16": 1, "f32": 1, "f64": 1}[path]
    eb = {"split_fp16": 2, "bf16": 2, "f32": 4, "f64": 8}[path]
    gb = {"split_fp16": 8, "bf16": 4, "f32": 4, "f64": 8}[path]
    bytes_ = n_a * gemm_rows * Kp * eb + n_f * B * Kp * eb + B * rows * gb
    sec = gemm_ms / 1e3
    tc = path in ("split_fp16", "bf16")
    if tc:
        r = {"kernel": "tc_gemm_kernel (Abel GEMM, tcgen05)", "bound": "tensor",
             "achieved": useful / sec / 1e12, "peak": peak, "unit": "TFLOP/s",
             "peak_source": "%s bf16_tflops (dense FP16 rate = BF16 rate)" % peak_src}
    else:
        fp = {"f32": 152 * 128 * 2 * 2.07e9 / 1e12, "f64": 1.25}[path]
        r = {"kernel": "simt_gemm_kernel (Abel GEMM, CUDA cores)", "bound": "alu",
             "achieved": useful / sec / 1e12, "peak": fp, "unit": "TFLOP/s",
             "peak_source": "derived: FP32 152 SMs x 128 lanes x 2 FLOP x 2.07 GHz; FP64 nominal 1.25 TFLOP/s"}
    r["frac"] = r["achieved"] / r["peak"]
    r.update({"ms": gemm_ms, "flops_per_launch": useful, "executed_flops_per_launch": executed,
              "executed_tflops": executed / sec / 1e12, "executed_frac": executed / sec / 1e12 / r["peak"],
              "algorithmic_bytes_per_launch": bytes_, "hbm_gbs": bytes_ / sec / 1e9,
              "hbm_frac": bytes_ / sec / 1e9 / hbm,
              "traffic": traffic.get(("abel_gemm", path, name))})
    return r


def fft_roofline(B, M, N, rows, path, fft_ms, peaks, peak_src, traffic, name, sine=False):
    """The transform stage: bound by FP32 (double-float) or FP64 arithmetic at
    the precision the split / FP64 paths need, by HBM for the FP32 path."""
    hbm = peaks.get("hbm_gbs", 6800.0)
    gbytes = {"split_fp16": 8, "f64": 8, "f32": 4, "bf16": 4}[path]
    bytes_ = B * rows * gbytes + B * N * (8 if path == "f64" else 4)
    sec = fft_ms / 1e3
    hbm_gbs = bytes_ / sec / 1e9
    kern = "dst16_forward_kernel (sine form)" if sine else "dct16_forward_kernel (real-even)"
    if path in ("split_fp16", "f64"):
        # double-float: FP32 operations; FP64: one operation per FP64 add or multiply
        ops = (dst_fp32_ops(M, N, path == "f64") if sine else fft_fp32_ops(M, N, path == "f64")) * B
        peak = ALU_PEAK_TOPS["f64" if path == "f64" else "f32"]
        r = {"kernel": kern, "bound": "alu", "achieved": ops / sec / 1e12, "peak": peak, "unit": "Tops/s",
             "ops_per_launch": ops, "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz max SM clock"
             if path != "f64" else "nominal FP64 1.25 TFLOP/s"}
        r["frac"] = r["achieved"] / peak
    else:
        r = {"kernel": kern if sine else "fft_forward_kernel (Stockham, FP32)", "bound": "hbm", "achieved": hbm_gbs,
             "peak": hbm, "unit": "GB/s", "frac": hbm_gbs / hbm, "peak_source": "%s hbm_gbs" % peak_src}
    r.update({"ms": fft_ms, "bytes_per_launch": bytes_, "hbm_gbs": hbm_gbs, "hbm_frac": hbm_gbs / hbm,
              "traffic": traffic.get(("fft_sine" if sine else "fft", path, name))})
    return r


# ------------------------------------------------------------------ GPU helpers
def time_steps(torch, fn, flush, steps, warmup, clocks=None):
    """CUDA-event times (ms) of fn() over `steps` calls, L2 flushed before each
    (flush None: L2 left warm).  All steps are queued before one synchronise,
    so the device never waits for the host inside a timed interval (a host
    stall between an event and the launches after it would be counted)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
        clocks.wait_first()
    evs = []
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        evs.append((e0, e1))
    torch.cuda.synchronize()
    ts = [e0.elapsed_time(e1) for e0, e1 in evs]
    clk = clocks.stop() if clocks is not None else None
    return ts, clk


def sample_rows(B, tn, extra, seed):
    """Functions to check: the first and last of every function tile of width
    tn, plus `extra` drawn at random."""
    idx = set()
    for t0 in range(0, B, tn):
        idx.add(t0)
        idx.add(min(B, t0 + tn) - 1)
    rng = np.random.default_rng(seed)
    rest = np.setdiff1d(np.arange(B), sorted(idx))
    if rest.size:
        idx.update(int(i) for i in rng.choice(rest, size=min(extra, rest.size), replace=False))
    return np.array(sorted(idx))


class Dense:
    """One dense sampled workload on the GPU: plans per path built from one
    FP64 operator, resident inputs, and the oracle reference on sampled rows."""

    def __init__(self, leg, torch, name, rank, with_ref, extra=24):
        self.leg, self.torch, self.name = leg, torch, name
        cfg = workloads.CONFIGS[name]
        self.B, self.K, self.N, self.M = cfg["B"], cfg["K"], cfg["N"], cfg["M"]
        self.rows = self.M // 2 + 1
        self.Kp = (self.K + 31) // 32 * 32
        self.f_np = workloads.workload_inputs(name, salt=rank)
        self.plans = {}
        self.plan_s = {}
        t0 = time.time()
        self.plans["split_fp16"] = leg.Plan(self.N, self.M, self.K, 0, leg.SPLIT_FP16)
        torch.cuda.synchronize()
        self.plan_s["split_fp16"] = time.time() - t0
        self.f32 = torch.from_numpy(self.f_np).cuda()
        self.tn = self.plans["split_fp16"].tile_info(self.B)["tn"]
        self.sample = sample_rows(self.B, self.tn, extra, 7 + rank)
        self.ref = None
        if with_ref:
            from oracle import oracle as O
            self.ref = oracle_coeffs(O, name, self.f_np[self.sample].astype(np.float64))

    def plan(self, path):
        if path not in self.plans:
            t0 = time.time()
            self.plans[path] = self.leg.Plan.like(self.plans["split_fp16"], PATHS[path])
            self.torch.cuda.synchronize()
            self.plan_s[path] = time.time() - t0
        return self.plans[path]

    def autotune(self, path):
        """leg_plan_autotune on this batch: GEMM tile width and transform kernel."""
        plan = self.plan(path)
        c = self.torch.empty((self.B, self.N), dtype=plan.io_dtype, device="cuda")
        choice = plan.autotune(self.inputs(path), c)
        if path == "split_fp16":
            self.retile()
        return choice

    def retile(self):
        """Sampled rows for the split plan's current tile width."""
        tn = self.plans["split_fp16"].tile_info(self.B)["tn"]
        if tn != self.tn:
            self.tn = tn
            self.sample = sample_rows(self.B, self.tn, 36, 7)
            if self.ref is not None:
                from oracle import oracle as O
                self.ref = oracle_coeffs(O, self.name, self.f_np[self.sample].astype(np.float64))

    def inputs(self, path):
        torch = self.torch
        if path == "f64":
            if not hasattr(self, "f64"):
                self.f64 = self.f32.double()
            return self.f64
        return self.f32

    def run(self, path, flush, steps, warmup, peaks, peak_src, clocks=None, transform=None, stages=10,
            warm_steps=0):
        leg, torch = self.leg, self.torch
        plan = self.plan(path)
        prev = plan.transform
        if transform is not None:
            plan.set_transform(transform)
        f = self.inputs(path)
        c = torch.empty((self.B, self.N), dtype=plan.io_dtype, device="cuda")
        plan.reserve(self.B)
        ts, clk = time_steps(torch, lambda: plan.forward(f, c), flush, steps, warmup, clocks)
        st = []
        for _ in range(min(stages, steps)):
            flush.zero_()
            st.append(plan.forward_profiled(f, c))
        warm = None
        if warm_steps:
            # back to back between one event pair: no flush, no host gap between steps
            for _ in range(2):
                plan.forward(f, c)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(warm_steps):
                plan.forward(f, c)
            e1.record()
            e1.synchronize()
            tw = e0.elapsed_time(e1) / warm_steps
            warm = {"value": self.B * self.N / (tw / 1e3), "ms_per_step": tw, "steps": warm_steps,
                    "l2": "not flushed; steps back to back between one pair of events"}
        plan.status()
        ms = float(np.mean(ts))
        prep_ms, gemm_ms, fft_ms = (float(v) for v in np.mean(np.array(st), 0))
        out = {"value": self.B * self.N / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
               "steps": steps, "plan_build_s": self.plan_s.get(path),
               "stages_ms": {"input_split": prep_ms, "abel_gemm": gemm_ms, "transform": fft_ms},
               "gemm_roofline": gemm_roofline(self.B, self.rows, self.K, self.Kp, path, gemm_ms, peaks, peak_src,
                                              TRAFFIC, self.name),
               "transform_roofline": fft_roofline(self.B, self.M, self.N, self.rows, path, fft_ms, peaks, peak_src,
                                                  TRAFFIC, self.name, sine=plan.transform == leg.TRANSFORM_SINE),
               "gpu_launches_per_step": LAUNCHES[path]}
        if warm is not None:
            out["l2_warm"] = warm
        if self.ref is not None:
            got = c[torch.from_numpy(self.sample).cuda()].double().cpu().numpy()
            out["max_rel_err"] = relerr(got, self.ref)
            out["err_sample"] = "%d functions (first and last of every %d-function GEMM tile, the rest random)" \
                                % (len(self.sample), self.tn)
        if transform is not None:
            plan.set_transform(prev)
        out["_ts"], out["_clk"], out["_stage"] = ts, clk, (prep_ms, gemm_ms, fft_ms)
        return out


def strip(d):
    return {k: v for k, v in d.items() if not k.startswith("_")}


# ------------------------------------------------------------------ other workloads
def plain_method(leg, torch):
    """The plain method (closed form at the quadrature points, FP64) on the
    generating function t = 0.5: c_n = 0.5^n to 1e-12; latency of one call."""
    cfg = workloads.CONFIGS["genfn_plain_n64"]
    plan = leg.Plan(cfg["N"], cfg["M"], 17, cfg["Q"], leg.F64)
    params = torch.tensor([cfg["t"]], dtype=torch.float64, device="cuda")
    c = torch.empty((1, cfg["N"]), dtype=torch.float64, device="cuda")
    for _ in range(5):
        plan.plain_forward(leg.FAMILY_GENFN, params, c)
    torch.cuda.synchronize()
    ts = []
    for _ in range(50):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.plain_forward(leg.FAMILY_GENFN, params, c)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    err = float(np.max(np.abs(c.cpu().numpy()[0] - cfg["t"] ** np.arange(cfg["N"]))))
    return {"N": cfg["N"], "M": cfg["M"], "Q": cfg["Q"], "t": cfg["t"], "max_abs_err_vs_t_pow_n": err,
            "tolerance": 1e-12, "ms_per_call": float(np.median(ts)), "launches_per_call": 2}


def table1_plain(leg, torch, O):
    """Table 1's test function |x|^{3/2} on the plain method with the sine-form
    transform (Eq. 2.13) at several (M, Q): parity against the oracle's route 3
    at the same (M, Q), and the method error against the true column (Eq. 2.15)."""
    true = {}
    with open(os.path.join(ROOT, "tests", "golden", "table1_abs_x_3_2.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                n, t, _ = line.split()
                true[int(n)] = float(t)
    out = []
    N = 32
    for M, Q in ((256, 64), (1024, 256), (1024, 1024), (4096, 4096)):
        plan = leg.Plan(N, M, 17, Q, leg.F64, flags=leg.FLAG_SINE_FORM)
        c = plan.plain_forward(leg.FAMILY_ABSPOW, torch.tensor([1.5], dtype=torch.float64, device="cuda"))
        got = c.cpu().numpy()[0]
        ref = O.coeffs_sine(N, M, Q, f=lambda omx: np.abs(1 - omx) ** 1.5)[0]
        out.append({"M": M, "Q": Q, "parity_vs_oracle_route3": float(np.max(np.abs(got - ref)) / np.max(np.abs(ref))),
                    "max_abs_err_vs_table1_true": max(abs(got[n] - t) for n, t in true.items())})
    return out


def ragged(leg, torch, flush, rank, peaks, peak_src, with_ref, steps=20, warmup=3, tile=None, transform=None):
    """The ragged workload: 10,000 closed-form functions in 9 size buckets,
    one grouped persistent GEMM launch, replayed as a CUDA graph."""
    cfg = workloads.CONFIGS["ragged_10000"]
    rng = np.random.default_rng(workloads.SEED_BASE + 3 + 1000 * rank)
    fam, par, n = workloads.ragged_spec(cfg["count"], rng, cfg["Nmin"], cfg["Nmax"])
    lay = workloads.ragged_layout(fam, par, n, rng)
    t0 = time.time()
    plans = [leg.Plan(*workloads.bucket_sizes(Nb), dtype=leg.SPLIT_FP16) for Nb in lay["buckets"]]
    torch.cuda.synchronize()
    setup = time.time() - t0
    # each bucket's transform (kernel and radix) timed on a batch of its size,
    # before the batch captures its launches
    tr = {}
    for b, (Nb, p) in enumerate(zip(lay["buckets"], plans)):
        if transform is not None:   # fixed from the command line
            if p.M >= 256 or transform[0] != leg.TRANSFORM_SINE:
                p.set_transform(*transform)
        else:
            Bb = int(np.sum(lay["bidx"] == b))
            p.autotune(torch.randn((Bb, p.K), dtype=torch.float32, device="cuda"))
        tr[str(Nb)] = "%s, radix %d" % (["real-even", "Stockham", "sine form"][p.transform], p.transform_radix)
    batch = leg.Ragged(plans, lay["bidx"], n, lay["in_off"], lay["out_off"])
    torch.cuda.synchronize()
    dev = lambda a, dt: torch.tensor(a, dtype=dt, device="cuda")
    f = torch.empty(lay["n_in"], dtype=torch.float32, device="cuda")
    leg.sample_cl(dev(fam, torch.int32), dev(par, torch.float64), dev(lay["K"], torch.int32),
                  dev(lay["in_off"], torch.int64), f, coef=dev(lay["coef"], torch.float64),
                  coef_off=dev(lay["coef_off"], torch.int64))
    c = torch.empty(lay["n_out"], dtype=torch.float32, device="cuda")
    model_tn = batch.tile_info()["tn"]
    if tile is not None:
        batch.set_tile(tile)
        tuned_tn = batch.tile_info()["tn"]
    else:
        tuned_tn = batch.autotune(f, c)   # the grouped launch's tile width, timed on this batch
    ts, _ = time_steps(torch, lambda: batch.forward(f, c), flush, steps, warmup)
    st = []
    for _ in range(min(5, steps)):
        flush.zero_()
        st.append(batch.forward_profiled(f, c))
    batch.forward(f, c)
    batch.status()
    ms = float(np.mean(ts))
    split_ms, gemm_ms, fft_ms = (float(v) for v in np.mean(np.array(st), 0))
    # grouped GEMM roofline: useful FLOP over all buckets
    useful, executed, abytes = 0.0, 0.0, 0.0
    for b, Nb in enumerate(lay["buckets"]):
        N, M, K, Q = workloads.bucket_sizes(Nb)
        Bb = int(np.sum(lay["bidx"] == b))
        rows, Kp = M // 2 + 1, (K + 31) // 32 * 32
        useful += 2.0 * Bb * rows * K
        executed += 8 * 2.0 * Bb * (rows - 1) * Kp
        abytes += 3 * (rows - 1) * Kp * 2 + 7 * Bb * Kp * 2 + Bb * rows * 8
    peak = peaks.get("bf16_tflops", 1900.0)
    sec = gemm_ms / 1e3
    roof = {"kernel": "tc_gemm_kernel (grouped Abel GEMM over all buckets)", "bound": "tensor",
            "achieved": useful / sec / 1e12, "peak": peak, "unit": "TFLOP/s", "frac": useful / sec / 1e12 / peak,
            "executed_tflops": executed / sec / 1e12, "executed_frac": executed / sec / 1e12 / peak,
            "flops_per_launch": useful, "executed_flops_per_launch": executed,
            "algorithmic_bytes_per_launch": abytes, "hbm_gbs": abytes / sec / 1e9,
            "peak_source": "%s bf16_tflops" % peak_src, "traffic": TRAFFIC.get(("abel_gemm", "split_fp16", "ragged"))}
    out = {"value": float(np.sum(n)) / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "functions": cfg["count"],
           "coefficients": int(np.sum(n)), "buckets": lay["buckets"], "plan_build_s": setup,
           "stages_ms": {"input_split": split_ms, "grouped_gemm": gemm_ms, "transforms": fft_ms},
           "roofline": roof, "tile_width": tuned_tn, "tile_width_cost_model": model_tn,
           "tile_chosen_by": "leg_ragged_autotune (timed candidates: the cost model's width and 128..64)",
           "bucket_transforms": tr,
           "gpu_launches_per_step": 2 + len(lay["buckets"]), "cuda_graph": True}
    if with_ref:
        from oracle import oracle as O
        f_host, c_host = f.cpu().numpy(), c.cpu().numpy()
        worst, count = 0.0, 0
        for b, Nb in enumerate(lay["buckets"]):
            N, M, K, Q = workloads.bucket_sizes(Nb)
            idx = np.where(lay["bidx"] == b)[0]
            pick = sorted({int(idx[0]), int(idx[-1])})
            fk = np.stack([f_host[lay["in_off"][i]:lay["in_off"][i] + K].astype(np.float64) for i in pick])
            if 2 * Q >= K and M > N + K - 1:
                refs = O.coeffs_direct(N, (K + N) // 2 + 4, f_cl=fk)
            else:
                refs = O.coeffs_abel(N, M, Q, f_cl=fk)
            for i, r in zip(pick, refs):
                r = r[:n[i]]
                g = c_host[lay["out_off"][i]:lay["out_off"][i] + n[i]]
                worst = max(worst, float(np.max(np.abs(g - r)) / np.max(np.abs(r))))
                count += 1
        out["max_rel_err"] = worst
        out["err_sample"] = ("%d functions, the first and last of every bucket, vs the oracle at the bucket's "
                             "(N, M, K, Q): route 1 where exact, else route 2" % count)
    del batch, plans, f, c
    return out


def differentiation(leg, torch, flush, rank, peaks, peak_src, with_ref, steps=20, warmup=3, transform=None):
    """B=1024, K=4097, N=2048, M=8192: forward + backward of the split path
    (leg_forward, leg_backward) against the FP64 GPU path, errors of both
    directions against the oracle (route 1 and route 1 transposed)."""
    name = "cheb_b1024_k4097_n2048_m8192"
    d = Dense(leg, torch, name, rank, with_ref, extra=12)
    split = d.plan("split_fp16")
    f64p = d.plan("f64")
    B, N, K = d.B, d.N, d.K
    x = d.f32
    c = torch.empty((B, N), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(workloads.SEED_BASE + 4 + 1000 * rank)
    v_np = rng.standard_normal((B, N)).astype(np.float32)
    v = torch.from_numpy(v_np).cuda()
    df = torch.empty_like(x)
    split.reserve(B)
    if transform is None:
        tuned = split.autotune(x)   # the forward's GEMM tile width and transform kernel, timed on this batch
    else:                           # fixed from the command line
        split.set_transform(transform)
        tuned = {"tn": 0, "fft": split.transform}

    def fwd_bwd():
        split.forward(x, c)
        split.backward(v, df)
    ts, _ = time_steps(torch, fwd_bwd, flush, steps, warmup)
    tf, _ = time_steps(torch, lambda: split.forward(x, c), flush, steps, warmup)
    tb, _ = time_steps(torch, lambda: split.backward(v, df), flush, steps, warmup)
    split.status()
    x64, v64 = x.double(), v.double()
    c64 = torch.empty((B, N), dtype=torch.float64, device="cuda")
    df64 = torch.empty_like(x64)

    def fwd_bwd64():
        f64p.forward(x64, c64)
        f64p.backward(v64, df64)
    t64, _ = time_steps(torch, fwd_bwd64, flush, 3, 1)
    ms, ms64 = float(np.mean(ts)), float(np.mean(t64))
    out = {"value": B * N / (ms / 1e3), "unit": UNIT + " (forward + backward)", "ms_per_step": ms,
           "forward_ms": float(np.mean(tf)), "backward_ms": float(np.mean(tb)),
           "f64_gpu_path": {"value": B * N / (ms64 / 1e3), "ms_per_step": ms64},
           "speedup_vs_fp64_gpu_path": ms64 / ms, "plan_build_s": d.plan_s.get("split_fp16"),
           "tuned": {"tn": tuned["tn"], "transform": TRANSFORM_NAMES[tuned["fft"]]},
           "gpu_launches_per_step": 3 + 3}
    if with_ref:
        from oracle import oracle as O
        sel = torch.from_numpy(d.sample).cuda()
        split.forward(x, c)
        out["forward_max_rel_err"] = relerr(c[sel].double().cpu().numpy(), d.ref)
        split.backward(v, df)
        ref_b = O.adjoint_direct(oracle_quadrature_points(workloads.CONFIGS[name]), K,
                                 v_np[d.sample].astype(np.float64))
        out["backward_max_rel_err"] = relerr(df[sel].double().cpu().numpy(), ref_b)
        f64p.forward(x64, c64)
        f64p.backward(v64, df64)
        out["f64_gpu_path"]["forward_max_rel_err"] = relerr(c64[sel].cpu().numpy(), d.ref)
        out["f64_gpu_path"]["backward_max_rel_err"] = relerr(df64[sel].cpu().numpy(), ref_b)
        out["err_sample"] = ("%d functions; forward vs oracle route 1, backward df = L^T v (v ~ N(0,1)) vs the "
                             "oracle's route 1 transposed" % len(d.sample))
    del d, split, f64p
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


def ragged_line(args, leg, torch, dist, flush, rank, world, peaks, peak_src):
    """--workload ragged_10000: the ragged batch as the timed workload."""
    fixed = None
    if args.transform is not None:
        fixed = ({"reg": leg.TRANSFORM_REG, "stockham": leg.TRANSFORM_STOCKHAM, "sine": leg.TRANSFORM_SINE}[
            args.transform], args.radix)
    r = ragged(leg, torch, flush, rank, peaks, peak_src, rank == 0, steps=args.steps, warmup=args.warmup,
               tile=args.tile, transform=fixed)
    ms = max_over_ranks(torch, dist, r["ms_per_step"], "cuda")
    if rank == 0:
        line = {"metric": METRIC, "value": whole_job_rate(world, r["coefficients"], ms), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_STR["split_fp16"],
                "data": "synthetic",
                "config": {"workload": "ragged_10000", "functions": r["functions"], "buckets": r["buckets"],
                           "l2": "flushed (512 MiB write) before every timed step"},
                "max_rel_err": r.get("max_rel_err"), "err_sample": r.get("err_sample"), "roofline": r["roofline"],
                "stages_ms": r["stages_ms"], "tile_width": r["tile_width"], "bucket_transforms": r["bucket_transforms"],
                "gpu_launches": r["gpu_launches_per_step"] * args.steps}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def differentiation_line(args, leg, torch, dist, flush, rank, world, peaks, peak_src):
    """--workload diff_b1024_k4097: forward + backward (leg_forward, leg_backward)
    at B=1024, K=4097, N=2048, M=8192 as the timed workload."""
    fixed = None
    if args.transform is not None:
        fixed = {"reg": leg.TRANSFORM_REG, "stockham": leg.TRANSFORM_STOCKHAM, "sine": leg.TRANSFORM_SINE}[args.transform]
    r = differentiation(leg, torch, flush, rank, peaks, peak_src, rank == 0, steps=args.steps, warmup=args.warmup,
                        transform=fixed)
    ms = max_over_ranks(torch, dist, r["ms_per_step"], "cuda")
    if rank == 0:
        line = {"metric": METRIC + " (forward + backward)", "value": whole_job_rate(world, 1024 * 2048, ms),
                "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_STR["split_fp16"],
                "data": "synthetic",
                "config": {"workload": "cheb_b1024_k4097_n2048_m8192", "B": 1024, "K": 4097, "N": 2048, "M": 8192,
                           "step": "forward + backward", "l2": "flushed (512 MiB write) before every timed step"},
                "gpu_launches": r["gpu_launches_per_step"] * args.steps}
        line.update({k: r[k] for k in r if k not in ("value", "unit", "ms_per_step", "gpu_launches_per_step")})
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def gpu_arm(args, rank, world, local_rank):
    import torch
    import paper_1106_0463_gb300 as leg

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    name = args.workload
    peaks, peak_src = load_peaks()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    with_ref = rank == 0
    if name == "ragged_10000":
        ragged_line(args, leg, torch, dist, flush, rank, world, peaks, peak_src)
        return
    if name == "diff_b1024_k4097":
        differentiation_line(args, leg, torch, dist, flush, rank, world, peaks, peak_src)
        return

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # ---------------- the headline: tuned, then the timed region on the selected path
    head = Dense(leg, torch, name, rank, with_ref, extra=36)
    B, N = head.B, head.N
    if args.tile is not None and args.transform is not None:
        plan = head.plan(args.path)
        if args.path in ("split_fp16", "bf16"):
            plan.set_tile(args.tile)
        plan.set_transform({"reg": leg.TRANSFORM_REG, "stockham": leg.TRANSFORM_STOCKHAM,
                            "sine": leg.TRANSFORM_SINE}[args.transform])
        tuned = {"tn": args.tile, "fft": plan.transform, "source": "command line"}
        if args.radix:
            plan.set_transform(plan.transform, args.radix)
        if args.path == "split_fp16":
            head.retile()
    else:
        tuned = head.autotune(args.path)   # GEMM tile width and transform kernel, timed on this batch
        tuned["source"] = "leg_plan_autotune on this batch"
    barrier()
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    phys = vis.split(",")[local_rank].strip() if vis else str(local_rank)
    # one batch at a time (L2 flushed before each), with the error, stage times and rooflines
    res = head.run(args.path, flush, args.steps, args.warmup, peaks, peak_src, clocks=ClockSampler(phys),
                   warm_steps=min(args.steps, 50))
    barrier()
    single_ms = max_over_ranks(torch, dist, float(np.sum(res["_ts"])), "cuda") / args.steps
    single = {"value": whole_job_rate(world, B * N, single_ms), "ms_per_step": single_ms, "steps": args.steps,
              "api": "leg_forward, one batch per step, each step between its own pair of events",
              "l2": "flushed (512 MiB write) before every step", "clocks": res["_clk"]}

    # the timed region: `steps` batches of the workload in one leg_forward_batches
    # call (batch b = the workload's batch times 1 + b/64, distinct device buffers
    # holding more bytes than L2); for split-FP16 plans batch b's transform runs
    # beside batch b+1's split and GEMM
    plan = head.plan(args.path)
    f1 = head.inputs(args.path)
    scale = 1.0 + torch.arange(args.steps, device="cuda", dtype=f1.dtype) / 64.0
    fb = (f1.unsqueeze(0) * scale.view(-1, 1, 1)).contiguous()
    cb = torch.empty((args.steps, B, N), dtype=plan.io_dtype, device="cuda")
    nw = min(max(args.warmup, 2), args.steps)
    plan.forward_batches(fb[:nw], cb[:nw])
    barrier()
    clk = ClockSampler(phys)
    clk.start()
    clk.wait_first()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.forward_batches(fb, cb)
    e1.record()
    e1.synchronize()
    batches_clk = clk.stop()
    barrier()
    ms_per_step = max_over_ranks(torch, dist, e0.elapsed_time(e1) / args.steps, "cuda")
    value = whole_job_rate(world, B * N, ms_per_step)
    same = all(bool(torch.equal(cb[b], plan.forward(fb[b]))) for b in sorted({0, 1, args.steps - 1}))
    # stage times inside the pipeline (events on each stage's stream), for the rooflines
    pms = plan.forward_batches_profiled(fb, cb)
    plan.status()
    pipe_stages = {"input_split": pms[0], "abel_gemm": pms[1], "transform": pms[2],
                   "how": "mean per batch over a leg_forward_batches_profiled call on the timed region's batches: "
                          "CUDA events on each stage's own stream inside the pipeline; the transform runs at low "
                          "priority on the SMs the next batch's GEMM leaves free, so its span covers most of that "
                          "GEMM (its kernel efficiency is in transform_roofline, timed on the whole GPU)"}
    pipe_roof = gemm_roofline(B, head.rows, head.K, head.Kp, args.path, pms[1], peaks, peak_src, TRAFFIC, name)
    batches_in_mb = fb.numel() * fb.element_size() / 1e6
    del fb, cb

    # ---------------- e2e through the public API with pinned host buffers.
    # (1) the timed region's batches from host memory: one
    # leg_forward_host_batches call on `steps` batches (batch b = the workload's
    # batch times 1 + b/64), each batch's input copied by a copy engine while
    # the batches before it compute, its coefficients written into host memory
    # by its transform; (2) leg_forward_host calls back to back with
    # leg_plan_set_host_overlap(plan, 1); (3) one leg_forward_host call at a
    # time in the default ordering, L2 flushed before each.
    plan = head.plan(args.path)
    f1 = head.inputs(args.path)
    scale = 1.0 + torch.arange(args.steps, device="cuda", dtype=f1.dtype) / 64.0
    fbh = (f1.unsqueeze(0) * scale.view(-1, 1, 1)).cpu().pin_memory()
    cbh = torch.empty((args.steps, B, N), dtype=plan.io_dtype).pin_memory()
    nw = min(max(args.warmup, 2), args.steps)
    plan.forward_host_batches(fbh[:nw], cbh[:nw], sync=False)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.forward_host_batches(fbh, cbh, sync=False)
    e1.record()
    e1.synchronize()
    batches_ms = max_over_ranks(torch, dist, e0.elapsed_time(e1) / args.steps, "cuda")
    same_b = all(bool(torch.equal(cbh[b], plan.forward(fbh[b].cuda()).cpu())) for b in sorted({0, args.steps - 1}))
    del fbh, cbh

    f_host = torch.from_numpy(head.f_np).to(plan.io_dtype).pin_memory()
    c_host = torch.empty((B, N), dtype=plan.io_dtype).pin_memory()
    single_ts, _ = time_steps(torch, lambda: plan.forward_host(f_host, c_host, sync=False), flush, args.steps,
                              args.warmup)
    plan.set_host_overlap(True)
    for _ in range(args.warmup):
        plan.forward_host(f_host, c_host, sync=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        plan.forward_host(f_host, c_host, sync=False)
    e1.record()
    e1.synchronize()
    calls_ms = max_over_ranks(torch, dist, e0.elapsed_time(e1) / args.steps, "cuda")
    plan.set_host_overlap(False)
    f_dev = head.inputs(args.path)
    same = bool(torch.equal(c_host, plan.forward(f_dev).cpu()))
    c_dev = torch.empty((B, N), dtype=plan.io_dtype, device="cuda")
    copy_ms = {}
    for direction, dst, src in (("h2d", f_dev.clone(), f_host), ("d2h", c_host, c_dev)):
        ts, _ = time_steps(torch, lambda: dst.copy_(src, non_blocking=True), flush, 10, 2)
        copy_ms[direction] = float(np.mean(ts))
    single_step = max_over_ranks(torch, dist, float(np.mean(single_ts)), "cuda")
    staged = args.path in ("split_fp16", "bf16")
    e2e = {"value": whole_job_rate(world, B * N, batches_ms), "unit": UNIT,
           "h2d_bytes_per_step": f_host.numel() * f_host.element_size(),
           "d2h_bytes_per_step": c_host.numel() * c_host.element_size(),
           "api": ("leg_forward_host_batches on pinned host buffers (%d batches of %d functions, one call): each "
                   "batch's f crosses the host link by a copy engine into a device staging buffer while the "
                   "batches before it compute, and its transform writes c into the pinned host buffer"
                   % (args.steps, B) if args.path == "split_fp16" else
                   "leg_forward_host_batches on pinned host buffers (leg_forward_host on each batch in turn)"),
           "timing": "one call between a pair of CUDA events, every batch's copies inside; the %d batches' f "
                     "(%.0f MB, in distinct host buffers) and the operator planes exceed L2"
                     % (args.steps, args.steps * f_host.numel() * f_host.element_size() / 1e6),
           "ms_per_step": batches_ms, "bit_identical_to_leg_forward": same_b and same, "bare_copy_ms": copy_ms,
           "note": "the host link's %.1f MB per batch (bare copies %.0f + %.0f us) run during the GEMMs of the "
                   "batches in flight, so the figure comes out near the device-resident one; the single-call "
                   "figure below shows the copies exposed" % (
                       (f_host.numel() * f_host.element_size() + c_host.numel() * c_host.element_size()) / 1e6,
                       copy_ms["h2d"] * 1e3, copy_ms["d2h"] * 1e3),
           "calls_with_host_overlap": {
               "value": whole_job_rate(world, B * N, calls_ms), "ms_per_step": calls_ms,
               "api": ("leg_forward_host calls back to back with leg_plan_set_host_overlap(plan, 1): each call's "
                       "f copied into a staging buffer during the previous call's kernels"
                       if staged else "leg_forward_host calls back to back")},
           "single_call": {"value": whole_job_rate(world, B * N, single_step), "ms_per_step": single_step,
                           "api": "leg_forward_host, default ordering (each call after the work queued before "
                                  "it; pinned buffers read and written in place by the kernels)",
                           "l2": "flushed (512 MiB write) before every call"}}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return

    roof = pipe_roof   # the GEMM: the pipeline's critical path
    single["stages_ms"] = res["stages_ms"]
    single["gemm_roofline"] = res["gemm_roofline"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPE_STR[args.path], "data": "synthetic",
        "config": {"workload": name, "B": B, "K": head.K, "N": N, "M": head.M, "Q": (head.K + 1) // 2,
                   "path": args.path, "tile_width": head.tn,
                   "launch_settings": {"tile_width_setting": tuned["tn"],
                                       "transform": TRANSFORM_NAMES[tuned["fft"]],
                                       "transform_radix": head.plan(args.path).transform_radix,
                                       "chosen_by": tuned["source"]},
                   "schedule": ("%d batches of %d functions in one leg_forward_batches call: each batch's input "
                                "split and Abel GEMM on a high-priority stream, the previous batch's transform on "
                                "a low-priority one (the SMs the GEMM's CTA pairs leave free); every kernel is "
                                "leg_forward's for one batch" % (args.steps, B)
                                if args.path == "split_fp16" else
                                "%d batches of %d functions in one leg_forward_batches call (leg_forward on each "
                                "in turn)" % (args.steps, B)),
                   "l2": "not flushed between batches: inputs larger than L2 (the %d batches' f, %.0f MB in "
                         "distinct buffers, and the operator planes, %.0f MB); the single_batch figure flushes "
                         "L2 before every step" % (args.steps, batches_in_mb, 3 * (head.rows - 1) * head.Kp * 2 / 1e6),
                   "inputs": "random decaying Chebyshev series sampled at CL nodes, FP32, seeded; batch b of the "
                             "timed region is that batch times 1 + b/64"},
        "max_rel_err": res.get("max_rel_err"), "tolerance": 1e-6,
        "err_sample": (res.get("err_sample", "") + " vs the FP64 oracle " + oracle_route_name(name) +
                       "; the timed region's batches 0, 1 and last equal leg_forward on them bit for bit: %s"
                       % same),
        "roofline": roof, "stages_ms": pipe_stages,
        "transform_roofline": res["transform_roofline"], "plan_build_s": head.plan_s.get(args.path),
        "e2e": e2e, "clocks": batches_clk or res["_clk"], "gpu_launches": LAUNCHES[args.path] * args.steps,
        "l2_warm": res.get("l2_warm"), "single_batch": single,
    }
    wl = {}
    if not args.no_extras:
        # precision sweep and the sine form on the headline workload
        # every path one batch per step, L2 flushed before each (like with like)
        sweep = {args.path: {"value": single["value"] / world, "ms_per_step": single["ms_per_step"],
                             "max_rel_err": line["max_rel_err"]}}
        for p in ("f64", "f32", "bf16", "split_fp16"):
            if p == args.path:
                continue
            r = head.run(p, flush, 3 if p == "f64" else 10, 2, peaks, peak_src)
            sweep[p] = {"value": r["value"], "ms_per_step": r["ms_per_step"], "max_rel_err": r.get("max_rel_err"),
                        "stages_ms": r["stages_ms"]}
        wl["precision_sweep_" + name] = sweep
        if args.path == "split_fp16":
            # ablation: the collapsed operator L = R A (N x K, built once in FP64) in one
            # split GEMM with no transform, on the same inputs
            t0 = time.time()
            coll = leg.Plan(N, head.M, head.K, 0, leg.SPLIT_FP16, flags=leg.FLAG_COLLAPSED)
            torch.cuda.synchronize()
            build_s = time.time() - t0
            fin = head.inputs("split_fp16")
            cc = torch.empty((B, N), dtype=torch.float32, device="cuda")
            coll_tile = coll.autotune(fin)   # the GEMM tile width, timed on this batch
            ts, _ = time_steps(torch, lambda: coll.forward(fin, cc), flush, 20, 3)
            coll.status()
            ms = float(np.mean(ts))
            ent = {"value": B * N / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "launches_per_step": 2,
                   "plan_build_s": build_s, "tuned": coll_tile,
                   "useful_gemm_tflops": 2.0 * B * N * head.K / (ms / 1e3) / 1e12,
                   "note": "ablation, not the paper's route: L = R A multiplied out at plan time"}
            if head.ref is not None:
                ent["max_rel_err"] = relerr(cc[torch.from_numpy(head.sample).cuda()].double().cpu().numpy(),
                                            head.ref)
            wl["collapsed_split_fp16_" + name] = ent
            del coll
        line["speedup_vs_fp64_gpu_path"] = sweep[args.path]["value"] / sweep["f64"]["value"]
        line["speedup_basis"] = "one batch per step on both paths, L2 flushed before each (single_batch)"
        other = leg.TRANSFORM_REG if tuned["fft"] == leg.TRANSFORM_SINE else leg.TRANSFORM_SINE
        r = head.run(args.path, flush, 20, 3, peaks, peak_src, transform=other)
        wl[("real_even_transform_" if other == leg.TRANSFORM_REG else "sine_form_") + name] = strip(r)
        del head
        # the B=4096, K=1025 workload: split, plain FP32, FP64, collapsed
        c2name = "cheb_b4096_k1025_n512_m2048"
        c2 = Dense(leg, torch, c2name, rank, with_ref, extra=24)
        sub = {}
        sub["split_fp16"] = strip(c2.run("split_fp16", flush, 50, 3, peaks, peak_src, warm_steps=50))
        sub["split_fp16_sine_form"] = strip(c2.run("split_fp16", flush, 50, 3, peaks, peak_src,
                                                   transform=leg.TRANSFORM_SINE))
        # the same as a stream of 20 batches (distinct buffers, 336 MB) through leg_forward_batches
        p2, nb2 = c2.plan("split_fp16"), 20
        fb2 = c2.inputs("split_fp16").unsqueeze(0).expand(nb2, -1, -1).contiguous()
        cb2 = torch.empty((nb2, c2.B, c2.N), dtype=torch.float32, device="cuda")
        p2.forward_batches(fb2[:3], cb2[:3])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        p2.forward_batches(fb2, cb2)
        e1.record()
        e1.synchronize()
        ms2 = e0.elapsed_time(e1) / nb2
        sub["split_fp16_sine_form_batches"] = {
            "value": c2.B * c2.N / (ms2 / 1e3), "ms_per_step": ms2, "batches": nb2,
            "api": "leg_forward_batches (each batch's transform beside the next batch's split and GEMM)",
            "bit_identical_to_leg_forward": bool(torch.equal(cb2[nb2 - 1], p2.forward(fb2[nb2 - 1])))}
        del fb2, cb2
        sub["f32"] = strip(c2.run("f32", flush, 20, 3, peaks, peak_src))
        sub["f32_sine_form"] = strip(c2.run("f32", flush, 20, 3, peaks, peak_src, transform=leg.TRANSFORM_SINE))
        sub["f64"] = strip(c2.run("f64", flush, 3, 1, peaks, peak_src))
        sub["speedup_vs_fp64_gpu_path"] = sub["split_fp16"]["value"] / sub["f64"]["value"]
        coll = leg.Plan(c2.N, c2.M, c2.K, 0, leg.SPLIT_FP16, flags=leg.FLAG_COLLAPSED)
        cc = torch.empty((c2.B, c2.N), dtype=torch.float32, device="cuda")
        ts, _ = time_steps(torch, lambda: coll.forward(c2.f32, cc), flush, 20, 3)
        coll.status()
        sub["collapsed_split_fp16"] = {"value": c2.B * c2.N / (np.mean(ts) / 1e3), "ms_per_step": float(np.mean(ts)),
                                       "launches_per_step": 2}
        if c2.ref is not None:
            sub["collapsed_split_fp16"]["max_rel_err"] = relerr(
                cc[torch.from_numpy(c2.sample).cuda()].double().cpu().numpy(), c2.ref)
        if rank == 0 and args.cpu_route2:   # minutes of CPU time for the operator build
            sub["cpu_baseline_route2_explicit_operator"] = oracle_route2_operator_rate(c2name)
        wl[c2name] = sub
        del c2, coll
        wl["ragged_10000"] = ragged(leg, torch, flush, rank, peaks, peak_src, with_ref)
        wl["cheb_b1024_k4097_n2048_m8192"] = differentiation(leg, torch, flush, rank, peaks, peak_src, with_ref)
        wl["genfn_plain_n64"] = plain_method(leg, torch)
        from oracle import oracle as O
        wl["table1_abs_x_3_2_plain_sine_form"] = table1_plain(leg, torch, O)
        line["workloads"] = wl
    if not args.no_cpu_baseline:
        line["cpu_baseline"], _, _ = oracle_rate(name)
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
