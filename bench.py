"""Benchmark of the GSW hologram engine (one JSON line on stdout).

Workload (default): rand100_512 -- a 512 x 512 SLM, 100 traps with x, y ~ U[-40, 40] um and
z ~ U[-10, 10] um (seed 0), 30 GSW iterations with fast sincos, 8-bit phase output.
One step = upload of the starting phases (device to device) + hot_gsw(30) + the 8-bit
encoding of the result, i.e. one complete hologram.

Metric: GSW pixel-trap updates per second (one update = one (pixel, trap) pair through one
full iteration, forward field and back-projection), summed over all GPUs; holograms/s is
reported beside it.  --gpus N > 1 runs N independent replicas (one per rank; the path has
no exchange step), timed between barriers, max over ranks.

--impl reference times the FP64 CPU oracle on the host cores instead (bounded sample).
--single K runs hot_gsw(K) once on the workload (no timing): the program that the ncu
summaries under profiles/ capture.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "GSW pixel-trap updates/s (512x512 px, M=100, 30 iterations)"
UNIT = "updates/s"
SFU_LANES_PER_SM = 16          # sin.approx / cos.approx results per clock per SM (sm_103a)
SFU_OPS_PER_UPDATE = 4         # one sin + one cos in the forward field, one each in back-projection
SFU_OPS_PER_UPDATE_ONCE = 2    # one-exponential step: one sin + one cos per pair and iteration
FMA_LANES_PER_SM = 128         # FP32 FMA results per clock per SM (sm_103a)
FMA_OPS_PER_UPDATE = 8         # separable mode: one complex multiply-add (4 FMA) in each step
TC_FLOPS_PER_UPDATE = 48       # tensor mode: 2 complex MACs (16 flops) x 3 MMAs per product (hi/lo split)
F16_PER_BF16 = 1.0             # nominal dense FP16 / BF16 tensor rate (GB300): the same
L2_FLUSH_BYTES = 256 << 20     # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="engine", choices=["engine", "reference"])
    ap.add_argument("--workload", default="rand100_512")
    ap.add_argument("--precision", default=None, choices=["accurate", "fast", "separable", "tensor"],
                    help="override the workload's mode (separable: its own FP32-FMA roofline; "
                         "tensor: the FP16 tensor-core roofline)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision-report", action="store_true",
                    help="errors of the four precision modes against the FP64 oracle, per result")
    ap.add_argument("--m-sweep", action="store_true",
                    help="time per GSW iteration vs trap count M = 1..4096 on a 768^2 SLM (Fig. 5 analogue)")
    ap.add_argument("--grid-sweep", action="store_true",
                    help="efficiency and uniformity vs trap count on n x n grids (n = 2..9, 768^2 SLM)")
    ap.add_argument("--single", type=int, default=0, metavar="K",
                    help="run hot_gsw(K) once on the workload and print e, u (no timing; for profilers)")
    ap.add_argument("--merge", type=int, default=1, choices=[1, 2, 4],
                    help="with --single: schedule blocks per launched block of the GSW step "
                         "(hot_set_block_merge; the timed runs let the autotuner choose)")
    ap.add_argument("--direct", action="store_true",
                    help="with --single: the direct step kernels even where the one-exponential step "
                         "applies (hot_set_once(0))")
    ap.add_argument("--cpu-sample-iters", type=int, default=0,
                    help="GSW iterations of the CPU-baseline sample (0: the workload's own count)")
    return ap.parse_args()


def workload_config(w, extra=None):
    cfg = {"workload": f"{w.name}: {w.W}x{w.H} px, M={w.M} traps, {w.iters} GSW iterations, "
                       f"{w.precision} sincos" + (", 8-bit output" if w.quantize else ""),
           "W": w.W, "H": w.H, "M": w.M, "iters": w.iters, "precision": w.precision,
           "output": "u8" if w.quantize else "f32", "seed": 0}
    if extra:
        cfg.update(extra)
    return cfg


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first_sample(self, timeout: float = 5.0):
        """Blocks until nvidia-smi has printed one sample (so the timed region is covered)."""
        t0 = time.time()
        while self.proc and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.01)

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle (CPU)

def cpu_baseline(w, iters: int):
    """The FP64 oracle as it stands, on this host's cores, over `iters` full GSW iterations of
    the workload (a bounded sample of its `w.iters`)."""
    import oracle
    cores = oracle.set_threads()
    t0 = time.perf_counter()
    oracle.gsw(w.geom, w.xyz, iters, w.phi0, w.w0)
    dt = time.perf_counter() - t0
    return {"value": w.N * w.M * iters / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{iters} of {w.iters} GSW iterations of {w.name} (FP64, all {w.N} pixels, "
                      f"all {w.M} traps, plus one final forward), {dt:.2f} s"}


def run_reference(args):
    from paper_0907_4027_gb300 import workloads as wl
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = wl.NAMED[args.workload]()
    iters = 2
    for _ in range(args.warmup):
        cpu_baseline(w, iters)
    times, cores = [], None
    t_all = time.perf_counter()
    for _ in range(args.steps):
        r = cpu_baseline(w, iters)
        times.append(w.N * w.M * iters / r["value"])
        cores = r["cores"]
    total = time.perf_counter() - t_all
    value = w.N * w.M * iters * args.steps / sum(times)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        "config": workload_config(w, {"reference_step": f"{iters} GSW iterations (bounded sample)"}),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{iters} of {w.iters} GSW iterations of {w.name} per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- engine (GPU)

def kernel_source_hash(kernel: str = "step") -> str:
    """First 16 hex digits of the SHA-256 of the kernels' source with comments and blank space
    removed (so that a profile stays matched to code whose comments alone changed)."""
    name = "tc_kernels.cuh" if kernel == "tc" else "gsw_kernels.cuh"
    src = open(os.path.join(ROOT, "paper_0907_4027_gb300", "csrc", name)).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    src = " ".join(src.split())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def profiled_traffic(workload: str, kernel: str = "step"):
    """DRAM bytes per launch of the fused step kernel (gsw_step / gsw_sep), or per iteration of
    the tensor mode's three kernels (gsw_tc), from the committed ncu summary, if the summary was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"gsw_{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not h or not b or h.group(1) != kernel_source_hash(kernel):
        return None
    return float(b.group(1))


def run_engine(args):
    import torch
    import torch.distributed as dist

    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot, sharded, workloads as wl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    w = wl.NAMED[args.workload]()
    if args.precision:
        w.precision = args.precision
    sep = w.precision == "separable"
    tensor = w.precision == "tensor"
    stream = torch.cuda.current_stream()
    h = hot.Hologram(w.W, w.H, w.pitch, w.wavelength, w.focal, stream.cuda_stream, w.precision)
    h.set_traps(w.xyz, w.w0)
    phi0 = torch.tensor(w.phi0, dtype=torch.float32, device="cuda")
    out = torch.empty(w.N, dtype=torch.uint8 if w.quantize else torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    fmt = "u8" if w.quantize else "f32"

    def step():
        h.set_phase(phi0)
        h.gsw(w.iters, metrics=False)
        h.phase(fmt, out=out)

    # tiling picked by the autotuner (untimed setup; phases and weights are kept)
    h.set_phase(phi0)
    t_tune = time.perf_counter()
    if tensor:  # fixed tiles: nothing to tune
        tuned = {"rows": None, "blocks_per_sm": None, "chunk": None, "merge": None, "once": False,
                 "us_per_iter": None}
    else:
        tuned = h.autotune(w.iters)
    tuned["seconds"] = time.perf_counter() - t_tune

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # timed region: per-step events, L2 flushed between steps (outside the events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = h.launches
    with ClockSampler(local) as clk:
        clk.wait_first_sample()
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    launches = h.launches - launches0
    if world > 1:
        dist.barrier()
    # Dominant kernel: one step-kernel launch per GSW iteration.  Its duration in the real
    # (graph-replayed, programmatically dependent) pipeline is the marginal time of an
    # iteration: CUDA events around hot_gsw(K) and hot_gsw(K_small) on the launching stream.
    k_small = max(1, w.iters // 3)
    n_roof = min(args.steps, 50)
    evk = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(n_roof)]
    for i in range(n_roof):
        flush.fill_(float(i))
        h.set_phase(phi0)
        evk[i][0].record(stream)
        h.gsw(w.iters, metrics=False)
        evk[i][1].record(stream)
        flush.fill_(float(i))
        h.set_phase(phi0)
        evk[i][2].record(stream)
        h.gsw(k_small, metrics=False)
        evk[i][3].record(stream)
    torch.cuda.synchronize()
    per_iter = sorted((e[0].elapsed_time(e[1]) - e[2].elapsed_time(e[3])) / (w.iters - k_small) for e in evk)
    iter_ms = per_iter[len(per_iter) // 2]
    # per-kernel device times: the same steps again, kernels launched one by one between
    # CUDA events on the launching stream (the timed region above replays CUDA graphs)
    n_prof = min(args.steps, 20)
    h.profile(True)
    for i in range(n_prof):
        flush.fill_(float(i))
        step()
    prof = h.profile_read()
    h.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sharded.max_over_ranks(sum(step_ms))  # replicas: the slowest rank's timed region
    updates_per_step = w.N * w.M * w.iters
    value = world * updates_per_step * args.steps / (total_ms * 1e-3)

    # roofline of the dominant kernel (weight update + back-projection + forward field of one
    # GSW iteration per launch)
    # Dominant kernel: the fused step kernel, one launch per GSW iteration (one unit of work
    # per pair).  Its duration in the real pipeline (graph replay, each launch a programmatic
    # dependent of the previous one) is the marginal time of an iteration; the profiled pass
    # (launches one by one between CUDA events) gives the unpipelined duration and the shares.
    step_kernel_ms, step_kernel_n = prof["step"]
    units_per_launch = 1.0
    avg_launch_s = iter_ms * 1e-3
    achieved = w.N * w.M * units_per_launch / avg_launch_s
    dev = torch.cuda.get_device_properties(local)
    sm_max_mhz = 2070.0
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        sm_max_mhz = float(json.load(open(peaks_path)).get("sm_max_mhz", sm_max_mhz))
    once = bool(tuned.get("once"))  # the one-exponential step (hot_set_once), if the autotuner kept it
    if sep or tensor:
        lanes, ops, pipe = FMA_LANES_PER_SM, FMA_OPS_PER_UPDATE, "FP32 FMA"
    else:
        lanes, ops, pipe = SFU_LANES_PER_SM, SFU_OPS_PER_UPDATE_ONCE if once else SFU_OPS_PER_UPDATE, "SFU"
    peak = dev.multi_processor_count * lanes * sm_max_mhz * 1e6 / ops
    peak_direct = dev.multi_processor_count * SFU_LANES_PER_SM * sm_max_mhz * 1e6 / SFU_OPS_PER_UPDATE
    lanes_measured = hot.hot_sfu_rate(3 if sep or tensor else 0)[0]
    traffic = profiled_traffic(args.workload, "tc" if tensor else "sep" if sep else "once" if once else "step")
    kernel_share = {k: round(v[0] / max(sum(x[0] for x in prof.values()), 1e-12), 4)
                    for k, v in prof.items()}

    # end to end through the public API with host buffers
    xyz = w.xyz.copy()
    phi_host = torch.tensor(w.phi0, dtype=torch.float32).pin_memory()
    g_host = torch.empty(w.N, dtype=torch.uint8 if w.quantize else torch.float32).pin_memory()
    phi_np, g_np = phi_host.numpy(), g_host.numpy()

    def e2e_step():
        h.set_traps(xyz, w.w0)
        h.set_phase(phi_np)
        e, u = h.gsw(w.iters, metrics=True)
        h.phase(fmt, out=g_np)
        return e, u

    from paper_0907_4027_gb300.hot import hot_phase_out, HOT_FMT_U8, HOT_FMT_F32  # noqa: F401
    for _ in range(2):
        e2e_step()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    n_e2e = min(args.steps, 200)
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        eu = e2e_step()
    torch.cuda.synchronize()
    e2e_s = sharded.max_over_ranks(time.perf_counter() - t0)
    e2e_value = world * updates_per_step * n_e2e / e2e_s
    h2d = w.N * 4 + w.M * 3 * 8 + w.M * 8
    d2h = w.N * (1 if w.quantize else 4) + 16

    launch_timing = (f"marginal iteration time of graph-replayed hot_gsw({w.iters}) vs hot_gsw({k_small}), "
                     f"CUDA events, median of {n_roof}")
    if tensor:
        # three launches per iteration (operand P, back-projection GEMM, forward GEMM); the
        # GEMMs' algorithmic FP16 MMA work is 48 flops per pair (no padding counted)
        bf16 = float(json.load(open(peaks_path))["bf16_tflops"]) if os.path.exists(peaks_path) else 1900.0
        tc_peak = bf16 * F16_PER_BF16
        tc_achieved = TC_FLOPS_PER_UPDATE * w.N * w.M / avg_launch_s / 1e12
        roofline = {"bound": "tensor", "achieved": tc_achieved, "peak": tc_peak, "unit": "TFLOP/s",
                    "frac": tc_achieved / tc_peak, "traffic": traffic,
                    "kernel": "tc_prep_kernel + tc_gemm_kernel<back> + tc_gemm_kernel<fwd> (one GSW iteration)",
                    "peak_basis": f"measured bf16 burst {bf16:.1f} TFLOP/s (MEASURED_PEAKS.json); FP16 "
                                  f"runs at the bf16 rate (nominal ratio {F16_PER_BF16:.1f})",
                    "flops_per_update": TC_FLOPS_PER_UPDATE, "avg_iteration_us": avg_launch_s * 1e6,
                    "frac_of_value": TC_FLOPS_PER_UPDATE * value / world / 1e12 / tc_peak,
                    "updates_per_s": achieved,
                    "fp32_fma_roofline_updates_per_s": peak, "launch_timing": launch_timing,
                    "avg_iteration_us_unpipelined": step_kernel_ms * 1e3 / max(step_kernel_n, 1)}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "updates/s",
                    "frac": achieved / peak, "traffic": traffic,
                    "frac_of_value": value / world / peak,
                    "frac_of_value_note": "the bench value (whole step: forward of the starting phases, "
                                          "iterations, finalize, 8-bit encoding) over the same peak",
                    "kernel": ("gsw_sep_kernel<back, fwd>" if sep else
                               f"gsw_once_kernel<{w.precision}, back>" if once else
                               f"gsw_step_kernel<{w.precision}, back, fwd>") + " (one GSW iteration per launch)",
                    "peak_basis": f"{dev.multi_processor_count} SMs x {lanes} {pipe} "
                                  f"lanes/clk x {sm_max_mhz:.0f} MHz / {ops} "
                                  f"{pipe} ops per update",
                    "lanes_per_clk_per_sm_measured": round(lanes_measured, 2),
                    **({"frac_direct_form": achieved / peak_direct,
                        "frac_direct_form_note": "the same rate over the direct method's bound (two "
                                                 "exponentials per pair and iteration, 4 SFU ops per update); "
                                                 "the one-exponential step evaluates each pair's exponential "
                                                 "once, so its own bound is half as many SFU ops"}
                       if once else {}),
                    "avg_launch_us": avg_launch_s * 1e6,
                    "units_per_launch": units_per_launch,
                    "launch_timing": launch_timing,
                    "avg_launch_us_unpipelined": step_kernel_ms * 1e3 / max(step_kernel_n, 1)}
    if rank == 0:
        metric = METRIC if args.workload == "rand100_512" else \
            f"GSW pixel-trap updates/s ({w.W}x{w.H} px, M={w.M}, {w.iters} iterations)"
        line = {
            "metric": metric, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16x3" if tensor else "f32", "data": "synthetic",
            "config": workload_config(w, {
                "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                "l2": "flushed between steps (256 MB write outside the step events)",
                "tiling": {k: tuned[k] for k in ("rows", "blocks_per_sm", "chunk", "merge", "once")},
                "autotune": {"us_per_iter": tuned["us_per_iter"], "seconds": round(tuned["seconds"], 3),
                             "search": "the one-exponential step against a coordinate search over "
                                       "rows/blocks_per_sm/chunk/merge of the direct kernels, best of 3 graph replays"},
                "timing": "CUDA events per step on the launching stream, summed; hot_gsw replays "
                          "one CUDA graph per call; roofline kernel times from a second pass of "
                          "the same steps with per-launch events"}),
            "holograms_per_s": world * args.steps / (total_ms * 1e-3),
            "roofline": roofline,
            # per step: the dominant kernel's time in the real pipeline (iterations x marginal
            # iteration time; at most ms_per_step) and the rest of the step
            "kernel_time_ms": {"step_kernel_pipelined": round(w.iters * iter_ms, 4),
                               "rest_of_step": round(total_ms / args.steps - w.iters * iter_ms, 4)},
            # shares of device time from a second pass with every launch bracketed by its own
            # events (launches serialised: per-launch times there exceed the pipelined ones)
            "kernel_time_share_unpipelined": kernel_share,
            "kernel_time_ms_unpipelined": {k: round(v[0] / n_prof, 4) for k, v in prof.items()},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "api": "hot_set_traps + hot_set_phase (pinned host) + hot_gsw + hot_phase_out (host)",
                    "final_e": eu[0], "final_u": eu[1]},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, args.cpu_sample_iters or w.iters)
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_adam(args):
    """Differentiable form (diff256_1024): Adam on the phases for the trap-intensity loss
    L = -sum log|V_m|^2 + 10 var|V_m|^2, 200 steps, lr 1.0, in the fast, separable and accurate
    modes (--precision picks one), three ways: (a) the autograd Function over the
    forward-field and adjoint kernels with the loss in PyTorch; (b) the loss and its gradient from
    one library call (hot_intensity_loss) with PyTorch's fused Adam; (c) (b) with each step
    captured in a CUDA graph (three library kernels and the fused Adam update, no host work per
    step).  Beside plain GSW on the same traps and phi0 at the same mode.  The line's value is (c)
    in the workload's mode."""
    import torch
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import autograd as ag, hot, workloads as wl

    base = wl.NAMED[args.workload]()
    modes = [args.precision] if args.precision else ["fast", "separable", "accurate"]
    stream = torch.cuda.current_stream()
    beta = 10.0

    def eu(V):
        I = (V.abs() ** 2).double()
        return float(I.sum()), float(1 - (I.max() - I.min()) / (I.max() + I.min()))

    def timed(run, n_steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        run(n_steps)
        ev[1].record(stream)
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1])

    results = {}
    for mode in modes:
        w = wl.NAMED[args.workload]()
        w.precision = mode
        h = hot.Hologram(w.W, w.H, w.pitch, w.wavelength, w.focal, stream.cuda_stream, w.precision)
        h.set_traps(w.xyz, w.w0)
        out = {}

        # (a) autograd, loss in PyTorch
        phi = torch.tensor(w.phi0, dtype=torch.float32, device="cuda", requires_grad=True)
        opt = torch.optim.Adam([phi], lr=1.0)

        def step_a(n):
            for _ in range(n):
                opt.zero_grad(set_to_none=True)
                ag.trap_intensity_loss(ag.trap_fields(h, phi), beta).backward()
                opt.step()
        step_a(3)
        with torch.no_grad():
            phi.copy_(torch.tensor(w.phi0, dtype=torch.float32, device="cuda"))
        opt = torch.optim.Adam([phi], lr=1.0)
        ms = timed(step_a, w.iters)
        with torch.no_grad():
            out["autograd"] = {"steps_per_s": w.iters / (ms * 1e-3), "ms_per_step": ms / w.iters,
                               "e_u": eu(ag.trap_fields(h, phi))}

        # (b) library loss and gradient, fused Adam
        phi = torch.tensor(w.phi0, dtype=torch.float32, device="cuda", requires_grad=True)
        opt = torch.optim.Adam([phi], lr=1.0, fused=True)

        def step_b(n):
            for _ in range(n):
                opt.zero_grad(set_to_none=True)
                ag.intensity_loss(h, phi, beta).backward()
                opt.step()
        step_b(3)
        with torch.no_grad():
            phi.copy_(torch.tensor(w.phi0, dtype=torch.float32, device="cuda"))
        opt = torch.optim.Adam([phi], lr=1.0, fused=True)
        ms = timed(step_b, w.iters)
        with torch.no_grad():
            out["library"] = {"steps_per_s": w.iters / (ms * 1e-3), "ms_per_step": ms / w.iters,
                              "e_u": eu(ag.trap_fields(h, phi))}

        # (c) the library step captured in a CUDA graph (a hologram on the capture stream)
        cap = torch.cuda.Stream()
        hc = hot.Hologram(w.W, w.H, w.pitch, w.wavelength, w.focal, cap.cuda_stream, w.precision)
        hc.set_traps(w.xyz, w.w0)
        phi = torch.tensor(w.phi0, dtype=torch.float32, device="cuda", requires_grad=True)
        phi.grad = torch.zeros_like(phi)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        opt = torch.optim.Adam([phi], lr=1.0, fused=True, capturable=True)

        def step_c():
            hot.hot_intensity_loss(hc.ctx, phi.detach(), beta, loss, phi.grad)
            opt.step()
        cap.wait_stream(stream)
        with torch.cuda.stream(cap):
            for _ in range(3):      # warm-up: optimizer state, the library's buffers
                step_c()
        stream.wait_stream(cap)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            step_c()
        with torch.no_grad():
            phi.copy_(torch.tensor(w.phi0, dtype=torch.float32, device="cuda"))
        for st in opt.state.values():
            for k in ("exp_avg", "exp_avg_sq"):
                st[k].zero_()
            st["step"].zero_()
        torch.cuda.synchronize()
        ms = timed(lambda n: [g.replay() for _ in range(n)], w.iters)
        with torch.no_grad():
            out["library_graph"] = {"steps_per_s": w.iters / (ms * 1e-3), "ms_per_step": ms / w.iters,
                                    "e_u": eu(ag.trap_fields(h, phi)), "loss": float(loss.item())}
        hc.close()

        # plain GSW from the same starting phases
        phi0 = torch.tensor(w.phi0, dtype=torch.float32, device="cuda")
        gsw = {}
        for K in (5, 10, 30):
            h.set_phase(phi0)
            h.set_weights(np.ones(w.M))
            h.gsw(K)
            h.set_phase(phi0)
            h.set_weights(np.ones(w.M))
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            ge, gu = h.gsw(K)
            ev[1].record(stream)
            torch.cuda.synchronize()
            gsw[str(K)] = {"ms": ev[0].elapsed_time(ev[1]), "e": ge, "u": gu}
        out["gsw_same_traps"] = gsw
        h.close()
        results[mode] = out
    main = results[modes[0]]
    line = {
        "metric": "Adam steps/s on -sum log I + 10 var I (1024x1024 px, M=256)",
        "value": main["library_graph"]["steps_per_s"], "unit": "steps/s", "n_gpus": 1, "steps": base.iters,
        "warmup": 3, "ms_per_step": main["library_graph"]["ms_per_step"], "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "path": "hot_intensity_loss (forward field; loss and adjoint coefficients; adjoint) + torch fused Adam, "
                "each step one CUDA graph replay",
        "config": {"workload": f"{base.name}: {base.W}x{base.H} px, M={base.M} traps, {base.iters} Adam steps on "
                               f"the phases, {modes[0]} mode", "W": base.W, "H": base.H, "M": base.M,
                   "steps": base.iters, "precision": modes[0], "seed": 0,
                   "optimizer": "Adam lr 1.0 (the best of 1e-2, 3e-2, 0.1, 0.3, 1.0 for this loss; torch defaults "
                                "otherwise)"},
        "modes": results,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_m_sweep(args):
    """Fig. 5 analogue (time per trap per GSW iteration vs M): 768 x 768 SLM, random 3-D traps
    (seed 0), M = 1 .. 4096, in the fast, separable and tensor modes (--precision picks one).
    Per point: the marginal time of one iteration (graph-replayed hot_gsw(K) minus hot_gsw(K/4),
    CUDA events, median of 5) and the time of the forward field alone (hot_gsw(0): F(phi0) and
    the Eq. 4 metrics).  A least-squares line t = a + b M over M >= 16 gives the fixed cost a and
    the cost per trap b, beside the SFU bound of the direct evaluation (4 SFU ops per pixel-trap
    pair)."""
    import torch
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot, workloads as wl

    W = H = 768
    Ms = [1, 2, 4, 8, 16, 32, 64, 100, 128, 256, 512, 1024, 2048, 4096]
    modes = [args.precision] if args.precision else ["fast", "separable", "tensor"]
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sfu_us_per_trap = W * H * SFU_OPS_PER_UPDATE / (sms * SFU_LANES_PER_SM * 2070e6) * 1e6

    def timed(h, phi0, k, reps=5):
        out = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            h.set_phase(phi0)
            a.record(stream)
            h.gsw(k, metrics=False)
            b.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b) * 1e3)
        return statistics.median(out)

    results = {}
    for mode in modes:
        rows = []
        for M in Ms:
            w = wl.random_case(W, H, M, seed=0, precision=mode)
            with hot.Hologram.from_workload(w, stream.cuda_stream) as h:
                phi0 = torch.tensor(w.phi0, dtype=torch.float32, device="cuda")
                K = 20 if M <= 1024 else 8
                h.gsw(K, metrics=False)
                h.gsw(K // 4, metrics=False)
                h.gsw(0, metrics=False)
                t_iter = (timed(h, phi0, K) - timed(h, phi0, K // 4)) / (K - K // 4)
                t_fwd = timed(h, phi0, 0)
            rows.append({"M": M, "us_per_iteration": round(t_iter, 3), "us_forward_only": round(t_fwd, 3),
                         "us_per_trap_per_iteration": round(t_iter / M, 5),
                         "updates_per_s": W * H * M / (t_iter * 1e-6)})
        fit = [r for r in rows if r["M"] >= 16]
        xs = np.array([r["M"] for r in fit], dtype=np.float64)
        ys = np.array([r["us_per_iteration"] for r in fit])
        b, a = np.polyfit(xs, ys, 1)
        results[mode] = {"points": rows, "fit_M_ge_16": {"fixed_us": round(float(a), 3),
                                                         "us_per_trap": round(float(b), 5)}}
    print(json.dumps({"metric": "time per GSW iteration vs trap count (768x768 SLM)", "W": W, "H": H,
                      "sfu_bound_us_per_trap": round(sfu_us_per_trap, 5),
                      "paper_context": "0.44 ms per trap per iteration on a GTX 260 (SLM size not stated)",
                      "results": results}), flush=True)
    return 0


def run_grid_sweep(args):
    """Sec. 5 / Fig. 7 analogue: e and u of n x n square grids (spacing 4 um, n = 2..9) on a
    768 x 768 SLM at a fixed 20 Hz frame rate.  Per grid: the random superposition (SR, seeded
    theta_m), then GSW started from it with (a) the iteration count the paper's GPU affords at
    20 Hz (0.44 ms per trap per iteration: K = floor(50 ms / (0.44 ms M)), at least 1) and
    (b) the count this GPU affords in 50 ms (measured, capped at 1000); (a) is checked against
    the FP64 oracle.  Fast sincos, FP32."""
    import torch
    import oracle
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot, workloads as wl

    stream = torch.cuda.current_stream()
    rows, worst = [], {"e": 0.0, "u": 0.0}
    for n in range(2, 10):
        w = wl.paper_grid(n, 768)
        w.precision = "fast"
        theta = np.random.default_rng(n).uniform(0.0, 2.0 * np.pi, w.M)
        coef = np.exp(1j * theta)
        k_paper = max(1, int(50.0 / (0.44 * w.M)))
        with hot.Hologram.from_workload(w, stream.cuda_stream) as h:
            h.superposition(coef)
            phi_sr = h.phase("f32")
            e_sr, u_sr = h.gsw(0)
            e_p, u_p = h.gsw(k_paper)
            # this GPU's iteration budget in 50 ms (time per iteration from a 20-iteration run)
            h.set_phase(phi_sr)
            h.set_weights(np.ones(w.M))
            h.gsw(20, metrics=False)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            h.set_phase(phi_sr)
            h.set_weights(np.ones(w.M))
            ev[0].record(stream)
            h.gsw(20, metrics=False)
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms_iter = ev[0].elapsed_time(ev[1]) / 20
            k_ours = int(min(1000, 50.0 / ms_iter))
            h.set_phase(phi_sr)
            h.set_weights(np.ones(w.M))
            e_o, u_o = h.gsw(k_ours)
        ref_sr = oracle.metrics(oracle.forward(w.geom, w.xyz, oracle.backproject(w.geom, w.xyz, coef)))
        ref = oracle.gsw(w.geom, w.xyz, k_paper, phi_sr.astype(np.float64))
        worst["e"] = max(worst["e"], abs(e_p - ref["e"]), abs(e_sr - ref_sr[0]))
        worst["u"] = max(worst["u"], abs(u_p - ref["u"]), abs(u_sr - ref_sr[1]))
        rows.append({"n": n, "M": w.M, "sr": {"e": e_sr, "u": u_sr},
                     "paper_20hz": {"iters": k_paper, "e": e_p, "u": u_p, "oracle_e": ref["e"], "oracle_u": ref["u"]},
                     "gb300_20hz": {"iters": k_ours, "e": e_o, "u": u_o, "ms_per_iter": ms_iter}})
    line = {"metric": "GSW efficiency and uniformity vs trap count at 20 Hz (n x n grids, 768^2 SLM)",
            "unit": "e, u", "n_gpus": 1, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper_grid n = 2..9: n x n traps, 4 um spacing, z = 0, 768 x 768 px, "
                                   "GSW started from a seeded random superposition, fast sincos"},
            "sweep": rows, "max_abs_diff_vs_oracle": worst,
            "paper_context": "efficiency never below 85 %; u = 0.36 for 9 x 9 with one iteration; "
                             "SR: e about 70 %, u a few percent (Sec. 5, GTX 260)"}
    print(json.dumps(line), flush=True)
    return 0


def run_precision_report(args):
    """Errors of HOT_PREC_ACCURATE, HOT_PREC_FAST, HOT_PREC_SEPARABLE and HOT_PREC_TENSOR against
    the FP64 oracle, per result, on grid16_256 and rand100_512, with the time per GSW iteration of
    each mode."""
    import torch
    import oracle
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot, workloads as wl

    stream = torch.cuda.current_stream()
    out = {}
    for name in ("grid16_256", "rand100_512"):
        base = wl.NAMED[name]()
        K = base.iters
        r1 = oracle.gsw(base.geom, base.xyz, 1, base.phi0)
        rK = oracle.gsw(base.geom, base.xyz, K, base.phi0)
        for prec in ("accurate", "fast", "separable", "tensor"):
            w = wl.NAMED[name]()
            w.precision = prec
            h = hot.Hologram.from_workload(w, stream.cuda_stream)
            h.gsw(1)
            V1, _ = h.fields()
            h.set_phase(w.phi0)
            h.set_weights(np.ones(w.M))
            h.gsw(K - 1)
            VK, wK1 = h.fields()
            e, u = h.gsw(1)
            phiK = h.phase("f32").astype(np.float64)
            g = h.phase("u8")
            # time per iteration (marginal, graph replay)
            phi0 = torch.tensor(w.phi0, dtype=torch.float32, device="cuda")
            ts = []
            for _ in range(5):
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                h.set_phase(phi0); ev[0].record(stream); h.gsw(K, metrics=False); ev[1].record(stream)
                h.set_phase(phi0); ev[2].record(stream); h.gsw(1, metrics=False); ev[3].record(stream)
                torch.cuda.synchronize()
                ts.append((ev[0].elapsed_time(ev[1]) - ev[2].elapsed_time(ev[3])) / (K - 1))
            h.close()
            _, coef = oracle.update_weights(VK, wK1)
            ophi, S = oracle.backproject(w.geom, w.xyz, coef, want_S=True)
            dphi = np.abs(np.angle(np.exp(1j * (phiK - ophi))))
            cond = np.abs(S) * dphi / np.sum(np.abs(coef))
            og = oracle.quantize(ophi)
            q = ophi / (2 * np.pi / 256)
            near = np.abs(q - (np.floor(q) + 0.5)) * (2 * np.pi / 256) < 1e-4
            out[f"{name}/{prec}"] = {
                "V1_max_rel_err": float(np.max(np.abs(np.abs(V1) - np.abs(r1["V"])) / np.abs(r1["V"]))),
                "V1_max_abs_err": float(np.max(np.abs(V1 - r1["V"]))),
                "e_abs_err": abs(e - rK["e"]), "u_abs_err": abs(u - rK["u"]),
                "phase_err_rad_median": float(np.median(dphi)), "phase_err_rad_p99": float(np.percentile(dphi, 99)),
                "phase_err_conditioned_max": float(cond.max()),
                "u8_differ": int(np.sum(g != og)), "u8_differ_not_near_boundary": int(np.sum((g != og) & ~near)),
                "us_per_iteration": 1e3 * float(np.median(ts)),
            }
    print(json.dumps({"metric": "precision report (GPU vs FP64 oracle)", "results": out}), flush=True)
    return 0


def run_batch(args):
    """Batched form (batch64): 64 holograms, sizes from {512^2, 1024^2, 1920x1152}, M ~ U{8..2000},
    30 GSW iterations per hologram in one CUDA graph, in the fast direct mode (shortest-first
    groups, one launch per group and iteration, autotuned tiling) and in the tensor mode (each
    member's own launch sequence on 8 concurrent chains); --precision picks one mode.
    Holograms/s and per-hologram latency (device timer stamps from the start of the graph to each
    hologram's completion), beside the same holograms run one by one through hot_gsw in the same
    mode.  The line's value is the fastest batched mode; best_one_by_one is the fastest mode run
    one by one."""
    import torch
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot, workloads as wl

    stream = torch.cuda.current_stream()
    modes = [args.precision] if args.precision else ["fast", "tensor"]
    K = wl.batch64()[0].iters
    results = {}
    for mode in modes:
        ws = wl.batch64()
        for w in ws:
            w.precision = mode
        holos = [hot.Hologram.from_workload(w, stream.cuda_stream) for w in ws]
        pairs = sum(w.N * w.M for w in ws) * K

        def reset():
            for h, w in zip(holos, ws):
                h.set_phase(w.phi0)
                h.set_weights(np.ones(w.M))

        batch = hot.Batch(holos, stream.cuda_stream)
        t_tune = time.perf_counter()
        tuned = batch.autotune(2) if mode != "tensor" else None
        t_tune = time.perf_counter() - t_tune
        tiling = batch.tiling()
        reps = max(1, min(args.steps, 5))
        total, lats = [], []
        for i in range(reps + 1):
            reset()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            batch.gsw(K)
            ev[1].record(stream)
            torch.cuda.synchronize()
            if i:  # i = 0: graph capture and warm-up
                total.append(ev[0].elapsed_time(ev[1]))
                lats.append(batch.latency())
        batch_ms = float(np.median(total))
        lat = np.concatenate(lats)
        eu_batch = batch.metrics()
        batch.close()
        # the same holograms one by one (each its own hot_gsw graph, default tiling), in the given order
        for h in holos:
            h.gsw(K, metrics=False)
        reset()
        torch.cuda.synchronize()
        ev_all = [torch.cuda.Event(enable_timing=True) for _ in range(len(holos) + 1)]
        ev_all[0].record(stream)
        for i, h in enumerate(holos):
            h.gsw(K, metrics=False)
            ev_all[i + 1].record(stream)
        torch.cuda.synchronize()
        seq_lat = np.array([ev_all[0].elapsed_time(ev_all[i + 1]) for i in range(len(holos))])
        eu_seq = [h.metrics() for h in holos]
        for h in holos:
            h.close()
        results[mode] = {
            "batch": {"holograms_per_s": len(ws) / (batch_ms * 1e-3), "ms": batch_ms,
                      "updates_per_s": pairs / (batch_ms * 1e-3),
                      "latency_ms_p50": float(np.percentile(lat, 50)),
                      "latency_ms_p99": float(np.percentile(lat, 99)),
                      "tiling": tiling,
                      "autotune": dict(tuned, seconds=t_tune, iters=2) if tuned else None},
            "sequential": {"holograms_per_s": len(ws) / (seq_lat[-1] * 1e-3), "ms": float(seq_lat[-1]),
                           "updates_per_s": pairs / (seq_lat[-1] * 1e-3),
                           "latency_ms_p50": float(np.percentile(seq_lat, 50)),
                           "latency_ms_p99": float(np.percentile(seq_lat, 99))},
            "batch_vs_sequential_max_abs_diff": {"e": max(abs(x[0] - y[0]) for x, y in zip(eu_batch, eu_seq)),
                                                 "u": max(abs(x[1] - y[1]) for x, y in zip(eu_batch, eu_seq))},
        }
    best = max(modes, key=lambda m: results[m]["batch"]["holograms_per_s"])
    best_seq = max(modes, key=lambda m: results[m]["sequential"]["holograms_per_s"])
    line = {
        "metric": "holograms/s, batch of 64 uneven holograms (30 GSW iterations each)",
        "value": results[best]["batch"]["holograms_per_s"], "unit": "holograms/s", "n_gpus": 1,
        "steps": max(1, min(args.steps, 5)), "higher_is_better": True,
        "dtype": "f16x3" if best == "tensor" else "f32", "data": "synthetic",
        "config": {"workload": "batch64: 64 holograms, sizes from {512^2, 1024^2, 1920x1152}, M ~ U{8..2000}, "
                               "30 GSW iterations in one CUDA graph", "seed": 0, "batched_mode": best},
        "best_one_by_one": {"mode": best_seq, "holograms_per_s": results[best_seq]["sequential"]["holograms_per_s"]},
        "modes": results,
        "latency": "device %globaltimer: start of the batch's first launch to each hologram's finalize; "
                   "one by one: CUDA events from the first hot_gsw to each hologram's end",
    }
    print(json.dumps(line), flush=True)
    return 0


def run_single(args):
    """One hot_gsw(K) call on the workload (trap tables, starting phases, K iterations, e and u)."""
    import torch
    from paper_0907_4027_gb300 import _build
    _build.build()
    from paper_0907_4027_gb300 import hot, workloads as wl
    w = wl.NAMED[args.workload]()
    if args.precision:
        w.precision = args.precision
    with hot.Hologram.from_workload(w, torch.cuda.current_stream().cuda_stream) as h:
        if args.merge > 1:
            h.set_block_merge(args.merge)
        if args.direct:
            h.set_once(False)
        e, u = h.gsw(args.single)
        print(json.dumps({"workload": w.name, "precision": w.precision, "iters": args.single, "e": e, "u": u,
                          "kernels": h.launches, "tiling": h.tiling()}), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.single:
        return run_single(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.grid_sweep:
        return run_grid_sweep(args)
    if args.m_sweep:
        return run_m_sweep(args)
    if args.precision_report:
        return run_precision_report(args)
    if args.workload == "diff256_1024":
        return run_adam(args)
    return run_engine(args)


if __name__ == "__main__":
    sys.exit(main())
