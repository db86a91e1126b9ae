#!/usr/bin/env python
"""Benchmark of the path-CV hot path on one GB300 (or N independent walkers on N GPUs).

Workload (the headline: the largest configuration that fits one GPU): N = 5000 atoms,
M = 2000 landmarks along a synthetic path (120 MB in FP32 storage, beyond what L2 holds
with the frames streaming through), a batch of F = 10,000 FP32 frames (600 MB) drifting
along the path with N(0, 0.05 nm) noise; floating close structure with eps = 0.05 nm^2
(Algorithm 2).  One step evaluates s, z and their coordinate derivatives ds/dx, dz/dx for
the whole batch: frame centring, close-structure decisions, exact alignments at
reassignments, approximate MSDs, path CVs and the adjoint.  The close-structure state is
reset at the start of every step so each step does the same work.  The step is timed with
per-kernel profiling off; a separate pass of the same steps with per-launch CUDA events
gives the kernel shares and the dominant kernel's roofline.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on the box's
host cores (OpenMP) on a bounded sample of the same workload.
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
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "path-CV frames/s and aligned MSDs/s on 1 GB300; % of HBM/L2 roofline"
# headline workload: N atoms, M landmarks, F frames per step, eps, frame noise, seed
N_ATOMS, N_LANDMARKS, N_FRAMES = 5000, 2000, 10_000
EPS, SEED = 0.05, 5

# FP32 ALU peak of one GB300: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.070 GHz (max SM clock)
SMS, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.070
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * SM_MAX_GHZ / 1e3

# algorithmic FP32 flops per (frame, landmark, atom) of each pair kernel (FMA = 2 flops)
FLOPS_PER_UNIT = {
    "approx_pair": 6,         # deviation form: dx . d (3 FMA); the norms are O(N) per frame / landmark
    "approx_pair_mma": 6,     # the same cross term on the tensor cores (3 FP16 MMAs per product, h h' + h l' + l h')
    "exact_pair": 45,         # pass 1: 9 FMA; pass 2: R a (9 FMA), 3 sub, 3 FMA
    "adjoint_beta_pair": 36,  # beta^s, beta^z += gamma R_i a (2 x 9 FMA), per-pair rotations
    "adjoint_beta_seg": 12,   # beta^s, beta^z += gamma b_i (2 x 3 FMA), b_i shared by a segment
    "adjoint_beta_mma": 12,   # the same product on the tensor cores (3 FP16 MMAs per product, h l' + l h' + h h')
}
# tensor-core kernels: operand kind (the peak is the measured bf16 rate, scaled for TF32)
TENSOR_KERNELS = {"adjoint_beta_mma": "f16", "approx_pair_mma": "f16"}
# DRAM bytes per unit of work from ncu captures of the current kernels, with the workload
# geometry they were taken on (atoms, landmarks); used only on that geometry (the units:
# approximate MSDs for the MSD kernels, frames for the adjoint)
DRAM_BYTES_PER_UNIT = {
    # approx_cross_mma on the first 2000 frames of the 5000-atom / 2000-landmark trajectory:
    # 1.2077 GB read + 0.0182 GB written for 3,986,000 approximate MSDs (the same segment
    # lengths as the full step, so the same traffic per approximate MSD)
    ("approx_pair_mma", 5000, 2000): 1.225962e9 / 3_986_000,
}
TF32_PER_BF16 = 1.1 / 2.25


def measured_peaks() -> dict:
    """Peaks measured on this GPU pool (HBM copy bandwidth, bf16 cuBLAS burst and sustained)."""
    path = ROOT / "MEASURED_PEAKS.json"
    try:
        return json.loads(path.read_text())
    except (OSError, ValueError):
        return {}


# side measurements: name -> (function, keyword arguments); see run_ours
DETAILS = {
    "c1_exact_fp64": ("config", dict(label="exact path CV, FP64, N=22, M=20, F=1000 (reflecting walk)", seed=1, n=22,
                                     m=20, f=1000, eps=-1.0, grad=False, precision="fp64", noise=0.02, steps=10,
                                     schedule="walk")),
    "c4_exact_grad": ("config", dict(label="exact path CV with gradients, FP32, N=1000, M=500, F=4096", seed=4,
                                     n=1000, m=500, f=4096, eps=-1.0, grad=True, precision="fp32")),
    "c3_group": ("group", dict()),
    "c5_stream_fp32": ("stream", dict(precision="fp32")),
    "c5_stream_fp16": ("stream", dict(precision="fp16")),
    # one frame per call at the size of the paper's first data set (24 atoms, 521 landmarks,
    # no neighbour list, eps = 0.01 nm^2): the per-step latency of the call
    "step_latency_n24_m521_fp64": ("stream", dict(precision="fp64", n=24, m=521, eps=0.01, seed=6)),
    "step_latency_n24_m521_fp32": ("stream", dict(precision="fp32", n=24, m=521, eps=0.01, seed=6)),
    "step_latency_n24_m521_fp32_grad": ("stream", dict(precision="fp32", n=24, m=521, eps=0.01, seed=6, grad=True)),
    "c5_batched_fp32": ("config", dict(label="close-structure path CV, N=5000, M=2000, F=10000, fp32 landmark storage",
                                       seed=5, n=5000, m=2000, f=10_000, eps=0.05, grad=False, precision="fp32",
                                       steps=1)),
    "c5_batched_fp16": ("config", dict(label="close-structure path CV, N=5000, M=2000, F=10000, fp16 landmark storage",
                                       seed=5, n=5000, m=2000, f=10_000, eps=0.05, grad=False, precision="fp16",
                                       steps=1)),
    # the first 2000 frames of the headline workload (its geometry and segment lengths; about
    # 2 GB on the device): the case the ncu captures of its kernels run on
    "c5_f2000_grad": ("config", dict(label="close-structure path CV with gradients, N=5000, M=2000, the first 2000 "
                                           "of 10000 frames, fp32 landmark storage", seed=5, n=5000, m=2000, f=2000,
                                     f_gen=10_000, eps=0.05, grad=True, precision="fp32", steps=1)),
    # the headline workload with FP16-stored landmarks (the headline itself is FP32 storage)
    "c5_batched_fp16_grad": ("config", dict(label="close-structure path CV with gradients, N=5000, M=2000, F=10000, "
                                                  "fp16 landmark storage", seed=5, n=5000, m=2000, f=10_000,
                                            eps=0.05, grad=True, precision="fp16", steps=2)),
    # the paper's second data set in size (304 atoms, 2120 landmarks, a neighbour list of 50
    # updated every 50 steps): the original method with and without the list, and the
    # close structure with the list
    "nl_exact_m2120": ("config", dict(label="exact path CV with gradients, N=304, M=2120, F=10000, FP32, "
                                            "neighbour list 50 every 50 steps", seed=8, n=304, m=2120, f=10_000,
                                      eps=-1.0, grad=True, precision="fp32", nl=(50, 50))),
    "nl_exact_m2120_nolist": ("config", dict(label="exact path CV with gradients, N=304, M=2120, F=10000, FP32, "
                                                   "no neighbour list", seed=8, n=304, m=2120, f=10_000, eps=-1.0,
                                             grad=True, precision="fp32")),
    "nl_close_m2120": ("config", dict(label="close-structure path CV with gradients, N=304, M=2120, F=10000, FP32, "
                                            "eps=0.05, neighbour list 50 every 50 steps", seed=8, n=304, m=2120,
                                      f=10_000, eps=0.05, grad=True, precision="fp32", nl=(50, 50))),
    # the consumer of s, z and their derivatives: Gaussian-hill bias and force on the frames of
    # the headline workload's size
    "metad_bias_f100k": ("metad", dict(f=100_000, n=300, hills=2000, stride=500)),
    "nl_close_m2120_nolist": ("config", dict(label="close-structure path CV with gradients, N=304, M=2120, F=10000, "
                                                   "FP32, eps=0.05, no neighbour list", seed=8, n=304, m=2120,
                                             f=10_000, eps=0.05, grad=True, precision="fp32")),
}


# details run only on request (--detail NAME): the small cases of the profiler captures
PROFILE_ONLY = {"c5_f2000_grad"}


def run_detail(pcv, name: str, calls: int = 200) -> dict:
    kind, kw = DETAILS[name]
    if kind == "stream":
        return time_stream(pcv, calls=calls, **kw)
    if kind == "metad":
        return time_metad(pcv, **kw)
    if kind == "group":
        return time_group(pcv, **kw)
    return time_config(pcv, **kw)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--eps", type=float, default=EPS)
    ap.add_argument("--frames", type=int, default=N_FRAMES)
    ap.add_argument("--no-details", action="store_true", help="skip the exact-mode / eps-sweep side measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    ap.add_argument("--detail", default=None, choices=sorted(DETAILS),
                    help="run one side measurement alone and print it (for profiling)")
    ap.add_argument("--calls", type=int, default=200, help="frames fed one per call in the streaming measurements")
    return ap.parse_args()


def workload_config(args):
    lm_mb = N_LANDMARKS * N_ATOMS * 3 * 4 / 1e6
    fr_mb = args.frames * N_ATOMS * 3 * 4 / 1e6
    return {
        "workload": f"close-structure path CV with gradients, N={N_ATOMS} atoms, M={N_LANDMARKS} landmarks "
                    f"(FP32 storage), F={args.frames} frames per step, eps={args.eps} nm^2: s, z, ds/dx, dz/dx",
        "atoms": N_ATOMS, "landmarks": N_LANDMARKS, "frames_per_step": args.frames, "eps_nm2": args.eps,
        "precision": "fp32 (compensated sums, FP32 eigen-solve + direct MSD; FP64 refresh re-checks)",
        "l2": f"inputs larger than L2: frames {fr_mb:.0f} MB per step and landmarks {lm_mb:.0f} MB vs 126 MB L2 "
              "(no flush needed)",
        "data": "synthetic: seeded self-avoiding chains, interpolated path, drift + N(0,0.05) noise",
    }


def make_inputs(frames: int):
    from paper_1801_02362_gb300 import synth

    lm, fr = synth.make_problem(SEED, n_atoms=N_ATOMS, n_landmarks=N_LANDMARKS, n_frames=frames, frame_noise=0.05)
    return lm, np.ascontiguousarray(fr, dtype=np.float32)


# ------------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "100"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in Path(self.path).read_text().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        import torch

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(value: float, pg, device):
    if pg is None:
        return value
    import torch

    t = torch.tensor([value], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def barrier(pg):
    if pg is not None:
        pg.barrier()


# ------------------------------------------------------------------------------------------
def lambda_from_gpu(pcv, lm):
    """lambda = 2.3 / mean D(a_k, a_{k+1}), the adjacent-landmark MSDs computed by the library."""
    import torch

    ctx = pcv.PathCV(lm, 1.0, eps=-1.0, precision="fp32")
    out = ctx.evaluate(torch.tensor(lm, dtype=torch.float32, device="cuda"), msd=True)
    d = out["msd"].cpu().numpy()
    ctx.close()
    return 2.3 / float(np.mean(np.diagonal(d, offset=1)))


def time_config(pcv, label: str, seed: int, n: int, m: int, f: int, eps: float, grad: bool, precision: str,
                noise: float = 0.05, steps: int = 3, schedule: str = "drift", nl=None, f_gen: int | None = None) -> dict:
    """One side measurement: a fresh context on seeded synthetic inputs of the given sizes,
    2 untimed evaluations, then `steps` timed ones (CUDA events on the context's stream).
    nl = (M_nl, L): neighbour list of M_nl landmarks updated every L steps.  f_gen: generate
    that many frames of trajectory and evaluate the first f (the same drift rate, hence the
    same close-structure segments, as the f_gen-frame workload)."""
    import torch
    from paper_1801_02362_gb300 import synth

    dt = torch.float64 if precision == "fp64" else torch.float32
    sdt = np.float64 if precision == "fp64" else np.float32
    ldt = np.float16 if precision == "fp16" else sdt
    lm, fr = synth.make_problem(seed, n_atoms=n, n_landmarks=m, n_frames=f_gen or f, frame_noise=noise,
                                schedule=schedule, frame_dtype=sdt, landmark_dtype=ldt)
    fr = fr[:f]
    lam = lambda_from_gpu(pcv, lm)
    ctx = pcv.PathCV(lm, lam, eps=eps, precision=precision, neighbor_list=nl)
    frames = torch.tensor(np.ascontiguousarray(fr), dtype=dt, device="cuda")
    for _ in range(2):
        pcv.pcv_reset_close_state(ctx.ctx)
        ctx.evaluate(frames, grad=grad)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        pcv.pcv_reset_close_state(ctx.ctx)
        ctx.evaluate(frames, grad=grad)
    b.record(stream)
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / steps
    # kernel times from a separate pass with per-launch events
    ctx.set_profiling(True)
    ctx.profile()
    for _ in range(steps):
        pcv.pcv_reset_close_state(ctx.ctx)
        ctx.evaluate(frames, grad=grad)
    pr = ctx.profile()
    st = ctx.stats()
    ctx.close()
    out = {"workload": label, "atoms": n, "landmarks": m, "frames": f, "eps_nm2": eps, "precision": precision,
           "gradients": grad, "ms_per_step": t, "frames_per_s": f / (t / 1e3),
           "msds_per_s": (st["landmark_alignments"] + st["approx_msds"]) / (t / 1e3),
           "exact_msds": st["landmark_alignments"], "approx_msds": st["approx_msds"],
           "kernel_ms": {k: round(v[0] / steps, 4) for k, v in pr.items()}}
    if nl is not None:
        out["neighbor_list"] = {"size": nl[0], "stride": nl[1]}
        # algorithmic FP32 work of the list kernels against the FP32 peak: frames between
        # updates x listed landmarks x atoms (exact: 45 flop, approximate: 27 flop -- R a,
        # 3 sub, 3 FMA -- per unit); the adjoint over every frame's own landmarks (36 flop:
        # beta^s and beta^z, 2 x 9 FMA)
        m_nl = nl[0]
        if eps < 0:
            n_upd = (st["landmark_alignments"] - m_nl * f) / (m - m_nl)
            pair_flop = 45
        else:
            nref = st["landmark_alignments"] / m
            n_uapp = (st["approx_msds"] - m_nl * (f - nref)) / (m - m_nl)
            n_upd = nref + n_uapp
            pair_flop = 27
        n_between = f - n_upd
        work = {"nl_pair": n_between * m_nl * n * pair_flop}
        if grad:
            work["nl_beta"] = (n_upd * m + n_between * m_nl) * n * 36
        roof = {}
        for name, flop in work.items():
            if name in pr:
                ms = pr[name][0] / steps
                tf = flop / (ms / 1e3) / 1e12
                roof[name] = {"ms": round(ms, 4), "TFLOP_s": round(tf, 2), "frac_fp32_peak": round(tf / FP32_PEAK_TFLOPS, 4)}
        out["list_kernels"] = roof
    # expensive distance computations per step (the cost model of the paper's Section 6.2)
    out["expensive_per_step"] = (st["xy_alignments"] + st["landmark_alignments"]) / f
    if nl is None and any(k in pr for k in FLOPS_PER_UNIT):
        out["roofline"] = kernel_roofline(pr, steps, f, n, m, st["landmark_alignments"], st["approx_msds"])
    return out


def time_stream(pcv, precision: str, n: int = 5000, m: int = 2000, calls: int = 200, eps: float = 0.05,
                seed: int = 5, grad: bool = False) -> dict:
    """Per-MD-step use: close-structure evaluation fed one frame per call (no gradients).
    Reports the time per call and, for the landmark-streaming kernels, bytes of landmarks
    read per launch / the kernel's average launch time against the measured HBM peak."""
    import torch
    from paper_1801_02362_gb300 import synth

    ldt = np.float16 if precision == "fp16" else (np.float64 if precision == "fp64" else np.float32)
    fdt = np.float64 if precision == "fp64" else np.float32
    lm, fr = synth.make_problem(seed, n_atoms=n, n_landmarks=m, n_frames=10_000, frame_noise=0.05,
                                landmark_dtype=ldt, frame_dtype=fdt)
    fr = torch.tensor(np.ascontiguousarray(fr[:calls + 8]), dtype=torch.float64 if precision == "fp64" else torch.float32,
                      device="cuda")
    lam = lambda_from_gpu(pcv, lm)
    ctx = pcv.PathCV(lm, lam, eps=eps, precision=precision)
    s = torch.empty(1, dtype=torch.float64, device="cuda")
    z = torch.empty_like(s)
    gs = torch.empty_like(fr[0]) if grad else None
    gz = torch.empty_like(fr[0]) if grad else None
    P = lambda t: None if t is None else t.data_ptr()
    for t in range(8):  # warm-up calls
        pcv.pcv_evaluate(ctx.ctx, 1, P(fr[t]), P(s), P(z), P(gs), P(gz), None, None)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    state = pcv.pcv_save_state(ctx.ctx)  # the profiled pass below replays the same calls
    a.record(stream)
    for t in range(8, 8 + calls):  # timed without per-launch profiling events
        pcv.pcv_evaluate(ctx.ctx, 1, P(fr[t]), P(s), P(z), P(gs), P(gz), None, None)
    b.record(stream)
    torch.cuda.synchronize()
    per_call_ms = a.elapsed_time(b) / calls
    # kernel times: the same calls again from the same close-structure state, with events
    pcv.pcv_load_state(ctx.ctx, state)
    ctx.set_profiling(True)
    ctx.profile()
    st0 = ctx.stats()
    for t in range(8, 8 + calls):
        pcv.pcv_evaluate(ctx.ctx, 1, P(fr[t]), P(s), P(z), P(gs), P(gz), None, None)
    torch.cuda.synchronize()
    pr = ctx.profile()
    st = ctx.stats()
    ctx.close()
    elem = {"fp16": 2, "fp32": 4, "fp64": 8}[precision]
    set_bytes = m * n * 3 * elem
    hbm = measured_peaks().get("hbm_gbs", 6793.8)
    # calls whose frame refreshed ran the exact kernel, the others the approximate one; each
    # such launch reads the whole landmark set once
    n_ref = (st["refreshes_threshold"] + st["refreshes_initial"]) - (st0["refreshes_threshold"] +
                                                                      st0["refreshes_initial"])
    work = {"exact_pair": n_ref, "approx_pair": calls - n_ref}
    kern = {}
    for name, n_work in work.items():
        if name in pr and n_work > 0:
            ms = pr[name][0]
            gbs = n_work * set_bytes / (ms / 1e3) / 1e9
            kern[name] = {"launches_with_work": n_work, "ms_per_launch": ms / n_work, "landmark_GB_per_s": gbs,
                          "frac_of_hbm_peak": gbs / hbm}
    return {"workload": f"close-structure path CV one frame per call, N={n}, M={m}, eps={eps}, {precision} landmark "
                        "storage",
            "landmark_set_MB": set_bytes / 1e6, "l2_resident": set_bytes < 126e6, "calls": calls,
            "ms_per_call": per_call_ms, "frames_per_s": 1e3 / per_call_ms,
            "refreshes": st["refreshes_threshold"] - st0["refreshes_threshold"],
            "kernels": kern, "hbm_peak_GB_per_s": hbm,
            "kernel_ms": {k: round(v[0] / calls, 4) for k, v in pr.items()}}


def time_metad(pcv, f: int, n: int, hills: int, stride: int, seed: int = 9, steps: int = 10) -> dict:
    """Metadynamics bias (Eq. vbias) on F steps: `hills` hills held before the call, a hill
    every `stride` steps; s, z a seeded walk along a 200-landmark path, ds/dx, dz/dx seeded
    FP32 arrays of N atoms.  Times the bias alone (hill sums) and with the force (the
    chain-rule pass over F x N x 3 derivatives, HBM-bound)."""
    import torch

    rng = np.random.default_rng(seed)
    s = torch.tensor(np.clip(1 + np.cumsum(rng.normal(scale=0.05, size=f)) % 199, 1, 200), device="cuda")
    z = torch.tensor(rng.uniform(0.0, 0.02, size=f), device="cuda")
    g = torch.Generator(device="cuda").manual_seed(seed)
    dsdx = torch.randn((f, n, 3), generator=g, device="cuda", dtype=torch.float32)
    dzdx = torch.randn((f, n, 3), generator=g, device="cuda", dtype=torch.float32)
    h0 = np.stack([rng.uniform(1, 200, hills), rng.uniform(0, 0.02, hills)], axis=1)
    mt = pcv.Metad(1.0, 0.3, 0.002, stride, max_hills=hills + (steps + 4) * (f // stride + 1))
    stream = torch.cuda.current_stream()
    out = {}
    for label, with_force in (("bias_only", False), ("bias_and_force", True)):
        mt.set_hills(h0, 1)
        for _ in range(2):
            mt.apply(s, z, dsdx if with_force else None, dzdx if with_force else None)
        mt.set_hills(h0, 1)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            mt.apply(s, z, dsdx if with_force else None, dzdx if with_force else None)
        b.record(stream)
        torch.cuda.synchronize()
        out[label] = a.elapsed_time(b) / steps
    n_end = mt.hills()[0].shape[0]
    mt.close()
    # hills seen per step, averaged over the timed calls (the hill set grows by f/stride per call)
    avg_hills = (hills + n_end) / 2.0
    evals = f * avg_hills
    flops = evals * 14  # per hill: 2 sub, 2 mul + FMA (argument), exp (~4 flop), mul, add, 2 x (mul, FMA)
    force_bytes = f * n * 3 * 4 * 3  # read ds/dx, dz/dx, write the force (FP32)
    t_force = max(out["bias_and_force"] - out["bias_only"], 1e-9)
    hbm = measured_peaks().get("hbm_gbs", 6793.8)
    return {"workload": f"metadynamics bias on {f} steps, {hills}+ hills, a hill every {stride} steps, N={n} "
                        "FP32 derivatives", "ms_bias_only": out["bias_only"], "ms_bias_and_force": out["bias_and_force"],
            "steps_per_s": f / (out["bias_and_force"] / 1e3), "hill_evaluations_per_s": evals / (out["bias_only"] / 1e3),
            "bias_TFLOP_s": flops / (out["bias_only"] / 1e3) / 1e12,
            "bias_frac_fp32_peak": flops / (out["bias_only"] / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
            "force_GB_s": force_bytes / (t_force / 1e3) / 1e9,
            "force_frac_hbm_peak": force_bytes / (t_force / 1e3) / 1e9 / hbm}


def time_group(pcv, n_inst: int = 256, f: int = 512, seed: int = 7, steps: int = 5) -> dict:
    """Batched multiple walkers: n_inst independent instances, N ~ U[50, 2000] atoms,
    M ~ U[50, 1000] landmarks, f frames each, FP32 exact mode.  One group call (three
    persistent launches, replayed from a captured graph after the first call) against one
    pcv_evaluate per instance, on the same contexts and buffers."""
    import torch
    from paper_1801_02362_gb300 import synth

    rng = np.random.default_rng(seed)
    ctxs, bufs, pairs = [], [], 0
    for k in range(n_inst):
        n = int(rng.integers(50, 2001))
        m = int(rng.integers(50, 1001))
        lm, fr = synth.make_problem(1000 + k, n_atoms=n, n_landmarks=m, n_frames=f, frame_noise=0.05)
        lam = lambda_from_gpu(pcv, lm)
        ctx = pcv.PathCV(lm, lam, eps=-1.0, precision="fp32")
        x = torch.tensor(np.ascontiguousarray(fr), dtype=torch.float32, device="cuda")
        bufs.append({"x": x, "s": torch.empty(f, dtype=torch.float64, device="cuda"),
                     "z": torch.empty(f, dtype=torch.float64, device="cuda")})
        ctxs.append(ctx)
        pairs += f * m * n
    P = lambda t: t.data_ptr()
    ios = [{"F": f, "frames": P(b["x"]), "s": P(b["s"]), "z": P(b["z"])} for b in bufs]
    handles = [c.ctx for c in ctxs]
    stream = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)

    def per_instance():
        for c, io in zip(ctxs, ios):
            pcv.pcv_evaluate(c.ctx, f, io["frames"], io["s"], io["z"], None, None, None, None)

    def group():
        pcv.pcv_evaluate_group(handles, ios)

    out = {}
    for name, fn in (("per_instance_launches", per_instance), ("group_persistent_graph", group)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(steps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        out[name] = a.elapsed_time(b) / steps
    tuned = pcv.pcv_group_tuning(handles[0])
    for c in ctxs:
        c.close()
    t = out["group_persistent_graph"]
    flops = 45.0 * pairs  # exact tiles: 9 FMA (pass 1) + 9 FMA + 3 sub + 3 FMA (pass 2) per atom pair
    return {"workload": f"{n_inst} independent instances, N~U[50,2000], M~U[50,1000], {f} frames each, "
                        "FP32 exact mode",
            "instances": n_inst, "frames_per_step": n_inst * f, "atom_landmark_frame_triples": pairs,
            "ms_per_step_group": t, "ms_per_step_per_instance": out["per_instance_launches"],
            "group_speedup": out["per_instance_launches"] / t, "frames_per_s": n_inst * f / (t / 1e3),
            "achieved_TFLOP_s": flops / (t / 1e3) / 1e12, "fp32_peak_TFLOP_s": FP32_PEAK_TFLOPS,
            "frac_of_fp32_peak": flops / (t / 1e3) / 1e12 / FP32_PEAK_TFLOPS,
            "autotuned": {"tile_frames": tuned[0], "tile_landmarks": tuned[1], "persistent_ctas": tuned[2]}}


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_sample(lm, fr, lam, eps, seconds: float, probe: int = 4):
    """Frames n such that the oracle's close-structure run over fr[:n] (with gradients)
    takes about `seconds`: the run from frame 0 includes the initial assignment and the
    reassignments in proportion to the workload's own rate once n spans a few gaps."""
    import oracle

    t0 = time.perf_counter()
    oracle.close(fr[:probe], lm, lam, eps, want_grad=True, want_D=False)
    per = (time.perf_counter() - t0) / probe
    return int(max(probe, min(len(fr), seconds / max(per, 1e-9))))


def cpu_baseline(lm, fr, lam, eps, seconds: float) -> dict:
    """The FP64 oracle as it stands on the host cores (OpenMP over the landmarks and atoms of
    each frame; Algorithm 2 itself is sequential over frames), on the first frames of the
    workload."""
    import oracle

    oracle.build()
    n = oracle_sample(lm, fr, lam, eps, seconds)
    t0 = time.perf_counter()
    r = oracle.close(fr[:n], lm, lam, eps, want_grad=True, want_D=False)
    dt = time.perf_counter() - t0
    n_ref = int((r["refreshed"] == 1).sum())
    return {"value": n / dt, "unit": "frames/s", "cores": oracle.threads(), "host_cores": host_cores(),
            "kind": "oracle",
            "sample": f"first {n} frames of the workload ({n_ref} reassignments + the initial assignment), close "
                      f"structure eps={eps} with gradients, {dt:.1f} s on {oracle.threads()} OpenMP threads"}


def run_reference(args):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    import oracle

    oracle.build()
    lm, fr = make_inputs(min(args.frames, 2000))
    lam = 2.3 / oracle.mean_adjacent_msd(lm)
    # bounded sample per step: ~2 s of oracle time from frame 0 of the workload
    n = oracle_sample(lm, fr, lam, args.eps, 2.0)
    for _ in range(args.warmup):
        oracle.close(fr[:n], lm, lam, args.eps, want_grad=True, want_D=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.close(fr[:n], lm, lam, args.eps, want_grad=True, want_D=False)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": oracle.threads(), "host_cores": host_cores(),
                         "kind": "oracle",
                         "sample": f"first {n} frames of the workload per step, close structure with gradients "
                                   f"(Algorithm 2 is sequential over frames; OpenMP over landmarks and atoms)"},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def kernel_roofline(prof: dict, steps: int, F: int, n: int, m: int, exact_msds: int, approx_msds: int) -> dict:
    """Roofline of the dominant kernel (by device time among the kernels with a work model)
    from a profiled pass of `steps` steps: algorithmic flops per launch / average launch
    time against the FP32 pipe or the TF32 tensor peak."""
    share = {k: v[0] for k, v in prof.items()}
    total_ms = sum(share.values())
    dom = max((k for k in prof if k in FLOPS_PER_UNIT), key=lambda k: prof[k][0])
    dom_ms, dom_launches = prof[dom]
    per_launch_ms = dom_ms / dom_launches
    launches_per_step = dom_launches / steps
    if dom.startswith("approx_pair"):
        units = approx_msds / launches_per_step * n
    elif dom == "exact_pair":
        units = exact_msds / launches_per_step * n
    else:
        units = F * m * n / launches_per_step
    flops = FLOPS_PER_UNIT[dom] * units
    achieved = flops / (per_launch_ms / 1e3) / 1e12
    if dom in TENSOR_KERNELS:
        peaks = measured_peaks()
        bf16 = peaks.get("bf16_tflops_sustained")
        src = "measured" if bf16 else "fallback"
        bound = "tensor"
        if TENSOR_KERNELS[dom] == "tf32":
            peak = (bf16 if bf16 else 1700.0) * TF32_PER_BF16
            peak_source = (f"TF32 dense: {src} sustained bf16 cuBLAS rate x 1.1/2.25 (nominal TF32/bf16); 3xTF32 issues "
                           "3 MMAs per algorithmic product, so frac <= 1/3")
        else:
            peak = bf16 if bf16 else 1700.0
            peak_source = (f"FP16 dense = bf16 dense: {src} sustained bf16 cuBLAS rate; the split operands issue 3 MMAs "
                           "per algorithmic product, so frac <= 1/3")
    else:
        peak, bound = FP32_PEAK_TFLOPS, "alu"
        peak_source = "152 SMs x 128 FP32 lanes x 2 flop x 2.070 GHz max clock (derived; FP32 FMA pipe)"
    traffic = None
    per_unit = DRAM_BYTES_PER_UNIT.get((dom, n, m))
    if per_unit is not None:
        work = approx_msds if dom.startswith("approx_pair") else F
        traffic = per_unit * work / launches_per_step
    return {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "peak_source": peak_source,
            "per_launch_ms": per_launch_ms, "flops_per_launch": flops,
            "timing": "per-launch CUDA events on the library's stream, in a separate pass of the same steps "
                      "(the headline's timed region runs without them)",
            "kernel_share": {k: round(v / total_ms, 4) for k, v in sorted(share.items(), key=lambda kv: -kv[1])}}


def c2_details(pcv, dev, stream) -> dict:
    """The 300-atom, 200-landmark, 100k-frame workload (FP32, gradients) across the
    close-structure thresholds and in exact mode, each with its dominant kernel's roofline."""
    import torch
    from paper_1801_02362_gb300 import synth

    n, m, F = 300, 200, 100_000
    lm, fr = synth.make_problem(1, n_atoms=n, n_landmarks=m, n_frames=F, frame_noise=0.05)
    fr = np.ascontiguousarray(fr, dtype=np.float32)
    lam = lambda_from_gpu(pcv, lm)
    frames = torch.from_numpy(fr).to(dev)
    ctx = pcv.PathCV(lm, lam, eps=0.05, precision="fp32", device=dev.index)
    pcv.pcv_set_stream(ctx.ctx, stream.cuda_stream)
    s = torch.empty(F, dtype=torch.float64, device=dev)
    z = torch.empty(F, dtype=torch.float64, device=dev)
    gs = torch.empty_like(frames)
    gz = torch.empty_like(frames)
    P = pcv._ptr
    out = {}
    for label, eps, grad in (("c2_close_eps0.05_grad", 0.05, True), ("c2_close_eps0.01_grad", 0.01, True),
                             ("c2_close_eps0.1_grad", 0.1, True), ("c2_close_eps0.05_fwd_only", 0.05, False),
                             ("c2_exact_grad", -1.0, True)):
        pcv.pcv_set_close_threshold(ctx.ctx, eps)

        def step():
            pcv.pcv_reset_close_state(ctx.ctx)
            pcv.pcv_evaluate(ctx.ctx, F, P(frames), P(s), P(z), P(gs) if grad else None, P(gz) if grad else None,
                             None, None)

        for _ in range(2):
            step()
        torch.cuda.synchronize(dev)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        k = 3
        a.record(stream)
        for _ in range(k):
            step()
        b.record(stream)
        torch.cuda.synchronize(dev)
        t = a.elapsed_time(b) / k
        ctx.set_profiling(True)
        ctx.profile()
        for _ in range(k):
            step()
        pr = ctx.profile()
        ctx.set_profiling(False)
        st = ctx.stats()
        out[label] = {"workload": f"N={n}, M={m}, F={F}, FP32, eps={eps}" + (", gradients" if grad else ""),
                      "ms_per_step": t, "frames_per_s": F / (t / 1e3),
                      "refreshes": st["refreshes_threshold"], "exact_msds": st["landmark_alignments"],
                      "approx_msds": st["approx_msds"],
                      "roofline": kernel_roofline(pr, k, F, n, m, st["landmark_alignments"], st["approx_msds"]),
                      "kernel_ms": {kk: round(v[0] / k, 4) for kk, v in pr.items()}}
    ctx.close()
    return out


def run_ours(args):
    import torch

    from paper_1801_02362_gb300 import pcv

    if args.detail:
        pcv.load()
        print(json.dumps({"detail": args.detail, **run_detail(pcv, args.detail, args.calls)}), flush=True)
        return
    world, rank, local, pg = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pcv.load()
    lm, fr = make_inputs(args.frames)
    F = fr.shape[0]
    lam = lambda_from_gpu(pcv, lm)
    frames = torch.from_numpy(fr).to(dev)
    stream = torch.cuda.current_stream(dev)
    ctx = pcv.PathCV(lm, lam, eps=args.eps, precision="fp32", device=local)
    s = torch.empty(F, dtype=torch.float64, device=dev)
    z = torch.empty(F, dtype=torch.float64, device=dev)
    gs = torch.empty_like(frames)
    gz = torch.empty_like(frames)
    P = pcv._ptr

    def step():
        pcv.pcv_reset_close_state(ctx.ctx)
        pcv.pcv_evaluate(ctx.ctx, F, P(frames), P(s), P(z), P(gs), P(gz), None, None)

    pcv.pcv_set_stream(ctx.ctx, stream.cuda_stream)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(pg)
    torch.cuda.synchronize(dev)
    st0 = ctx.stats()
    launches0, syncs0 = st0["kernel_launches"], st0["host_syncs"]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(pg)
    clk = clocks.stop()
    ms_local = e0.elapsed_time(e1)
    st = ctx.stats()
    launches = st["kernel_launches"] - launches0
    ms = max_over_ranks(ms_local, pg, dev)
    frames_total = F * args.steps * world
    value = frames_total / (ms / 1e3)
    # per-step counts of exact and approximate MSDs (the stats reset with the state each step)
    exact_msds_step = st["landmark_alignments"]
    approx_msds_step = st["approx_msds"]
    msds = (exact_msds_step + approx_msds_step) * args.steps * world / (ms / 1e3)

    # kernel shares and the dominant kernel's roofline: a separate pass of the same steps
    # with per-launch events on the library's stream
    prof_steps = max(1, min(args.steps, 5))
    ctx.set_profiling(True)
    ctx.profile()  # clear
    for _ in range(prof_steps):
        step()
    prof = ctx.profile()
    ctx.set_profiling(False)
    roofline = kernel_roofline(prof, prof_steps, F, N_ATOMS, N_LANDMARKS, exact_msds_step, approx_msds_step)

    # end to end through the host entry point: H2D of the frames, evaluation, D2H of s, z, gradients
    host_fr = torch.from_numpy(fr).pin_memory()
    hs = torch.empty(F, dtype=torch.float64).pin_memory()
    hz = torch.empty(F, dtype=torch.float64).pin_memory()
    hgs = torch.empty_like(host_fr).pin_memory()
    hgz = torch.empty_like(host_fr).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    pcv.pcv_reset_close_state(ctx.ctx)
    pcv.pcv_evaluate_host(ctx.ctx, F, P(host_fr), P(hs), P(hz), P(hgs), P(hgz), None, None)
    barrier(pg)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        pcv.pcv_reset_close_state(ctx.ctx)
        pcv.pcv_evaluate_host(ctx.ctx, F, P(host_fr), P(hs), P(hz), P(hgs), P(hgz), None, None)
    e2e_s = max_over_ranks(time.perf_counter() - t0, pg, dev)
    e2e = {"value": F * e2e_steps * world / e2e_s, "unit": "frames/s", "h2d_bytes_per_step": int(fr.nbytes),
           "d2h_bytes_per_step": int(2 * F * 8 + 2 * fr.nbytes), "api": "pcv_evaluate_host"}
    ctx.close()

    details = {}
    if not args.no_details and rank == 0:
        details.update(c2_details(pcv, dev, stream))
        for name in DETAILS:
            if name not in PROFILE_ONLY:
                details[name] = run_detail(pcv, name, args.calls)
        if "c5_stream_fp32" in details and "c5_stream_fp16" in details:
            details["c5_fp16_vs_fp32_speedup"] = {
                "stream_per_call": details["c5_stream_fp32"]["ms_per_call"] / details["c5_stream_fp16"]["ms_per_call"],
                "batched_per_step": details["c5_batched_fp32"]["ms_per_step"] / details["c5_batched_fp16"]["ms_per_step"]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(lm, fr, lam, args.eps, args.cpu_seconds)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(args),
            "msds_per_s": msds, "exact_msds_per_step": exact_msds_step, "approx_msds_per_step": approx_msds_step,
            "refreshes_per_step": st["refreshes_threshold"], "fp64_rechecks_per_step": st["fp64_rechecks"],
            "host_syncs_per_step": (st["host_syncs"] - syncs0) / args.steps, "lambda": lam,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "details": details,
        }
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
