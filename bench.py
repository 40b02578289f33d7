#!/usr/bin/env python
"""Benchmark: batched FWI gradient (32 shots, 512 x 256 at 6.25 m, nt = 4000)
on one GB300 per rank, through libwave's C ABI.

A step is one full gradient evaluation of the 32-shot batch: forward sweep
(source injection, receiver gather), misfit, adjoint sweep with the fused
zero-lag imaging condition, binomial-checkpoint recomputation, and the shot
sum.  ``value`` is shot-gradients per second over all ranks; grid-point
updates per second, the plain one-shot-at-a-time rate, the BF16-store rate,
an end-to-end rate through host buffers, the roofline of the dominant stencil
kernel and the FP64 oracle on the host cores are reported beside it.

    python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-pt updates/s & shot-gradients/s (batched vs plain, ≤1e-3 rel L2); HBM roofline %"
UNIT = "shot-gradients/s"
WORKLOAD = ("2D FWI gradient, 32 shots: 512x256 at 6.25 m, layered 1500-3500 m/s + 5% Gaussian-random "
            "perturbation (100 m), 512 receivers, 20 Hz Ricker, nt=4000 at dt=0.5 ms, 40-cell sponge, FP32, "
            "binomial checkpointing")
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes per launch from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum, caches
# flushed before the launch, so the reads are cold and the dirty lines a launch leaves in L2 are not
# counted), keyed by (kernel, SHA-256 prefix of that kernel's source text plus the shared stencil
# header) at capture time; a kernel whose source has changed since gets null.
VARIANT_KERNEL = {(0, 18): ("k_step2d_sgt", "k_step2d_sgt<16,8,2,0,fwd>"),
                  (0, 27): ("k_step2d_sgt", "k_step2d_sgt<16,8,2,1,fwd>"),
                  (1, 16): ("k_step2d_sgt", "k_step2d_sgt<16,8,2,0,adj>"),
                  (1, 25): ("k_step2d_sgt", "k_step2d_sgt<16,8,2,1,adj>")}
# shot-group TMA kernels with deeper rings and the adjoint's forward level by TMA
for _k, _fl, _g in ((39, 9, 2), (40, 9, 4), (41, 17, 4), (42, 9, 8), (43, 17, 8), (44, 41, 4), (45, 33, 2), (46, 41, 8), (47, 49, 4)):
    VARIANT_KERNEL[(0, _k)] = ("k_step2d_sgt", "k_step2d_sgt<16,8,%d,%d,fwd>" % (_g, _fl))
for _k, _fl, _g in ((37, 5, 2), (38, 13, 2), (39, 13, 4), (40, 5, 4), (41, 69, 4), (42, 101, 4), (43, 37, 4), (44, 101, 8), (45, 45, 4), (46, 101, 2)):
    VARIANT_KERNEL[(1, _k)] = ("k_step2d_sgt", "k_step2d_sgt<16,8,%d,%d,adj>" % (_g, _fl))
# the z-window kernels (step2d_zw.cu): (TZ, BZ, G) of forward variants 33-38 and adjoint variants 31-36
for _i, _c in enumerate([(16, 4, 2), (16, 4, 4), (16, 2, 2), (32, 8, 2), (32, 4, 2), (16, 8, 2)]):
    for _which, _base, _tag in ((0, 33, "fwd"), (1, 31, "adj")):
        VARIANT_KERNEL[(_which, _base + _i)] = ("k_step2d_zw", "k_step2d_zw<%d,%d,%d,%s>" % (*_c, _tag),
                                                "step2d_zw.cu")
TRAFFIC = {("k_step2d_sgt<16,8,4,41,fwd>", "2663cea1310bc711"): 53.40e6,
           ("k_step2d_sgt<16,8,4,101,adj>", "2663cea1310bc711"): 87.59e6,
           ("k_step3d_tma<8,76,8,fwd>", "773f3f582c635e7a"): 1386.69e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nsnap", type=int, default=1536,
                    help="checkpoint slots (two FP32 fields per shot each; 1536 = 80 GB for the 32-shot survey)")
    ap.add_argument("--nshot", type=int, default=32)
    ap.add_argument("--nt", type=int, default=4000)
    ap.add_argument("--only-main", action="store_true", help="timed gradient steps only (for launch lists)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--variants", default=None,
                    help="FWD,ADJ 2D kernel variants to use instead of running the autotuner")
    ap.add_argument("--only-3d", type=int, default=0, metavar="NT",
                    help="run only the config-3 3D forward for NT steps and print its line (for profiling)")
    ap.add_argument("--variant-3d", type=int, default=-1, help="3D kernel variant (-1: library default)")
    ap.add_argument("--only-fno", action="store_true",
                    help="run only the FNO training/inference measurement and print its line (for profiling)")
    ap.add_argument("--only-batch", action="store_true",
                    help="run only the config-4 uneven batch and print its line (for profiling)")
    ap.add_argument("--batch-nshot", type=int, default=64, help="problems in the uneven batch")
    ap.add_argument("--batch-scale", type=float, default=1.0,
                    help="grid and nt scale of the uneven batch (1 = config 4; smaller for profiling)")
    ap.add_argument("--batch-quick", action="store_true",
                    help="uneven batch: only the BF16 batched call (for profiling)")
    return ap.parse_args()


def kernel_hash(func: str, file: str = "kernels.cu") -> str:
    """SHA-256 prefix of a kernel's definition (from its name to the closing
    brace at column 0) in a csrc file, plus stencil.cuh."""
    csrc = os.path.join(ROOT, "paper_2304_05592_gb300", "csrc")
    with open(os.path.join(csrc, file)) as f:
        text = f.read()
    i = text.find(f" {func}(")
    if i < 0:
        return ""
    j = text.find("\n}\n", i)
    with open(os.path.join(csrc, "stencil.cuh")) as f:
        body = text[i:j] + f.read()
    return hashlib.sha256(body.encode()).hexdigest()[:16]


def step_bytes(kind: str, npts: int, nshot: int, store: str = "fp32") -> dict:
    """Algorithmic DRAM bytes of one 2D step launch over nshot shots of npts
    padded points each: every field read or written once, the model (and the
    gradient accumulator) once per launch because the shots share them
    ("amortised"), and the per-point figure of the survey's table ("nominal":
    16 B forward, 28 B adjoint with imaging, the model read once per shot)."""
    if kind == "fwd":
        per_shot = 12 + (2 if store == "bf16" else 0)  # u, u_prev read; u_next (+ BF16 copy) written
        return {"amortised": npts * (per_shot * nshot + 4), "nominal": npts * nshot * (16 + per_shot - 12)}
    per_shot = 16 - (2 if store == "bf16" else 0)      # mu^{k+1}, mu^{k+2}, u^k read; mu^k written
    return {"amortised": npts * (per_shot * nshot + 4 + 8), "nominal": npts * nshot * (28 - (16 - per_shot))}


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def make_problem(nshot: int, nt: int, rank: int = 0, world: int = 1):
    """The 32-shot gradient workload; with world > 1 ranks the survey has
    nshot * world sources spread over the same 50-3150 m line and
    this rank gets its contiguous shard of nshot of them."""
    from paper_2304_05592_gb300 import synth
    from paper_2304_05592_gb300.dist import shard

    p = synth.config2(nshot=32, nt=nt)
    if world > 1:
        total = nshot * world
        xs = np.linspace(50.0, 3150.0, total)  # the 32-shot line, refined
        mine = np.asarray(list(shard(total, rank, world)))
        p = p.with_shots(np.zeros(len(mine), dtype=int))
        p.src[:, 0, 0] = xs[mine]
    elif nshot != 32:
        p = p.with_shots(np.arange(nshot) % 32)
    from scipy.ndimage import gaussian_filter

    v0 = gaussian_filter(p.vel.astype(np.float64), 8.0).astype(np.float32)  # smooth starting model
    return p, v0


# ---------------------------------------------------------------------------
# Reference arm: the FP64 oracle on the host cores.


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    p, v0 = make_problem(1, args.nt)
    g = oracle.Grid(2, p.nx, p.nz, p.h, p.dt, p.nt, p.nb, vref=p.vref)
    q = oracle.ricker(p.f0, p.dt, p.nt)[None, :, None]
    dobs = oracle.forward(g, p.vel, p.src, q, p.rec)
    times = []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        oracle.gradient(g, v0, p.src, q, p.rec, dobs)
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
    tot = sum(times)
    value = args.steps / tot
    sample = f"1 of the 32 shots per step (full nt={p.nt}, full grid), FP64, OpenMP over grid rows"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "nshot_per_step": 1, "nt": p.nt},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Our arm.


def cpu_baseline(nt: int):
    """The FP64 oracle on the host cores: one shot of the 32-shot gradient (the
    headline sample), plus the survey's timing plan -- config 1 (full) at one
    thread and at all cores, and config 2 at one thread on a shortened record
    (nt = 400, scaled to the full record: the oracle's cost is linear in nt)."""
    import oracle
    from paper_2304_05592_gb300 import synth

    oracle.build()
    cores = oracle.threads()

    def grad_time(p, vel, nt_run=None):
        if nt_run:
            p = p.with_nt(nt_run)
        g = oracle.Grid(2, p.nx, p.nz, p.h, p.dt, p.nt, p.nb, vref=p.vref)
        q = oracle.ricker(p.f0, p.dt, p.nt)[None, :, None]
        src, rec = p.src[:1], p.rec[:1]
        dobs = oracle.forward(g, p.vel, src, q, rec)
        t = time.perf_counter()
        oracle.gradient(g, vel, src, q, rec, dobs)
        return time.perf_counter() - t, 2.0 * (p.nt - 1) * p.padded_points

    p, v0 = make_problem(1, nt)
    el, _ = grad_time(p, v0)
    out = {"value": 1.0 / el, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"1 shot of the 32 (full grid, nt={nt}), one gradient, FP64, {el:.1f} s"}
    plan = {}
    c1 = synth.config1()
    v1 = (c1.vel * 1.03).astype(np.float32)
    for th in (1, cores):
        oracle.set_threads(th)
        e, ups = grad_time(c1, v1)
        plan[f"config1_gradient_{th}_threads"] = {"s": e, "pt_updates_per_s": ups / e, "shot_gradients_per_s": 1 / e}
    oracle.set_threads(1)
    e, ups = grad_time(p, v0, 400)
    full = e * (nt - 1) / 399
    plan["config2_gradient_1_thread"] = {"s_at_nt_400": e, "pt_updates_per_s": ups / e,
                                         "shot_gradients_per_s_extrapolated": 1 / full}
    oracle.set_threads(cores)
    plan["config2_gradient_all_threads"] = {"s": el, "shot_gradients_per_s": 1 / el,
                                            "pt_updates_per_s": 2.0 * (nt - 1) * p.padded_points / el}
    out["plan"] = plan
    return out


def _variant3d(v: int) -> str:
    """Label of a 3D step variant; -1 is the library default, variant 16 (TMA plane
    ring, 8-row tiles, 76 planes per CTA, 8 ring slots), whose traffic was captured."""
    return "16 (k_step3d_tma<8,76,8>)" if v in (-1, 16) else str(v)


def config3_forward(dev, peak, nt: int = 200, variant: int = -1):
    """3D config-3 forward (400 x 400 x 300 at 10 m, 160 000 receivers), nt steps.
    The step launches are timed as one run between CUDA events (the average
    includes the gaps between launches), as the 2D steps are."""
    import torch

    from paper_2304_05592_gb300 import synth, wave
    from paper_2304_05592_gb300.wave import Grid

    p = synth.config3(nt=nt)
    g = Grid.of(p)
    v = torch.from_numpy(p.vel).to(dev)
    q = wave.wave_ricker(p.f0, p.dt, p.nt, device=dev)[None, :, None].contiguous()
    wave.wave_forward(g, v, p.src, q, p.rec)
    torch.cuda.synchronize()
    wave.wave_profile_start(0)
    t = time.perf_counter()
    wave.wave_forward(g, v, p.src, q, p.rec)
    torch.cuda.synchronize()
    el = time.perf_counter() - t
    fms, fn, _, _ = wave.wave_profile_stop()
    avg = fms / max(fn, 1) / 1e3
    N = p.padded_points
    ach = 16 * N / avg / 1e9
    return {"workload": "3D forward 400x400x300 at 10 m + 40-cell sponge (480x480x380 padded), 160000 receivers, "
                        f"{p.nt} of the 2000 steps", "pt_updates_per_s": N * (p.nt - 1) / el,
            "kernel": f"3D step variant {_variant3d(variant)}", "avg_launch_us": avg * 1e6,
            "achieved_gbs": ach, "frac": ach / peak,
            "traffic": TRAFFIC.get(("k_step3d_tma<8,76,8,fwd>", kernel_hash("k_step3d_tma")))
            if variant in (-1, 16) else None,
            "bound": "hbm", "bytes_per_point": 16}


def fno_preconditioner(dev):
    """The learned preconditioner's FNO (4 Fourier layers, width 32, hidden 64,
    16 x 16 modes on 256 x 512): FP32 training steps (forward, backward, MSE,
    Adam) and inference with FP32 or BF16 activations, batch 8, random inputs."""
    import torch

    from paper_2304_05592_gb300 import fno

    net = fno.FNO2d(fno.FNOConfig(), 256, 512, dev, seed=0)
    B = 8
    gen = torch.Generator(device=dev).manual_seed(0)
    x = torch.randn((B, 3, 256, 512), generator=gen, device=dev)
    y = torch.randn((B, 1, 256, 512), generator=gen, device=dev)

    def timed(fn, n):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(n):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / n

    t_train = timed(lambda: net.train_step(x, y, 1e-4), 10)
    t_f32 = timed(lambda: net.forward(x, train=False), 20)
    fno.fno_set_tensor_cores(False)
    t_b16_cc = timed(lambda: net.forward(x, train=False, bf16=True), 20)
    fno.fno_set_tensor_cores(True)
    t_b16 = timed(lambda: net.forward(x, train=False, bf16=True), 20)
    tc_status = fno.fno_tensor_core_status()
    # algorithmic FLOPs of one forward per pixel: per layer 2 W^2 (channel mix) + 2 W 2mx (x transform)
    # + 2 W 2mx (inverse in the fused kernel) + 16 W KZ mx Nz / (Nz Nx) (z transforms) + 8 W^2 KZ mx / (Nz Nx)
    # (mode mix); lift 2 cin W; projection 2 W H + 2 H
    W, H, KZ, mx, Nz, Nx, cin = 32, 64, 32, 16, 256, 512, 3
    per_layer = 2 * W * W + 4 * W * 2 * mx + 16 * W * KZ * mx / Nx + 8 * W * W * KZ * mx / (Nz * Nx)
    flop = (4 * per_layer + 2 * cin * W + 2 * W * H + 2 * H) * Nz * Nx
    # FP32 CUDA-core peak from unit counts and clocks: 152 SMs x 128 FMA lanes x 2 x 2.07 GHz
    alu_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    ach = flop * B / t_f32 / 1e12
    return {"workload": "FNO 4 layers, width 32, hidden 64, 16x16 modes, 256x512, batch 8",
            "train_samples_per_s": B / t_train, "infer_samples_per_s_fp32": B / t_f32,
            "infer_samples_per_s_bf16_tensor_cores": B / t_b16,
            "infer_samples_per_s_bf16_cuda_cores": B / t_b16_cc, "tensor_core_status": tc_status,
            "bf16_tensor_core_forward_tflops": flop * B / t_b16 / 1e12, "forward_gflop_per_sample": flop / 1e9,
            "forward_roofline": {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
                                 "frac": ach / alu_peak, "peak_kind": "derived: 152 SM x 128 FP32 lanes x 2 x 2.07 GHz"}}


def uneven_batch(dev, nshot: int = 64, scale: float = 1.0, full: bool = True):
    """Config 4: 64 shots of different grids, models and nt.  The batched
    gradient (two persistent sweeps under a CUDA graph, sweep kernel chosen by
    wave_autotune_batch on this batch) is timed directly with the BF16 store,
    through the torch.autograd.Function (BatchMisfit: misfits forward,
    velocity gradients backward) with the BF16 and the FP32 store, and against
    one wave_gradient call per shot with autotuned step kernels."""
    import torch

    from paper_2304_05592_gb300 import autograd, synth, wave
    from paper_2304_05592_gb300.wave import BatchProblem, Grid

    probs = synth.uneven_batch(seed=4, nshot=nshot, scale=scale)
    bps = []
    pts = 0
    for pb in probs:
        g = Grid.of(pb)
        q = wave.wave_ricker(pb.f0, pb.dt, pb.nt, device=dev)[:, None].contiguous()
        v = torch.from_numpy(pb.vel).to(dev)
        dob = wave.wave_forward(g, v, pb.src, q[None].contiguous(), pb.rec)[0].contiguous()
        bps.append(BatchProblem(g, (v * 1.02).contiguous(), pb.src[0], q, pb.rec[0], dob))
        pts += 2 * (pb.nt - 1) * pb.padded_points
    out = {"workload": "64 2D shots, nx 256-768, nz 128-384, h 6.25-12.5 m, nt 1500-4000, layered models"
           if nshot == 64 and scale == 1.0 else f"{nshot} 2D shots of the config-4 recipe scaled by {scale}",
           "batched": "2 persistent sweeps in a CUDA graph"}

    def timed(fn):
        fn()  # first call: set-up, graph capture
        torch.cuda.synchronize()
        t = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t

    for store, name in ((wave.STORE_BF16, "bf16"), (wave.STORE_FP32, "fp32")):
        if store == wave.STORE_FP32 and not full:
            continue
        ws = wave.wave_workspace_size_batch(bps, store)
        work = torch.empty(ws, dtype=torch.uint8, device=dev)
        vf, va = wave.wave_autotune_batch(bps, store=store, steps=200, work=work)
        grads = [torch.empty(b.grid.phys_shape, dtype=torch.float32, device=dev) for b in bps]
        el = timed(lambda: wave.wave_gradient_batch(bps, store=store, grads=grads, work=work))
        del work
        torch.cuda.empty_cache()
        vels = [b.vel.requires_grad_(True) for b in bps]

        def via_autograd():
            m = autograd.batch_misfit(bps, store=store)
            m.sum().backward()
            for v in vels:
                v.grad = None

        el_ag = timed(via_autograd) if full else None
        for b in bps:
            b.vel.requires_grad_(False)
        torch.cuda.empty_cache()
        out[name] = {"shot_gradients_per_s_batched": len(bps) / el, "pt_updates_per_s_batched": pts / el,
                     "shot_gradients_per_s_autograd": len(bps) / el_ag if el_ag else None,
                     "sweep_variants": {"forward": vf, "adjoint": va, "chosen_by": "wave_autotune_batch"},
                     "workspace_gb": ws / 1e9}
    if full:
        # one call per shot, each shape's step kernels autotuned first (BF16 store, as the batched line)
        for bp in bps:
            wave.wave_autotune(bp.grid, bp.vel, bp.src[None], bp.wavelet[None].contiguous(), bp.rec[None], steps=10)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for bp in bps:
            wave.wave_gradient(bp.grid, bp.vel, bp.src[None], bp.wavelet[None].contiguous(), bp.rec[None],
                               bp.d_obs[None].contiguous(), store=wave.STORE_BF16)
        torch.cuda.synchronize()
        out["shot_gradients_per_s_one_call_per_shot"] = len(bps) / (time.perf_counter() - t)
        out["one_call_per_shot"] = "wave_gradient per problem, BF16 store, step kernels from wave_autotune per shape"
    # bytes of the sweeps at the BF16 store: 18 B per forward update, 26 B per adjoint update
    b16 = out["bf16"]
    half = b16["pt_updates_per_s_batched"] / 2
    b16["achieved_gbs_at_22_b_per_update"] = half * (18 + 26) / 1e9
    return out


def lsrtm_config2(dev, iters: int = 2):
    """Least-squares RTM (CGLS: one Born modelling and one J' per iteration) on
    the 32-shot config-2 survey, data from a known squared-slowness
    perturbation (two Gaussian blobs) of the smooth starting model."""
    import torch

    from paper_2304_05592_gb300 import lsrtm, wave
    from paper_2304_05592_gb300.wave import Grid

    p, v0 = make_problem(32, 4000)
    g = Grid.of(p)
    vel = torch.from_numpy(v0).to(dev)
    q = wave.wave_ricker(p.f0, p.dt, p.nt, device=dev)[None, :, None].repeat(p.nshot, 1, 1).contiguous()
    zz, xx = np.meshgrid(np.arange(p.nz), np.arange(p.nx), indexing="ij")
    m0 = 1.0 / v0.astype(np.float64) ** 2
    dm = 0.03 * m0 * (np.exp(-((zz - 120) ** 2 + (xx - 200) ** 2) / 200.0)
                      - np.exp(-((zz - 180) ** 2 + (xx - 330) ** 2) / 150.0))
    dd = wave.wave_born(g, vel, p.src, q, p.rec, torch.from_numpy(dm.astype(np.float32)).to(dev))
    lsrtm.lsrtm_cgls(g, vel, p.src, q, p.rec, dd, 1, nsnap=1536)  # warm-up
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, hist = lsrtm.lsrtm_cgls(g, vel, p.src, q, p.rec, dd, iters, nsnap=1536)
    torch.cuda.synchronize()
    el = time.perf_counter() - t
    return {"workload": "LSRTM (CGLS) on the 32-shot config-2 survey, Born data of a known perturbation",
            "iterations_per_s": iters / el, "iterations_timed": iters,
            "residual_ratio": hist.rnorm[-1] / hist.rnorm[0],
            "per_iteration": "1 wave_born + 1 wave_jacobian_adjoint (checkpointed, 1536 slots) + 3 dot products"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__

    __graft_entry__.build()
    if args.only_fno:
        print(json.dumps({"fno_preconditioner": fno_preconditioner(dev)}))
        return 0
    if args.only_batch:
        print(json.dumps({"uneven_batch": uneven_batch(dev, args.batch_nshot, args.batch_scale,
                                                       full=not args.batch_quick)}))
        return 0
    if args.only_3d:
        from paper_2304_05592_gb300 import wave as _w

        _w.wave_set_variant(2, args.variant_3d)
        print(json.dumps({"config3_forward": config3_forward(dev, hbm_peak()[0], args.only_3d, args.variant_3d)}))
        return 0
    from paper_2304_05592_gb300 import wave
    from paper_2304_05592_gb300.wave import Grid

    p, v0 = make_problem(args.nshot, args.nt, rank, world)
    grid = Grid.of(p)
    vel_true = torch.from_numpy(p.vel).to(dev)
    vel = torch.from_numpy(v0).to(dev)
    q1 = wave.wave_ricker(p.f0, p.dt, p.nt, device=dev)
    wavelet = q1[None, :, None].repeat(p.nshot, 1, 1).contiguous()
    d_obs = wave.wave_forward(grid, vel_true, p.src, wavelet, p.rec)
    store = wave.STORE_CHECKPOINT
    if args.variants:
        tuned = tuple(int(x) for x in args.variants.split(","))
        wave.wave_set_variant(0, tuned[0])
        wave.wave_set_variant(1, tuned[1])
        chosen_by = "--variants"
    else:
        tuned = wave.wave_autotune(grid, vel, p.src, wavelet, p.rec, steps=40)
        chosen_by = "wave_autotune"
    nbytes = wave.wave_workspace_size(grid, wave.OP_GRADIENT, p.src, p.rec, store, args.nsnap)
    work = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    grad = torch.empty(grid.phys_shape, dtype=torch.float32, device=dev)

    from paper_2304_05592_gb300.dist import sharded_gradient

    def grad_fn(shots):
        # this rank's shard is fixed: p holds exactly its shots
        phi, g, _ = wave.wave_gradient(grid, vel, p.src, wavelet, p.rec, d_obs, store=store, nsnap=args.nsnap,
                                       grad=grad, work=work)
        return phi, g

    def step():
        # one gradient of the whole survey: this rank's shots, then one all-reduce when world > 1
        phi, _ = sharded_gradient(grad_fn, p.nshot * world)
        return phi

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = wave.wave_launch_count()
    # every run of consecutive step launches of one kind is timed as a whole, so launches
    # inside a run overlap as they do unmeasured (programmatic dependent launch)
    wave.wave_profile_start(0)
    barrier()
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
    fwd_ms, fwd_n, adj_ms, adj_n = wave.wave_profile_stop()
    launches = wave.wave_launch_count() - launches0
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    sec = ms / 1e3
    value = p.nshot * args.steps * world / sec
    N = p.padded_points
    updates = 2.0 * (p.nt - 1) * N * p.nshot * args.steps * world  # forward + adjoint steps (recompute excluded)
    sched_steps, _ = wave.wave_checkpoint_schedule(p.nt, args.nsnap)

    # roofline of the dominant stencil kernel (CUDA events around runs of consecutive launches,
    # on the launching stream, inside the timed region)
    peak, peak_kind = hbm_peak()
    f_avg = fwd_ms / max(fwd_n, 1) / 1e3
    a_avg = adj_ms / max(adj_n, 1) / 1e3
    n_fwd_launch = sched_steps * args.steps
    n_adj_launch = (p.nt - 1) * args.steps
    fb, ab = step_bytes("fwd", N, p.nshot), step_bytes("adj", N, p.nshot)
    kern = {"fwd": {"name": f"2D forward step, variant {tuned[0]}", "bytes": fb, "avg_s": f_avg, "n": fwd_n,
                    "total_s": f_avg * n_fwd_launch, "launches": n_fwd_launch},
            "adj": {"name": f"2D adjoint step + imaging, variant {tuned[1]}", "bytes": ab, "avg_s": a_avg,
                    "n": adj_n, "total_s": a_avg * n_adj_launch, "launches": n_adj_launch}}
    dom = max(kern, key=lambda k: kern[k]["total_s"])
    traffic = {}
    for k in kern:
        vk = VARIANT_KERNEL.get((0 if k == "fwd" else 1, tuned[0] if k == "fwd" else tuned[1]))
        traffic[k] = TRAFFIC.get((vk[1], kernel_hash(vk[0], vk[2] if len(vk) > 2 else "kernels.cu"))) if vk else None
    kd = kern[dom]
    achieved = kd["bytes"]["amortised"] / kd["avg_s"] / 1e9 if kd["avg_s"] > 0 else None
    tr = traffic[dom]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": tr,
                "kernel": kd["name"], "peak_kind": peak_kind,
                "bytes_per_launch": kd["bytes"]["amortised"],
                "bytes_model": "amortised: each field once, model (and gradient accumulator) once per launch",
                "avg_launch_us": kd["avg_s"] * 1e6,
                "timing": "CUDA events around each run of consecutive launches of one kind in the timed region "
                          f"({kd['n']} launches covered)",
                "achieved_nominal_gbs": kd["bytes"]["nominal"] / kd["avg_s"] / 1e9 if kd["avg_s"] else None,
                "achieved_dram_gbs": tr / kd["avg_s"] / 1e9 if tr and kd["avg_s"] else None,
                "other": {k: {"kernel": v["name"], "avg_launch_us": v["avg_s"] * 1e6,
                              "achieved_gbs": v["bytes"]["amortised"] / v["avg_s"] / 1e9 if v["avg_s"] else None,
                              "frac": v["bytes"]["amortised"] / v["avg_s"] / 1e9 / peak if v["avg_s"] else None,
                              "traffic": traffic[k],
                              "share_of_timed_region": v["total_s"] / sec if sec else None}
                          for k, v in kern.items()}}
    # the whole timed region, as one rate: bytes of all step launches of the gradients / wall time
    step_level = {"amortised_gbs": (n_fwd_launch * fb["amortised"] + n_adj_launch * ab["amortised"]) / sec / 1e9,
                  "nominal_gbs": (n_fwd_launch * fb["nominal"] + n_adj_launch * ab["nominal"]) / sec / 1e9}
    if traffic["fwd"] and traffic["adj"]:
        step_level["dram_gbs"] = (n_fwd_launch * traffic["fwd"] + n_adj_launch * traffic["adj"]) / sec / 1e9
    for k in list(step_level):
        step_level[k.replace("_gbs", "_frac")] = step_level[k] / peak
    roofline["step_level"] = step_level

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nshot_per_gpu": p.nshot, "nt": p.nt, "grid": f"{p.nx}x{p.nz}",
                       "padded_points": N, "store": "checkpoint", "nsnap": args.nsnap,
                       "forward_steps_per_gradient": sched_steps,
                       "kernel_variants": {"forward": tuned[0], "adjoint": tuned[1], "chosen_by": chosen_by},
                       "l2": "inputs larger than L2 (d_obs %.0f MB, checkpoints %.1f GB per GPU)" % (
                           d_obs.numel() * 4 / 1e6, nbytes / 1e9),
                       "parallelism": f"shots x{world}, gradient all-reduce" if world > 1 else "single GPU"},
            "pt_updates_per_s": updates / sec,
            "roofline": roofline, "gpu_launches": int(launches), "clocks": clk.summary()}

    if not args.only_main and rank == 0:
        del work
        torch.cuda.empty_cache()
        # plain: one shot per call, step kernels autotuned for the one-shot shape
        plain_tuned = wave.wave_autotune(grid, vel, p.src[:1], wavelet[:1].contiguous(), p.rec[:1], steps=40)
        nplain = min(4, p.nshot)
        wb = wave.wave_workspace_size(grid, wave.OP_GRADIENT, p.src[:1], p.rec[:1], store, args.nsnap)
        w1 = torch.empty(wb, dtype=torch.uint8, device=dev)
        g1 = torch.empty_like(grad)

        def plain(i):
            wave.wave_gradient(grid, vel, p.src[i:i + 1], wavelet[i:i + 1], p.rec[i:i + 1], d_obs[i:i + 1],
                               store=store, nsnap=args.nsnap, grad=g1, work=w1)

        plain(0)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(nplain):
            plain(i)
        e1.record(stream)
        torch.cuda.synchronize()
        line["plain_shot_gradients_per_s"] = nplain / (e0.elapsed_time(e1) / 1e3)
        line["plain_kernel_variants"] = {"forward": plain_tuned[0], "adjoint": plain_tuned[1],
                                         "chosen_by": "wave_autotune (one-shot shape)"}
        del w1
        torch.cuda.empty_cache()
        # BF16 full storage
        wb = wave.wave_workspace_size(grid, wave.OP_GRADIENT, p.src, p.rec, wave.STORE_BF16, 1)
        wbf = torch.empty(wb, dtype=torch.uint8, device=dev)
        g2 = torch.empty_like(grad)
        wave.wave_gradient(grid, vel, p.src, wavelet, p.rec, d_obs, store=wave.STORE_BF16, grad=g2, work=wbf)
        torch.cuda.synchronize()
        e0.record(stream)
        nb = 2
        for _ in range(nb):
            wave.wave_gradient(grid, vel, p.src, wavelet, p.rec, d_obs, store=wave.STORE_BF16, grad=g2, work=wbf)
        e1.record(stream)
        torch.cuda.synchronize()
        line["bf16_store_shot_gradients_per_s"] = nb * p.nshot / (e0.elapsed_time(e1) / 1e3)
        line["bf16_store_vs_checkpoint_rel_l2"] = float((g2 - grad).norm() / grad.norm())
        del wbf
        torch.cuda.empty_cache()
        # end to end through host buffers (pinned), same checkpointed gradient
        work = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        h_vel = vel.cpu().pin_memory()
        h_wav = wavelet.cpu().pin_memory()
        h_obs = d_obs.cpu().pin_memory()
        h_grad = torch.empty(grid.phys_shape, dtype=torch.float32).pin_memory()
        h2d = (h_vel.numel() + h_wav.numel() + h_obs.numel()) * 4
        d2h = h_grad.numel() * 4 + 8

        def e2e_step():
            dv = h_vel.to(dev, non_blocking=True)
            dw = h_wav.to(dev, non_blocking=True)
            do = h_obs.to(dev, non_blocking=True)
            phi, g, _ = wave.wave_gradient(grid, dv, p.src, dw, p.rec, do, store=store, nsnap=args.nsnap,
                                           grad=grad, work=work)
            h_grad.copy_(g, non_blocking=True)
            torch.cuda.synchronize()
            return phi

        e2e_step()
        t0 = time.perf_counter()
        ne = max(2, args.steps // 2)
        for _ in range(ne):
            e2e_step()
        el = time.perf_counter() - t0
        line["e2e"] = {"value": ne * p.nshot / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h}
        del work
        torch.cuda.empty_cache()
        line["config3_forward"] = config3_forward(dev, peak)
        torch.cuda.empty_cache()
        line["uneven_batch"] = uneven_batch(dev)
        torch.cuda.empty_cache()
        line["lsrtm"] = lsrtm_config2(dev)
        line["fno_preconditioner"] = fno_preconditioner(dev)
        torch.cuda.empty_cache()
        if world == 1 and not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(p.nt)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
