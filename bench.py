#!/usr/bin/env python
"""Throughput of the per-keyframe latent-feature optimisation step (LatentAM, arxiv 2602.12314).

One step = one fwd+bwd+Adam iteration of the whole hot path on one keyframe through the
C ABI (latentam_step, iters = 1, queries learnable = Stage I with R1 = 1): projection,
binning + depth sort, query splatting, dictionary decode, feature loss with the trust
region, decode backward, splat backward, Adam on (f, K, V).

Workload (the single-keyframe room configuration): 300k Gaussians on the surfaces of a
6x5x3 m room with 20 boxes, 640x480 pinhole view, d = 32, M = 256, D = 512, FP32 end to
end; seeded synthetic data standing in for the paper's RGB-D + CLIP/SAM keyframes.

  python bench.py [--gpus N --steps K --warmup W] [--precision both|fp32|bf16] [--impl reference]

By default every precision form runs: the FP32 form gives the headline value (its decode on the
tcgen05 tensor cores with each FP32 operand split into a BF16 hi and lo term, three MMAs per
product, FP32 accumulation), and the FP32 form on the FMA pipes, the BF16, BF16-batched and FP8
tensor-core forms, the mask-pooled forms and the full Stage I objective are reported under
"forms".

Under torchrun (N > 1) every rank optimises its own keyframe (replicas, weak scaling); the
timed region is bracketed by a barrier and a device synchronisation and the slowest rank's
time is used.  Rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd latent optim iters/sec at 640x480,D=512 (FP32 vs BF16 batched); % roofline"
WORKLOAD = ("room keyframe: 300k Gaussians (6x5x3 m room, 20 boxes), 640x480, d=32, M=256, D=512; "
            "one fwd+bwd+Adam iteration incl. projection and depth/tile sort (Stage I, R1=1)")
SM_FP32_LANES = 128  # FP32 FMA lanes per SM

# DRAM traffic (read + write bytes) of the decode stage per pixel, from one ncu capture of every
# decode launch of a step on the 480x360 crop (172,800 pixels), keyed by a hash of the kernel
# sources it was taken on: once they change, the figure no longer describes the kernels and the
# roofline reports no traffic.
_DECODE_TRAFFIC = {"bf16": ("ba5351875c7c97d7", 1224.157e6 / 172800), "fp32_fma": ("6c2f4b1cc96cf828", 3359.43e6 / 172800),
                   "fp32": ("ba5351875c7c97d7", 2391.129e6 / 172800)}
_DECODE_SOURCES = {"bf16": ("decode_tc.cu", "tc_gemm.cuh", "tc_common.cuh"), "fp32_fma": ("decode_f32.cu",),
                   "fp32": ("decode_tc.cu", "tc_gemm.cuh", "tc_common.cuh")}
# bytes each splat kernel must move per unit (render forward: per pair 24 B of conic, mean and
# opacity + 4d B of query staged once per tile, per pixel 4d B of Q + 8 B of T and count; render
# backward: per pixel 4d B of dQ, per pair 24 B, per Gaussian 4d B of df)
SPLAT_FWD_BYTES = lambda P, n, N, d: P * (24 + 4 * d) + n * (4 * d + 8)  # noqa: E731
SPLAT_BWD_BYTES = lambda P, n, N, d: n * 4 * d + P * 24 + N * 4 * d  # noqa: E731


def _decode_sources_hash(form="bf16"):
    import hashlib
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2602_12314_gb300", "csrc")
    h = hashlib.sha256()
    for f in _DECODE_SOURCES[form]:
        with open(os.path.join(src, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--batch", type=int, default=6, help="keyframes of the batched form (B + 1, B = 5 in Sec. IV-A)")
    p.add_argument("--precision", choices=["both", "fp32", "fp32_fma", "bf16", "fp8", "bf16_batch", "fp32_batch",
                                          "fp32_masks", "bf16_masks", "fp32_full"], default="both",
                   help="both: the FP32 form is the headline value, the BF16 tensor-core form is reported beside it")
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--workload", choices=["room", "tiny", "precision", "batch8", "building"], default="room",
                   help="room (the headline run); the others print their own line")
    p.add_argument("--crop", type=int, nargs=2, metavar=("W", "H"), default=None,
                   help="profiling only: the central W x H crop of the keyframe (all Gaussians kept)")
    return p.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"latentam_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower() in ("active", "1"):
                        reasons.add(name)
        except Exception:
            return None
        if not sm:
            return None
        hi = max(mx)
        loaded = [s for s in sm if s > 0.5 * hi] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": hi, "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_barrier(dist):
    """Barrier over the ranks of a multi-GPU run (no-op for one process)."""
    if dist is not None:
        dist.barrier()


def max_ms_over_ranks(dist, ms: float, device: str) -> float:
    """The slowest rank's time: every rank's step time is reduced with MAX (the job is as
    fast as its slowest replica)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, frames_per_step: int, steps: int, ms: float) -> float:
    """Whole-job keyframe-iterations per second: all ranks' work over the slowest rank's time."""
    return world * frames_per_step * steps / (ms / 1e3)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _scene(seed, crop=None):
    from workloads import room_scene
    s = room_scene(seed)
    if crop:
        w, h = crop
        s = s.crop((s.camera.width - w) // 2, (s.camera.height - h) // 2, w, h)
    return s


def _workload(args):
    if not args.crop:
        return WORKLOAD
    return WORKLOAD.replace("640x480", "central %dx%d crop of the 640x480 frame" % tuple(args.crop))


def _config(args, scene, world, precision):
    return {"workload": _workload(args), "precision": precision, "global_batch": world,
            "n_pixels": scene.camera.n_pixels, "gaussians": scene.n, "d": scene.d, "M": scene.M, "D": scene.D,
            "l2": "inputs larger than L2 (target features %.0f MB FP32 / %.0f MB BF16 per step)"
                  % (scene.F.nbytes / 1e6, scene.F.nbytes / 2e6),
            "parallelism": f"replicas x{world}",
            "fp32_form": "decode contractions on tcgen05: each FP32 operand split into BF16 hi + lo, three MMAs per "
                         "product (hi hi + hi lo + lo hi), FP32 accumulation; softmax and loss in FP32 (held to the "
                         "FP32 parity bars: 1e-4 on features, 1e-3 on gradients)"}


def _oracle_iteration(scene, cfg):
    """One oracle iteration: forward, backward and the Adam update of f, K, V."""
    import numpy as np

    import oracle
    out = oracle.iteration(scene, cfg)
    for name, x, g in (("f", scene.f, out["df"]), ("K", scene.K, out["dK"]), ("V", scene.V, out["dV"])):
        p = x.astype(np.float64).copy()
        m, v = np.zeros_like(p), np.zeros_like(p)
        oracle.adam(p.reshape(-1), g.reshape(-1), m.reshape(-1), v.reshape(-1), 1, 0.01)
    return out


def _cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def run_reference(args, world, rank):
    """The oracle (plain FP64 C, OpenMP over independent outputs) as it stands, timed on this
    machine's host cores: every step is one whole oracle iteration (render, decode, loss,
    backward, Adam) of the full 640x480 room keyframe with its 300k Gaussians.  Under torchrun
    only rank 0 runs it."""
    if rank != 0:
        return
    import oracle
    s = _scene(args.seed, args.crop)
    cfg = oracle.LossConfig()
    oracle.build()
    for _ in range(max(args.warmup, 0)):
        _oracle_iteration(s, cfg)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _oracle_iteration(s, cfg)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    sample = (f"{args.steps} whole oracle iterations (fwd, bwd, Adam) of the {s.camera.width}x{s.camera.height} "
              f"keyframe with all {s.n} Gaussians, {dt:.1f} s on {_cores()} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(args, s, world, args.precision),
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": _cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def decode_flops(n, M, D, d):
    """Algorithmic FLOPs of decode + loss + decode backward (direct form, attention kept):
    S (2nMd) + Fhat (2nMD) + dA (2nMD) + dQ (2nMd) + dV (2nMD) + dK (2nMd)."""
    return 6.0 * n * M * D + 6.0 * n * M * d


def _pipelined_e2e(st, host, get, put, steps, barrier, max_over_ranks, world, n_frames):
    """End-to-end timing through the public API with every step's inputs copied from pinned
    host memory: two device input sets, the copies of step i + 1 issued on a second stream while
    step i computes (the copy stream starts after the timed region opens and the last step waits
    for its own copies), each step's loss read back.  get(name) / put(name, tensor) access the
    step's input tensors."""
    import torch

    bufs = [{k: torch.empty_like(get(k)) for k in host}, {k: torch.empty_like(get(k)) for k in host}]
    copy_stream = torch.cuda.Stream()
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    compute = torch.cuda.current_stream()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(compute)

    def issue(i):
        b = i % 2
        with torch.cuda.stream(copy_stream):
            for k, t in host.items():
                bufs[b][k].copy_(t, non_blocking=True)
            ready[b].record(copy_stream)

    copy_stream.wait_event(e0)
    issue(0)
    for i in range(steps):
        b = i % 2
        if i + 1 < steps:
            issue(i + 1)  # the buffer set it fills was last read by step i - 1, already finished
        compute.wait_event(ready[b])
        for k in host:
            put(k, bufs[b][k])
        st.step(1, learn_f=True, want_loss=True)  # reads the loss back (synchronises the compute stream)
    e1.record(compute)
    torch.cuda.synchronize()
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1))
    return job_throughput(world, n_frames, steps, ms)


def _measure(args, world, rank, local, scene, prec, dist, views=None, masks=None, full=None):
    """Time args.steps steps of one precision form; returns its numbers (rank 0 view).  With
    `views`, a step is one iteration of the batched step over all those keyframes and the
    value counts keyframe-iterations per second.  With `masks`, the step is mask-pooled (one
    decoded row and target per SAM-style mask)."""
    import numpy as np
    import torch

    from paper_2602_12314_gb300 import _lib as L
    from paper_2602_12314_gb300 import api

    ctx = api.Context(local)
    target_dtype = torch.float32 if prec in (api.FP32, api.FP32_FMA) else torch.bfloat16
    if full is not None:  # the whole Stage I objective: geometry, colour and depth too
        st = api.LatentStepFull(ctx, scene, *full)
    elif views is None:
        st = api.LatentStep(ctx, scene, precision=prec, target_dtype=target_dtype, masks=masks)
    else:
        st = api.LatentBatchStep(ctx, views, precision=prec, target_dtype=target_dtype)
    n_frames = 1 if views is None else len(views)
    for _ in range(max(args.warmup, 3)):
        st.step(1, learn_f=True, want_loss=False)
    torch.cuda.synchronize()

    def barrier():
        rank_barrier(dist)

    def max_over_ranks(ms):
        return max_ms_over_ranks(dist, ms, "cuda")

    # ---- device-resident timed region (iterations replayed as CUDA graphs) -----------------
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = L.load().latentam_launch_count()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        st.step(1, learn_f=True, want_loss=False)
    ev1.record()
    torch.cuda.synchronize()
    barrier()
    launches = L.load().latentam_launch_count() - launches0
    ms = max_over_ranks(ev0.elapsed_time(ev1))
    clk = clocks.stop()
    value = job_throughput(world, n_frames, args.steps, ms)

    # ---- per-stage CUDA-event timers over a second pass (plain launches) --------------------
    prof_steps = max(1, min(args.steps, 10))
    ctx.profile(True)
    ctx.profile_read(reset=True)
    for _ in range(prof_steps):
        st.step(1, learn_f=True, want_loss=False)
    prof = ctx.profile_read(reset=True)
    ctx.profile(False)

    # ---- end to end through the public API, host buffers ----------------------------------
    e2e = None
    if not args.no_e2e and full is not None:
        host = {k: torch.as_tensor(np.ascontiguousarray(getattr(scene, k)), dtype=torch.float32).pin_memory()
                for k in ("means", "quats", "scales", "opacities")}
        host["colours"] = torch.as_tensor(full[0]).pin_memory()
        host.update({"F": torch.as_tensor(scene.F, dtype=torch.float32).pin_memory(),
                     "mask": torch.as_tensor(scene.mask, dtype=torch.uint8).pin_memory(),
                     "image": torch.as_tensor(full[1]).pin_memory(), "depth": torch.as_tensor(full[2]).pin_memory()})
        geo = ("means", "quats", "scales", "opacities", "colours")

        def get(k):
            return st.p[k] if k in geo else getattr(st, k)

        def put(k, t):
            if k in geo:
                st.p[k].copy_(t)  # the optimised state takes the new keyframe's values
            else:
                setattr(st, k, t)

        h2d = sum(t.numel() * t.element_size() for t in host.values())
        e2e_value = _pipelined_e2e(st, host, get, put, args.steps, barrier, max_over_ranks, world, n_frames)
        e2e = {"value": e2e_value, "unit": "iters/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 8 * L.FULL_LOSS_PARTS, "pipelined": True}
    elif not args.no_e2e:
        if views is None:
            host = {k: torch.as_tensor(np.ascontiguousarray(getattr(scene, k)), dtype=torch.float32).pin_memory()
                    for k in ("means", "quats", "scales", "opacities")}
            if masks is None:
                host["F"] = torch.as_tensor(scene.F, dtype=torch.float32).to(target_dtype).pin_memory()
                host["mask"] = torch.as_tensor(scene.mask, dtype=torch.uint8).pin_memory()
            else:
                host["F"] = torch.as_tensor(masks.F, dtype=torch.float32).to(target_dtype).pin_memory()
                host["mask"] = torch.as_tensor(masks.valid, dtype=torch.uint8).pin_memory()
                host["mask_offsets"] = torch.as_tensor(masks.offsets).pin_memory()
                host["mask_pixels"] = torch.as_tensor(masks.pixels).pin_memory()
        else:  # the keyframes' targets (the map's geometry stays on the device)
            host = {"F": torch.cat([torch.as_tensor(v.F) for v in views]).to(target_dtype).pin_memory(),
                    "mask": torch.cat([torch.as_tensor(v.mask) for v in views]).pin_memory()}
        h2d = sum(t.numel() * t.element_size() for t in host.values())
        d2h = 8 * L.LOSS_PARTS
        e2e_value = _pipelined_e2e(st, host, lambda k: getattr(st, k), lambda k, t: setattr(st, k, t), args.steps,
                                   barrier, max_over_ranks, world, n_frames)
        e2e = {"value": e2e_value, "unit": "iters/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "pipelined": True}
    ctx_pairs = None
    if full is None:
        ctx_pairs = _pair_counts(ctx, views if views is not None else [scene])
    tuned = _tune_summary(ctx.autotune_choices())
    ctx.close()

    # ---- roofline of the dominant stage (decode + loss + decode backward) -------------------
    peaks, peak_src = _peaks()
    n, M, D, d = scene.camera.n_pixels * n_frames, scene.M, scene.D, scene.d
    if views is not None:
        n = sum(v.camera.n_pixels for v in views)
    if masks is not None:
        n = masks.n_masks
    if full is not None:
        return {"value": value, "ms_per_step": ms / args.steps, "gpu_launches": int(launches), "e2e": e2e,
                "keyframes_per_step": n_frames, "roofline": None, "splat_roofline": None, "clocks": clk,
                "stages_ms_per_step": {k: v[0] / prof_steps for k, v in prof.items()}, "dtype": "f32",
                "autotune": tuned}
    dec_ms, dec_cnt = prof["decode"]
    dec_avg_s = dec_ms / max(dec_cnt, 1) / 1e3
    flops = decode_flops(n, M, D, d)
    props = torch.cuda.get_device_properties(local)
    split = prec == api.FP32 and M <= 1024 and D <= 1024
    form = "fp32" if split else "fp32_fma" if prec in (api.FP32, api.FP32_FMA) else "bf16"
    key, per_pixel = _DECODE_TRAFFIC[form]
    traffic = per_pixel * n if key and key == _decode_sources_hash(form) and masks is None and \
        prec != api.FP8 else None
    src = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of every decode launch of one step on the 480x360 "
           "crop, scaled by pixel count") if traffic else None
    if form == "fp32_fma":
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        peak = props.multi_processor_count * SM_FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
        roof = {"bound": "alu", "kernel": "decode stage on the FMA pipes (attention rows, tiled FP32 GEMMs)",
                "achieved": flops / dec_avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"FP32 FMA: {props.multi_processor_count} SMs x {SM_FP32_LANES} lanes x 2 x "
                               f"{sm_mhz:.0f} MHz (max SM clock)"}
    elif form == "fp32":
        peak = float(peaks["bf16_tflops_sustained"]) / 3.0
        roof = {"bound": "tensor", "kernel": "decode stage: the six contractions on tcgen05 (for M <= 512 four GEMM "
                                             "kernels, dQ and dK as trailing products of the dA -> dS kernel; six "
                                             "above), operands split "
                                             "into BF16 hi/lo planes, three MMAs per FP32 product",
                "achieved": flops / dec_avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"bf16 sustained ({peak_src}) / 3: each FP32 product is three BF16 MMAs",
                "executed_bf16_tflops": 3.0 * flops / dec_avg_s / 1e12}
    else:
        peak = float(peaks["bf16_tflops_sustained"])
        roof = {"bound": "tensor", "kernel": "decode stage (tcgen05 GEMM kernels + their epilogues; for M <= 512 "
                                             "dQ and dK as trailing products of the dA -> dS kernel)",
                "achieved": flops / dec_avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"bf16 sustained ({peak_src})" + (
                    "; the FP8 form is quoted against this BF16 peak: five of its six contractions are BF16 and no "
                    "FP8 peak was measured on this pool" if prec == api.FP8 else "")}
    roof.update({"traffic": traffic, "traffic_source": src, "algorithmic_per_launch": flops})
    roof["frac"] = roof["achieved"] / roof["peak"]
    return {"value": value, "ms_per_step": ms / args.steps, "gpu_launches": int(launches), "e2e": e2e,
            "keyframes_per_step": n_frames, "roofline": roof,
            "splat_roofline": _splat_roofline(ctx_pairs, prof, prof_steps, peaks, peak_src, d),
            "clocks": clk, "stages_ms_per_step": {k: v[0] / prof_steps for k, v in prof.items()},
            "dtype": {api.FP32: "f32", api.FP32_FMA: "f32", api.BF16: "bf16", api.FP8: "bf16+e4m3"}[prec],
            "autotune": tuned}


def _tune_summary(choices):
    """The autotuner's choices for the pixel reductions of the decode backward, readable."""
    names = {5: "dV = A^T dFhat", 6: "dK = c dS^T Q"}
    tiles = {5: ("256 atoms x 256 features per CTA", "128 atoms x 256 features per CTA"), 6: ("128 atoms x 64",)}
    out = []
    for c in choices:
        r = c["reduction"] % 16
        out.append({"reduction": names.get(r, str(r)), "form": "fp32 split" if c["reduction"] >= 16 else "bf16",
                    "pixels": c["n"], "M": c["M"], "D": c["D"], "tile": tiles.get(r, ("?",) * 2)[c["tile"]],
                    "pixel_split": c["split"], "ms": round(c["ms"], 4)})
    return out


def _pair_counts(ctx, scenes):
    """(pairs P, pixels n, Gaussians N) of each keyframe: one binning through the C ABI."""
    from paper_2602_12314_gb300 import api
    out = []
    for s in scenes:
        proj = api.project(ctx, s.means, s.quats, s.scales, s.opacities, s.camera)
        bins = api.sort(ctx, proj, s.camera)
        out.append((int(bins.num_pairs), s.camera.n_pixels, int(s.means.shape[0])))
    return out


def _splat_roofline(pairs, prof, prof_steps, peaks, peak_src, d):
    """Render forward and backward against the HBM roofline: the algorithmic bytes of the
    keyframes of one step (SPLAT_FWD_BYTES / SPLAT_BWD_BYTES) over each stage's device time per
    step (CUDA-event stage timers)."""
    if not pairs:
        return None
    out = {}
    for stage, fn in (("render_fwd", SPLAT_FWD_BYTES), ("render_bwd", SPLAT_BWD_BYTES)):
        ms = prof[stage][0] / prof_steps
        if ms <= 0:
            continue
        b = sum(fn(P, n, N, d) for P, n, N in pairs)
        a = b / (ms / 1e3) / 1e9
        out[stage] = {"bound": "hbm", "achieved": a, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                      "frac": a / float(peaks["hbm_gbs"]), "algorithmic_bytes_per_step": b, "ms_per_step": ms,
                      "peak_source": f"hbm copy ({peak_src})", "pairs": [p[0] for p in pairs]}
    return out


def _measure_kmeans(args, local, scene, masks):
    """Device time of one streaming K-means dictionary update (5 micro-clusters, 10 + 10 Lloyd
    iterations, K = M slots half occupied) from the keyframe's mask targets and from its
    per-pixel targets (CUDA events, median of 5 calls after 2 warm-up calls)."""
    import numpy as np
    import torch

    from paper_2602_12314_gb300 import api

    ctx = api.Context(local)
    rng = np.random.default_rng(args.seed)
    out = {}
    for name, F, valid in (("mask_targets", masks.F, masks.valid), ("per_pixel_targets", scene.F, scene.mask)):
        Fd = torch.as_tensor(F, dtype=torch.float32, device="cuda")
        vd = torch.as_tensor(valid, dtype=torch.uint8, device="cuda")
        init = rng.choice(np.flatnonzero(valid), size=5, replace=False).astype(np.int32)
        V0 = torch.as_tensor(scene.V, device="cuda")
        w0 = torch.zeros(scene.M, device="cuda")
        w0[: scene.M // 2] = 10.0
        times = []
        for it in range(7):
            V, w = V0.clone(), w0.clone()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            api.stream_kmeans(ctx, Fd, V, w, init, valid=vd)
            e1.record()
            torch.cuda.synchronize()
            if it >= 2:
                times.append(e0.elapsed_time(e1))
        out[name] = {"rows": int(F.shape[0]), "ms": float(np.median(times))}
    ctx.close()
    out["K"], out["D"], out["k_micro"] = scene.M, scene.D, 5
    return out


def _prec_of(api, form):
    if form.startswith("fp32_fma"):
        return api.FP32_FMA
    return api.FP32 if form.startswith("fp32") else api.FP8 if form == "fp8" else api.BF16


def run_ours(args, world, rank, local):
    import torch

    from paper_2602_12314_gb300 import api

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    scene = _scene(args.seed + rank, args.crop)
    forms = (["fp32", "fp32_fma", "bf16", "bf16_batch", "fp8", "fp32_masks", "bf16_masks", "fp32_full"]
             if args.precision == "both" else [args.precision])
    res = {}
    masks = None
    for f in forms:
        views = None
        if f.endswith("_batch"):
            from workloads import room_views
            views = room_views(args.seed + rank, n_views=args.batch)
        if f.endswith("_masks") and masks is None:
            from workloads import sam_masks
            masks = sam_masks(scene, overlap=True, seed=args.seed + rank)
        full = None
        if f.endswith("_full"):
            from workloads import room_rgbd
            full = room_rgbd(args.seed + rank, scene)
        prec = _prec_of(api, f)
        res[f] = _measure(args, world, rank, local, scene, prec, dist,
                          views, masks if f.endswith("_masks") else None, full)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    head = res[forms[0]]
    n = scene.camera.n_pixels
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        times = []
        for _ in range(3):
            t0 = time.perf_counter()
            _oracle_iteration(scene, oracle.LossConfig())
            times.append(time.perf_counter() - t0)
        cpu = {"value": 1.0 / min(times), "unit": "iters/s", "cores": _cores(), "kind": "oracle",
               "sample": f"whole FP64 oracle iterations (fwd, bwd, Adam) of the {scene.camera.width}x"
                         f"{scene.camera.height} keyframe with all {scene.n} Gaussians: best of 3 "
                         f"({', '.join(f'{t:.2f}' for t in times)} s)"}
    line = {
        "metric": METRIC, "value": head["value"], "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": head["dtype"], "data": "synthetic",
        "config": _config(args, scene, world, args.precision),
        "e2e": head["e2e"], "gpu_launches": head["gpu_launches"], "roofline": head["roofline"],
        "splat_roofline": head["splat_roofline"], "cpu_baseline": cpu,
        "clocks": head["clocks"], "stages_ms_per_step": head["stages_ms_per_step"],
        "autotune": head.get("autotune"),
    }
    if len(forms) > 1:
        line["forms"] = {f: {k: res[f][k] for k in ("value", "ms_per_step", "dtype", "e2e", "roofline",
                                                    "splat_roofline", "gpu_launches", "clocks",
                                                    "stages_ms_per_step", "keyframes_per_step", "autotune")}
                         for f in forms}
        line["forms"]["fp32_fma"]["workload"] = (
            "the room keyframe, FP32 form with every decode contraction on the FMA pipes (CUDA cores)")
        line["forms"]["bf16_batch"]["workload"] = (
            f"{args.batch} keyframes of the room (the new keyframe + {args.batch - 1} history keyframes) "
            "sharing the map and the dictionary, one latentam_step_batch iteration; value = keyframe-iterations/s")
        line["forms"]["fp32_full"]["workload"] = (
            "the room keyframe with the whole Stage I objective (Eq. full_obj): queries, colours and depth "
            "rendered together, feature loss, L1 + SSIM against a ray-cast RGB image, depth L1, gradients of "
            "every Gaussian attribute and the dictionary, one Adam update of all eight groups (plain launches, "
            "one host synchronisation per iteration for the pair count)")
        for f in ("fp32_masks", "bf16_masks"):
            line["forms"][f]["workload"] = (
                f"the room keyframe with SAM-style mask targets ({masks.n_masks} masks: 80x60-pixel cells of "
                "the surface regions plus the whole regions, overlapping), queries mask-pooled before the "
                "decode; the roofline is the decode stage on the pooled rows, a small part of this step")
        line["kmeans"] = _measure_kmeans(args, local, scene, masks)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _building_keyframe(args, ctx):
    """The large-map workload: the 2M-Gaussian two-floor building in a voxel-hashed map with a
    host-resident store (5 cm voxels), the active set within 5 m of a 1296 x 968 camera gathered
    on the GPU, synthetic per-pixel targets (64 segment embeddings, one per 32 x 32 block, plus
    N(0, 0.02^2), l2-normalised), d = 32, M = 1024, D = 768.  Returns the keyframe as a scene and
    the gather time."""
    import time as _t

    import numpy as np
    import torch

    from paper_2602_12314_gb300 import api
    from workloads import Scene, building_gaussians
    from workloads.scenes import _look_camera

    g = building_gaussians(args.seed)
    vmap = api.VoxelMap(ctx, 32, table_log2=24, voxel_size=0.05, capacity=1 << 21, host_store=True)
    vmap.insert(*[g[k] for k in ("means", "quats", "scales", "opacities", "f")])
    cam = _look_camera((7.5, 7.5, 1.5), (1.0, 0.0, 0.0), (0, 0, -1), 1000.0, 1000.0, 648.0, 484.0, 1296, 968)
    torch.cuda.synchronize()
    t0 = _t.perf_counter()
    loc = vmap.sync([7.5, 7.5, 1.5], 5.0)
    gather_ms = (_t.perf_counter() - t0) * 1e3
    H, W, D, M = 968, 1296, 768, 1024
    gen = torch.Generator(device="cuda").manual_seed(args.seed)
    emb = torch.randn((64, D), generator=gen, device="cuda")
    yy, xx = torch.meshgrid(torch.arange(H, device="cuda"), torch.arange(W, device="cuda"), indexing="ij")
    lab = ((yy // 32) * ((W + 31) // 32) + xx // 32) % 64
    F = emb[lab.reshape(-1)] + 0.02 * torch.randn((H * W, D), generator=gen, device="cuda")
    F = F / F.norm(dim=1, keepdim=True)
    rng = np.random.default_rng(args.seed)
    K = (rng.normal(size=(M, 32)) / np.sqrt(32)).astype(np.float32)
    V = (rng.normal(size=(M, D)) / np.sqrt(32)).astype(np.float32)
    scene = Scene(name="building keyframe", means=loc["means"], quats=loc["quats"], scales=loc["scales"],
                  opacities=loc["opacities"], f=loc["f"], K=K, V=V, V0=V.copy(), F=F,
                  mask=torch.ones(H * W, dtype=torch.uint8, device="cuda"), camera=cam)
    return scene, gather_ms, vmap


def run_workloads(args, world, rank, local):
    """The other workloads of the step (their numbers are reported beside the headline run):
    tiny, precision (500k Gaussians, M = 512, D = 1024), batch8 (eight keyframes of uneven
    resolution with their own maps, M = 512, D = 768) and building (the large map)."""
    import torch

    from paper_2602_12314_gb300 import api
    from workloads import keyframe_batch, precision_scene, tiny_scene

    torch.cuda.set_device(local)
    args.no_e2e = True
    res, extra = {}, {}
    views = None
    if args.workload == "tiny":
        scene, forms = tiny_scene(args.seed), ("fp32", "bf16")
        desc = "tiny keyframe: 2,000 Gaussians, 64x48, d=16, M=64, D=512"
    elif args.workload == "precision":
        scene, forms = precision_scene(args.seed), ("fp32", "bf16", "fp8")
        desc = "room keyframe at larger dims: 500k Gaussians, 640x480, d=32, M=512, D=1024"
    elif args.workload == "batch8":
        sizes = ((320, 240), (640, 480), (640, 480), (640, 480), (848, 480), (848, 480), (1200, 680), (1200, 680))
        ns = (100_000, 150_000, 250_000, 300_000, 400_000, 500_000, 700_000, 1_000_000)
        views = keyframe_batch(args.seed, sizes=sizes, ns=ns, d=32, M=512, D=768)
        scene, forms = views[0], ("bf16_batch", "fp32_batch")
        desc = ("eight keyframes of uneven resolution (320x240, 640x480 x3, 848x480 x2, 1200x680 x2; 3,444,480 pixels), "
                "each with its own room and 100k-1M Gaussians, one shared dictionary d=32, M=512, D=768")
    else:
        ctx = api.Context(local)
        scene, gather_ms, vmap = _building_keyframe(args, ctx)
        extra = {"gather_ms": gather_ms, "local_gaussians": int(scene.means.shape[0]), "map_gaussians_inserted": None}
        forms = ("bf16",)
        desc = ("large map: 2M-Gaussian two-floor building in a voxel-hashed map (5 cm voxels, host-resident store), "
                "the active set within 5 m gathered on the GPU, one 1296x968 keyframe, d=32, M=1024, D=768, "
                "10 iterations per keyframe")
        args.steps = 10
    for f in forms:
        prec = _prec_of(api, f)
        res[f] = _measure(args, world, rank, local, scene, prec, None, views if f.endswith("_batch") else None)
    line = {"workload": args.workload, "description": desc, "steps": args.steps,
            "forms": {f: {k: r[k] for k in ("value", "ms_per_step", "dtype", "roofline", "splat_roofline", "clocks",
                                            "stages_ms_per_step", "keyframes_per_step")} for f, r in res.items()}}
    line.update(extra)
    print(json.dumps(line), flush=True)


def main():
    args = _args()
    world, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload != "room":
        run_workloads(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
