#!/usr/bin/env python3
"""Benchmark: rays/s and geodesic steps/s of the 1024 x 1024 analytic Kerr image
(a = 0.9375, i = 60 deg, r_cam = 1000 M, +-20 M, 230 GHz), mixed FP32/FP64 path against
the plain FP64 path on the same GPU, with the FP64 CPU oracle timed on a bounded sample.

One "step" = one complete render of the image (camera, adaptive RK4 geodesics, plasma,
emissivity, backward transfer, deterministic flux reduction) through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun each rank renders its own full image (independent units, weak scaling, no
collective on the data path); the max over ranks of the timed region is reported.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "kerr_analytic_1024x1024_a0.9375_i60_230GHz"
METRIC = "rays/s and geodesic steps/s at 1024^2 Kerr image, mixed+MLP vs FP64 at <=1e-3 flux"
CPU_SAMPLE_STRIDE = 8  # oracle traces every 8th pixel in each direction (128 x 128 rays)
PROFILED_RENDERS = 2   # renders of the separate pass that records per-kernel times
# DRAM bytes (read + write) of one launch of a kernel at the headline size, from the ncu
# capture summarised in profiles/launches_kerr_analytic_1024_mlp_df.md (null for kernels
# without a capture of their current source)
DRAM_BYTES_PER_LAUNCH = {"mixed_fp64_long": 1955072}
# hardware counters of the same kernel at 512^2 (profiles/k_mixed_fp64_df64_passes_512.md):
# FP32 (FMA) pipe busy and issue-active fractions beside the algorithmic-flop roofline
NCU_PIPES = {"mixed_fp64_long": {"fma_pipe": 0.162, "issue_active": 0.501, "at": "512^2, ncu"}}
FINAL_LINE_MAX = 2000  # bytes: the last stdout line carries the headline only


def _env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def max_over_ranks(value, dist, device="cuda"):
    """The maximum of a per-rank number over all ranks: a replicated job takes as long as its
    slowest rank."""
    import torch

    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world, units_per_step_per_rank, ms_per_step):
    """Whole-job throughput of `world` replicas, each processing units_per_step_per_rank per
    step, timed by the slowest rank's ms per step (weak scaling)."""
    return world * units_per_step_per_rank / (ms_per_step * 1e-3)


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [l.strip().split(", ") for l in open(self.f.name) if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(cam: dict, freqs, stride: int, threads: int = 0):
    """Time the FP64 CPU oracle on the strided pixel subset of the workload."""
    import oracle
    from paper_1801_10452_b300 import scenes

    s = oracle.scene(a=cam["spin"], incl_deg=cam["incl_deg"], r_cam=cam["r_cam"], nx=cam["nx"] // stride,
                     ny=cam["ny"] // stride, amin=cam["alpha_min"], amax=cam["alpha_max"], bmin=cam["beta_min"],
                     bmax=cam["beta_max"], eps=cam["eps"], r_stop_factor=cam["r_stop_factor"], r_esc=cam["r_escape"],
                     mass_msun=cam["mass_msun"], dist_pc=cam["distance_pc"], **{
                         "n0": scenes.ANALYTIC_PLASMA["n0"], "n_pow": scenes.ANALYTIC_PLASMA["n_pow"],
                         "the0": scenes.ANALYTIC_PLASMA["the0"], "the_pow": scenes.ANALYTIC_PLASMA["the_pow"],
                         "B0": scenes.ANALYTIC_PLASMA["B0_gauss"], "B_pow": scenes.ANALYTIC_PLASMA["B_pow"]})
    # The strided camera keeps the full-size pixel pitch: cover every `stride`-th pixel
    # centre of the full image.
    da = (cam["alpha_max"] - cam["alpha_min"]) / cam["nx"]
    db = (cam["beta_max"] - cam["beta_min"]) / cam["ny"]
    n_s = cam["nx"] // stride
    # pixel j of the sample = full pixel stride*j + stride//2
    off = (stride // 2 + 0.5) * da - 0.5 * stride * da
    s.amin = cam["alpha_min"] + off
    s.amax = s.amin + n_s * stride * da
    offb = (stride // 2 + 0.5) * db - 0.5 * stride * db
    s.bmin = cam["beta_min"] + offb
    s.bmax = s.bmin + (cam["ny"] // stride) * stride * db
    oracle.lib()
    t0 = time.perf_counter()
    img, steps, status = oracle.render(s, freqs, nthreads=threads)
    dt = time.perf_counter() - t0
    # rescale the per-pixel Jy to the full-size pixel solid angle
    img = img / (stride * stride)
    return dict(seconds=dt, rays=img[0].size * len(freqs) / len(freqs), steps=int(steps.sum()), img=img,
                cores=oracle.num_threads() if threads <= 0 else threads)


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores, a bounded sample per step."""
    rank, _, world = _env_rank()
    if rank != 0:
        return
    from paper_1801_10452_b300 import scenes

    cam = scenes.HEADLINE
    for _ in range(max(0, min(args.warmup, 1))):
        oracle_sample(cam, scenes.HEADLINE_FREQS, CPU_SAMPLE_STRIDE * 2)
    secs, rays, steps = 0.0, 0, 0
    for _ in range(args.steps):
        r = oracle_sample(cam, scenes.HEADLINE_FREQS, CPU_SAMPLE_STRIDE * 2)
        secs += r["seconds"]
        rays += r["rays"]
        steps += r["steps"]
    v = rays / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (analytic plasma, deterministic)",
        "config": {"workload": WORKLOAD, "sample": f"every {CPU_SAMPLE_STRIDE * 2}th pixel per axis per step"},
        "steps_per_s": steps / secs,
        "cpu_baseline": {"value": v, "unit": "rays/s", "cores": r["cores"], "kind": "oracle",
                         "sample": f"{int(rays / args.steps)} rays per step (strided subset of the 1024^2 image)"},
        "e2e": {"value": v, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _time_render(ctx, torch, freqs, image, flush_buf, n, stream):
    """n renders, L2 flushed before each, device time of the renders only (CUDA events)."""
    tot = 0.0
    for _ in range(n):
        flush_buf.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.render(freqs, image=image, flux=False, stream=stream)
        b.record(stream)
        b.synchronize()
        tot += a.elapsed_time(b)
    return tot


def train_surrogate(R, torch, cam, steps, n_train, handoff=60):
    """Train the learned far-field surrogate on integrator-generated rays (not timed as part
    of a render step), for a hand-off after `handoff` steps; returns its parameters and a
    summary."""
    ctx = R.Context(R.camera_desc(**cam, precision=R.MIXED_MLP))
    ctx.load_plasma(R.plasma_desc(**scenes_mod().ANALYTIC_PLASMA))
    ctx.surrogate_handoff(handoff)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, y = ctx.surrogate_generate(n_train, seed=0x1801104520000005)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    ctx.surrogate_init(y, seed=7)
    t1 = time.perf_counter()
    ctx.surrogate_train(x, y, steps, lr=2e-3, lr_final=2e-5, seed=11)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    xh, yh = ctx.surrogate_generate(100_000, seed=0x1801104520000006)
    err = np.abs(ctx.surrogate_eval(xh).cpu().numpy() - yh.cpu().numpy())
    names = ["dt", "ln_r", "theta", "phi", "k_theta", "k_r"]
    summ = {"rays": n_train, "steps": steps, "batch": 4096, "handoff_steps": handoff, "generate_s": t_gen, "train_s": t_train,
            "heldout_median_abs_err": dict(zip(names, np.median(err, 0).tolist())),
            "heldout_p99_abs_err": dict(zip(names, np.percentile(err, 99, axis=0).tolist())),
            "range": "alpha, beta in +-20 M; a in [0, 0.99]; i in [5, 85] deg"}
    return ctx.surrogate_get(), summ


def _timed_path(R, torch, cam, prec, freqs, args, flush, stream, world, dist, sample_clocks, params=None, flags=0,
                plasma=None, fields=None, steps=None):
    """Warm up, then time `steps` (default args.steps) renders of one path; returns
    measurements.  plasma/fields: a grid scene (default: the analytic plasma)."""
    ctx = R.Context(R.camera_desc(**cam, precision=prec, flags=flags))
    if plasma is None:
        ctx.load_plasma(R.plasma_desc(**scenes_mod().ANALYTIC_PLASMA))
    else:
        ctx.load_plasma(R.plasma_desc(**plasma), fields=fields)
    n_steps = args.steps if steps is None else steps
    if params is not None:
        ctx.surrogate_set(params)
    image = torch.empty((len(freqs), cam["ny"], cam["nx"]), dtype=torch.float64, device="cuda")
    tuned = None if args.no_autotune else ctx.autotune(freqs, stream=stream)
    for _ in range(args.warmup):
        ctx.render(freqs, image=image, flux=False, stream=stream)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if sample_clocks else None
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    ctx.stats_reset()
    ctx.profile(False)
    wall0 = time.perf_counter()
    dev_ms = _time_render(ctx, torch, freqs, image, flush, n_steps, stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    st = ctx.stats_ex()
    if world > 1:
        dev_ms = max_over_ranks(dev_ms, dist)
    # per-kernel breakdown in a separate pass with the library's per-launch events on (the
    # timed renders above run without them)
    ctx.stats_reset()
    ctx.profile(True)
    prof_ms = _time_render(ctx, torch, freqs, image, flush, PROFILED_RENDERS, stream)
    prof = ctx.profile_read()
    timeline = ctx.profile_timeline()
    ctx.profile(False)
    st_prof = ctx.stats_ex()
    _, flux = ctx.render(freqs, image=image, stream=stream)
    torch.cuda.synchronize()
    return dict(ctx=ctx, image=image, ms=dev_ms / n_steps, wall=wall, clocks=clocks, prof=prof, stats=st, flux=flux,
                tuned=tuned, st_prof=st_prof, prof_ms=prof_ms / PROFILED_RENDERS, timeline=timeline)


def _lightcurve_extra(R, torch, args, stream, params, n=100, size=256):
    """Slow-light light curve: n snapshots of the torus 10 M apart (noise advected at the
    Keplerian rate), n frames of size^2 at 230 GHz in one persistent launch sequence per
    path, against n per-frame fast-light renders (frame f on snapshot f)."""
    from paper_1801_10452_b300 import scenes

    fields, meta = scenes.torus_snapshots(n, dt_snap=10.0, device="cuda", seed=scenes.SLOW["seed"])
    cam = dict(scenes.HEADLINE, nx=size, ny=size)
    freqs = [230e9]
    t_obs = 10.0 * np.arange(n)
    out = {"workload": f"grid_torus_lightcurve_{n}x{size}x{size}_230GHz",
           "frames": n, "rays_per_lightcurve": n * size * size,
           "snapshots": f"{n} x 2 MiB, 10 M apart, noise rotated at the local Keplerian rate"}

    def make(prec, flags, slow):
        ctx = R.Context(R.camera_desc(**cam, precision=prec, flags=flags))
        ctx.load_plasma(R.plasma_desc(**scenes.grid_plasma(meta, scenes.DISK_MODEL, slow, -50.0)), fields=fields)
        if prec == R.MIXED_MLP:
            ctx.surrogate_set(params)
        return ctx

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / reps

    paths = [("mlp_df", R.MIXED_MLP, R.FLAG_INNER_DF64)] if params is not None else []
    paths += [("mixed_df", R.MIXED, R.FLAG_INNER_DF64), ("fp64", R.FP64, 0)]
    for name, prec, flags in paths:
        slow = make(prec, flags, 1)
        reps = 1 if prec == R.FP64 else 2
        ms_lc = timed(lambda: slow.lightcurve(freqs, t_obs, stream=stream), reps)
        fl = slow.lightcurve(freqs, t_obs, stream=stream)
        entry = {"ms_per_lightcurve": ms_lc, "rays_per_s": n * size * size / (ms_lc * 1e-3),
                 "flux_jy_min_max": [float(fl.min()), float(fl.max())]}
        slow.close()
        if prec != R.FP64:
            fast = make(prec, flags, 0)
            img = torch.empty((1, size, size), dtype=torch.float64, device="cuda")

            def frames():
                for f in range(n):
                    fast.render(freqs, image=img, flux=False, snap=f, stream=stream)

            ms_pf = timed(frames, 1)
            entry["per_frame_fast_light_ms"] = ms_pf
            entry["per_frame_rays_per_s"] = n * size * size / (ms_pf * 1e-3)
            fast.close()
        out[name] = entry
    return out


def _disk_extra(R, torch, stream, fma64, reps=2):
    """Thin-disk line emitter (sec. 4.2.1): the paper's five spins at 1024^2, i = 30 deg,
    FP64 rays with Newton-refined equatorial crossings and the first-order line spectrum.
    Roofline: the geodesic step's algorithmic flops (step size + RK4; counted from the
    source) x steps / kernel time against the FP64 FMA-chain peak."""
    from paper_1801_10452_b300 import flopcount, scenes

    geo = flopcount.flops_per_step(1, "analytic")["geodesic_only"]
    cam0 = scenes.THIN_DISK
    out = {"workload": f"thin_disk_{cam0['nx']}x{cam0['ny']}_i{cam0['incl_deg']:g}_rin_isco_rout15_q2",
           "spins": scenes.THIN_DISK_SPINS, "per_spin": {}}
    tot_ms = tot_rays = 0.0
    for a in scenes.THIN_DISK_SPINS:
        ctx = R.Context(R.camera_desc(**dict(cam0, spin=a)))
        res = ctx.disk_render(**scenes.THIN_DISK_GEOM, stream=stream)
        torch.cuda.synchronize()
        ctx.stats_reset()
        ctx.profile(True)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            res = ctx.disk_render(**scenes.THIN_DISK_GEOM, stream=stream)
        t1.record(stream)
        t1.synchronize()
        ms = t0.elapsed_time(t1) / reps
        prof = ctx.profile_read()
        ctx.profile(False)
        st = ctx.stats()
        order = res["order"].cpu().numpy()
        spec = res["spectrum"]
        edges = res["edges"]
        centres = 0.5 * (edges[1:] + edges[:-1])
        rays = cam0["nx"] * cam0["ny"]
        steps = st["steps"] / reps
        k_ms = prof["disk"][0] / reps
        ach = geo * steps / (k_ms * 1e-3) / 1e12
        out["per_spin"][f"{a:g}"] = {
            "ms": ms, "rays_per_s": rays / (ms * 1e-3), "steps_per_ray": steps / rays,
            "hit_fraction_first_order": float((order == 1).mean()), "hit_fraction_any": float((order > 0).mean()),
            "line_peak_E_ratio": float(centres[int(np.argmax(spec))]),
            "line_mean_E_ratio": float((spec * centres).sum() / spec.sum()),
            "roofline": {"bound": "alu", "pipe": "fp64", "achieved": ach, "peak": fma64, "unit": "TFLOP/s",
                         "frac": ach / fma64, "flops_per_step": geo}}
        tot_ms += ms
        tot_rays += rays
        ctx.close()
    out["rays_per_s_all_spins"] = tot_rays / (tot_ms * 1e-3)
    return out


def _learned_disk_extra(R, torch, stream, bf16_peak, steps, n_train, reps=3):
    """The surrogate's equatorial outputs: a crossing network (4 -> 256 -> 256 -> 256 -> 16)
    trained on n_train integrator rays over the learned workload's range, its held-out
    accuracy, and the learned thin disk against the FP64 disk at 1024^2 (i = 30 deg, +-16 M)
    for the disk workload's five spins (the negative ones from a second network trained on
    a in [-0.99, 0]).  Network roofline: its
    algorithmic flops (2 x (4 x 256 + 2 x 256^2 + 256 x 16) per ray) over its profiled time
    against the measured BF16 peak."""
    from paper_1801_10452_b300 import scenes

    cam_t = dict(scenes.SMALL)
    ctx = R.Context(R.camera_desc(**cam_t))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, y = ctx.crossings_generate(n_train, seed=0x1801104520000005)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    ctx.crossings_init(y, seed=7)
    t1 = time.perf_counter()
    ctx.crossings_train(x, y, steps, lr=2e-3, lr_final=2e-5, seed=11)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    del x, y
    P = ctx.crossings_get()
    # retrograde spins of the disk workload: a second network over a in [-0.99, 0]
    t2 = time.perf_counter()
    xr, yr = ctx.crossings_generate(n_train, seed=0x1801104520000007, spin=(-0.99, 0.0))
    ctx.crossings_init(yr, seed=7, inputs=xr)
    ctx.crossings_train(xr, yr, steps, lr=2e-3, lr_final=2e-5, seed=11)
    torch.cuda.synchronize()
    t_retro = time.perf_counter() - t2
    del xr, yr
    P_retro = ctx.crossings_get()
    ctx.crossings_set(P)
    xh, _, zh = ctx.crossings_generate(100_000, seed=0x1801104520000006, raw=True)
    ph = ctx.crossings_eval(xh).cpu().numpy()
    zh = zh.cpu().numpy()
    pres_t, pres_p = zh[:, 0::4] > 0.5, ph[:, 0::4] > 0.5
    both = pres_t & pres_p
    rel_r = np.abs(ph[:, 1::4][both] / zh[:, 1::4][both] - 1)
    rel_l = np.abs(ph[:, 2::4][both] / zh[:, 2::4][both] - 1)
    rat = both & np.isfinite(zh[:, 3::4]) & (zh[:, 1::4] >= 6.0)
    rel_g = np.abs(ph[:, 3::4][rat] / zh[:, 3::4][rat] - 1)
    out = {"training": {"rays": n_train, "steps": steps, "batch": 4096, "generate_s": t_gen, "train_s": t_train,
                        "range": "alpha, beta in +-20 M; a in [0, 0.99]; i in [5, 85] deg",
                        "heldout_rays": 100_000,
                        "heldout_count_accuracy": float(np.mean(np.all(pres_t == pres_p, axis=1))),
                        "heldout_r_rel_err_median": float(np.median(rel_r)),
                        "heldout_r_rel_err_p99": float(np.quantile(rel_r, 0.99)),
                        "heldout_lambda_rel_err_p99": float(np.quantile(rel_l, 0.99)),
                        "heldout_ratio_rel_err_median_r_ge_6": float(np.median(rel_g)),
                        "heldout_ratio_rel_err_p99_r_ge_6": float(np.quantile(rel_g, 0.99)),
                        "note": "held-out rays over the whole range, critical-curve band included"},
           "training_retrograde": {"rays": n_train, "steps": steps, "range": "a in [-0.99, 0]",
                                   "generate_and_train_s": t_retro}}
    ctx.close()
    flops_ray = 2 * (4 * 256 + 2 * 256 * 256 + 256 * 16)
    cam0 = scenes.THIN_DISK
    out["workload"] = f"learned_thin_disk_{cam0['nx']}x{cam0['ny']}_i{cam0['incl_deg']:g}_rin_isco_rout15_q2"
    out["per_spin"] = {}

    def timed(ctx, learned):
        r = ctx.disk_render(**scenes.THIN_DISK_GEOM, stream=stream, learned=learned)
        torch.cuda.synchronize()
        ctx.profile(True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            r = ctx.disk_render(**scenes.THIN_DISK_GEOM, stream=stream, learned=learned)
        e1.record(stream)
        e1.synchronize()
        prof = ctx.profile_read()
        ctx.profile(False)
        return e0.elapsed_time(e1) / reps, {k: v.cpu().numpy() if hasattr(v, "cpu") else v for k, v in r.items()}, prof

    # (suffix, band, double-float fallback, confidence margins: presence logit, ln r)
    variants = [("", 1.0, True, (2.0, 0.01)), ("_noconfidence", 1.0, True, (0.0, 0.0)),
                ("_fp64fallback", 1.0, False, (2.0, 0.01)), ("_band0.5", 0.5, True, (2.0, 0.01))]
    for a in scenes.THIN_DISK_SPINS:
        ctx = R.Context(R.camera_desc(**dict(cam0, spin=a)))
        ctx.crossings_set(P if a >= 0.0 else P_retro)
        ms_f, f, _ = timed(ctx, False)
        # retrograde: a larger critical curve, whose strongly deflected surroundings need a
        # 1.5 M band at a = -0.99 to keep every pixel within 1e-2 (measured; 1.0 M reported too)
        for suffix, band, df, conf in (variants if a >= 0.0 else [("", 1.5, True, (2.0, 0.01)),
                                                                   ("_band1", 1.0, True, (2.0, 0.01))]):
            ctx.crossings_config(fallback_band=band, fallback_df64=df)
            ctx.crossings_confidence(*conf)
            ms_l, g, prof = timed(ctx, True)
            fb = g["steps"] > 0
            nb = ~fb
            hit = nb & (f["order"] > 0) & (g["order"] == f["order"])
            rel = np.abs(g["ratio"][hit] / f["ratio"][hit] - 1)
            fbh = fb & (f["order"] > 0) & (g["order"] == f["order"])
            rel_fb = np.abs(g["ratio"][fbh] / f["ratio"][fbh] - 1)
            # every learned pixel, misclassified ones included: intensity error relative to
            # the larger of the two intensities (a false hit or a false miss counts as 1)
            Il, If = g["intensity"][nb], f["intensity"][nb]
            big = np.maximum(np.abs(Il), np.abs(If))
            rel_all = np.where(big > 0, np.abs(Il - If) / np.where(big > 0, big, 1.0), 0.0)
            sf, sg = f["spectrum"], g["spectrum"]
            rays = cam0["nx"] * cam0["ny"]
            mlp_ms = prof["surrogate_mlp"][0] / reps
            ach = flops_ray * rays / (mlp_ms * 1e-3) / 1e12
            w = np.nonzero(hit)
            out["per_spin"][f"{a:g}{suffix}"] = {
                "fallback_band_M": band, "fallback_arithmetic": "double-float" if df else "fp64",
                "confidence_margins": list(conf),
                "order_mismatch_learned_pixels": int((g["order"][nb] != f["order"][nb]).sum()),
                "intensity_rel_err_max_all_learned": float(rel_all.max()) if rel_all.size else 0.0,
                "intensity_rel_err_p99_all_learned": float(np.quantile(rel_all, 0.99)) if rel_all.size else 0.0,
                "intensity_pixels_over_1e-2_all_learned": int((rel_all > 1e-2).sum()),
                "ms_learned": ms_l, "ms_fp64": ms_f, "speedup": ms_f / ms_l, "rays_per_s_learned": rays / (ms_l * 1e-3),
                "fallback_fraction": float(fb.mean()),
                "fallback_order_agreement": float((g["order"][fb] == f["order"][fb]).mean()),
                "fallback_ratio_rel_err_max": float(rel_fb.max()) if rel_fb.size else 0.0,
                "order_agreement_outside_fallback": float((g["order"][nb] == f["order"][nb]).mean()),
                "ratio_rel_err_max": float(rel.max()), "ratio_rel_err_p99": float(np.quantile(rel, 0.99)),
                "pixels_compared": int(hit.sum()), "pixels_over_1e-2": int((rel > 1e-2).sum()),
                "worst_pixel_alpha_beta": [float(cam0["alpha_min"] + (w[1][np.argmax(rel)] + 0.5) *
                                                 (cam0["alpha_max"] - cam0["alpha_min"]) / cam0["nx"]),
                                           float(cam0["beta_min"] + (w[0][np.argmax(rel)] + 0.5) *
                                                 (cam0["beta_max"] - cam0["beta_min"]) / cam0["ny"])],
                "spectrum_total_rel_err": float(sg.sum() / sf.sum() - 1),
                "spectrum_l1_normalised": float(np.abs(sg / sg.sum() - sf / sf.sum()).sum()),
                "stage_ms": {k: v[0] / reps for k, v in prof.items() if v[1]},
                "network_roofline": {"bound": "tensor", "kernel": "k_mlp_tc12<16> + k_mlp_tc34<16> (tcgen05; mma.sync if selected)", "achieved": ach,
                                     "peak": bf16_peak, "unit": "TFLOP/s", "frac": ach / bf16_peak,
                                     "flops_per_ray": flops_ray}}
        ctx.close()
    out["heldout_ratio_note"] = "held-out ratios compared where r >= 6 M (outside every prograde ISCO)"
    return out


def _verlet_extra(R, torch, stream, fma64, flush, reps=2):
    """The FP64 path with the velocity-Verlet integrator (sec. 2.2.2) on the headline image,
    with and without the re-evaluation, beside RK4, and RK4 with the forward formal-solution
    transfer (sec. 3): time per render, rays/s, steps/s, flux against RK4, and the FP64
    roofline (algorithmic flops per step, counted from the source, x steps / kernel time
    against the FP64 FMA-chain peak)."""
    from paper_1801_10452_b300 import flopcount, scenes

    fl = flopcount.flops_per_step(1, "analytic")
    cam = scenes.HEADLINE
    freqs = scenes.HEADLINE_FREQS
    out = {"workload": "kerr_analytic_1024x1024_a0.9375_i60_230GHz_fp64", "per_integrator": {}}
    flux_rk4 = None
    for name, flags, fps in (("rk4", 0, fl["fp64_step"]), ("verlet", R.FLAG_VERLET, fl["verlet_step"]),
                             ("verlet_reeval", R.FLAG_VERLET_REEVAL, fl["verlet_reeval_step"]),
                             ("rk4_forward_transfer", R.FLAG_FORWARD_RT, fl["fp64_step"])):
        ctx = R.Context(R.camera_desc(**cam, flags=flags))
        ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA))
        img = torch.empty((1, cam["ny"], cam["nx"]), dtype=torch.float64, device="cuda")
        _, flux = ctx.render(freqs, image=img, stream=stream)
        ctx.stats_reset()
        ctx.profile(True)
        ms = []
        for _ in range(reps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.render(freqs, image=img, flux=False, stream=stream)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        prof = ctx.profile_read()
        ctx.profile(False)
        st = ctx.stats()
        t = float(np.mean(ms))
        steps = st["steps"] / reps
        k_ms = prof["render_fp64"][0] / reps
        ach = fps * steps / (k_ms * 1e-3) / 1e12
        if flux_rk4 is None:
            flux_rk4 = flux[0]
        out["per_integrator"][name] = {
            "ms": t, "rays_per_s": cam["nx"] * cam["ny"] / (t * 1e-3), "geodesic_steps_per_s": steps / (t * 1e-3),
            "steps_per_ray": steps / (cam["nx"] * cam["ny"]), "flux_rel_vs_rk4": float(flux[0] / flux_rk4 - 1),
            "roofline": {"bound": "alu", "pipe": "fp64", "achieved": ach, "peak": fma64, "unit": "TFLOP/s",
                         "frac": ach / fma64, "flops_per_step": fps}}
        ctx.close()
    return out


def _emissivity_extra(R, torch, stream, size=256):
    """Emissivity options on the spectral scene (a = 0.9375, i = 60 deg, eight frequencies
    1e10-1e13 Hz) through the FP64 path: the flux change from the exact K2 (sec. 4.2.2 expects
    a few per cent at most) and from the Theta_e fit-validity mask at 0.5 (the fit's stated
    limit) and 2, per frequency, with the render times."""
    from paper_1801_10452_b300 import scenes

    cam = dict(scenes.SPECTRAL, spin=0.9375, nx=size, ny=size)
    freqs = scenes.SPECTRAL_FREQS
    out = {"workload": f"kerr_analytic_{size}x{size}_a0.9375_i60_8freq_fp64", "freqs_hz": freqs}
    base = None
    for name, flags, mask in (("k2_fit", 0, 0.0), ("k2_exact", R.FLAG_K2_EXACT, 0.0), ("mask_0.5", 0, 0.5),
                              ("mask_2", 0, 2.0)):
        ctx = R.Context(R.camera_desc(**cam, flags=flags))
        ctx.load_plasma(R.plasma_desc(**scenes.ANALYTIC_PLASMA, theta_e_min=mask))
        img = torch.empty((len(freqs), size, size), dtype=torch.float64, device="cuda")
        ctx.render(freqs, image=img, stream=stream)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _, fl = ctx.render(freqs, image=img, stream=stream)
        b.record(stream)
        b.synchronize()
        if base is None:
            base = fl
        out[name] = {"ms": a.elapsed_time(b), "flux_jy": [float(v) for v in fl],
                     "flux_rel_vs_fit": [float(v / w - 1) if w > 0 else 0.0 for v, w in zip(fl, base)]}
        ctx.close()
    return out


def scenes_mod():
    from paper_1801_10452_b300 import scenes

    return scenes


def run_native(args):
    import torch

    import paper_1801_10452_b300 as R
    from paper_1801_10452_b300 import build, scenes

    rank, local_rank, world = _env_rank()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    build.build()
    stream = torch.cuda.current_stream()
    cam = dict(scenes.HEADLINE, nx=args.size, ny=args.size)
    freqs = scenes.HEADLINE_FREQS
    npix = cam["nx"] * cam["ny"]
    paths = [p for p in args.paths.split(",") if p]
    workload = WORKLOAD if args.size == 1024 else WORKLOAD.replace("1024x1024", f"{args.size}x{args.size}")
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > L2
    rays_step = npix * len(freqs)

    params, sur, params_grid = None, None, None
    if any(p.startswith("mlp") for p in paths):
        params, sur = train_surrogate(R, torch, cam, args.train_steps, args.train_rays)
        if not (args.no_grid and args.no_lightcurve):
            # the torus's fine structure wants the earlier hand-off (smaller angular error of
            # the learned start states; measured per pixel in the grid workload)
            params_grid, sur_grid = train_surrogate(R, torch, cam, args.train_steps, args.train_rays, handoff=30)
            sur = {"analytic": sur, "grid": sur_grid}
    res = {}
    for pth in paths:
        prec = {"mlp": R.MIXED_MLP, "mixed": R.MIXED, "fp64": R.FP64, "mlp_df": R.MIXED_MLP, "mixed_df": R.MIXED}[pth]
        flags = R.FLAG_INNER_DF64 if pth.endswith("_df") else 0
        res[pth] = _timed_path(R, torch, cam, prec, freqs, args, flush, stream, world, dist,
                               sample_clocks=(rank == 0 and pth == paths[0]),
                               params=params if pth.startswith("mlp") else None, flags=flags)
    # ---- the grid workload (synthetic FM torus snapshot, 256^2 MKS cells) at the same size ----
    grid = None
    if not args.no_grid:
        fields, meta = scenes.torus_snapshots(1)
        gplasma = scenes.grid_plasma(meta, scenes.DISK_MODEL)
        gres = {}
        for pth in ("mlp_df", "mixed_df", "fp64"):
            prec = {"mlp_df": R.MIXED_MLP, "mixed_df": R.MIXED, "fp64": R.FP64}[pth]
            if prec == R.MIXED_MLP and params_grid is None:
                continue
            gres[pth] = _timed_path(R, torch, cam, prec, freqs, args, flush, stream, world, dist, sample_clocks=False,
                                    params=params_grid if prec == R.MIXED_MLP else None,
                                    flags=R.FLAG_INNER_DF64 if pth.endswith("_df") else 0, plasma=gplasma,
                                    fields=fields, steps=2 if pth == "fp64" else None)
        grid = {"workload": workload.replace("kerr_analytic", "grid_torus"),
                "snapshot": "Fishbone-Moncrief torus x lognormal noise, 256 x 256 MKS cells, 2 MiB (L2-resident)"}
        for pth, r in gres.items():
            st = r["stats"]
            n_r = args.steps if pth != "fp64" else 2
            samples_s = (st["steps"] / n_r) / (r["ms"] * 1e-3)
            grid[pth] = {"ms_per_step": r["ms"], "rays_per_s": aggregate_rate(world, rays_step, r["ms"]),
                         "geodesic_steps_per_s": world * samples_s, "flux_jy": float(r["flux"][0]),
                         "grid_sample_GBps": samples_s * 128 / 1e9,
                         "grid_sample_note": "128 B of FP32 fields per plasma sample (4 corners x 8 fields), "
                                             "served from L2: the snapshot is 2 MiB"}
        if "fp64" in gres:
            ref = gres["fp64"]["image"].cpu().numpy()[0]
            band = _band_mask(cam)
            pk = np.abs(ref).max()
            m = ~band & (np.abs(ref) >= 1e-6 * pk)
            for pth in gres:
                if pth != "fp64":
                    grid[pth]["flux_rel_err_vs_fp64"] = float(abs(gres[pth]["flux"][0] / gres["fp64"]["flux"][0] - 1))
                    rel = np.abs(gres[pth]["image"].cpu().numpy()[0] - ref) / np.maximum(np.abs(ref), 1e-300)
                    grid[pth]["pixels_vs_fp64_outside_band"] = {
                        "compared": int(m.sum()), "max_rel": float(rel[m].max()),
                        "p999_rel": float(np.quantile(rel[m], 0.999)), "over_1e-2": int((rel[m] > 1e-2).sum()),
                        "note": "pixels above 1e-6 of the peak, more than 0.5 M from the critical curve"}
        for r in gres.values():
            r["ctx"].close()
    # ---- the slow-light light curve (100 snapshots 10 M apart, 100 frames of 256^2) ----
    lcurve = None
    if not args.no_lightcurve:
        lcurve = _lightcurve_extra(R, torch, args, stream, params_grid)
    # ---- the FP64 path with the velocity-Verlet integrator (sec. 2.2.2) ----
    verlet = None
    if not args.no_verlet and rank == 0:
        verlet = _verlet_extra(R, torch, stream, R.measure_fma_peak(True), flush)
    # ---- emissivity options: exact K2 and the Theta_e validity mask ----
    emis = None
    if not args.no_emissivity and rank == 0:
        emis = _emissivity_extra(R, torch, stream)
    # ---- the thin-disk line emitter (sec. 4.2.1), five spins ----
    disk = None
    if not args.no_disk and rank == 0:
        disk = _disk_extra(R, torch, stream, R.measure_fma_peak(True))
    ldisk = None
    if not args.no_disk and not args.no_learned_disk and rank == 0:
        ldisk = _learned_disk_extra(R, torch, stream, _peaks().get("bf16_tflops", 1800.0), args.train_steps,
                                   args.train_rays)
    main = res[paths[0]]
    ms_step = main["ms"]
    value = aggregate_rate(world, rays_step, ms_step)
    st = main["stats"]
    steps_per_s = world * (st["steps"] / args.steps) / (ms_step * 1e-3)
    # kernel launches per render (counted by the library in the profiled pass) x timed renders
    launches_per_render = sum(v[1] for v in main["prof"].values()) / PROFILED_RENDERS
    launches = int(round(launches_per_render * args.steps))

    # ---- end to end through the C ABI with host buffers --------------------------------
    e2e = None
    if not args.no_e2e:
        ctx = main["ctx"]
        img_bytes = 8 * rays_step
        host_img = R.pinned_host_array((len(freqs), cam["ny"], cam["nx"]))
        ctx.render_host(freqs, out=host_img)
        e2e_t = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx.render_host(freqs, out=host_img)
            e2e_t.append(time.perf_counter() - t0)
        e2e = {"value": world * rays_step / float(np.mean(e2e_t)), "unit": "rays/s", "h2d_bytes_per_step": 8 * len(freqs),
               "d2h_bytes_per_step": int(img_bytes) + 8 * len(freqs)}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- rooflines: algorithmic flops (from the kernel source) / measured FMA peaks -------
    fma32 = R.measure_fma_peak(False)
    fma64 = R.measure_fma_peak(True)
    roofs = _rooflines(res, fma32, fma64, npix)
    dom = _dominant_kernel(main["prof"], paths[0], roofs)
    roof = dict(roofs[paths[0] + ":" + dom])
    df_ipf = roof.get("df64_instructions_per_flop")
    if roof["bound"] == "tensor":
        src = "MEASURED_PEAKS.json bf16_tflops_sustained"
    elif df_ipf:
        src = f"FP32 FMA-chain probe {fma32:.1f} TFLOP/s / (2 x {df_ipf:.2f} FP32 instr per flop, double-float)"
    else:
        src = f"{roof['pipe'].upper()} FMA-chain probe, this run"
    traffic = DRAM_BYTES_PER_LAUNCH.get(dom) if args.size == 1024 else None
    roof.update({"kernel": dom, "traffic": traffic, "peak_source": src})

    # ---- CPU oracle on a bounded sample of the same workload -----------------------------
    cpu, parity = None, {}
    if not args.no_cpu_baseline:
        r = oracle_sample(cam, freqs, CPU_SAMPLE_STRIDE)
        cpu = {"value": r["rays"] / r["seconds"], "unit": "rays/s", "cores": r["cores"], "kind": "oracle",
               "sample": f"{int(r['rays'])} rays: every {CPU_SAMPLE_STRIDE}th pixel per axis of the {args.size}^2 image",
               "steps_per_s": r["steps"] / r["seconds"]}
        # and on one core (a sparser sample of the same image)
        r1 = oracle_sample(cam, freqs, CPU_SAMPLE_STRIDE * 4, threads=1)
        cpu["single_thread"] = {"value": r1["rays"] / r1["seconds"], "steps_per_s": r1["steps"] / r1["seconds"],
                                "sample": f"{int(r1['rays'])} rays: every {CPU_SAMPLE_STRIDE * 4}th pixel per axis"}
        o = r["img"]
        h = CPU_SAMPLE_STRIDE // 2
        sl = (slice(None), slice(h, None, CPU_SAMPLE_STRIDE), slice(h, None, CPU_SAMPLE_STRIDE))
        big = np.abs(o) >= 1e-6 * np.abs(o).max()
        for pth, rr in res.items():
            g = rr["image"].cpu().numpy()[sl]
            den = np.maximum(np.abs(o), 1e-12 * np.abs(o).max())
            e = np.abs(g - o) / den
            parity[pth] = {"max_rel_err_sampled": float(e.max()), "max_rel_err_sampled_bright": float(e[big].max()),
                           "flux_rel_err_sampled": float(abs(g.sum() / o.sum() - 1))}

    dtype = {"mlp": "f32+f64+bf16", "mixed": "f32+f64", "fp64": "f64", "mlp_df": "f32+df64+bf16",
             "mixed_df": "f32+df64"}[paths[0]]
    detail = {
        "headline": {"workload": workload, "precision": paths[0], "ms_per_step": ms_step, "value": value,
                     "steps_per_ray": st["steps"] / (args.steps * npix),
                     "fp64_step_fraction": st["fp64_steps"] / max(st["steps"], 1),
                     "stats_per_render": {k: v / args.steps for k, v in st.items()},
                     "launch": main["tuned"], "wall_s_timed_region": main["wall"],
                     "fma_peaks_tflops": {"fp32": fma32, "fp64": fma64}},
        "kernels": {pth: {"profiled_ms_per_render": r["prof_ms"],
                          "kernel_ms_per_render": {k: v[0] / PROFILED_RENDERS for k, v in r["prof"].items() if v[1]},
                          "launches_per_render": {k: v[1] / PROFILED_RENDERS for k, v in r["prof"].items() if v[1]},
                          "timeline_last_render": _timeline_summary(r["timeline"])}
                    for pth, r in res.items()},
        "rooflines": roofs,
        "paths": {pth: {"ms_per_step": r["ms"], "rays_per_s": world * rays_step / (r["ms"] * 1e-3),
                        "geodesic_steps_per_s": world * (r["stats"]["steps"] / args.steps) / (r["ms"] * 1e-3),
                        "flux_jy": float(r["flux"][0])} for pth, r in res.items()},
        "cpu_baseline": cpu, "oracle_parity_sampled": parity,
        "surrogate": sur, "grid_workload": grid, "lightcurve_workload": lcurve, "thin_disk_workload": disk,
        "learned_thin_disk_workload": ldisk, "verlet_workload": verlet, "emissivity_options": emis,
    }
    if "fp64" in res:
        detail["flux_rel_err_vs_fp64"] = {pth: float(abs(r["flux"][0] / res["fp64"]["flux"][0] - 1))
                                          for pth, r in res.items() if pth != "fp64"}
    # the side workloads and the breakdown: one line each before the headline, and a file
    for name, obj in detail.items():
        if obj is not None:
            print(json.dumps({"bench_part": name, "data": obj}), flush=True)
    if args.detail_json:
        with open(args.detail_json, "w") as f:
            json.dump(detail, f, indent=1)

    line = {
        "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic (analytic plasma, deterministic)",
        "config": {"workload": workload, "precision": paths[0], "pixels": npix, "freqs_hz": freqs,
                   "parallelism": f"replicas x{world}", "l2": "flushed (256 MB write) before every timed render"},
        "geodesic_steps_per_s": steps_per_s,
        "roofline": {k: _round(roof.get(k)) for k in ("bound", "kernel", "pipe", "achieved", "peak", "unit", "frac",
                                                       "traffic", "peak_source")},
        "cpu_baseline": None if cpu is None else {k: _round(cpu[k]) for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": None if e2e is None else {k: _round(v) for k, v in e2e.items()},
        "gpu_launches": launches,
        "clocks": None if main["clocks"] is None else {k: main["clocks"][k] for k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "rays_per_s": {pth: _round(world * rays_step / (r["ms"] * 1e-3)) for pth, r in res.items()},
    }
    if roof.get("frac_of_fp64_native") is not None:
        line["roofline"]["frac_of_fp64_native"] = _round(roof["frac_of_fp64_native"])
    if dom in NCU_PIPES:
        line["roofline"]["counters"] = NCU_PIPES[dom]
    if "flux_rel_err_vs_fp64" in detail:
        line["flux_rel_err_vs_fp64"] = {k: _round(v) for k, v in detail["flux_rel_err_vs_fp64"].items()}
    if parity:
        line["oracle_max_rel_err_sampled"] = {k: _round(v["max_rel_err_sampled"]) for k, v in parity.items()}
    line["detail"] = "bench_part lines above" + (f"; {os.path.basename(args.detail_json)}" if args.detail_json else "")
    print(_final_line(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# keys of the headline line that may be dropped, in this order, to keep it under
# FINAL_LINE_MAX bytes (the rest is the contract and is always printed)
OPTIONAL_KEYS = ("oracle_max_rel_err_sampled", "rays_per_s", "detail", "flux_rel_err_vs_fp64")


def _final_line(line):
    """The headline JSON line, at most FINAL_LINE_MAX bytes: optional keys are dropped in
    the order of OPTIONAL_KEYS until it fits."""
    out = json.dumps(line)
    for k in OPTIONAL_KEYS:
        if len(out) <= FINAL_LINE_MAX:
            break
        line.pop(k, None)
        out = json.dumps(line)
    return out


def _band_mask(cam, width=0.5):
    """Pixel centres within `width` M of the critical curve (Bardeen's closed form, nearest
    vertex of a densely sampled curve)."""
    from scipy.spatial import cKDTree

    a, inc = cam["spin"], np.radians(cam["incl_deg"])
    rp = 2 * (1 + np.cos(2 / 3 * np.arccos(-abs(a))))
    rm = 2 * (1 + np.cos(2 / 3 * np.arccos(abs(a))))
    r = np.linspace(rp, rm, 20000)
    xi = -(r**3 - 3 * r**2 + a * a * r + a * a) / (a * (r - 1))
    eta = r**3 * (4 * a * a - r * (r - 3) ** 2) / (a * a * (r - 1) ** 2)
    b2 = eta + a * a * np.cos(inc) ** 2 - xi * xi / np.tan(inc) ** 2
    ok = b2 >= 0
    al_c, be_c = -xi[ok] / np.sin(inc), np.sqrt(b2[ok])
    curve = np.concatenate([np.stack([al_c, be_c], 1), np.stack([al_c, -be_c], 1)])
    al = cam["alpha_min"] + (np.arange(cam["nx"]) + 0.5) * (cam["alpha_max"] - cam["alpha_min"]) / cam["nx"]
    be = cam["beta_min"] + (np.arange(cam["ny"]) + 0.5) * (cam["beta_max"] - cam["beta_min"]) / cam["ny"]
    A, B = np.meshgrid(al, be)
    d, _ = cKDTree(curve).query(np.stack([A.ravel(), B.ravel()], 1))
    return (d < width).reshape(A.shape)


def _round(v, digits=5):
    """Round floats to `digits` significant digits (compact output)."""
    if isinstance(v, float) and np.isfinite(v) and v != 0.0:
        return float(f"{v:.{digits}g}")
    return v


def _timeline_summary(tl):
    """Per-launch timeline of the last profiled render: (kernel, stream lane, start ms, ms)."""
    if not tl:
        return []
    # launches of the last render: from the last launch that starts a render (the first
    # kernel of the first lane after the previous render's flux reduction)
    starts = [i for i, e in enumerate(tl) if i > 0 and tl[i - 1][0] == "reduce" and e[0] != "reduce"]
    first = starts[-1] if starts else 0
    t0 = tl[first][2]
    return [[e[0], e[1], round(e[2] - t0, 4), round(e[3], 4)] for e in tl[first:]]


def _rooflines(res, fma32, fma64, npix):
    """Per path and kernel: algorithmic flops (counted from the kernel source, FMA = 2) x the
    steps the kernel took (device counters) / its CUDA-event time, against the measured
    FMA-chain peak of the pipe it runs on (FP32, FP64, or the double-float rate derived from
    the FP32 one); the network against the sustained BF16 figure of MEASURED_PEAKS.json."""
    from paper_1801_10452_b300 import flopcount as _fc

    peaks = _peaks()
    fl = _flops_per_step()["fp64_step"]
    df_ipf = _fc.df64_instructions_per_step(1, "analytic")["instructions_per_flop"]
    pk_df = fma32 / (2.0 * df_ipf)
    roofs = {}
    for pth, r in res.items():
        prof, s = r["prof"], r["st_prof"]
        df = pth.endswith("_df")
        for kname, (kms, kn) in prof.items():
            if kn == 0 or kname in ("reduce", "trace", "load", "peak", "surrogate"):
                continue
            if kname == "surrogate_mlp":
                # the two 256 x 256 hidden layers on the tensor cores: 2 x 2 x 256^2 flops per ray
                per_ms = kms / PROFILED_RENDERS
                ach = 2.0 * 2 * 256 * 256 * npix / (per_ms * 1e-3) / 1e12
                pkb = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1400.0))
                roofs[pth + ":" + kname] = {"bound": "tensor", "pipe": "bf16 tcgen05", "achieved": ach, "peak": pkb,
                                            "unit": "TFLOP/s", "frac": ach / pkb, "kernel_ms_per_render": per_ms}
                continue
            entry = {"bound": "alu", "unit": "TFLOP/s"}
            if kname == "render_fp64":
                steps_k, pk, pipe = s["steps"], fma64, "fp64"
            elif kname in ("mixed_fp64", "mixed_fp64_long"):
                # mixed_fp64: the first stream's passes; mixed_fp64_long: the near-critical
                # rays' FP64 phase on the second stream
                n_long = s.get("fp64_steps_long", 0)
                steps_k = s["fp64_steps"] - n_long if kname == "mixed_fp64" else n_long
                pk, pipe = (pk_df, "fp32 (double-float)") if df else (fma64, "fp64")
                if df:
                    entry["df64_instructions_per_flop"] = df_ipf
            else:
                steps_k = s["fp32_steps_in"] if kname == "mixed_fp32_in" else s["fp32_steps_out"]
                pk, pipe = fma32, "fp32"
            ach = fl * steps_k / (kms * 1e-3) / 1e12
            entry.update({"pipe": pipe, "achieved": ach, "peak": pk, "frac": ach / pk,
                          "kernel_ms_per_launch": kms / kn, "launches_per_render": kn / PROFILED_RENDERS,
                          "steps_per_render": steps_k / PROFILED_RENDERS, "flops_per_step": fl})
            if pipe.startswith("fp32 (double"):
                entry["frac_of_fp64_native"] = ach / fma64
            roofs[pth + ":" + kname] = entry
    return roofs


def _dominant_kernel(prof, path, roofs):
    """The kernel with the most device time per render among those with a roofline; on the
    mixed path the second stream's FP64 launch overlaps the first stream's, and each counts
    with its own CUDA-event duration."""
    cand = {k: v[0] for k, v in prof.items() if v[1] and (path + ":" + k) in roofs}
    return max(cand, key=lambda k: cand[k])


def _flops_per_step():
    """Algorithmic flops of one geodesic step with its transfer sample (analytic plasma, one
    frequency), counted from the kernel source: see the flop-count table in the design notes."""
    from paper_1801_10452_b300 import flopcount

    return flopcount.flops_per_step(1, "analytic")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--size", type=int, default=1024, help="image side (profiling runs use a smaller case)")
    ap.add_argument("--paths", default="mlp_df,mlp,mixed_df,mixed,fp64",
                    help="comma list of paths to time (first = value): mlp, mixed, fp64, mlp_df, mixed_df")
    ap.add_argument("--no-grid", action="store_true", help="skip the grid (torus snapshot) workload")
    ap.add_argument("--no-lightcurve", action="store_true", help="skip the slow-light light-curve workload")
    ap.add_argument("--no-disk", action="store_true", help="skip the thin-disk line-emitter workload")
    ap.add_argument("--no-learned-disk", action="store_true", help="skip the crossing network and the learned thin disk")
    ap.add_argument("--no-verlet", action="store_true", help="skip the FP64 velocity-Verlet workload")
    ap.add_argument("--no-emissivity", action="store_true", help="skip the exact-K2 / Theta_e-mask comparison")
    ap.add_argument("--detail-json", default=None, help="also write the side workloads and breakdown to this file")
    ap.add_argument("--train-steps", type=int, default=16000)
    ap.add_argument("--train-rays", type=int, default=10_000_000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
