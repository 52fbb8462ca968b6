#!/usr/bin/env python3
"""Benchmark of the delivery-state renderer (one JSON line on stdout).

Default workload: batched forward + backward training step on 250,000
Gaussians (rank-2 temporal basis, 64 clusters x 4 layers), 64 delivery states
per step at 512x512 on 8 ring cameras: render every state, per-state FP64 MSE
against the teacher render of its view (loss = mean over states), adjoint
render to scene gradients.  A step runs the whole hot path: closure, masked
prefix decode, Eq. 1 deformation, EWA projection, binning, the two radix
sorts, tile ranges, compositing, MSE, backward compositing, backward
projection.

``--impl reference`` times the FP64 CPU oracle on the same workload (bounded
pixel sample per step, extrapolated to states/s).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "delivery-state renders/s and Mpix/s, batched fwd+bwd vs plain per-state, ≤1e-4 err"
UNIT = "states/s"
# Roofline of the raster kernels as the measurement plan defines it: every
# (pixel, Gaussian, state) evaluation the oracle counts costs 17 FP32
# operations and one MUFU exp, forward and adjoint alike.  The FP32 peak counts
# an FMA as two operations (148 SMs x 128 lanes x 2 x clock), so the FP32
# fraction is a lower bound; the MUFU peak is the measured ex2.approx rate of
# this GPU (32 per SM per clock).
FP32_OPS_PER_EVAL = 17
MUFU_OPS_PER_EVAL = 1
MUFU_EX2_PER_SM_CLK = 32
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum, one pass); valid only for the
# kernel source it was taken on (sha1 of csrc/raster.cu), the workload at full size
# and the sort tile side in pixels.
MEASURED_TRAFFIC = {
    ("raster_bwd", "c3_fwdbwd_250k", 32): (805_345_280 + 78_024_448, "743ee6f557420f32b4f7d1e189fac67d23338d5e"),
    ("raster_fwd", "c3_fwdbwd_250k", 32): (441_935_360 + 183_101_184, "743ee6f557420f32b4f7d1e189fac67d23338d5e"),
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def rank_states(w, rank):
    """Weak scaling: rank r renders its own batch of delivery states (rank 0
    keeps the workload's masks, others draw prefix masks with seed 10000 + r)."""
    from paper_2606_17212_b300 import synth
    if rank == 0:
        return w.states.masks
    rng = np.random.default_rng(10_000 + rank)
    d = synth.prefix_states(w.states.n, w.scene.n_clusters, w.scene.n_layers, rng)
    return synth._pack(synth.depths_to_bits(d, w.scene.n_layers))


def max_over_ranks(x, device=None):
    """Max of a float over the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def flat_gradients(grads, device=None):
    """Place every scene-gradient tensor in one flat buffer (each slice 16-byte
    aligned) so that data-parallel ranks can sum them with one all-reduce.
    Returns (views keyed as grads, flat buffer)."""
    import torch
    sizes = {k: v.numel() for k, v in grads.items()}
    pad = lambda n: (n + 3) // 4 * 4
    flat = torch.zeros(sum(pad(n) for n in sizes.values()), dtype=torch.float32,
                       device=device if device is not None else next(iter(grads.values())).device)
    views, off = {}, 0
    for k, v in grads.items():
        views[k] = flat[off:off + sizes[k]].view(v.shape)
        off += pad(sizes[k])
    return views, flat


def reduce_gradients(flat):
    """Data-parallel training step: each rank's scene gradient covers its own
    states; their sum over the process group is the gradient of the loss over
    all ranks' states (one all-reduce; identity without a group)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}, "fallback"


def raster_roofline(name, evals, ms_per_launch, sms, sm_mhz, traffic=None):
    """Roofline entry of a raster kernel under the measurement plan's count:
    17 FP32 operations and one MUFU exp per oracle-counted (pixel, Gaussian,
    state) evaluation, against the FP32 FMA peak (an FMA counted as two, so
    the fraction is a lower bound) and the measured ex2 rate."""
    t = ms_per_launch / 1e3
    fp32_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    mufu_peak = sms * MUFU_EX2_PER_SM_CLK * sm_mhz * 1e6 / 1e12
    achieved = FP32_OPS_PER_EVAL * evals / t / 1e12
    mufu = MUFU_OPS_PER_EVAL * evals / t / 1e12
    return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak, "traffic": traffic, "traffic_unit": "bytes per launch (ncu)",
            "peak_kind": "FP32 FMA peak from unit counts and clock: %d SMs x 128 lanes x 2 x %.0f MHz (derived)"
                         % (sms, sm_mhz),
            "per_eval": "%d FP32 ops + %d MUFU exp per oracle-counted (pixel, Gaussian, state) evaluation"
                        % (FP32_OPS_PER_EVAL, MUFU_OPS_PER_EVAL),
            "mufu": {"achieved": mufu, "peak": mufu_peak, "unit": "T ex2/s", "frac": mufu / mufu_peak,
                     "peak_kind": "measured ex2.approx rate: %d per SM per clock" % MUFU_EX2_PER_SM_CLK},
            "ms_per_launch": ms_per_launch, "evals_per_launch": evals}


def hbm_entry(name, nbytes, ms, peak_gbs, what):
    """Achieved algorithmic bandwidth of an HBM-bound kernel (group) against the measured copy peak."""
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": gbs, "peak": peak_gbs, "unit": "GB/s",
            "frac": gbs / peak_gbs, "bytes_per_step": nbytes, "ms_per_step": ms, "bytes": what}


def scene_bytes(sc):
    """Bytes of a scene's attributes: base (mean, temporal coefficients, log-scale,
    quaternion, opacity logit, colour) and every refinement layer."""
    nc = sc.colour.shape[1]
    per = 4 * (3 + 3 * sc.temporal_rank + 3 + 4 + 1 + nc) + 4 * (sc.n_layers - 1) * (11 + nc)
    return per * sc.n


class ClockSampler:
    """SM clock and throttle-reason sampling (read-only NVML queries) every
    20 ms on a background thread during the timed region."""

    REASONS = {"hw_slowdown": ("nvmlClocksEventReasonHwSlowdown", 0x8),
               "hw_thermal_slowdown": ("nvmlClocksEventReasonHwThermalSlowdown", 0x40),
               "sw_thermal_slowdown": ("nvmlClocksEventReasonSwThermalSlowdown", 0x20),
               "sw_power_cap": ("nvmlClocksEventReasonSwPowerCap", 0x4)}

    def __init__(self, index=0):
        import threading
        self.samples, self.max_mhz, self.reasons = [], None, set()
        self.stop_flag = False
        try:
            import pynvml
            pynvml.nvmlInit()
            self.nv = pynvml
            self.h = pynvml.nvmlDeviceGetHandleByIndex(index)
            self.max_mhz = pynvml.nvmlDeviceGetMaxClockInfo(self.h, pynvml.NVML_CLOCK_SM)
        except Exception as e:   # no NVML binding: poll nvidia-smi instead
            self.nv, self.err = None, str(e)
            self.index = index
            self.th = threading.Thread(target=self._run_smi, daemon=True)
            self.th.start()
            return
        self.th = threading.Thread(target=self._run, daemon=True)
        self.th.start()

    def _run_smi(self):
        import subprocess
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        while not self.stop_flag:
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip().split(",")
                self.samples.append(float(out[0]))
                self.max_mhz = float(out[1])
                for nm, v in zip(names, out[2:6]):
                    if v.strip().lower() == "active":
                        self.reasons.add(nm)
            except Exception:
                pass
            time.sleep(0.02)

    def _run(self):
        nv = self.nv
        while not self.stop_flag:
            try:
                self.samples.append(nv.nvmlDeviceGetClockInfo(self.h, nv.NVML_CLOCK_SM))
                r = nv.nvmlDeviceGetCurrentClocksEventReasons(self.h)
                for name, (const, default) in self.REASONS.items():
                    if r & getattr(nv, const, default):
                        self.reasons.add(name)
            except Exception:
                pass
            time.sleep(0.02)

    def stop(self):
        self.stop_flag = True
        self.th.join(timeout=10)
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(self.reasons), "samples": len(self.samples)}


def oracle_sample(w, states, n_bands=16, band_rows=2, n_pix=1024, seed=0, want_backward=True):
    """Time the FP64 oracle as it stands on a bounded sample of the given
    states (one protocol for the CPU baseline and the reference arm).
    Forward: the projection (once per state) plus n_bands bands of band_rows
    whole rows at random heights, rendered as in the full image (row filter),
    extrapolated to all rows.  Adjoint: its fixed part (projection and the
    per-record chain rule, timed with dL/dI = 0) plus the adjoint of n_pix
    random pixels, extrapolated to all pixels.  Returns a dict: seconds per
    full state (extrapolated), the measured seconds of the sampled work, the
    extrapolation factor, evaluations per pixel, threads and a description."""
    import oracle
    sc = w.scene
    rng = np.random.default_rng(seed)
    D = oracle.state_depths(w.states, sc.n_clusters, sc.n_layers)
    H, W = w.cams[0].height, w.cams[0].width
    tot_t, tot_meas, tot_eval, tot_px = 0.0, 0.0, 0, 0
    rows = min(band_rows, H)
    for s in states:
        cam = w.cams[int(w.states.cam[s])]
        t = float(w.states.t[s])
        t0 = time.perf_counter()
        oracle.project(sc, D[s], t, cam)
        t_proj = time.perf_counter() - t0
        t_rows, n_rows, meas = 0.0, 0, t_proj
        for y0 in rng.integers(0, H - rows + 1, size=n_bands):
            t0 = time.perf_counter()
            _, _, ne = oracle.render_rows(sc, D[s], t, cam, w.bg, int(y0), int(y0) + rows)
            dt = time.perf_counter() - t0
            meas += dt
            t_rows += max(dt - t_proj, 0.0)
            n_rows += rows
            tot_eval += ne
            tot_px += rows * W
        fwd = t_proj + t_rows * H / n_rows
        bwd = 0.0
        if want_backward:
            dL = np.zeros((H, W, 3))
            t0 = time.perf_counter()
            oracle.render_backward(sc, D[s], t, cam, w.bg, dL)
            t_fix = time.perf_counter() - t0
            flat = rng.choice(H * W, size=min(n_pix, H * W), replace=False)
            dL[flat // W, flat % W] = rng.normal(size=(flat.size, 3))
            t0 = time.perf_counter()
            oracle.render_backward(sc, D[s], t, cam, w.bg, dL)
            dt = time.perf_counter() - t0
            meas += t_fix + dt
            bwd = t_fix + max(dt - t_fix, 0.0) * (H * W) / flat.size
        tot_t += fwd + bwd
        tot_meas += meas
    threads = os.cpu_count() or 1
    n = max(len(states), 1)
    desc = ("%d state(s), each: projection once + %d bands of %d whole rows (FP64 forward on %d threads, row "
            "filter as in the full image) extrapolated to %d rows%s" % (
                len(states), n_bands, rows, threads, H,
                "; adjoint (1 thread): fixed part once + %d random pixels extrapolated to %dx%d" % (n_pix, W, H)
                if want_backward else ""))
    return {"sec_per_state": tot_t / n, "sampled_s": tot_meas, "extrapolation": tot_t / max(tot_meas, 1e-12),
            "evals_per_px": tot_eval / max(tot_px, 1), "threads": threads, "desc": desc}


def t_interval(samples):
    """Student-t 95% confidence interval of the mean of per-step times (ms),
    with the sample count; None for fewer than two samples."""
    x = np.asarray(samples, np.float64)
    if x.size < 2:
        return None
    from scipy import stats
    h = float(stats.t.ppf(0.975, x.size - 1) * x.std(ddof=1) / np.sqrt(x.size))
    return {"lo": float(x.mean() - h), "hi": float(x.mean() + h), "n": int(x.size),
            "what": "rank-local per-step device times of the headline path"}


def workload_config(w, ws, views, path):
    return {"workload": w.name, "gaussians": w.scene.n, "clusters": w.scene.n_clusters,
            "layers": w.scene.n_layers, "temporal_rank": w.scene.temporal_rank,
            "states_per_step": w.states.n, "resolution": [w.cams[0].width, w.cams[0].height],
            "cameras": len(w.cams), "view_groups": len(views),
            "l2": "flushed between timed steps (256 MB write)", "parallelism": "dp%d" % ws, "path": path}


def reference_arm(args, w):
    """The FP64 oracle on the host cores, the same sampling protocol as the
    CPU baseline of the GPU arm: each step samples one state (16 bands of 2
    rows forward, 1,024 adjoint pixels) and extrapolates it to whole states.
    ms_per_step is the measured time of the sampled work; value is the
    extrapolated states/s."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    views = sorted(set(zip(w.states.cam.tolist(), w.states.t.tolist())))
    cfg = workload_config(w, ws, views, "fp64_oracle_cpu")
    sec_states, sampled = [], []
    last = None
    for k in range(args.warmup + args.steps):
        r = oracle_sample(w, [k % w.states.n], seed=k, want_backward=w.target_scene is not None)
        if k >= args.warmup:
            sec_states.append(r["sec_per_state"])
            sampled.append(r["sampled_s"])
        last = r
    sec_per_state = float(np.mean(sec_states))
    value = 1.0 / sec_per_state
    meas_ms = float(np.mean(sampled)) * 1e3
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": meas_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference", "config": cfg,
            "extrapolated": True,
            "extrapolation_factor": sec_per_state * 1e3 / meas_ms,
            "step_what": "one sampled state per step; ms_per_step is the measured time of that sample, value the "
                         "states/s it extrapolates to",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": last["threads"], "kind": "oracle",
                             "sample": "per step: " + last["desc"], "extrapolated": True},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_mix(args):
    """Serving-shaped uneven mix: 48 scenes (SH degree 3, 50k-2.7M Gaussians,
    256^2 / 512^2 / 960x540), 64 states each; one step = the training step
    (render, MSE against the scene's complete render at the state's view,
    adjoint) of every scene.  Headline = the faster of the context calls and
    one CUDA graph holding every scene's plan (plans share one arena)."""
    import torch
    from paper_2606_17212_b300 import dgs, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    R = dgs.Renderer(0)
    R.set_tile_size(args.tile_size)
    specs = synth.mix_specs(scale=args.scale)
    scenes = []
    t_gen = time.perf_counter()
    evals_total = 0.0
    oracle_sec = 0.0
    oracle_meas = 0.0
    threads = None
    for spec in specs:
        w = synth.mix_workload(spec)
        sc = dgs.DeviceScene.from_host(w.scene, device=dev)
        st = dgs.DeviceStates.from_host(w.states)
        views = sorted(set(zip(w.states.cam.tolist(), w.states.t.tolist())))
        ridx = np.array([views.index(v) for v in zip(w.states.cam.tolist(), w.states.t.tolist())], np.int32)
        full = torch.full((len(views), st.masks.shape[1]), -1, dtype=torch.int32, device=dev)
        fv = dgs.DeviceStates(full, np.array([v[1] for v in views], np.float32),
                              np.array([v[0] for v in views], np.int32))
        targets = R.render_states_batched(sc, fv, w.cams, w.bg)
        S, H, W = st.n, w.cams[0].height, w.cams[0].width
        # oracle on a bounded sample of this scene: evaluations per pixel and CPU time per state
        if not args.no_oracle_sample:
            r = oracle_sample(w, [0], n_bands=4, n_pix=64, seed=spec.index, want_backward=True)
            evals_total += r["evals_per_px"] * H * W * S
            oracle_sec += r["sec_per_state"] * S
            oracle_meas += r["sampled_s"]
            threads = r["threads"]
        scenes.append(dict(spec=spec, w_t=w.states.t, w_cam=w.states.cam, cams=w.cams, bg=w.bg, sc=sc, st=st,
                           ridx=ridx, targets=targets, S=S, H=H, W=W,
                           host_masks=torch.from_numpy(np.ascontiguousarray(w.states.masks).view(np.int32)).pin_memory(),
                           images=torch.empty((S, H, W, 3), device=dev), grads=sc.zeros_like_grads()))
        del w
    t_gen = time.perf_counter() - t_gen
    total_states = sum(c["S"] for c in scenes)
    total_px = sum(c["S"] * c["H"] * c["W"] for c in scenes)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def eager_step():
        out = []
        for c in scenes:
            R.render_states_batched(c["sc"], c["st"], c["cams"], c["bg"], out=c["images"])
            mse, _, dL = R.image_mse(c["images"], c["targets"], c["ridx"], weight=1.0 / c["S"], want_grad=True)
            for g in c["grads"].values():
                g.zero_()
            R.render_backward(c["sc"], c["st"], c["cams"], c["bg"], dL, c["grads"], images=c["images"])
            out.append(mse)
        return out

    def timed(fn, K):
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        torch.cuda.synchronize()
        for k in range(K):
            flush.fill_(float(k))
            starts[k].record()
            fn()
            ends[k].record()
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / K

    for _ in range(args.warmup):
        eager_step()
    clocks = ClockSampler(0)
    R.reset_kernel_launches()
    R.profile(True)
    eager_ms = timed(eager_step, args.steps)
    eager_launches = R.kernel_launches()
    prof = R.profile_read()
    R.profile(False)

    # scene waves: dgs_render_scenes_batched / dgs_render_scenes_backward over
    # groups of scenes, one forward and one adjoint raster launch per group (a
    # renderer of its own: its per-scene workspaces are freed before the plans)
    R2 = dgs.Renderer(0)
    R2.set_tile_size(args.tile_size if args.tile_size else 32)
    wave = max(1, args.mix_wave)
    waves = [scenes[k:k + wave] for k in range(0, len(scenes), wave)]

    def waves_step():
        out = []
        for grp in waves:
            jobs = [(c["sc"], c["st"], c["cams"], c["bg"], c["images"]) for c in grp]
            R2.render_scenes_batched(jobs)
            dls = []
            for c in grp:
                mse, _, dL = R2.image_mse(c["images"], c["targets"], c["ridx"], weight=1.0 / c["S"], want_grad=True)
                for g in c["grads"].values():
                    g.zero_()
                out.append(mse)
                dls.append(dL)
            R2.render_scenes_backward(jobs, dls, [c["grads"] for c in grp])
        return out

    waves_ms = None
    waves_launches = 0
    waves_prof = {}
    try:
        for _ in range(args.warmup):
            waves_step()
        R2.reset_kernel_launches()
        R2.profile(True)
        waves_ms = timed(waves_step, args.steps)
        waves_launches = R2.kernel_launches()
        waves_prof = R2.profile_read()
        R2.profile(False)
        waves_err = None
    except RuntimeError as e:            # e.g. a group's workspaces do not fit
        waves_err = str(e).splitlines()[0]
    R2.close()
    torch.cuda.empty_cache()

    # graph: one plan per scene in a shared arena, the whole step captured once
    arena = dgs.Arena(R)
    for c in scenes:
        c["plan"] = dgs.Plan(R, c["sc"], c["st"], c["cams"], c["bg"], dgs.PLAN_RENDER, ref_index=c["ridx"],
                             n_refs=int(c["targets"].shape[0]), entry_headroom=args.entry_headroom, arena=arena)
        c["g_masks"] = c["st"].masks.clone()
        c["g_mse"] = torch.empty(c["S"], dtype=torch.float64, device=dev)
        c["g_psnr"] = torch.empty_like(c["g_mse"])
        c["g_dL"] = torch.empty_like(c["images"])

    def plan_step():
        for c in scenes:
            for g in c["grads"].values():
                g.zero_()
            c["plan"].render(c["g_masks"], c["images"])
            c["plan"].image_mse(c["images"], c["targets"], c["g_mse"], c["g_psnr"], c["g_dL"], weight=1.0 / c["S"])
            c["plan"].backward(c["g_dL"], c["grads"], images=c["images"])

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan_step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    R.reset_kernel_launches()
    with torch.cuda.graph(graph):
        plan_step()
    launches_per_step = R.kernel_launches()
    for _ in range(args.warmup):
        graph.replay()
    graph_ms = timed(graph.replay, args.steps)
    for c in scenes:
        c["plan"].status()
    clk = clocks.stop()
    use_graph = graph_ms < eager_ms
    ms = graph_ms if use_graph else eager_ms
    value = total_states / (ms / 1e3)
    use_waves = waves_ms is not None and waves_ms < ms
    if use_waves:              # the headline path; the end-to-end run below uses it too
        ms = waves_ms
        value = total_states / (ms / 1e3)
        graph = None           # the plans' memory goes back before the scene workspaces return
        for c in scenes:
            c.pop("plan").close()
        arena.close()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        R2 = dgs.Renderer(0)
        R2.set_tile_size(args.tile_size if args.tile_size else 32)

    # end to end: every scene's masks H2D from pinned memory, every MSE D2H, per step
    res_host = [torch.empty(c["S"], dtype=torch.float64).pin_memory() for c in scenes]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if use_waves:
        waves_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
    for _ in range(args.steps):
        if use_waves:
            for c in scenes:
                c["st"].masks.copy_(c["host_masks"], non_blocking=True)
            for m, rh in zip(waves_step(), res_host):
                rh.copy_(m, non_blocking=True)
        elif use_graph:
            for c in scenes:
                c["g_masks"].copy_(c["host_masks"], non_blocking=True)
            graph.replay()
            for c, rh in zip(scenes, res_host):
                rh.copy_(c["g_mse"], non_blocking=True)
        else:
            for c in scenes:
                c["st"].masks.copy_(c["host_masks"], non_blocking=True)
            for m, rh in zip(eager_step(), res_host):
                rh.copy_(m, non_blocking=True)
        torch.cuda.synchronize()
    e2e_value = total_states / ((time.perf_counter() - t0) / args.steps)
    h2d = sum(c["host_masks"].numel() * 4 + c["w_t"].nbytes + c["w_cam"].nbytes for c in scenes)
    d2h = total_states * 8

    pk, pk_kind = _peaks()
    sm_mhz = pk.get("sm_max_mhz", 2032.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roof = None
    if "raster_bwd" in prof and evals_total > 0:
        bms, bn = prof["raster_bwd"]
        # every scene's backward launch of a step together: evaluations per step / time per step
        roof = raster_roofline("raster_bwd", evals_total, bms / args.steps, sms, sm_mhz)
        roof["launches_per_step"] = bn / args.steps
        roof["what"] = "all scenes' backward launches of one step together"
    cpu = None if (args.no_cpu_baseline or oracle_sec == 0) else {
        "value": total_states / oracle_sec, "unit": UNIT, "cores": threads, "kind": "oracle",
        "sampled_s": oracle_meas, "extrapolated": True, "extrapolation_factor": oracle_sec / max(oracle_meas, 1e-12),
        "sample": "per scene, 1 state: projection + 4 bands of 2 whole rows (FP64 forward on %s threads), "
                  "adjoint fixed part + 64 random pixels (1 thread), extrapolated to the scene's 64 states"
                  % threads}
    sizes = [c["spec"].n for c in scenes]
    cfg = {"workload": "c5_mix_48", "scenes": len(scenes), "gaussians_total": int(sum(sizes)),
           "gaussians_min": int(min(sizes)), "gaussians_max": int(max(sizes)), "sh_degree": 3,
           "states_per_step": total_states, "states_per_scene": 64,
           "resolutions": sorted({"%dx%d" % (c["W"], c["H"]) for c in scenes}),
           "pixels_per_step": int(total_px), "l2": "flushed between timed steps (256 MB write)",
           "parallelism": "dp1",
           "path": "scene_waves" if use_waves else ("cuda_graph_arena_plans" if use_graph else "context_calls"),
           "generation_s": round(t_gen, 1)}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "mpix_per_s": total_px / (ms / 1e3) / 1e6,
            "eager_per_step": {"ms": eager_ms, "value": total_states / (eager_ms / 1e3), "unit": UNIT,
                               "what": "context calls, scene after scene"},
            "scene_waves_per_step": ({"ms": waves_ms, "value": total_states / (waves_ms / 1e3), "unit": UNIT,
                                      "what": "dgs_render_scenes_batched / dgs_render_scenes_backward over groups of "
                                              "%d scenes: one forward and one adjoint raster launch per group" % wave,
                                      "kernels_ms_per_step": {k: v[0] / args.steps for k, v in waves_prof.items()}}
                                     if waves_ms is not None else {"error": waves_err}),
            "graph_per_step": {"ms": graph_ms, "value": total_states / (graph_ms / 1e3), "unit": UNIT,
                               "what": "one CUDA graph of every scene's plan (one arena)"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": waves_launches if use_waves else
                            ((launches_per_step * args.steps) if use_graph else eager_launches),
            "clocks": clk, "roofline": roof, "cpu_baseline": cpu,
            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()}, "peaks": pk_kind}
    for c in scenes:
        if "plan" in c:
            c["plan"].close()
    if not use_waves:
        arena.close()
    else:
        R2.close()
    R.close()
    return line


def run_groups(args):
    """Utility table of the 2.7M-Gaussian sweep scene (Eq. 3 / Eq. 4): every
    completion group (64 clusters x 4 layers = 256 packets) over 64 sampled
    valid contexts, i.e. 2 x 256 x 64 = 32,768 rendered states per step (the
    state count of the paper's utility experiment), 480x270, one view."""
    import torch
    from paper_2606_17212_b300 import dgs, synth
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    w = synth.config("c4_utility_2p7m", scale=args.scale, n_states=1)
    sc_h = w.scene
    groups = np.array([(c, l) for c in range(sc_h.n_clusters) for l in range(sc_h.n_layers)], np.int32)
    M = 64
    ctx = synth.group_contexts(groups, M, sc_h.n_clusters, sc_h.n_layers, np.random.default_rng(2104))
    G = len(groups)
    states = synth.States(ctx, np.full(G * M, 0.25, np.float32), np.zeros(G * M, np.int32))
    R = dgs.Renderer(0)
    R.set_tile_size(args.tile_size)
    scene = dgs.DeviceScene.from_host(sc_h, device=dev)
    dst = dgs.DeviceStates.from_host(states)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        R.group_utility(scene, dst, groups, M, w.cams, w.bg)
    clocks = ClockSampler(0)
    R.reset_kernel_launches()
    R.profile(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record()
        R.group_utility(scene, dst, groups, M, w.cams, w.bg)
        ends[k].record()
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / args.steps
    launches = R.kernel_launches()
    prof = R.profile_read()
    R.profile(False)
    clk = clocks.stop()
    n_states = 2 * G * M
    # end to end: contexts H2D from pinned memory, the utility table D2H
    host = torch.from_numpy(np.ascontiguousarray(ctx).view(np.int32)).pin_memory()
    out = torch.empty((G, 4), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        dst.masks.copy_(host, non_blocking=True)
        _, st = R.group_utility(scene, dst, groups, M, w.cams, w.bg)
        out.copy_(st, non_blocking=True)
        torch.cuda.synchronize()
    e2e = n_states / ((time.perf_counter() - t0) / args.steps)
    H, W = w.cams[0].height, w.cams[0].width
    line = {"metric": METRIC, "value": n_states / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c4_group_utility", "gaussians": sc_h.n, "groups": G, "contexts_per_group": M,
                       "states_per_step": n_states, "resolution": [W, H], "alpha": 0.25, "beta": 0.05, "q": 0.10,
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": "dp1"},
            "groups_per_s": G / (ms / 1e3), "mpix_per_s": n_states * H * W / (ms / 1e3) / 1e6,
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": host.numel() * 4 + states.t.nbytes +
                    states.cam.nbytes, "d2h_bytes_per_step": G * 32},
            "gpu_launches": launches, "clocks": clk,
            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()}}
    R.close()
    return line


def run_main(args, w):
    """The training step (or the distortion pass of a utility workload): eager
    context calls and, for training, one replayed CUDA graph of a capture-safe
    plan; the faster is the headline.  Returns the JSON line (rank 0) or None."""
    ws, rank, local = _dist()
    import torch
    from paper_2606_17212_b300 import dgs
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # weak scaling: every rank renders its own batch of states (different mask seed)
    w.states.masks = rank_states(w, rank)

    R = dgs.Renderer(local)
    R.set_tile_size(args.tile_size)
    scene = dgs.DeviceScene.from_host(w.scene, device=dev)
    states = dgs.DeviceStates.from_host(w.states)
    S = states.n
    H, W = w.cams[0].height, w.cams[0].width
    training = w.target_scene is not None

    # targets: complete render of the teacher scene at every (camera, time) a state uses
    views = sorted(set(zip(w.states.cam.tolist(), w.states.t.tolist())))
    ref_index = np.array([views.index((c, t)) for c, t in zip(w.states.cam.tolist(), w.states.t.tolist())],
                         np.int32)
    if training:
        teacher = dgs.DeviceScene.from_host(w.target_scene, device=dev)
        full = torch.full((len(views), states.masks.shape[1]), -1, dtype=torch.int32, device=dev)
        tv = dgs.DeviceStates(full, np.array([v[1] for v in views], np.float32),
                              np.array([v[0] for v in views], np.int32))
        targets = R.render_states_batched(teacher, tv, w.cams, w.bg)
        del teacher
    images = torch.empty((S, H, W, 3), dtype=torch.float32, device=dev)
    grads, grad_flat = flat_gradients(scene.zeros_like_grads(), device=dev)
    loss_w = 1.0 / (S * ws)           # mean over the states of every rank
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > 126 MB L2

    def step(st):
        if training:
            R.render_states_batched(scene, st, w.cams, w.bg, out=images)
            if args.loss == "eq2":
                mse, _, dL = R.objective(images, targets, ref_index)
            else:
                mse, _, dL = R.image_mse(images, targets, ref_index, weight=loss_w, want_grad=True)
            grad_flat.zero_()
            R.render_backward(scene, st, w.cams, w.bg, dL, grads, images=images)
            reduce_gradients(grad_flat)
            return mse
        mse, _ = R.state_utility(scene, st, w.cams, w.bg)
        return mse

    for _ in range(args.warmup):
        step(states)
    torch.cuda.synchronize()

    def timed(run_one, K):
        """Device time of K calls of run_one on the current stream, L2 flushed
        (256 MB write) between calls outside the timed events; max over ranks."""
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for k in range(K):
            flush.fill_(float(k))
            starts[k].record()
            run_one()
            ends[k].record()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        per = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        step_ms[0] = per
        total = max_over_ranks(sum(per), device=dev)
        return total / K

    step_ms = [None]

    clocks = ClockSampler(local)
    # ---- eager path through the context calls; the library's event profiler
    # times every kernel on its launching stream
    R.reset_kernel_launches()
    R.profile(True)
    eager_ms = timed(lambda: step(states), args.steps)
    eager_steps = step_ms[0]
    eager_launches = R.kernel_launches()
    reuse = R.tile_reuse_stats() if not training else None     # the timed steps' distortion pass
    prof = R.profile_read()
    R.profile(False)
    eager_tile = R.last_tile_size()
    graph_tile = None

    # ---- graph path (training): a capture-safe plan, the whole step captured
    # once in a CUDA graph and replayed (masks live in a static device buffer)
    graph_ms = None
    if training:
        plan = dgs.Plan(R, scene, states, w.cams, w.bg, dgs.PLAN_RENDER, ref_index=ref_index,
                        n_refs=len(views), entry_headroom=args.entry_headroom)
        graph_tile = plan.tile_size()
        g_masks = states.masks.clone()
        g_mse = torch.empty(S, dtype=torch.float64, device=dev)
        g_psnr = torch.empty_like(g_mse)
        g_dL = torch.empty_like(images)
        if args.loss == "eq2":
            plan.set_objective()
            g_loss = torch.empty(1, dtype=torch.float64, device=dev)

        def plan_step():
            grad_flat.zero_()
            plan.render(g_masks, images)
            if args.loss == "eq2":
                plan.objective(images, targets, g_loss, g_mse, g_dL)
            else:
                plan.image_mse(images, targets, g_mse, g_psnr, g_dL, weight=loss_w)
            plan.backward(g_dL, grads, images=images)

        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(2):
                plan_step()
        torch.cuda.current_stream().wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        R.reset_kernel_launches()
        with torch.cuda.graph(graph):
            plan_step()
        launches_per_step = R.kernel_launches()

        def graph_step():
            graph.replay()
            reduce_gradients(grad_flat)     # outside the graph: NCCL between ranks

        for _ in range(args.warmup):
            graph_step()
        graph_ms = timed(graph_step, args.steps)
        graph_steps = step_ms[0]
        plan.status()
        launches = launches_per_step * args.steps
    else:
        launches = eager_launches
    clk = clocks.stop()
    # headline = the faster public path (both are reported)
    use_graph = graph_ms is not None and graph_ms < eager_ms
    ms_per_step = graph_ms if use_graph else eager_ms
    ci95 = t_interval(graph_steps if use_graph else eager_steps)
    value = ws * S / (ms_per_step / 1e3)
    if training and not use_graph:
        launches = eager_launches

    # ---- end to end through the public API: masks H2D from pinned memory, loss D2H
    host_masks = torch.from_numpy(np.ascontiguousarray(w.states.masks).view(np.int32)).pin_memory()
    res_host = torch.empty(S, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        if use_graph:
            g_masks.copy_(host_masks, non_blocking=True)
            graph_step()
            res_host.copy_(g_mse, non_blocking=True)
        else:
            dev_masks = states.masks
            dev_masks.copy_(host_masks, non_blocking=True)
            mse = step(states)
            res_host.copy_(mse, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_value = ws * S / e2e_s
    h2d = host_masks.numel() * 4 + w.states.t.nbytes + w.states.cam.nbytes
    d2h = S * 8

    # ---- plain per-state path (one state per launch sequence, synchronized)
    plain = None
    plain_rounds = []
    if not args.no_plain and rank == 0:
        n_plain = S if training else min(S, 256)     # distortion workloads: a bounded sample of states

        def plain_state(s):
            # one state per call sequence, with the same arguments for forward and
            # backward so the backward reuses the forward's projection and lists
            m = states.masks[s:s + 1]
            cam = w.cams[int(w.states.cam[s])]
            st1 = dgs.DeviceStates(m, w.states.t[s:s + 1], np.zeros(1, np.int32))
            if training:
                R.render_state(scene, m[0], float(w.states.t[s]), cam, w.bg, out=images[s])
                _, _, dL = R.image_mse(images[s:s + 1], targets, ref_index[s:s + 1], weight=1.0 / S,
                                       want_grad=True)
                R.render_backward(scene, st1, [cam], w.bg, dL, grads, images=images[s:s + 1])
            else:
                R.state_utility(scene, st1, [cam], w.bg)
            torch.cuda.synchronize()

        for s in range(3):
            plain_state(s)
        plain_rounds = []          # three rounds over the states; their median is reported
        for _ in range(3):
            t0 = time.perf_counter()
            for s in range(n_plain):
                plain_state(s)
            plain_rounds.append(n_plain / (time.perf_counter() - t0))
        plain = float(np.median(plain_rounds))

    # ---- roofline of the dominant kernel, from the live events
    pk, pk_kind = _peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][0]) if prof else ("none", (0.0, 1))
    dom_name, (dom_ms, dom_n) = dom
    dom_ms_per_launch = dom_ms / max(dom_n, 1)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = pk.get("sm_max_mhz", 2032.0)
    cpu = None
    roof = None
    kernels_roof = None
    if rank == 0 and not args.no_oracle_sample:
        samp = oracle_sample(w, list(range(2 if training else 4)), want_backward=training)
        if not args.no_cpu_baseline:
            cpu = {"value": 1.0 / samp["sec_per_state"], "unit": UNIT, "cores": samp["threads"], "kind": "oracle",
                   "sample": samp["desc"], "sampled_s": samp["sampled_s"], "extrapolated": True,
                   "extrapolation_factor": samp["extrapolation"]}
        evals_per_state = samp["evals_per_px"] * H * W
        reuse_frac = 1.0
        if not training:
            # tile reuse: only the rendered (state, tile) pairs are raster work
            pairs, rendered, _ = reuse
            reuse_frac = rendered / max(pairs, 1)

        def raster_entry(name):
            ms_k, n_k = prof[name]
            per_launch = evals_per_state * S * reuse_frac / max(n_k / max(args.steps, 1), 1.0)
            traffic = None
            rec = MEASURED_TRAFFIC.get((name, w.name, eager_tile))
            if rec is not None and args.scale == 1.0 and args.states is None:
                import hashlib
                src = os.path.join(ROOT, "paper_2606_17212_b300", "csrc", "raster.cu")
                if hashlib.sha1(open(src, "rb").read()).hexdigest() == rec[1]:
                    traffic = rec[0]
            return raster_roofline(name, per_launch, ms_k / max(n_k, 1), sms, sm_mhz, traffic)

        if dom_name.startswith("raster"):
            roof = raster_entry(dom_name)
        kernels_roof = [raster_entry(k) for k in ("raster_fwd", "raster_fwd_mse", "raster_bwd")
                        if k in prof and k != dom_name]
        if training and graph_ms is not None:
            n_rec, n_ent = plan.status()
            hb = pk.get("hbm_gbs", 6400.0)
            per = lambda k: prof[k][0] / args.steps if k in prof else None
            if per("radix_depth"):
                kernels_roof.append(hbm_entry(
                    "radix_depth", n_rec * 16, per("radix_depth"), hb,
                    "each record's depth key and slot read once and written once (%d records)" % n_rec))
            if per("radix_tile"):
                kernels_roof.append(hbm_entry(
                    "radix_tile", n_rec * 16 + n_ent * 8, per("radix_tile"), hb,
                    "each record's tile rectangle read once, each (view group | tile key, record slot) entry "
                    "written once (%d entries)" % n_ent))
            if per("project"):
                kernels_roof.append(hbm_entry(
                    "project", scene_bytes(w.scene) + n_rec * 56, per("project"), hb,
                    "scene read once, 48 B record and 8 B depth key/slot written per record"))
            if per("image_mse"):
                kernels_roof.append(hbm_entry(
                    "image_mse", S * H * W * 24, per("image_mse"), hb,
                    "image read and gradient written, 12 B per pixel each (targets L2-resident)"))
    cfg = workload_config(w, ws, views, "cuda_graph_plan" if use_graph else "context_calls")
    cfg["tile_px"] = {"context_calls": eager_tile, "cuda_graph_plan": graph_tile}
    if training:
        cfg["loss"] = "mean MSE" if args.loss == "mse" else "Eq. 2: MSE + 0.2 (1 - SSIM), 0.3 CVaR_0.05 tail"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "mpix_per_s": value * H * W / 1e6,
            "eager_per_step": {"ms": eager_ms, "value": ws * S / (eager_ms / 1e3), "unit": UNIT,
                               "what": "context calls, no graph"},
            "graph_per_step": None if graph_ms is None else {
                "ms": graph_ms, "value": ws * S / (graph_ms / 1e3), "unit": UNIT,
                "what": "capture-safe plan, whole step replayed as one CUDA graph"},
            "ms_per_step_ci95": ci95,
            "plain_per_state": {"value": plain, "unit": UNIT, "rounds": plain_rounds,
                                "what": "median of three rounds over the step's states"} if plain else None,
            "batched_vs_plain": (value / ws / plain) if plain else None,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clk, "roofline": roof, "roofline_kernels": kernels_roof,
            "cpu_baseline": cpu,
            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in prof.items()},
            "kernels_note": "per-kernel times from the eager path's live events (same kernels as the graph)",
            "peaks": pk_kind}
    if not training:
        pairs, rendered, rounds = reuse
        line["tile_reuse"] = {"pairs": pairs, "rendered": rendered, "rounds": rounds,
                              "what": "(state, tile) pairs scored per step and how many were rendered; the rest "
                                      "took the partial of a state with the same depths on every cluster the "
                                      "tile's walk reached (bit-identical)"}
    R.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return line if rank == 0 else None


def run_others(args):
    """The utility sweep (2.7M Gaussians, 32,768 states) and the serving mix (48
    SH3 scenes, forward + backward) in the default run, a few steps each and no
    oracle sampling; a summary of each (or the error it raised) goes into the
    default line."""
    import copy
    import gc
    import torch
    from paper_2606_17212_b300 import synth
    out = {}
    for name in ("c4_utility_2p7m", "c5_mix_48"):
        a2 = copy.copy(args)
        a2.workload, a2.steps, a2.warmup = name, 3, 3
        a2.no_cpu_baseline = True
        a2.no_oracle_sample = True
        a2.states = None
        t0 = time.perf_counter()
        try:
            line = run_mix(a2) if name == "c5_mix_48" else run_main(a2, synth.config(name))
            keep = ("value", "unit", "ms_per_step", "mpix_per_s", "plain_per_state", "batched_vs_plain",
                    "tile_reuse", "gpu_launches", "clocks", "e2e", "eager_per_step", "graph_per_step",
                    "scene_waves_per_step")
            summ = {k: line.get(k) for k in keep if line.get(k) is not None}
            summ["config"] = line["config"]
            summ["steps"], summ["warmup"] = a2.steps, a2.warmup
            summ["wall_s"] = round(time.perf_counter() - t0, 1)
            out[name] = summ
        except Exception as e:      # reported, never fatal to the headline line
            out[name] = {"error": "%s: %s" % (type(e).__name__, str(e)[:300])}
        gc.collect()
        torch.cuda.empty_cache()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3_fwdbwd_250k")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--states", type=int, default=None, help="override the workload's state count")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-others", action="store_true",
                    help="default workload only: skip the utility-sweep and serving-mix summaries")
    ap.add_argument("--tile-size", type=int, default=0, choices=[0, 16, 32],
                    help="sort tile side (0: the library chooses per batch shape)")
    ap.add_argument("--no-oracle-sample", action="store_true",
                    help="skip the oracle sample (no cpu_baseline and no evaluation count for the roofline)")
    ap.add_argument("--mix-wave", type=int, default=8,
                    help="serving mix: scenes per dgs_render_scenes_batched call in the scene-wave path")
    ap.add_argument("--entry-headroom", type=float, default=1.1,
                    help="plan path: tile-entry capacity as a multiple of the sizing run's entries")
    ap.add_argument("--loss", default="mse", choices=["mse", "eq2"],
                    help="training loss: mean MSE, or Eq. 2 (MSE + 0.2 (1 - SSIM), CVaR_0.05 tail)")
    args = ap.parse_args()
    assert args.warmup >= 3 or args.impl == "reference", "at least 3 warm-up steps"

    from paper_2606_17212_b300 import synth
    ws, rank, local = _dist()
    if args.workload == "c4_group_utility":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the utility-table mode has no reference-arm "
                              "mode; the oracle's Eq. 3/4 is checked in the tests"}), flush=True)
            return
        if rank == 0:
            print(json.dumps(run_groups(args)), flush=True)
        return
    if args.workload == "c5_mix_48":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the serving mix has no reference-arm mode; "
                              "its oracle baseline is the cpu_baseline of the ours arm"}), flush=True)
            return
        if rank == 0:
            print(json.dumps(run_mix(args)), flush=True)
        return
    w = synth.config(args.workload, scale=args.scale, n_states=args.states)
    if args.impl == "reference":
        reference_arm(args, w)
        return

    line = run_main(args, w)
    if line is not None:
        if not args.no_others and args.workload == "c3_fwdbwd_250k" and args.scale == 1.0 and ws == 1:
            line["other_workloads"] = run_others(args)
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
