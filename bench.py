#!/usr/bin/env python
"""Benchmark of 3DGS loop-edge registration on GB300.

Workload (one bench step = one loop edge): the room-scale registration of
LoopSplat's Sec. 3.2 at full size -- a 150,000-Gaussian room submap P and
its copy Q moved by a 10 deg / 15 cm rigid map, 8 keyframes of 1200x680 per
submap, 100 iterations of forward + backward + on-device pose update in both
directions (16 keyframe problems, 13.06 Mpx per iteration), the residual
pass and the Eq. 7 fusion.  Inputs are seeded and synthetic (no dataset).

Metric: registration steps/s (one step = one iteration over all 16
keyframes, forward + backward + update), whole job over N GPUs; plus Mpx/s
and the p50/p99 latency of a loop edge.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "registration steps/s"
UNIT = "steps/s"
ITERS = 100
WORKLOAD = ("room_150k: 150,000-Gaussian room submap pair (10 deg / 15 cm), 8+8 keyframes 1200x680, "
            "100 iterations fwd+bwd+update in both directions, residual + Eq. 7 fusion")
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
# FP32 operations of the dominant kernels per unit of work (FMA = 2) per
# (pixel, Gaussian) pair that passes the alpha test -- the work the method's
# arithmetic needs as implemented: the forward 41 (exponent 9, exp32 20,
# opacity x e^x 1, 1 - alpha 1, transmittance 1, weight 1, 4 blends 8), the
# adjoint 64 (exponent 9, exp32 20, opacity x e^x 1, transmittance by
# division 3, g . c 7, dL/dalpha 3, weight 1, the colour-behind scalar 2,
# depth 2, screen and 2D-covariance gradients 16).  Pairs walked and
# skipped are overhead (how many depends on how tight the tile lists and
# culls are), not counted.
FWD_FLOPS_CONTRIB = 41.0
BWD_FLOPS_CONTRIB = 64.0
# DRAM bytes per launch of the room workload from one ncu capture of the
# current kernel (the fused forward + adjoint that the timed calls run, and
# the two-kernel adjoint); None while the kernel has changed since the capture
FB_TRAFFIC_BYTES = 278.152448e6
BWD_TRAFFIC_BYTES = 185.502976e6
FP32_LANES = 128
PEAK_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def peaks():
    try:
        return json.load(open(PEAK_FILE))
    except (OSError, ValueError):
        return {}


def make_workload(gs, ctx, torch, seed=1001):
    from paper_2408_10154_gb300 import synth
    c = synth.room_150k(seed=seed)
    src = gs.Gaussians.from_numpy(c["gaussians"])
    tgt = gs.gs_transform(ctx, src, c["T_gt"])  # Q = T_gt P (Eq. 8/9), on the device
    I8 = torch.tensor(np.stack([np.eye(3, 4)] * 8).reshape(8, 12), dtype=torch.float32, device="cuda")
    rs = gs.gs_render(ctx, src, I8, c["src_cams"])
    rt = gs.gs_render(ctx, tgt, I8, c["tgt_cams"])
    sv = list(zip(c["src_cams"], [x.contiguous() for x in gs.split_views(rs["rgb"], c["src_cams"], 3)],
                  [x.contiguous() for x in gs.split_views(rs["depth"], c["src_cams"], 1)]))
    tv = list(zip(c["tgt_cams"], [x.contiguous() for x in gs.split_views(rt["rgb"], c["tgt_cams"], 3)],
                  [x.contiguous() for x in gs.split_views(rt["depth"], c["tgt_cams"], 1)]))
    px = sum(int(cam[4]) * int(cam[5]) for cam in list(c["src_cams"]) + list(c["tgt_cams"]))
    return c, src, tgt, sv, tv, px


def rot_err(P, T):
    R = np.asarray(P)[:, :3].T @ np.asarray(T)[:, :3]
    return math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(R) - 1) / 2)))), float(
        np.linalg.norm(np.asarray(P)[:, 3] - np.asarray(T)[:, 3]))


def run_reference(args):
    """The oracle as it stands (FP64, OpenMP over pixel rows and adjoint
    bands on every host core) on the room workload.  One timed step = one
    keyframe iteration at full size (1200x680 render + L1 loss + adjoint +
    pose step, alternating the two directions); the value is scaled to the
    metric's unit (a registration step covers 16 keyframe iterations)."""
    rank, world, _ = env_rank()
    if rank != 0:
        return 0
    import oracle as O
    from paper_2408_10154_gb300 import synth
    O.build()
    cores = O.set_threads(os.cpu_count() or 1)
    c = synth.room_150k()
    g_src = O.Gaussians.from_dict(c["gaussians"])
    g_tgt = O.transform(g_src, c["T_gt"])
    jobs = []
    for moving, fixed, cam in ((g_tgt, g_src, c["src_cams"][0]), (g_src, g_tgt, c["tgt_cams"][0])):
        tr = O.render(fixed, np.eye(3, 4), cam)
        jobs.append((moving, cam, tr["rgb"].astype(np.float32), tr["depth"].astype(np.float32), O.centroid(moving)))

    def one_keyframe_iteration(k):
        moving, cam, t_rgb, t_dep, piv = jobs[k % 2]
        pose = np.eye(3, 4)
        r = O.render(moving, pose, cam)
        L, gr, gd = O.loss(r["rgb"], r["depth"], t_rgb, t_dep)
        b = O.backward(moving, pose, cam, gr, gd, pivot=piv, params=False)
        O.pose_step(pose, np.zeros(13), b["twist"], piv, 0, ITERS)

    for k in range(args.warmup):
        one_keyframe_iteration(k)
    times = []
    for k in range(args.steps):
        t = time.perf_counter()
        one_keyframe_iteration(k)
        times.append(time.perf_counter() - t)
    per_kf = float(np.mean(times))
    value = 1.0 / (16.0 * per_kf)  # a registration step covers 16 keyframe iterations
    sample = ("one keyframe iteration per bench step (1200x680 render + L1 loss + adjoint + pose step of the room "
              "workload, the two directions alternating), scaled to registration steps (16 keyframe iterations)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_kf * 1000.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "iters_per_edge": ITERS,
                       "bench_step": "one keyframe iteration = 1/16 of a registration step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    device = torch.cuda.current_device()
    import paper_2408_10154_gb300 as gs
    ctx = gs.Context(device)
    c, src, tgt, sv, tv, px = make_workload(gs, ctx, torch)
    opt = gs.default_options(profile=1)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stats_cls = gs.gsreg.gs_stats_t
    import ctypes

    def stats():
        st = stats_cls()
        ctx.check(ctx._lib.gs_ctx_stats(ctx.handle, ctypes.byref(st)))
        return st

    for _ in range(max(args.warmup, 0)):
        gs.gs_register(ctx, src, tgt, sv, tv, ITERS, opt)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(device)
    sampler.start()
    times, phases, launches, pairs, contrib, dups, results = [], np.zeros(5), 0, 0, 0, 0, []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()  # evict L2 between timed calls (outside the timed region)
        ev0.record()
        res = gs.gs_register(ctx, src, tgt, sv, tv, ITERS, opt)
        ev1.record()
        ev1.synchronize()
        times.append(ev0.elapsed_time(ev1))
        st = stats()
        phases += np.array(list(st.phase_ms))
        launches += st.kernel_launches
        pairs += st.pairs
        dups = st.n_dups
        results.append(res)
    torch.cuda.synchronize()
    sampler.stop()
    # pairs passing the alpha test, from one untimed counting call (the
    # registration is bit-reproducible, so it walks the timed calls' pairs)
    gs.gs_register(ctx, src, tgt, sv, tv, ITERS, gs.default_options(profile=2))
    contrib = stats().contributing * len(times)
    total_ms = float(sum(times))
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
        torch.distributed.barrier()
    steps_total = world * args.steps * ITERS
    value = steps_total / (total_ms / 1000.0)
    # end to end: inputs from pinned host memory each step, result read back
    host = {k: getattr(src, k).cpu().pin_memory() for k in ("means4", "log_scales4", "quats4", "logits", "rgb4")}
    host_t = {k: getattr(tgt, k).cpu().pin_memory() for k in ("means4", "log_scales4", "quats4", "logits", "rgb4")}
    host_v = [(cam, r.cpu().pin_memory(), d.cpu().pin_memory()) for cam, r, d in list(sv) + list(tv)]
    # two device input sets: each step's upload (side stream) overlaps the
    # previous step's registration, as a pipelined caller would run it; the
    # timed region holds every step's upload (the first one exposed) and
    # every result read-back
    names_g = ("means4", "log_scales4", "quats4", "logits", "rgb4")
    sets = []
    for _ in range(2):
        dsrc = gs.Gaussians(*[torch.empty_like(getattr(src, k)) for k in names_g])
        dtgt = gs.Gaussians(*[torch.empty_like(getattr(tgt, k)) for k in names_g])
        dviews = [(cam, torch.empty_like(r, device="cuda"), torch.empty_like(d, device="cuda")) for cam, r, d in host_v]
        sets.append((dsrc, dtgt, dviews))
    h2d = sum(v.numel() * v.element_size() for v in list(host.values()) + list(host_t.values()))
    h2d += sum(r.numel() * r.element_size() + d.numel() * d.element_size() for _, r, d in host_v)
    d2h = 12 * 8 + 8 + 16 * 8 + 16 * 12 * 8
    side = torch.cuda.Stream()

    def upload(st):
        dsrc, dtgt, dviews = st
        with torch.cuda.stream(side):
            for k in host:
                getattr(dsrc, k).copy_(host[k], non_blocking=True)
                getattr(dtgt, k).copy_(host_t[k], non_blocking=True)
            for (cam, r, d), (_, hr, hd) in zip(dviews, host_v):
                r.copy_(hr, non_blocking=True)
                d.copy_(hd, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(side)
        return ev

    n_e2e = max(2, min(args.steps, 4))
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev = upload(sets[0])
    for k in range(n_e2e):
        torch.cuda.current_stream().wait_event(ev)
        if k + 1 < n_e2e:
            ev = upload(sets[(k + 1) % 2])
        dsrc, dtgt, dviews = sets[k % 2]
        gs.gs_register(ctx, dsrc, dtgt, dviews[:8], dviews[8:], ITERS, opt)  # returns T on the host
    e2e_times = [(time.perf_counter() - t0) * 1000.0 / n_e2e]
    e2e_value = world * ITERS / (np.mean(e2e_times) / 1000.0)

    pk = peaks()
    clocks = sampler.summary()
    # roofline of the dominant kernel, from the CUDA-event phase times of the timed calls
    names = ["project", "bin", "forward", "backward", "update"]
    calls = args.steps
    per_launch_ms = phases / (calls * ITERS)
    dom = int(np.argmax(per_launch_ms))
    pairs_per_launch = pairs / (calls * ITERS)
    contrib_per_launch = contrib / (calls * ITERS)
    # FP32 peak: measured by an FMA-loop probe on this device (the SM count
    # read from it), beside the figure derived from unit counts and clocks
    probe_tflops, sms = gs.gs_probe_fp32(ctx)
    derived_fp32 = sms * FP32_LANES * 2 * (pk.get("sm_max_mhz", 2070.0) * 1e6) / 1e12
    peak_fp32 = probe_tflops
    # with fused compositing (the default for the registration loss) the
    # forward phase is the one kernel k_fwdbwd and the backward phase is empty
    fused = bool(opt.fuse_compositing)
    peak_source = ("measured: FMA-loop probe (gs_probe_fp32, scalar and packed f32x2 FMAs) on this GPU, "
                   "%d SMs" % sms)

    def alu_roof(kernel, fc, ms, traffic):
        flops = fc * contrib_per_launch
        achieved = flops / (ms / 1000.0) / 1e12
        return {"kernel": kernel, "bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                "frac": achieved / peak_fp32, "traffic": traffic, "flops_per_launch": flops,
                "ms_per_launch": float(ms), "peak_source": peak_source, "peak_derived": derived_fp32,
                "frac_of_derived": achieved / derived_fp32}

    if names[dom] in ("backward", "forward"):
        if fused and names[dom] == "forward":
            roof = alu_roof("k_fwdbwd", FWD_FLOPS_CONTRIB + BWD_FLOPS_CONTRIB, per_launch_ms[dom], FB_TRAFFIC_BYTES)
        elif names[dom] == "backward":
            roof = alu_roof("k_backward2", BWD_FLOPS_CONTRIB, per_launch_ms[dom], BWD_TRAFFIC_BYTES)
        else:
            roof = alu_roof("k_forward", FWD_FLOPS_CONTRIB, per_launch_ms[dom], None)
    else:
        hbm = pk.get("hbm_gbs", 6800.0)
        roof = {"kernel": names[dom], "bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s", "frac": None,
                "traffic": None}
    # HBM-bound steps: algorithmic bytes per launch / CUDA-event time.
    # Projection: 56 B per Gaussian of each moving submap + 52 B (48 B
    # record + 4 B count) per visible (keyframe, Gaussian).  Tile lists:
    # 16 B entry read per visible record, 8 B written at placement and 8 B
    # read + 8 B written by the per-tile sort per duplicate, 8 B range per tile.
    I8 = torch.tensor(np.stack([np.eye(3, 4)] * 8).reshape(8, 12), dtype=torch.float32, device="cuda")
    vis = sum(int((gs.gs_project(ctx, g, I8, cams, with_aux=False)[2] > 0).sum())
              for g, cams in ((tgt, c["src_cams"]), (src, c["tgt_cams"])))
    tiles = 16 * ((1200 + 15) // 16) * ((680 + 15) // 16)
    hbm_peak = pk.get("hbm_gbs", 6800.0)
    hbm = {}
    for name, nbytes in (("project", 56.0 * (src.n + tgt.n) + 52.0 * vis),
                         ("bin", 16.0 * vis + 24.0 * dups + 8.0 * tiles)):
        ms = per_launch_ms[names.index(name)]
        gbs = nbytes / (ms / 1000.0) / 1e9
        hbm[name] = {"bytes_per_launch": nbytes, "ms_per_launch": float(ms), "achieved_gbs": gbs,
                     "peak_gbs": hbm_peak, "frac": gbs / hbm_peak}
    hbm["visible_records_at_start"] = vis
    # the same edge with the forward and the adjoint as two kernels (one
    # untimed profiled call; bit-identical results): their own times and
    # the adjoint's roofline
    two = None
    if fused:
        gs.gs_register(ctx, src, tgt, sv, tv, ITERS, gs.default_options(profile=1, fuse_compositing=0))
        ph = np.array(list(stats().phase_ms)) / ITERS
        two = {"phase_ms_per_iteration": {n: float(v) for n, v in zip(names, ph)},
               "adjoint_roofline": alu_roof("k_backward2", BWD_FLOPS_CONTRIB, ph[3], BWD_TRAFFIC_BYTES),
               "forward_roofline": alu_roof("k_forward", FWD_FLOPS_CONTRIB, ph[2], None)}
    hbm["peak_source"] = "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in pk else "fallback 6800 GB/s"
    lat = sorted(times)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "iters_per_edge": ITERS, "pixels_per_iteration": px,
                   "l2": "flushed between timed calls (256 MB write); per-iteration working set > 129 MB L2",
                   "bench_step": "one loop edge = 100 registration steps + residual + fusion"},
        "mpx_per_s": value * px / 1e6,
        "edge_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "phase_ms_per_iteration": {n: float(v) for n, v in zip(names, per_launch_ms)},
        "pairs_per_iteration": pairs_per_launch, "contributing_pairs_per_iteration": contrib_per_launch,
        "dups": int(dups),
        "roofline": roof,
        "two_kernels": two,
        "hbm": hbm,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "bench_step": "one loop edge (100 registration steps): the bytes are per edge"},
        "clocks": clocks,
        "gpu_launches": int(launches),
    }
    T = results[-1][0]
    ang, dt = rot_err(T, c["T_gt"])
    out["accuracy"] = {"rot_err_deg": ang, "trans_err_mm": dt * 1000.0,
                       "keyframes_converged": int(np.sum(np.asarray(results[-1][2]) < 0.01))}
    ctx.close()
    if world == 1 and not args.room_only:
        # the rest of the metric: batched vs plain, and serving p50/p99
        bctx = gs.Context(device, 96 << 30)
        out["batched_32"], _ = measure_batched(gs, bctx, torch, reps=1, warmup=1)
        bctx.close()
        torch.cuda.empty_cache()
        out["serving"] = measure_serve(args.serve_rate, args.serve_seconds, 64, args.max_kf, args.round_iters)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(c)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def cpu_baseline(c):
    """Times the FP64 oracle, as it stands, on the host cores: keyframe
    iterations (render + loss + adjoint + pose step) of the room workload at
    full size, alternating the two directions -- 8 on all cores (OpenMP over
    pixel rows and adjoint bands) and 4 on one core -- scaled to
    registration steps/s (16 keyframe iterations per step)."""
    import oracle as O
    O.build()
    g_src = O.Gaussians.from_dict(c["gaussians"])
    g_tgt = O.transform(g_src, c["T_gt"])
    jobs = []
    for k in range(4):
        for moving, fixed, cam in ((g_tgt, g_src, c["src_cams"][k]), (g_src, g_tgt, c["tgt_cams"][k])):
            tr = O.render(fixed, np.eye(3, 4), cam)
            jobs.append((moving, cam, tr["rgb"].astype(np.float32), tr["depth"].astype(np.float32),
                         O.centroid(moving)))

    def timed(js):
        per = []
        for moving, cam, t_rgb, t_dep, piv in js:
            t = time.perf_counter()
            pose = np.eye(3, 4)
            r = O.render(moving, pose, cam)
            L, gr, gd = O.loss(r["rgb"], r["depth"], t_rgb, t_dep)
            b = O.backward(moving, pose, cam, gr, gd, pivot=piv, params=False)
            O.pose_step(pose, np.zeros(13), b["twist"], piv, 0, ITERS)
            per.append(time.perf_counter() - t)
        return float(np.mean(per)), float(sum(per))

    cores = O.set_threads(os.cpu_count() or 1)
    per_all, sec_all = timed(jobs)
    O.set_threads(1)
    per_one, sec_one = timed(jobs[:4])
    return {"value": 1.0 / (16.0 * per_all), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "8 keyframe iterations of the room workload at full size (4 per direction) on %d cores, "
                      "scaled to a 16-keyframe registration step" % cores,
            "seconds": sec_all,
            "single_core": {"value": 1.0 / (16.0 * per_one), "unit": UNIT, "cores": 1, "seconds": sec_one,
                            "sample": "4 of the same keyframe iterations on one core"},
            "host_cpus": os.cpu_count()}


def edge_problems(gs, ctx, torch, pairs):
    """Device problems (src, tgt = T_gt src, src keyframes, tgt keyframes,
    targets rendered on the device) of batched-workload pairs, and their
    pixels per iteration."""
    problems, px = [], 0
    for pr in pairs:
        src = gs.Gaussians.from_numpy(pr["gaussians"])
        tgt = gs.gs_transform(ctx, src, pr["T_gt"])
        k = len(pr["src_cams"])
        I = torch.tensor(np.stack([np.eye(3, 4)] * k).reshape(k, 12), dtype=torch.float32, device="cuda")
        rs = gs.gs_render(ctx, src, I, pr["src_cams"])
        rt = gs.gs_render(ctx, tgt, I, pr["tgt_cams"])
        sv = list(zip(pr["src_cams"], [x.contiguous() for x in gs.split_views(rs["rgb"], pr["src_cams"], 3)],
                      [x.contiguous() for x in gs.split_views(rs["depth"], pr["src_cams"], 1)]))
        tv = list(zip(pr["tgt_cams"], [x.contiguous() for x in gs.split_views(rt["rgb"], pr["tgt_cams"], 3)],
                      [x.contiguous() for x in gs.split_views(rt["depth"], pr["tgt_cams"], 1)]))
        problems.append((src, tgt, sv, tv))
        px += sum(int(c[4]) * int(c[5]) for c in list(pr["src_cams"]) + list(pr["tgt_cams"]))
    return problems, px


def measure_serve(rate, seconds, pool, max_kf, round_iters):
    """Serving stream (Poisson arrivals, 70 % frame-to-model tracking of a
    resident submap, 30 % loop edges; 40 / 100 iterations) through the
    continuous-batching server in real time, and the plain form: the same
    stream served one request at a time in arrival order (each request's
    gs_register time measured, FIFO queueing computed from the arrivals).
    Returns a dict with p50/p99 latencies and throughput of both."""
    import time
    import torch
    import paper_2408_10154_gb300 as gs
    from paper_2408_10154_gb300 import synth
    ctx = gs.Context(torch.cuda.current_device(), 64 << 30)
    st = synth.serving_stream(rate=rate, seconds=seconds, n_submaps=pool)
    edges, _ = edge_problems(gs, ctx, torch, synth.batched_pairs()["pairs"])
    tracks = []
    for sm in st["submaps"]:
        g = gs.Gaussians.from_numpy(sm["gaussians"])
        k = len(sm["cams"])
        I = torch.tensor(np.stack([np.eye(3, 4)] * k).reshape(k, 12), dtype=torch.float32, device="cuda")
        r = gs.gs_render(ctx, g, I, sm["cams"])
        rgb, dep = gs.split_views(r["rgb"], sm["cams"], 3), gs.split_views(r["depth"], sm["cams"], 1)
        tracks.append((g, [(sm["guesses"][f], rgb[f].contiguous(), dep[f].contiguous()) for f in range(k)]))
    arrivals = st["arrivals"]
    n = len(arrivals)

    # tracking requests: the tracking loss of Eq. 2 at the paper's tracking rates
    # (Supp. A: lambda_c 0.6, l_r 0.002, l_t 0.01 on TUM-RGBD / ScanNet)
    topt = gs.default_options(tracking_loss=1, lambda_c=0.6, lr_rot=0.002, lr_trans=0.01)

    def request(a):
        _, kind, idx, fr = a
        if kind == "track":
            g, fv = tracks[idx]
            return (g, g, [], [fv[fr]], topt), st["track_iters"], 640 * 480
        src, tgt, sv, tv = edges[idx]
        return edges[idx], st["edge_iters"], sum(int(c[4]) * int(c[5]) for c, _, _ in list(sv) + list(tv))

    # warm-up: one request of each kind through both forms
    for a in (next(x for x in arrivals if x[1] == "track"), next(x for x in arrivals if x[1] == "edge")):
        prob, iters, _ = request(a)
        gs.gs_register(ctx, *prob[:4], iters, *prob[4:])
        w = gs.Server(torch.cuda.current_device(), max_keyframes=max_kf, max_round_iters=round_iters)
        w.submit(*prob[:4], iters, *prob[4:])
        while w.counts()[1] or w.counts()[0]:
            w.step()
        w.close()
    torch.cuda.synchronize()
    # served: submit each request at its arrival time, one round per step
    srv = gs.Server(torch.cuda.current_device(), budget_bytes=160 << 30, max_keyframes=max_kf,
                    max_round_iters=round_iters)
    done_at, rid_of, i = {}, {}, 0
    t0 = time.perf_counter()
    while len(done_at) < n:
        now = time.perf_counter() - t0
        while i < n and arrivals[i][0] <= now:
            prob, iters, _ = request(arrivals[i])
            rid_of[srv.submit(*prob[:4], iters, *prob[4:])] = i
            i += 1
        waiting, inflight = srv.counts()[:2]
        if waiting == 0 and inflight == 0:
            time.sleep(max(0.0, arrivals[i][0] - (time.perf_counter() - t0)))
            continue
        for rid in srv.step():
            done_at[rid_of[rid]] = time.perf_counter() - t0
    served_T = {rid_of[r]: srv.poll(r)["T"] for r in rid_of}
    _, _, _, rounds, replans = srv.counts()
    srv.close()
    # plain: each request alone, FIFO in arrival order
    service, plain_T = [], {}
    for k, a in enumerate(arrivals):
        prob, iters, _ = request(a)
        torch.cuda.synchronize()
        t = time.perf_counter()
        plain_T[k] = gs.gs_register(ctx, *prob[:4], iters, *prob[4:])[0]
        service.append(time.perf_counter() - t)
    finish, tcur = [], 0.0
    for k, a in enumerate(arrivals):
        tcur = max(a[0], tcur) + service[k]
        finish.append(tcur)
    work = sum(request(a)[1] * request(a)[2] for a in arrivals)

    def summary(done):
        lat = {kind: [1000.0 * (done[k] - arrivals[k][0]) for k in range(n) if arrivals[k][1] == kind]
               for kind in ("track", "edge")}
        span = max(done[k] for k in range(n))
        out = {"makespan_s": span, "requests_per_s": n / span, "mpx_iter_per_s": work / span / 1e6}
        for kind, l in lat.items():
            if l:
                out[kind + "_latency_ms"] = {"p50": float(np.percentile(l, 50)), "p99": float(np.percentile(l, 99))}
        return out

    served = summary(done_at)
    plain = summary({k: finish[k] for k in range(n)})
    same = sum(int(np.array_equal(served_T[k], plain_T[k])) for k in range(n))
    ctx.close()
    return {"workload": "serving: Poisson %.0f/s for %.0f s (%d requests; 70 %% tracking 640x480 with the Eq. 2 "
                        "loss, 40 it, %d resident submaps of 50k-300k; 30 %% loop edges of the batched pool, 100 it)"
                        % (rate, seconds, n, pool),
            "rate_per_s": rate, "n_requests": n, "max_keyframes": max_kf, "round_iters": round_iters,
            "served": served, "plain": plain, "served_rounds": rounds, "served_replans": replans,
            "results_identical": same,
            "mean_plain_service_ms": 1000.0 * float(np.mean(service))}


def run_serve(args):
    """--workload serve: the serving record alone, as its own JSON line."""
    import torch
    torch.cuda.set_device(0)
    rec = measure_serve(args.rate, args.seconds, args.pool, args.max_kf, args.round_iters)
    out = {"metric": "serving requests/s", "value": rec["served"]["requests_per_s"], "unit": "requests/s",
           "n_gpus": 1, "steps": rec["n_requests"], "warmup": 2, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": {"workload": rec["workload"]},
           **{k: v for k, v in rec.items() if k != "workload"}}
    print(json.dumps(out), flush=True)
    return 0


def run_overlap(args):
    """Overlap ratio (loop filter) of the room submap pair under its ground
    truth: exact nearest neighbours both ways over 150k x 150k means (grid
    search).  Prints one JSON line (ms per call, queries per second)."""
    import torch
    torch.cuda.set_device(0)
    import paper_2408_10154_gb300 as gs
    from paper_2408_10154_gb300 import synth
    ctx = gs.Context(0)
    c = synth.room_150k()
    src = gs.Gaussians.from_numpy(c["gaussians"])
    tgt = gs.gs_transform(ctx, src, c["T_gt"])
    for _ in range(max(args.warmup, 1)):
        gs.gs_overlap_ratio(ctx, src, tgt, c["T_gt"])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(args.steps):
        r, k = gs.gs_overlap_ratio(ctx, src, tgt, c["T_gt"])
    ev1.record()
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    queries = float(src.n + tgt.n)
    out = {"metric": "overlap ratio calls/s", "value": 1000.0 / ms, "unit": "calls/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "overlap ratio of the room_150k pair (150,000 x 150,000 means, both directions)"},
           "overlap": r, "correspondences": k, "queries_per_s": queries / (ms / 1000.0),
           "brute_force_pairs_per_call": 2.0 * src.n * tgt.n,
           "roofline": None, "roofline_note": "grid search: latency-bound cell traversal, no dense work to count"}
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


def measure_batched(gs, ctx, torch, reps=1, warmup=1, problems=None, px=None, n_edges=None, T_gts=None):
    """Batched uneven registration: the pairs of the batched workload, each
    in both directions, registered (a) one pair per call ("plain",
    gs_register) and (b) all pairs in one batch (gs_register_batch).
    Returns (record dict, fused T and confidence of the last batch)."""
    from paper_2408_10154_gb300 import synth
    if problems is None:
        wl = synth.batched_pairs()
        problems, px = edge_problems(gs, ctx, torch, wl["pairs"])
        T_gts = [pr["T_gt"] for pr in wl["pairs"]]
    iters = ITERS
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        ev0.record()
        out = fn()
        ev1.record()
        ev1.synchronize()
        return ev0.elapsed_time(ev1), out

    def plain():
        lat = []
        for p in problems:
            t, _ = timed(lambda: gs.gs_register(ctx, *p, iters))
            lat.append(t)
        return lat

    def batched():
        return gs.gs_register_batch(ctx, problems, iters)

    for _ in range(max(warmup, 1)):
        batched()
        plain()
    plain_runs, batch_runs, res = [], [], None
    for _ in range(max(reps, 1)):
        plain_runs.append(plain())
        t, res = timed(batched)
        batch_runs.append(t)
    plain_ms = float(np.mean([sum(l) for l in plain_runs]))
    batch_ms = float(np.mean(batch_runs))
    lat_all = sorted(x for l in plain_runs for x in l)
    n = len(problems)
    rec = {"workload": "batched_32: %d uneven submap pairs (20k-400k Gaussians, 4-12 keyframes per submap at "
                       "640x480 / 1200x680), both directions, %d iterations" % (n, iters),
           "pixels_per_iteration": int(px),
           "batched": {"ms_per_batch": batch_ms, "steps_per_s": n * iters / (batch_ms / 1000.0),
                       "edges_per_s": n / (batch_ms / 1000.0),
                       "mpx_per_s": px * iters / (batch_ms / 1000.0) / 1e6},
           "plain": {"ms_per_batch": plain_ms, "steps_per_s": n * iters / (plain_ms / 1000.0),
                     "edges_per_s": n / (plain_ms / 1000.0),
                     "mpx_per_s": px * iters / (plain_ms / 1000.0) / 1e6,
                     "edge_latency_ms": {"p50": float(np.percentile(lat_all, 50)),
                                         "p99": float(np.percentile(lat_all, 99))}},
           "batched_over_plain": plain_ms / batch_ms,
           "step": "steps_per_s counts registration steps of single loop edges (one iteration of all the keyframe "
                   "problems of one edge, as in the headline), summed over the %d edges" % n}
    if T_gts is not None and res is not None:
        rec["batched"]["edges_within_1deg_2cm"] = int(sum(
            rot_err(res[0][k], T_gts[k])[0] < 1.0 and rot_err(res[0][k], T_gts[k])[1] < 0.02 for k in range(n)))
    return rec, res


def run_batched(args):
    """--workload batched_32: batched vs one-pair-per-call as its own JSON
    line; under torchrun the pairs are sharded (whole edges per rank, LPT on
    rendering work) and one result all-reduce gathers the fused transforms."""
    import torch
    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_2408_10154_gb300 as gs
    from paper_2408_10154_gb300 import shard, synth
    ctx = gs.Context(torch.cuda.current_device(), 96 << 30)
    wl = synth.batched_pairs()
    if args.pairs:
        wl["pairs"] = wl["pairs"][:args.pairs]  # a smaller batch (profiling captures only)
    costs = [shard.edge_cost(len(pr["gaussians"]["means4"]), len(pr["gaussians"]["means4"]), pr["src_cams"],
                             pr["tgt_cams"]) for pr in wl["pairs"]]
    mine = shard.lpt_partition(costs, world)[rank]
    problems, px = edge_problems(gs, ctx, torch, [wl["pairs"][i] for i in mine])
    rec, res = measure_batched(gs, ctx, torch, args.steps, args.warmup, problems, px)
    plain_ms, batch_ms = rec["plain"]["ms_per_batch"], rec["batched"]["ms_per_batch"]
    n_edges = len(wl["pairs"])
    rows = {i: np.concatenate([np.asarray(res[0][k], np.float64).reshape(12), [res[1][k]]])
            for k, i in enumerate(mine)}
    fused = shard.gather_results(rows, n_edges, 13, device="cuda")
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([plain_ms, batch_ms, px], dtype=torch.float64, device="cuda")
        tmax = t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(t)
        plain_ms, batch_ms, px = float(tmax[0]), float(tmax[1]), int(t[2])
    out = {"metric": METRIC, "value": n_edges * ITERS / (batch_ms / 1000.0), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": batch_ms, "higher_is_better": True,
           "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": rec["workload"], "pixels_per_iteration": px,
                      "step": "all %d loop edges, %d registration iterations" % (n_edges, ITERS)},
           "batched": rec["batched"], "plain": rec["plain"], "batched_over_plain": plain_ms / batch_ms,
           "edges_within_1deg_2cm": int(sum(
               rot_err(fused[i, :12].reshape(3, 4), pr["T_gt"])[0] < 1.0 and
               rot_err(fused[i, :12].reshape(3, 4), pr["T_gt"])[1] < 0.02 for i, pr in enumerate(wl["pairs"])))}
    if world > 1:
        out["config"]["sharding"] = "whole edges per rank by LPT on rendering work; one result all-reduce"
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--room-only", action="store_true",
                    help="the room line only (no batched and serving records)")
    ap.add_argument("--serve-rate", type=float, default=17.0,
                    help="arrivals per second of the serving record in the default line")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--workload", default="room_150k", choices=["room_150k", "batched_32", "serve", "overlap"],
                    help="room_150k: the benchmark line; batched_32: batched vs one-pair-per-call; "
                         "serve: continuous-batching server vs one request at a time")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: arrivals per second")
    ap.add_argument("--seconds", type=float, default=10.0, help="serve: length of the arrival stream")
    ap.add_argument("--pool", type=int, default=64, help="serve: resident tracking submaps")
    ap.add_argument("--max-kf", type=int, default=128, help="serve: keyframe problems in flight")
    ap.add_argument("--round-iters", type=int, default=10, help="serve: iterations per round")
    ap.add_argument("--pairs", type=int, default=0,
                    help="batched_32: register only the first N pairs (profiling captures; 0 = all 32)")
    ap.add_argument("--iters", type=int, default=ITERS,
                    help="iterations per loop edge (100 for the benchmark; fewer only for profiling captures)")
    args = ap.parse_args()
    globals()["ITERS"] = args.iters
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched_32":
        return run_batched(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "overlap":
        return run_overlap(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
