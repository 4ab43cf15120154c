#!/usr/bin/env python3
"""Throughput of the DIGS hot path on GB300: fwd+bwd projections/s on the synthetic 100k-Gaussian thorax
(256 x 256 detector, R = 3, 680 projections).

One step = one reconstruction iteration through the public C-ABI (``digs_step``): deform and project a
batch of B projections (B = --batch), L2 loss against the measured projections, the full backward to
Gaussians, control points and temporal weights, and the fused Adam update of every parameter group.

Prints ONE JSON line (rank 0).  ``value`` = projections processed by all ranks / max over ranks of the
summed device time of the timed steps (CUDA events around each step; L2 is flushed between steps by a
512 MB write outside the events).  ``e2e`` times the same steps end to end by the wall clock: every step's
host-to-device copy of the batch's measured projections from pinned memory (on a copy stream, double
buffered so that it overlaps the previous step), the step (replayed from a graph captured on the device
buffer its copy lands in, as in the device-timed loop; direct calls with --no-graph), and a
device-to-host read of its loss.
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same workload instead.
Multi-GPU (torchrun): every rank reconstructs its own independent scan (no data-path collective).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd projections/s (100k Gauss, 256²); % roofline; warm-start speedup"
UNIT = "projections/s"
# Algorithmic work, in FP32 lane operations (one FP32 result of one lane: an FMA counts once) and SFU
# operations, of the hot path's units:
#   per (pixel, Gaussian) pair inside the cutoff: forward ~18 FP32 + 2 SFU (rsqrt, exp2), backward ~46 FP32
#   + 2 SFU (the forward's terms recomputed, then the record-gradient sums);
#   per (projection, Gaussian): ~850 FP32 (deformation and projection set-up ~250, their adjoints ~600);
#   per Gaussian and step: the FFD, 64 x 12 R forward and 64 x 30 R backward;
#   algorithmic bytes per projection: parameters and FFD values read and gradients written,
#   2 N (11 + 12 R) 4 B, plus the measured and the rendered projection (2 x 4 B per pixel).
PAIR_WORK = {"raster_fwd": (18, 2), "raster_bwd": (46, 2)}
PROJ_GAUSS_OPS = 850
FFD_OPS_PER_RANK = 64 * 42


def step_work(pairs, B, N, R, npix):
    """(FP32 lane ops, SFU ops, algorithmic bytes) of one step over B projections with `pairs` in-cutoff
    (pixel, Gaussian) pairs in all."""
    fp32 = pairs * (PAIR_WORK["raster_fwd"][0] + PAIR_WORK["raster_bwd"][0]) + B * N * PROJ_GAUSS_OPS \
        + N * FFD_OPS_PER_RANK * R
    sfu = pairs * (PAIR_WORK["raster_fwd"][1] + PAIR_WORK["raster_bwd"][1])
    nbytes = B * (2 * N * (11 + 12 * R) * 4 + 2 * npix * 4)
    return fp32, sfu, nbytes


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=0, help="projections per step (0: autotuned over 8 ... 128)")
    ap.add_argument("--tile", type=int, default=0, help="raster tile edge (0: autotuned)")
    ap.add_argument("--lanes", type=int, default=0, help="backward lanes per Gaussian, 16 or 32 (0: autotuned)")
    ap.add_argument("--n", type=int, default=100_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time direct calls instead of graph replays")
    ap.add_argument("--no-batching", action="store_true", help="skip the four-scan batching measurement")
    ap.add_argument("--no-warmstart", action="store_true", help="skip the learned warm-start measurement")
    ap.add_argument("--only-cnn", action="store_true",
                    help="time only the weight-predictor CNN's training step and inference, print that line")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(pw) if pw else None}


def visible_gpu_index(local_rank):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip() != ""]
    if ids and all(v.strip().isdigit() for v in ids) and local_rank < len(ids):
        return int(ids[local_rank])
    return local_rank


def pipe_peaks(local):
    """Measured rates of the FP32 FMA pipe (scalar and packed FMA, the faster is the FP32 peak) and of the
    SFU (ex2 and rsqrt; one of each per pair, so the SFU peak for the pairs is their harmonic mean), in
    FP32 results per second, with the SM clocks sampled while they run."""
    from paper_2506_22280_gb300 import digs as D
    clocks = ClockSampler(visible_gpu_index(local))
    clocks.start()
    iters = {"ffma": 65536, "ffma2": 65536, "ex2": 16384, "rsqrt": 16384}
    rates = {k: D.pipe_rate(k, iters=iters[k]) for k in D.PIPES}
    clk = clocks.stop()
    out = {k + "_per_s": v for k, v in rates.items()}
    out["fp32_per_s"] = max(rates["ffma"], rates["ffma2"])
    out["sfu_per_s"] = 2.0 / (1.0 / rates["ex2"] + 1.0 / rates["rsqrt"])
    out["clocks"] = clk
    out["how"] = ("digs_pipe_bench: 2 CTAs of 1024 threads per SM, 8 independent chains per thread; best of 3 "
                  "launches timed with CUDA events; one FP32 result = one lane operation")
    return out


def kernel_roofline(kernel, pairs, ms, peaks, traffic=None):
    """Roofline of a raster kernel: its pairs' FP32 and SFU work at the measured pipe peaks; the slower
    pipe bounds it."""
    ops, sfu = PAIR_WORK[kernel]
    t_fp32 = pairs * ops / peaks["fp32_per_s"]
    t_sfu = pairs * sfu / peaks["sfu_per_s"]
    if t_fp32 >= t_sfu:
        pipe, work, peak = "fp32", pairs * ops, peaks["fp32_per_s"]
    else:
        pipe, work, peak = "sfu", pairs * sfu, peaks["sfu_per_s"]
    achieved = work / (ms / 1e3)
    return {"bound": "alu", "kernel": "k_" + kernel, "pipe": pipe, "achieved": achieved / 1e12, "peak": peak / 1e12,
            "unit": "T lane-ops/s", "frac": achieved / peak, "traffic": traffic,
            "peak_basis": "measured (digs_pipe_bench) FP32 FMA-pipe / SFU rate",
            "ops_per_pair": ops, "sfu_per_pair": sfu, "pairs_per_launch": pairs, "launch_ms": ms,
            "roofline_ms": max(t_fp32, t_sfu) * 1e3}


def adam_defaults(total):
    # per group: mu0 (mm), log-scale, quaternion, density pre-activation, phi (mm), w
    lr0 = [0.02, 0.005, 0.002, 0.01, 0.02, 0.01]
    lr1 = [x / 10 for x in lr0]
    return lr0, lr1, total


def batch_ids(step, B, n_proj):
    stride = max(n_proj // B, 1)
    return [int((step * 7 + j * stride) % n_proj) for j in range(B)]


def render_measured(pkg, wl, device):
    """Measured projections of all views, rendered from the ground truth by the forward model."""
    import torch
    gt = wl.extra["gt"]
    f = lambda a: torch.as_tensor(a, dtype=torch.float32, device=device).contiguous()
    ins = [f(gt["mu0"]), f(gt["scale"]), f(gt["quat"]), f(gt["rho"]), f(gt["phi"])]
    out = torch.empty(len(wl.views), wl.views[0]["nv"], wl.views[0]["nu"], device=device)
    for s in range(0, len(wl.views), 128):
        ids = list(range(s, min(s + 128, len(wl.views))))
        pj = pkg.Projector(wl.lattice, [wl.views[i] for i in ids])
        pj.forward(*ins, f(gt["w"][ids]), out=out[s:s + len(ids)])
    torch.cuda.synchronize()
    return out


def traffic_for(kernel, projections, tile, lanes):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was taken on the current
    source of that kernel with the same tile and backward lanes (else None).  The capture holds fewer
    projections than a bench launch: its records, tile counts and images all grow in proportion to the
    projections of the launch, so its bytes are scaled by projections / captured projections."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path)).get(kernel)
        src = open(os.path.join(ROOT, "paper_2506_22280_gb300", "csrc", rec["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest() != rec["sha256"]:
            return None
        if int(rec["tile"]) != tile or int(rec["bwd_lanes"]) != lanes:
            return None
        return float(rec["bytes_per_launch"]) * projections / float(rec["projections"])
    except Exception:
        return None


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline(wl):
    """The FP64 oracle, as it stands, on one projection of the full workload (fwd + bwd) on all host
    cores, and on one core for a 10,000-Gaussian sample of it."""
    import torch
    from oracle import digs_oracle as O
    import synth
    sub = wl.select_views([0])
    g = dict(mu0=sub.mu0, scale=sub.scale, quat=sub.quat, rho=sub.rho)
    gp = synth.random_grad_proj(1, sub.views[0]["nv"], sub.views[0]["nu"], seed=2)
    cores = torch.get_num_threads()
    t0 = time.perf_counter()
    O.project_vjp(g, sub.lattice, sub.phi, sub.w, sub.views, gp)
    dt = time.perf_counter() - t0
    n1 = min(10_000, wl.n)
    one = sub.subset(np.random.default_rng(3).choice(wl.n, n1, replace=False))
    torch.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        O.project_vjp(dict(mu0=one.mu0, scale=one.scale, quat=one.quat, rho=one.rho), one.lattice, one.phi, one.w,
                      one.views, gp)
        dt1 = time.perf_counter() - t0
    finally:
        torch.set_num_threads(cores)
    return {"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"1 projection of the {wl.n}-Gaussian thorax, FP64 oracle forward + backward (box mode), "
                      f"{dt:.1f} s on {cores} threads",
            "one_core": {"seconds": dt1, "gaussians": n1,
                         "sample": f"1 projection of a {n1}-Gaussian sample of the same thorax on 1 thread "
                                   f"({dt1:.1f} s; the oracle's cost is linear in the Gaussian count)"}}


def reduce_timings(values, world, device):
    """Max over ranks of each timed quantity: the job ends when the slowest replica's GPU does."""
    import torch
    import torch.distributed as dist
    red = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(red, op=dist.ReduceOp.MAX)
    return [float(x) for x in red.tolist()]


def whole_job_rate(world, B, K, max_ms):
    """Projections per second of the whole job: every rank's B x K projections over the slowest time."""
    return world * B * K / (max_ms / 1e3)


def make_rec_factory(pkg, D, wl, device, total=10_000, scan_sizes=None):
    lr0, lr1, _ = adam_defaults(total)

    def make(tile, lanes):
        return pkg.Reconstruction(wl["mu0"], wl["scale"], wl["quat"], wl["rho"], wl["phi"], wl["w"], wl["lattice"],
                                  D.adam_config(lr0, lr1, total), tile=tile, bwd_lanes=lanes, device=device,
                                  scan_sizes=scan_sizes)
    return make


def batching_measurement(pkg, D, device, steps=6, warmup=3):
    """Four thorax scans with uneven Gaussian counts in one state; each step renders 64 (scan, projection)
    items -- 16 distinct angles and times per scan -- with one launch per stage (a captured CUDA graph),
    against the plain method: one digs_step per projection on each scan's own state."""
    import torch
    import synth
    scans = synth.thorax_batch()
    sizes = [w.n for w in scans]
    meas = [render_measured(pkg, w, device) for w in scans]
    n_proj = len(scans[0].views)
    cat = lambda k: np.concatenate([getattr(w, k) for w in scans], 0)
    state = dict(mu0=cat("mu0"), scale=cat("scale"), quat=cat("quat"), rho=cat("rho"),
                 phi=np.stack([w.phi for w in scans], 0), w=cat("w"), lattice=scans[0].lattice)
    def items(step, per_scan=16):
        out = []
        for s in range(len(scans)):
            for j in batch_ids(step * len(scans) + s, per_scan, n_proj):
                out.append((s, j))
        return out

    def make_batch(B, step):
        its = items(step, B // len(scans))
        M = torch.stack([meas[s][j] for s, j in its]).contiguous()
        return M, [n_proj * s + j for s, j in its], [dict(scans[s].views[j], scan=s) for s, j in its]

    from paper_2506_22280_gb300 import autotune
    make = make_rec_factory(pkg, D, state, device, scan_sizes=sizes)
    # items per step: 64 (the workload's figure) first, then 32 and 128 (DIGS_MAX_VIEWS)
    tuned = autotune.tune(make, make_batch, tiles=(8, 16, 32), lanes=(16, 32), batch_sizes=(64, 32, 128), steps=2,
                          warmup=1)
    rec = make(tuned["tile"], tuned["bwd_lanes"])
    B = tuned["batch"]
    per_scan = B // len(scans)
    for s in range(warmup):
        rec.step(*make_batch(B, s))
    batches = [make_batch(B, warmup + s) for s in range(steps)]
    graphs = rec.capture(batches)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for g in graphs:
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    batched = steps * B / (e0.elapsed_time(e1) / 1e3)
    status = rec.status()
    del rec, graphs
    # plain: one projection per call on each scan's own state, same items
    plain_recs = []
    for s, w in enumerate(scans):
        st = dict(mu0=w.mu0, scale=w.scale, quat=w.quat, rho=w.rho, phi=w.phi, w=w.w, lattice=w.lattice)
        plain_recs.append(make_rec_factory(pkg, D, st, device)(16, 16))
    its = [it for k in range(warmup + steps) for it in items(k, per_scan)]
    for s, j in its[:len(scans) * 2]:
        plain_recs[s].step(meas[s][j:j + 1].contiguous(), [j], [scans[s].views[j]])
    torch.cuda.synchronize()
    timed = its[warmup * B:(warmup + steps) * B]
    e0.record()
    for s, j in timed:
        plain_recs[s].step(meas[s][j:j + 1].contiguous(), [j], [scans[s].views[j]])
    e1.record()
    torch.cuda.synchronize()
    plain = len(timed) / (e0.elapsed_time(e1) / 1e3)
    status = status or max(r.status() for r in plain_recs)
    return {"workload": f"4 synthetic thorax scans of {'/'.join(str(k // 1000) + 'k' for k in sizes)} Gaussians "
                        f"(per-scan surrogates, 680 projections each, 256x256); {B} (scan, projection) items per "
                        f"step (autotuned over 32, 64, 128), {per_scan} per scan, one launch per stage, "
                        "CUDA-graph-replayed step",
            "value": batched, "unit": UNIT, "plain_per_projection": plain, "speedup": batched / plain,
            "tile": tuned["tile"], "bwd_lanes": tuned["bwd_lanes"], "autotune_trials": tuned["trials"],
            "device_status": status}


def model_comparison(pkg, wl, device, tile, lanes, B=16, reps=10):
    """The exact line-integral model against the paper's 2D-Gaussian (EWA) model on one batch of the
    workload: forward + backward throughput (CUDA events; the backward reuses the forward's records) and
    the relative L2 difference of the two models' projections."""
    import torch
    f = lambda a: torch.as_tensor(a, dtype=torch.float32, device=device).contiguous()
    ids = batch_ids(0, B, len(wl.views))
    views = [wl.views[i] for i in ids]
    ins = [f(wl.mu0), f(wl.scale), f(wl.quat), f(wl.rho), f(wl.phi), f(wl.w[ids])]
    gp = torch.randn(B, 256, 256, device=device, generator=torch.Generator(device=device).manual_seed(0))
    out, imgs = {}, {}
    for name, ewa in (("exact", False), ("ewa", True)):
        pj = pkg.Projector(wl.lattice, views, tile=tile, device=device, bwd_lanes=lanes, ewa=ewa)
        I = pj.forward(*ins)
        pj.backward(*ins, gp, reuse=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            pj.forward(*ins, out=I)
            pj.backward(*ins, gp, reuse=True)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"proj_per_s_fwd_bwd": reps * B / (e0.elapsed_time(e1) / 1e3), "status": pj.status()}
        imgs[name] = I.clone()
    out["rel_l2_ewa_vs_exact"] = float((imgs["ewa"] - imgs["exact"]).norm() / imgs["exact"].norm())
    out["workload"] = f"{B} projections of the thorax workload, projector forward + backward"
    return out


def warmstart_measurement(pkg, D, wl, meas, device, tile, lanes, B=16, warmup_iters=150, max_iters=6000,
                          plateau_steps=504, plateau_rel=0.01, variants=((10_000, 3, 128),)):
    """Wall time for the plain batched optimisation to reach its plateau -- the full-scan loss changes by
    less than `plateau_rel` over `plateau_steps` steps -- against the learned warm start (render training
    pairs with the model, train the CNN, propose all weights, keep them if the scan loss falls) followed by
    the same optimisation until its scan loss is within 1 % of the plain plateau loss.  Both start from the
    same state after a short plain warm-up and share the learning-rate schedule (linear over max_iters);
    each variant (training pairs, epochs, render resolution) starts its own warm run from that state.
    Wall times exclude the scan-loss evaluations, which are timed and reported separately."""
    import torch
    import synth
    from paper_2506_22280_gb300 import warmstart as WS
    n_proj = len(wl.views)
    init = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho, phi=wl.phi, w=wl.w, lattice=wl.lattice)
    rec = make_rec_factory(pkg, D, init, device, total=warmup_iters + max_iters)(tile, lanes)
    plan = [batch_ids(s, B, n_proj) for s in range(warmup_iters + max_iters)]

    def step(r, s):
        ids = plan[s]
        r.step(meas[torch.as_tensor(ids, device=device)].contiguous(), ids, [wl.views[i] for i in ids])

    def timed_loss(r):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L = WS.scan_loss(r, meas, wl.views, r.w)
        return L, time.perf_counter() - t0

    for s in range(warmup_iters):
        step(rec, s)
    plain = rec.clone()
    chunk = n_proj // B                      # 42 steps: one pass over the scan
    every = max(1, plateau_steps // chunk)   # scan loss every 12 passes (504 steps)
    curve, t_plain, t_eval_plain, iters = [], 0.0, 0.0, 0
    torch.cuda.synchronize()
    while iters < max_iters:
        t0 = time.perf_counter()
        for k in range(iters, min(iters + chunk * every, max_iters)):
            step(plain, warmup_iters + k)
        torch.cuda.synchronize()
        t_plain += time.perf_counter() - t0
        iters = min(iters + chunk * every, max_iters)
        L, te = timed_loss(plain)
        t_eval_plain += te
        curve.append([iters, round(t_plain, 3), L])
        if len(curve) >= 2 and curve[-2][2] - L < plateau_rel * L:
            break
    final = curve[-1][2]
    target = 1.01 * final
    out = []
    for n_pairs, epochs, render_res in variants:
        warm = rec.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pred = pkg.WeightPredictor(int(wl.lattice["R"]), seed=0, input_scale=0.25)
        pitch = 1.6 * 256 / render_res  # the same 409.6 mm detector
        make_views = lambda a: synth.circular_views(a, 1000.0, 1500.0, render_res, render_res, pitch, pitch)
        imgs, cs, W = WS.render_training_pairs(warm, make_views, n_pairs, pred, seed=1)
        torch.cuda.synchronize()
        t_render = time.perf_counter() - t0
        sel = WS.train_and_propose(pred, imgs, cs, W, epochs, warm, meas, wl.views, np.asarray(wl.angles),
                                   batch=256, lr=3e-4)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0 - t_render
        losses = sel["history"]
        res = WS.warm_start(warm, pred, meas, wl.views, np.asarray(wl.angles), list(range(n_proj)),
                            proposal=sel["proposal"])
        torch.cuda.synchronize()
        t_cnn = time.perf_counter() - t0
        del imgs, cs, W
        t_warm, t_eval_warm, k, reached, wcurve = t_cnn, 0.0, 0, None, []
        while k < iters:
            t0 = time.perf_counter()
            for s in range(k, min(k + chunk, iters)):
                step(warm, warmup_iters + s)
            torch.cuda.synchronize()
            t_warm += time.perf_counter() - t0
            k = min(k + chunk, iters)
            L, te = timed_loss(warm)
            t_eval_warm += te
            wcurve.append([k, round(t_warm, 3), L])
            if L <= target:
                reached = k
                break
        status = max(plain.status(), warm.status())
        out.append({"protocol": (f"{warmup_iters} shared plain steps, then plain until the scan loss changes by < "
                                 f"{100 * plateau_rel:g} % over {chunk * every} steps vs CNN warm start ({n_pairs} pairs "
                                 f"rendered at {render_res}x{render_res}" + (", 2x2-averaged" if render_res == 256 else "")
                                 + f", up to {epochs} epochs at learning rate 3e-4, the epoch whose proposal has the "
                                 "lowest scan loss, BF16 inference, accept if the scan loss falls) + the same steps "
                                 f"until the scan loss is within 1% of the plain plateau; B = {B}, wall time; scan-loss "
                                 "evaluations excluded (reported as eval_s)"),
                    "plain_s": t_plain, "plain_steps": iters, "plain_final_scan_loss": final,
                    "warm_s": t_warm if reached else None, "cnn_s": t_cnn, "cnn_render_s": t_render,
                    "cnn_train_s": t_train, "warm_steps_to_target": reached,
                    "speedup": (t_plain / t_warm) if reached else None,
                    "eval_s": {"plain": t_eval_plain, "warm": t_eval_warm},
                    "accepted": res["accepted"], "scan_loss_before": res["loss_plain"],
                    "scan_loss_proposal": res["loss_proposal"], "proposal_epoch": sel["epoch"],
                    "cnn_epochs": losses, "plain_curve": curve,
                    "warm_curve": wcurve, "device_status": status})
        del warm, pred
    return out


def density_measurement(rec, plan, mb, views, varrs, T0, steps=8, quantile=0.9):
    """Adaptive density control on a copy of the bench state: the step with the statistic switched on
    against the same step without it, then one densify (plan, new cloud, moments) with the threshold at the
    statistic's 90th percentile; wall time around the densify, which reads the new size back to the host."""
    import torch
    r = rec.clone()
    r.enable_density_stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = {}
    for mode in ("with_statistic", "without_statistic"):
        if mode == "without_statistic":
            r.state.dens_grad = None
        torch.cuda.synchronize()
        e0.record()
        for s in range(steps):
            r.step(mb[T0 + s], plan[T0 + s], views[T0 + s], varr=varrs[T0 + s])
        e1.record()
        torch.cuda.synchronize()
        times[mode] = e0.elapsed_time(e1) / steps
    r.state.dens_grad = r.dens_grad.data_ptr()
    r.dens_projections = steps * len(plan[T0])  # the statistic summed over the first pass's projections
    stat = r.dens_grad / r.dens_projections
    tau = float(torch.quantile(stat, quantile).item())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = r.densify(tau=tau, s_split=4.0, rho_min=1e-5, generator=torch.Generator(device=r.mu0.device).manual_seed(0))
    torch.cuda.synchronize()
    t_dens = time.perf_counter() - t0
    loss = float(r.step(mb[T0], plan[T0], views[T0], varr=varrs[T0]).item())
    return {"step_ms_with_statistic": times["with_statistic"], "step_ms_without_statistic": times["without_statistic"],
            "densify_ms": t_dens * 1e3, "tau": tau, **info, "loss_after": loss, "device_status": r.status()}


def cnn_gemm_flops(B, R=3):
    """FLOPs of the weight-predictor CNN's GEMMs in one training step of batch B: the forward (four
    convolutions as im2col GEMMs, the 8194-wide and the R-wide layers), the weight gradients of all six
    and the data gradients of all but the first convolution."""
    ch, edge, k_feat, hid = [1, 32, 64, 128, 128], [128, 64, 32, 16, 8], 8194, 128
    fwd = dw = dx = 0
    for l in range(4):
        mnk = B * edge[l + 1] ** 2 * ch[l + 1] * 9 * ch[l]
        fwd += 2 * mnk
        dw += 2 * mnk
        dx += 2 * mnk if l > 0 else 0
    for a, b in ((k_feat, hid), (hid, R)):
        fwd += 2 * B * a * b
        dw += 2 * B * a * b
        dx += 2 * B * a * b
    return fwd + dw + dx


def cnn_measurement(pkg, device, B=256, R=3, reps=20):
    """CUDA-event times of one CNN training step (batch B) with the tensor-core GEMMs and with FP32 SIMT
    GEMMs, and of BF16 inference on 680 projections; the tensor-core step's GEMM work in TFLOP/s against
    the measured dense BF16 peak."""
    import torch
    rng = np.random.default_rng(0)
    img = torch.tensor(rng.uniform(size=(B, 128, 128)).astype(np.float32), device=device)
    cs = torch.tensor(rng.normal(size=(B, 2)).astype(np.float32), device=device)
    W = torch.tensor(rng.normal(size=(B, R)).astype(np.float32), device=device)
    out = {"batch": B}
    for tc in (True, False):
        net = pkg.WeightPredictor(R, seed=0, tensor_cores=tc, device=device)
        for _ in range(3):
            net.train_step(img, cs, W, 1e-3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            net.train_step(img, cs, W, 1e-3)
        e1.record()
        torch.cuda.synchronize()
        out["train_step_ms_tensor_cores" if tc else "train_step_ms_fp32_simt"] = e0.elapsed_time(e1) / reps
    imgs = torch.tensor(rng.uniform(size=(680, 128, 128)).astype(np.float32), device=device)
    css = torch.tensor(rng.normal(size=(680, 2)).astype(np.float32), device=device)
    net.predict(imgs, css)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    net.predict(imgs, css)
    e1.record()
    torch.cuda.synchronize()
    out["infer_680_ms"] = e0.elapsed_time(e1)
    flops = cnn_gemm_flops(B, R)
    achieved = flops / (out["train_step_ms_tensor_cores"] / 1e3) / 1e12
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = float(peaks.get("bf16_tflops", 1900.0))
    out["train_step_speedup"] = out["train_step_ms_fp32_simt"] / out["train_step_ms_tensor_cores"]
    out["roofline"] = {"bound": "tensor", "kernel": "k_gemm_tc (whole training step)", "achieved": achieved,
                       "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                       "peak_basis": "measured dense BF16 burst" if "bf16_tflops" in peaks else "fallback 1.9 PFLOP/s",
                       "flops_per_step": flops}
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    import paper_2506_22280_gb300 as pkg
    from paper_2506_22280_gb300 import digs as D
    from paper_2506_22280_gb300 import autotune
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if args.only_cnn:
        if rank == 0:
            print(json.dumps({"cnn": cnn_measurement(pkg, device)}), flush=True)
        return
    if world > 1:
        dist.init_process_group("nccl", device_id=device)
    pkg.lib()
    wl = synth.thorax(seed=1 + 101 * rank, n=args.n)
    n_proj = len(wl.views)
    meas = render_measured(pkg, wl, device)
    K, W = args.steps, args.warmup
    init = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho, phi=wl.phi, w=wl.w, lattice=wl.lattice)
    make = make_rec_factory(pkg, D, init, device)

    def tune_batch(b, s):
        ids = batch_ids(s, b, n_proj)
        return meas[torch.as_tensor(ids, device=device)].contiguous(), ids, [wl.views[i] for i in ids]

    # launch shape (tile, backward lanes, projections per step): the autotuner's pick unless given
    tuned = None
    if args.tile and args.lanes and args.batch:
        tile, lanes, B = args.tile, args.lanes, args.batch
    else:
        first = args.batch or 16
        tuned = autotune.tune(make, tune_batch, tiles=(args.tile,) if args.tile else (8, 16, 32),
                              lanes=(args.lanes,) if args.lanes else (16, 32),
                              batch_sizes=(first,) if args.batch else (16, 8, 32, 64, 128), steps=2, warmup=1)
        tile, lanes, B = tuned["tile"], tuned["bwd_lanes"], tuned["batch"]
    plan = [batch_ids(s, B, n_proj) for s in range(W + K + 8)]
    views = [[wl.views[i] for i in ids] for ids in plan]
    varrs = [D.views_array(v) for v in views]
    mb = [meas[torch.as_tensor(ids, device=device)].contiguous() for ids in plan]
    peaks = pipe_peaks(local)
    rec = make(tile, lanes)
    for s in range(W):
        rec.step(mb[s], plan[s], views[s], varr=varrs[s])
    torch.cuda.synchronize()
    if rec.status() != 0:
        raise RuntimeError("device status after warm-up: %d" % rec.status())
    # stage times (CUDA events around each stage, on the launching stream) from direct calls
    n_stage = min(K, 5)
    stages = {k: 0.0 for k in D.STAGES}
    l0 = D.kernel_launches()
    for s in range(n_stage):
        rec.step(mb[W + s], plan[W + s], views[W + s], time_stages=True, varr=varrs[W + s])
        st = D.stage_times()
        for k in stages:
            stages[k] += st[k] / n_stage
    launches_per_step = (D.kernel_launches() - l0) // n_stage
    T0 = W + n_stage
    use_graph = not args.no_graph
    if use_graph:
        graphs = rec.capture([(mb[T0 + s], plan[T0 + s], views[T0 + s]) for s in range(K)])
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    clocks = ClockSampler(visible_gpu_index(local))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.profiler.start()  # ncu --profile-from-start off captures the timed steps only
    t_wall0 = time.perf_counter()
    for s in range(K):
        flush.fill_(float(s))
        e0, e1 = ev[s]
        e0.record()
        if use_graph:
            graphs[s].replay()
        else:
            rec.step(mb[T0 + s], plan[T0 + s], views[T0 + s], varr=varrs[T0 + s])
        e1.record()
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    dev_ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    status = rec.status()
    # pair statistics of one forward of the last batch (for the roofline's algorithmic work)
    pj = pkg.Projector(wl.lattice, views[T0 + K - 1], tile=tile, device=device)
    ins = [rec.mu0, rec.scale, rec.quat, rec.rho, rec.phi,
           rec.w[torch.as_tensor(plan[T0 + K - 1], device=device)].contiguous()]
    pj.forward(*ins)
    pairs = D.pair_stats(pj.ws)
    # end to end: pinned host measured projections -> device, step, loss -> host
    e2e = None
    if not args.no_e2e:
        # every step copies its measured projections from pinned host memory (on a copy stream, into one of
        # two device buffers, so that step s + 1's copy overlaps step s) and reads its loss back to the host
        # (step s's loss is read once step s + 1 has been launched)
        host = [m.cpu().pin_memory() for m in mb[T0:T0 + K]]
        bufs = [torch.empty_like(mb[0]) for _ in range(2)]
        # as in the device-timed loop, each step is a replay of its captured graph (which reads the device
        # input buffer its copy lands in)
        graphs_e2e = rec.capture([(bufs[s % 2], plan[T0 + s], views[T0 + s]) for s in range(K)]) if use_graph else None
        loss_host = torch.empty(K, dtype=torch.float32).pin_memory()
        copy_stream = torch.cuda.Stream(device=device)
        main = torch.cuda.current_stream(device)
        copied = [torch.cuda.Event() for _ in range(2)]
        used = [torch.cuda.Event() for _ in range(2)]
        read = [torch.cuda.Event() for _ in range(K)]
        losses = []

        def copy_in(s):
            b = s % 2
            with torch.cuda.stream(copy_stream):
                if s >= 2:
                    copy_stream.wait_event(used[b])  # step s - 2 has finished with this buffer
                bufs[b].copy_(host[s], non_blocking=True)
                copied[b].record(copy_stream)

        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        copy_in(0)
        for s in range(K):
            if s + 1 < K:
                copy_in(s + 1)
            main.wait_event(copied[s % 2])
            if graphs_e2e is not None:
                graphs_e2e[s].replay()
                loss = rec.loss
            else:
                loss = rec.step(bufs[s % 2], plan[T0 + s], views[T0 + s], varr=varrs[T0 + s])
            used[s % 2].record(main)
            loss_host[s:s + 1].copy_(loss.reshape(-1)[:1], non_blocking=True)
            read[s].record(main)
            if s >= 1:
                read[s - 1].synchronize()
                losses.append(float(loss_host[s - 1]))
        read[K - 1].synchronize()
        losses.append(float(loss_host[K - 1]))
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        if not all(math.isfinite(v) for v in losses):
            raise RuntimeError("non-finite loss in the end-to-end steps")
    dev_ms, t_wall, e2e_s = reduce_timings([dev_ms, t_wall, e2e_s if not args.no_e2e else 0.0], world, device)
    batching = None
    if world == 1 and not args.no_batching:
        batching = batching_measurement(pkg, D, device)
    models = None
    if world == 1 and not args.no_batching:
        models = model_comparison(pkg, wl, device, tile, lanes, B=B)
    warm = warm_cfg = cnn = dens = None
    if world == 1 and not args.no_batching:
        dens = density_measurement(rec, plan, mb, views, varrs, T0)
    if world == 1 and not args.no_warmstart:
        # the bench's protocol (10k pairs rendered at the network's 128 x 128), then the workload's stated one
        # (20k pairs rendered at 256 x 256 and 2 x 2-averaged), both from the same plain run
        warm, warm_cfg = warmstart_measurement(pkg, D, wl, meas, device, tile, lanes,
                                               variants=((10_000, 4, 128), (20_000, 4, 256)))
        cnn = cnn_measurement(pkg, device)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    total_proj = world * B * K
    value = whole_job_rate(world, B, K, dev_ms)
    if not args.no_e2e:
        e2e = {"value": total_proj / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(mb[0].numel() * 4),
               "d2h_bytes_per_step": 4}
    # rooflines: each raster kernel against the measured FP32 / SFU peaks, and the whole step (fused
    # forward + backward) against the same peaks and the measured HBM bandwidth
    mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm = float(mp.get("hbm_gbs", 6800.0)) * 1e9
    kernels = {k: kernel_roofline(k, pairs["cutoff_pairs"], stages[k], peaks, traffic_for("k_" + k, B, tile, lanes))
               for k in ("raster_fwd", "raster_bwd")}
    dom = max(kernels, key=lambda k: stages[k])
    roofline = dict(kernels[dom], box_pairs_per_launch=pairs["box_pairs"], tile_pairs_per_launch=pairs["tile_pairs"])
    fp32_ops, sfu_ops, nbytes = step_work(pairs["cutoff_pairs"], B, args.n, int(wl.lattice["R"]),
                                          wl.views[0]["nu"] * wl.views[0]["nv"])
    times = {"fp32": fp32_ops / peaks["fp32_per_s"], "sfu": sfu_ops / peaks["sfu_per_s"], "hbm": nbytes / hbm}
    bound = max(times, key=times.get)
    step_roofline = {"bound": bound, "roofline_ms_per_step": times[bound] * 1e3, "ms_per_step": dev_ms / K,
                     "frac": times[bound] * 1e3 / (dev_ms / K), "fp32_ops_per_step": fp32_ops,
                     "sfu_ops_per_step": sfu_ops, "algorithmic_bytes_per_step": nbytes,
                     "pipe_ms": {k: v * 1e3 for k, v in times.items()},
                     "roofline_projections_per_s": B / times[bound],
                     "basis": ("FP32 and SFU peaks measured by digs_pipe_bench in this run; HBM = measured copy "
                               f"bandwidth {hbm / 1e9:.0f} GB/s; in-cutoff pairs counted by the forward raster")}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": dev_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": (f"synthetic thorax, {args.n} Gaussians, 256x256 detector (1.6 mm), R=3, "
                                    f"lattice 19^3 at 16 mm, 680-projection scan; {B} projections per step "
                                    "(fwd + bwd + Adam)"),
                       "batch_projections": B, "tile": tile, "bwd_lanes": lanes,
                       "launch": "CUDA-graph replay of the whole step" if use_graph else "direct calls",
                       "autotuned": tuned is not None, "l2": "flushed between steps (512 MB write)",
                       "parallelism": f"{world} independent scans (replicas)", "wall_s_timed": t_wall},
            "roofline": roofline, "step_roofline": step_roofline, "kernel_rooflines": kernels, "pipe_peaks": peaks,
            "e2e": e2e, "gpu_launches": launches_per_step * K, "clocks": clk,
            "stages_ms_per_step": stages, "device_status": status}
    if tuned is not None:
        line["config"]["autotune_trials"] = tuned["trials"]
    if batching is not None:
        line["batching"] = batching
        line["batching_speedup"] = batching["speedup"]
    if warm is not None:
        line["warm_start"] = warm
        line["warm_start_stated_protocol"] = warm_cfg
        line["warm_start_speedup"] = warm.get("speedup")
        line["warm_start_speedup_stated"] = warm_cfg.get("speedup")
    if cnn is not None:
        line["cnn"] = cnn
    if dens is not None:
        line["density_control"] = dens
    if models is not None:
        line["projection_models"] = models
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_reference(args):
    """The FP64 CPU oracle as it stands, timed on the machine's host cores: each step is one full projection
    (forward + backward) of the 100k-Gaussian thorax workload."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import torch
    import synth
    from oracle import digs_oracle as O
    wl = synth.thorax(seed=1, n=args.n)
    steps = []
    for s in range(args.warmup + args.steps):
        sub = wl.select_views([batch_ids(s, 1, len(wl.views))[0]])
        g = dict(mu0=sub.mu0, scale=sub.scale, quat=sub.quat, rho=sub.rho)
        gp = synth.random_grad_proj(1, 256, 256, seed=s)
        t0 = time.perf_counter()
        O.project_vjp(g, sub.lattice, sub.phi, sub.w, sub.views, gp)
        if s >= args.warmup:
            steps.append(time.perf_counter() - t0)
    t = sum(steps)
    value = len(steps) / t
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / len(steps), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"synthetic thorax, {args.n} Gaussians, 256x256 detector, R=3; one full "
                                   "projection fwd + bwd per step (nothing sampled or scaled)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"{len(steps)} steps x 1 projection x {args.n} Gaussians"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
