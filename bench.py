"""Benchmark: Stage-1 NTC training on the 250K-Gaussian, 20-view multi-view
video workload (1352x1014, 4 views per launch), plus the rasterizer
fwd+bwd throughput and the plain FP32 direct-optimisation path on the same
GPU, and the FP64 CPU oracle on a bounded sample.

One "step" is one Stage-1 iteration: NTC query of all Gaussians,
transformation, projection + binning + sort + compositing of a batch of 4
views, L1 + D-SSIM loss, backward into the hash table and MLP, Adam.  A
frame is 150 iterations (Section 5.2); the headline value is seconds per
frame.  Inputs are seeded synthetic scenes (the N3DV videos are not
available) resident in HBM; the per-iteration working set (pair buffers of
~0.5 GB) exceeds the 129 MB L2, so no flush is needed between iterations.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

METRIC = "NTC train s/frame @250K 3DGs, 20 views; raster fwd+bwd it/s vs FP32 plain"
ITERS_PER_FRAME = 150
CFG_INDEX = 3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=ITERS_PER_FRAME)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mlp", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-oracle-configs", action="store_true",
                    help="skip the oracle timings of the other workloads")
    ap.add_argument("--small", action="store_true",
                    help="100K Gaussians instead of 250K (smaller profiling captures)")
    ap.add_argument("--warm-iters", type=int, default=1000, help="NTC warm-up iterations (Eq. 7)")
    ap.add_argument("--eager", action="store_true", help="launch kernels one by one (no CUDA graph)")
    ap.add_argument("--no-converge", action="store_true", help="skip the equal-PSNR comparison")
    ap.add_argument("--no-render", action="store_true", help="skip the render-only measurement")
    ap.add_argument("--no-stage2", action="store_true", help="skip the Stage-2 measurement")
    ap.add_argument("--no-large", action="store_true", help="skip the 1M-Gaussian, 16-view run")
    ap.add_argument("--stream-frames", type=int, default=30,
                    help="frames of the streaming run (0: skip)")
    ap.add_argument("--bin", type=int, default=0,
                    help="bin side in tiles (0: autotune over 1, 2, 4, 8, 16)")
    ap.add_argument("--profile", action="store_true",
                    help="setup + timed steps only (for ncu launch lists)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(scene, n_sample_gauss=None, views=1):
    """Time the FP64 oracle's Stage-1 step on a bounded sample of the
    workload: every Gaussian through the cache and transformation, and the
    render + loss + backward of `views` of the 4 views of a batch.  Returns
    (seconds per full 4-view iteration, description, threads)."""
    import oracle
    oracle.build()
    cfg = scene.cfg
    g = scene.prev
    cams = scene.cams[:views]
    og = oracle.Grid()
    rng = np.random.default_rng(0)
    from paper_2403_01444_gb300 import scenes
    table = rng.uniform(-1e-4, 1e-4, size=(og.n_entries, 2))
    Ws = scenes.random_mlp([32, 64, 64, 7], rng)
    Ws[2][3] = np.abs(Ws[2][3]) + 1.0
    p = oracle.NTCParams(og, table, Ws)
    targets = np.random.default_rng(1).uniform(size=(views, 3, cfg.H, cfg.W))
    t0 = time.perf_counter()
    f = oracle.ntc_forward(p, g.mean, g.quat)
    t_ntc_f = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = oracle.render(g, cams, f["mean"], f["quat"])
    L, d_img, _ = oracle.loss_l1_dssim(r["img"], targets)
    grads = oracle.raster_bwd(r["proj"], cfg.W, cfg.H, r["T_final"], r["last"], d_img)
    dm, dq = oracle.project_bwd(g, cams, grads, mean=f["mean"], quat=f["quat"])
    t_view = (time.perf_counter() - t0) / views
    t0 = time.perf_counter()
    d_raw7 = oracle.apply_bwd(g.mean, g.quat, f["raw7"], og.aabb, dm, dq)
    dWs, d_enc = oracle.mlp_bwd(f["enc"], p.Ws, f["h1"], f["h2"], d_raw7)
    oracle.encode_bwd(og, g.mean, d_enc)
    t_ntc_b = time.perf_counter() - t0
    per_iter = t_ntc_f + t_ntc_b + cfg.views_per_batch * t_view
    desc = ("FP64 oracle, all %d Gaussians through NTC fwd/bwd + %d of the 4 views rendered, "
            "loss, backward (%.1f s); per-iteration time = NTC + 4 x per-view time"
            % (g.n, views, t_ntc_f + t_ntc_b + views * t_view))
    return per_iter, desc, oracle.num_threads()


def oracle_configs(budget_s=90.0):
    """The FP64 oracle on the other workloads, on the host cores: the plain
    method on the 4 096-Gaussian scene (all 50 direct-optimisation
    iterations), the cache on the 50K-Gaussian scene (one Stage-1 iteration,
    x 150 for a frame), and one 2-view forward + backward of the 500K and 1M
    Gaussian scenes.  Each entry says what it timed; entries are skipped once
    `budget_s` of CPU time is spent."""
    import oracle
    from paper_2403_01444_gb300 import scenes
    oracle.build()
    out = {"cores": oracle.num_threads()}
    spent = 0.0

    def fwd_bwd(g, cams, targets, mean=None, quat=None):
        r = oracle.render(g, cams, mean, quat)
        L, d_img, _ = oracle.loss_l1_dssim(r["img"], targets)
        gr = oracle.raster_bwd(r["proj"], cams[0].W, cams[0].H, r["T_final"], r["last"], d_img)
        return oracle.project_bwd(g, cams, gr, mean=mean, quat=quat)

    # config 1: plain FP32 method, every iteration
    sc = scenes.make_scene(1)
    g, cams = sc.prev, sc.cams
    tg = oracle.render(sc.target, cams)["img"]
    m, q = g.mean.astype(np.float64).copy(), g.quat.astype(np.float64).copy()
    mm, vm, mq, vq = (np.zeros_like(x) for x in (m, m, q, q))
    t0 = time.perf_counter()
    for it in range(sc.cfg.iters):
        dm, dq = fwd_bwd(g, cams, tg, m, q)
        oracle.adam(m, dm, mm, vm, it + 1, lr=0.0024, b2=0.999)
        oracle.adam(q, dq, mq, vq, it + 1, lr=0.015, b2=0.999)
    t = time.perf_counter() - t0
    spent += t
    out["plain-fp32-4k"] = {"s": t, "timed": "all %d direct-optimisation iterations, 4 views of "
                            "128x96, 4096 Gaussians" % sc.cfg.iters}
    # config 2: one Stage-1 iteration of the cache, a frame is 150
    sc = scenes.make_scene(2)
    og = oracle.Grid()
    rng = np.random.default_rng(0)
    p = oracle.NTCParams(og, rng.uniform(-1e-4, 1e-4, size=(og.n_entries, 2)),
                         scenes.random_mlp([32, 64, 64, 7], rng))
    p.Ws[2][3] = np.abs(p.Ws[2][3]) + 1.0
    tg = np.random.default_rng(1).uniform(size=(len(sc.cams), 3, sc.cfg.H, sc.cfg.W))
    t0 = time.perf_counter()
    oracle.stage1_loss_grads(p, sc.prev, sc.cams, tg)
    t = time.perf_counter() - t0
    spent += t
    out["ntc-50k-8v-480x360"] = {"s_per_iter": t, "s_per_frame": 150 * t,
                                 "timed": "one Stage-1 iteration (cache, 8 views, loss, backward); "
                                          "frame = 150 x"}
    # configs 4 and 5: one 2-view forward + backward
    for idx in (4, 5):
        name = scenes.CONFIGS[idx].name
        if spent > budget_s:
            out[name] = {"skipped": "CPU budget of %.0f s spent" % budget_s}
            continue
        sc = scenes.make_scene(idx)
        cams = sc.cams[:2]
        tg = np.random.default_rng(1).uniform(size=(2, 3, sc.cfg.H, sc.cfg.W))
        t0 = time.perf_counter()
        fwd_bwd(sc.prev, cams, tg)
        t = time.perf_counter() - t0
        spent += t
        out[name] = {"s": t, "timed": "one forward + backward of 2 views (%dx%d, %d Gaussians)"
                     % (sc.cfg.W, sc.cfg.H, sc.prev.n)}
    return out


def run_reference(args):
    """The reference arm: the FP64 oracle, as it stands, on the host cores.
    A Stage-1 iteration is split into five bounded units and each step runs
    one of them, in turn: the cache forward + backward of all Gaussians
    (steps k with k % 5 == 0), or the render, loss and backward of one view
    of the current 4-view batch (the batches cycle through the 20 cameras).
    An iteration is the mean cache unit plus four mean view units."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2403_01444_gb300 import scenes
    oracle.build()
    scene = scenes.make_scene(CFG_INDEX)
    cfg, g = scene.cfg, scene.prev
    Vb, nb = cfg.views_per_batch, cfg.n_cams // cfg.views_per_batch
    og = oracle.Grid()
    rng = np.random.default_rng(0)
    table = rng.uniform(-1e-4, 1e-4, size=(og.n_entries, 2))
    Ws = scenes.random_mlp([32, 64, 64, 7], rng)
    Ws[2][3] = np.abs(Ws[2][3]) + 1.0
    p = oracle.NTCParams(og, table, Ws)
    f_all = oracle.ntc_forward(p, g.mean, g.quat)           # set-up, not timed
    targets = np.random.default_rng(1).uniform(size=(cfg.n_cams, 3, cfg.H, cfg.W))
    grads_rng = np.random.default_rng(2)

    def step(k):
        unit = k % (Vb + 1)
        if unit == 0:
            dm, dq = grads_rng.normal(size=(g.n, 3)), grads_rng.normal(size=(g.n, 4))
            t0 = time.perf_counter()
            f = oracle.ntc_forward(p, g.mean, g.quat)
            d_raw7 = oracle.apply_bwd(g.mean, g.quat, f["raw7"], og.aabb, dm, dq)
            _, d_enc = oracle.mlp_bwd(f["enc"], p.Ws, f["h1"], f["h2"], d_raw7)
            oracle.encode_bwd(og, g.mean, d_enc)
            return 0, time.perf_counter() - t0
        v = ((k // (Vb + 1)) % nb) * Vb + unit - 1
        cam = [scene.cams[v]]
        t0 = time.perf_counter()
        r = oracle.render(g, cam, f_all["mean"], f_all["quat"])
        L, d_img, _ = oracle.loss_l1_dssim(r["img"], targets[v:v + 1])
        gr = oracle.raster_bwd(r["proj"], cfg.W, cfg.H, r["T_final"], r["last"], d_img)
        oracle.project_bwd(g, cam, gr, mean=f_all["mean"], quat=f_all["quat"])
        return 1, time.perf_counter() - t0

    for k in range(args.warmup):
        step(k)
    times = {0: [], 1: []}
    t_start = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        unit, t = step(k)
        times[unit].append(t)
    wall = time.perf_counter() - t_start
    if not times[0]:   # fewer steps than one cycle: time one cache unit
        times[0].append(step(0)[1])
    if not times[1]:
        times[1].append(step(1)[1])
    per_iter = float(np.mean(times[0])) + Vb * float(np.mean(times[1]))
    s_frame = per_iter * ITERS_PER_FRAME
    desc = ("FP64 oracle; %d steps, each one unit of a Stage-1 iteration on all %d Gaussians: "
            "the cache forward + backward, or one view's render + loss + backward; iteration = "
            "cache unit + %d view units; %.1f s of CPU" % (args.steps, g.n, Vb, wall))
    cores = oracle.num_threads()
    ms_step = 1e3 * wall / max(args.steps, 1)
    line = {"impl": "reference", "metric": METRIC, "value": s_frame, "unit": "s/frame",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "ms_per_iteration": per_iter * 1e3,
            "step": "one unit of a Stage-1 iteration (the cache forward + backward, or one "
                    "view's render + loss + backward); an iteration is %d units" % (Vb + 1),
            "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(scene, "single"),
            "cpu_baseline": {"value": s_frame, "unit": "s/frame", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": s_frame, "unit": "s/frame", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_dict(scene, parallelism):
    cfg = scene.cfg
    return {"workload": "ntc-stage1 250K Gaussians SH3, 20 cams 1352x1014, 4 views/launch, "
                        "150 it/frame (synthetic N3DV stand-in)",
            "gaussians": cfg.n_gauss, "sh_degree": cfg.sh_deg, "cameras": cfg.n_cams,
            "width": cfg.W, "height": cfg.H, "views_per_step": cfg.views_per_batch,
            "iters_per_frame": ITERS_PER_FRAME, "hash_grid": "16x2, 2^17, 16..1024",
            "mlp": "32-64-64-7", "parallelism": parallelism,
            "l2": "inputs larger than L2 (no flush)"}


def aggregate_timing(ms, world, device):
    """Max over ranks of the time per step (every rank has passed the same
    barrier-bracketed region) and the whole-job seconds per frame: each rank
    trains its own frames, so the job finishes world frames per max time."""
    import torch
    t = torch.tensor([float(ms)], device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, ms_max * ITERS_PER_FRAME / 1e3 / world


# ------------------------------------------------------------------ GPU arm
def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = "cuda"
    from paper_2403_01444_gb300 import build as _b
    _b.build()
    from paper_2403_01444_gb300 import gs3, scenes
    from paper_2403_01444_gb300.engine import (TargetFeeder, NTC, DirectOpt, Rasterizer, Renderer, Stage1,
                                               autotune_bin, warmup)

    if args.small:
        scene = scenes.make_scene(CFG_INDEX, n_gauss=100_000)
    else:
        scene = scenes.make_scene(CFG_INDEX)
    cfg = scene.cfg
    W, H, Vb = cfg.W, cfg.H, cfg.views_per_batch
    nb = cfg.n_cams // Vb
    G = gs3.Gaussians.from_numpy(scene.prev)
    Gt = gs3.Gaussians.from_numpy(scene.target)
    cams_dev = gs3.cameras_to_device(scene.cams)
    batch_cams = [gs3.camera_slice(cams_dev, b * Vb, Vb) for b in range(nb)]
    # ground-truth views (rendered once by the FP32 rasterizer)
    rt = Rasterizer(Gt.n, Vb, W, H, 1 << 24, dev)
    targets = torch.empty(cfg.n_cams, 3, H, W, device=dev)
    for b in range(nb):
        rt.fit_capacity(Gt, batch_cams[b], margin=1.2)
        targets[b * Vb:(b + 1) * Vb].copy_(rt.img)
    del rt
    torch.cuda.empty_cache()
    # NTC: I-NGP-style init, then the warm-up towards the identity (Eq. 7)
    precision = gs3.GS_MLP_BF16 if args.mlp == "bf16" else gs3.GS_MLP_FP32
    rng = np.random.default_rng(7)
    grid = gs3.hashgrid()
    entries = gs3.ntc_hashgrid_entries(grid)
    table = rng.uniform(-1e-4, 1e-4, size=(entries, 2)).astype(np.float32)
    Ws = [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
    ntc = NTC(table, Ws, grid, precision, dev)
    t0 = time.perf_counter()
    wl = warmup(ntc, G, iters=args.warm_iters)
    torch.cuda.synchronize()
    t_warm = time.perf_counter() - t0
    warm_table, warm_mlp = ntc.table.p.clone(), ntc.mlp.p.clone()
    # bin size: autotuned on the first batch's fwd + bwd of compositing
    tune = None
    if args.bin > 0:
        bin_side = args.bin
    else:
        tmp = Stage1(G, ntc, Vb, W, H, capacity=1 << 20)
        mt, qt = tmp.transform()
        tune_ms, bin_side = autotune_bin(G, batch_cams[0], Vb, W, H, mt.clone(), qt.clone())
        tune = {"bin_tiles": {str(k): round(v, 4) for k, v in tune_ms.items()}, "best": bin_side,
                "timed": "project + bin/sort + raster fwd + raster bwd + project bwd, one 4-view batch"}
        del tmp, mt, qt
        torch.cuda.empty_cache()
    st = Stage1(G, ntc, Vb, W, H, capacity=1 << 20, bin=bin_side)
    counts = []
    for b in range(nb):
        counts.append(st.raster.fit_capacity(G, batch_cams[b], *st.transform(), margin=1.0))
    st.raster.set_capacity(int(max(counts) * 1.3))
    ntc.reset_to(warm_table, warm_mlp)
    st.reset_state()

    # one CUDA graph of the whole iteration per view batch
    batches = [(batch_cams[b], targets[b * Vb:(b + 1) * Vb]) for b in range(nb)]
    graphs = st.capture(batches) if not args.eager else None
    ntc.reset_to(warm_table, warm_mlp)
    st.reset_state()
    stream = torch.cuda.current_stream()
    ev = {}
    stats = torch.zeros(4, dtype=torch.int64, device=dev)
    count_pairs = False

    def step(i, record=False):
        if i % ITERS_PER_FRAME == 0:
            # every frame starts from the warm-up parameters, its Adam step
            # count (bias correction, rate schedule) from 0
            ntc.reset_to(warm_table, warm_mlp)
            st.reset_state()
        b = i % nb
        cd, tg = batch_cams[b], targets[b * Vb:(b + 1) * Vb]
        if not record:
            if graphs is not None:
                graphs[b].replay()
            else:
                st.step(cd, tg)
            return
        E = lambda k: ev.setdefault(k, []).append(torch.cuda.Event(enable_timing=True)) or ev[k][-1].record(stream)
        E("t0")
        st.transform()
        E("t1")
        gs3.gs_project(G, cd, Vb, W, H, st.raster.proj, st.mean_t, st.quat_t, None, st.raster.d_err)
        E("t2")
        r = st.raster
        gs3.gs_bin_sort(r.proj, G.n, Vb, W, H, r.bin, r.capacity, r.vals, r.ranges, None, r.d_count, r.d_err, r.ws)
        E("t3")
        gs3.gs_raster_fwd(r.proj, G.n, Vb, W, H, r.bin, r.bg, r.vals, r.ranges, r.img, r.T_final, r.last,
                          stats[0:2] if count_pairs else None, lists=r.lists)
        E("t4")
        st.loss(r.img, tg)
        E("t5")
        gs3.gs_raster_bwd(r.proj, G.n, Vb, W, H, r.bin, r.bg, r.vals, r.ranges, r.T_final, r.last,
                          st.loss.d_img, r.grads, None, stats[2:4] if count_pairs else None, lists=r.lists)
        E("t6")
        gs3.gs_project_bwd(G, cd, Vb, W, H, r.grads, r.d_mean, r.d_quat, st.mean_t, st.quat_t)
        E("t7")
        if st.fused:
            gs3.ntc_fused_bwd(G.mean, G.quat, st.raw7, st.enc, G.n, ntc.grid, ntc.mlp_struct(), st.order,
                              r.d_mean, r.d_quat, st.loss_scale_view(), ntc.mlp.g, ntc.table.g)
        else:
            gs3.ntc_apply_bwd(G.mean, G.quat, st.raw7, G.n, st.aabb, st.order, r.d_mean, r.d_quat, st.d_raw7)
            gs3.ntc_active_rows(st.d_raw7, G.n, st.active, st.n_active)
            gs3.ntc_mlp_bwd(st.enc, G.n, ntc.mlp_struct(), st.d_raw7, st.loss_scale_view(), ntc.mlp.g, st.d_enc,
                            rows=st.active, d_rows=st.n_active)
            gs3.ntc_encode_bwd(G.mean, G.n, ntc.grid, st.d_enc, ntc.table.g, order=st.active, d_count=st.n_active)
        E("t8")
        st.update()
        E("t9")

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    gs3.lib().gs_launch_count.restype = ctypes_u64()
    l0 = gs3.lib().gs_launch_count()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.warmup, args.warmup + args.steps):
            step(i)
        e1.record(stream)
        torch.cuda.synchronize()
    launches = gs3.lib().gs_launch_count() - l0
    if graphs is not None:
        # replays do not pass through the library: count one eager iteration
        c0 = gs3.lib().gs_launch_count()
        st.step(*batches[0])
        torch.cuda.synchronize()
        launches = (gs3.lib().gs_launch_count() - c0) * args.steps
    ms = e0.elapsed_time(e1) / args.steps
    # one whole frame timed on its own, whatever K is: the reset to the
    # warm-up parameters and 150 iterations
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for i in range(ITERS_PER_FRAME):
        step(i)
    f1.record(stream)
    torch.cuda.synchronize()
    full_frame_s = f0.elapsed_time(f1) / 1e3
    if args.profile:
        if rank == 0:
            print(json.dumps({"profile_run": True, "ms_per_step": ms, "gpu_launches": int(launches),
                              "pairs": st.raster.count()}), flush=True)
        return
    st.raster.check()
    ms_max, s_per_frame = aggregate_timing(ms, world, dev)

    # per-stage breakdown (separate, instrumented pass)
    ev.clear()
    for i in range(args.warmup + args.steps, args.warmup + args.steps + 10):
        step(i, record=True)
    torch.cuda.synchronize()
    # (pixel, Gaussian) pairs the compositing kernels evaluate in one step
    ev_keep = {k: list(v) for k, v in ev.items()}
    stats.zero_()
    count_pairs = True
    step(args.warmup + args.steps + 10, record=True)
    count_pairs = False
    torch.cuda.synchronize()
    ev = ev_keep
    pair_counts = [int(x) for x in stats.cpu().tolist()]
    names = ["ntc_fwd", "project", "bin_sort", "raster_fwd", "loss", "raster_bwd", "project_bwd",
             "ntc_bwd", "adam"]
    stages = {}
    for k, nm in enumerate(names):
        a, b = ev["t%d" % k], ev["t%d" % (k + 1)]
        stages[nm] = statistics.mean(x.elapsed_time(y) for x, y in zip(a, b))
    pairs = int(st.raster.count())

    # rasterizer fwd+bwd it/s: project + bin/sort + raster fwd + raster bwd + project bwd
    raster_ms = sum(stages[k] for k in ("project", "bin_sort", "raster_fwd", "raster_bwd", "project_bwd"))

    # roofline of the dominant kernel group
    hbm, bf16, src = load_peaks()
    dom = max(stages, key=stages.get)
    sm_mhz = clk.summary().get("sm_mhz") or 2070.0
    n_sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    roof = roofline_for(dom, stages[dom], pairs, pair_counts, G.n, Vb, W, H, cfg, hbm, src, sm_mhz, n_sms)

    # the cache MLP on its own against the tensor peak: each launch timed
    # alone over all rows (the reverse dense, every row's gradient), tensor
    # FLOPs of the two BF16 hidden layers (32 -> 64 -> 64); the 64 -> 7
    # output layer runs in FP32 on the SIMT cores and is not counted
    mlp_roof = None
    if ntc.mlp_struct().precision == gs3.GS_MLP_BF16 and not st.fused:
        dW_keep = ntc.mlp.g.clone()
        d_enc_keep = st.d_enc.clone()

        def time_it(fn, reps=20):
            fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                fn()
            b.record(stream)
            torch.cuda.synchronize()
            return a.elapsed_time(b) / reps

        fwd_ms = time_it(lambda: gs3.ntc_mlp_fwd(st.enc, G.n, ntc.mlp_struct(), st.raw7, stream))
        bwd_ms = time_it(lambda: gs3.ntc_mlp_bwd(st.enc, G.n, ntc.mlp_struct(), st.d_raw7, st.loss_scale_view(),
                                                  ntc.mlp.g, st.d_enc))
        ntc.mlp.g.copy_(dW_keep)
        st.d_enc.copy_(d_enc_keep)
        f_fwd = 2 * (32 * 64 + 64 * 64) * G.n
        f_bwd = 2 * f_fwd   # input gradients and weight gradients of both layers
        mlp_roof = {"bound": "tensor", "dtype": "bf16", "peak": bf16, "unit": "TFLOP/s", "peak_source": src,
                    "rows": G.n, "fwd": {"ms": fwd_ms, "flops": f_fwd, "achieved": f_fwd / fwd_ms / 1e9,
                                         "frac": f_fwd / fwd_ms / 1e9 / bf16},
                    "bwd_dense": {"ms": bwd_ms, "flops": f_bwd, "achieved": f_bwd / bwd_ms / 1e9,
                                  "frac": f_bwd / bwd_ms / 1e9 / bf16},
                    "note": "latency-bound small GEMMs (K = 32/64 per row tile); ncu on the 100K case: "
                            "sm__pipe_tensor_cycles_active 6.6 % in the reverse"}

    # the rasterizer fwd+bwd against HBM: algorithmic bytes of projection,
    # binning/sort, compositing fwd/bwd and projection bwd, counted per
    # Gaussian, per (view, Gaussian, 16x16 tile) intersection and per pixel
    inter = int(st.raster.proj.tiles_touched.sum().item())
    K = (cfg.sh_deg + 1) ** 2
    per_g = (44 + 12 * K) * 2 + 28 + Vb * (44 + 32)   # params read twice (a4, a9), records, grads
    raster_bytes = G.n * per_g + inter * 124 + Vb * W * H * (20 + 32)
    raster_roof = {"bound": "hbm", "achieved": raster_bytes / (raster_ms * 1e-3) / 1e9, "peak": hbm,
                   "unit": "GB/s", "frac": raster_bytes / (raster_ms * 1e-3) / 1e9 / hbm,
                   "algorithmic_bytes": raster_bytes, "intersections": inter,
                   "bytes_per": {"gaussian": per_g, "intersection": 124, "pixel": 52},
                   "ms": raster_ms, "peak_source": src}

    # render-only: NTC query + transformation + projection + binning +
    # compositing of one 1352x1014 view, one CUDA graph per frame
    render_only = None
    if not args.no_render:
        ro_ms, ro_bin = autotune_bin(G, gs3.camera_slice(cams_dev, 0, 1),
                                     1, W, H, st.mean_t.clone(), st.quat_t.clone(), backward=False)
        rr = Renderer(G, ntc, 1, W, H, 1 << 20, bin=ro_bin)
        rr.raster.fit_capacity(G, gs3.camera_slice(cams_dev, 0, 1), *st.transform(), margin=1.3)
        views = [gs3.camera_slice(cams_dev, v, 1) for v in range(cfg.n_cams)]
        rgraphs = [rr.capture(v) for v in views] if not args.eager else None
        kr = 100
        for i in range(5):
            rgraphs[i % len(views)].replay() if rgraphs else rr.frame(views[i % len(views)])
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(kr):
            rgraphs[i % len(views)].replay() if rgraphs else rr.frame(views[i % len(views)])
        e1.record(stream)
        torch.cuda.synchronize()
        rr.raster.check()
        rms = e0.elapsed_time(e1) / kr
        render_only = {"ms_per_frame": rms, "fps": 1e3 / rms, "width": W, "height": H, "views": 1,
                       "gaussians": G.n, "bin_tiles": ro_bin,
                       "autotune_ms": {str(k): round(v, 4) for k, v in ro_ms.items()},
                       "includes": "NTC query (encode, BF16 MLP), transformation, projection, "
                                   "binning/sort, compositing; CUDA graph per frame"}
        del rr, rgraphs
        torch.cuda.empty_cache()

    # plain FP32 direct optimisation on the same inputs and rasterizer
    plain = None
    if not args.no_plain:
        do = DirectOpt(G, Vb, W, H, st.raster.capacity, device=dev, bin=bin_side)
        for i in range(3):
            do.step(batch_cams[i % nb], targets[(i % nb) * Vb:(i % nb + 1) * Vb])
        dgraphs = do.capture(batches) if not args.eager else None
        torch.cuda.synchronize()
        e0.record(stream)
        kp = max(10, args.steps // 2)
        for i in range(kp):
            b = i % nb
            if dgraphs is not None:
                dgraphs[b].replay()
            else:
                do.step(batch_cams[b], targets[b * Vb:(b + 1) * Vb])
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / kp
        plain = {"s_per_frame": pms * ITERS_PER_FRAME / 1e3, "ms_per_iter": pms, "iters": kp}
        del do, dgraphs

    converge = None
    if not args.no_converge and plain is not None:
        converge = equal_psnr(scene, G, Gt, ntc, warm_table, warm_mlp, st, batches, nb, Vb, W, H,
                              ms_max, plain["ms_per_iter"], dev)

    # end to end through the public API with host buffers: per step the batch's
    # target views go host->device from pinned memory (engine.TargetFeeder:
    # the next step's copy overlaps this step) and the loss comes back
    host_targets = targets.cpu().pin_memory()
    host_b = [host_targets[b * Vb:(b + 1) * Vb] for b in range(nb)]
    feeder = TargetFeeder(host_b, [targets[b * Vb:(b + 1) * Vb] for b in range(nb)])
    host_loss = torch.empty(1, pin_memory=True)
    ke = max(10, args.steps // 2)

    def e2e_step(i):
        b = i % nb
        feeder.before(b)
        if graphs is not None:
            graphs[b].replay()
        else:
            st.step(batch_cams[b], feeder.dev[b])
        feeder.after(b, (i + 1) % nb)
        host_loss.copy_(st.loss.d_loss, non_blocking=True)

    feeder.start(0)
    for i in range(2):
        e2e_step(i)
    torch.cuda.synchronize()
    e0.record(stream)
    feeder.start(0)
    for i in range(ke):
        if i % ITERS_PER_FRAME == 0:
            ntc.reset_to(warm_table, warm_mlp)
            st.reset_state()
        e2e_step(i)
    stream.wait_stream(feeder.copy_stream)   # the copies issued, one ahead, all inside
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / ke
    h2d = feeder.bytes_per_step

    cpu = None
    if converge is not None:
        # the paths' own final held-out PSNRs: does the plain path ever reach the cache's?
        n_fin = converge["ntc"]["final"]["heldout"]
        reach = [p["it"] for p in converge["direct"]["curve"][1:] if p["heldout"] >= n_fin - 0.05]
        converge["direct_reaches_ntc_final_psnr_within_frame"] = bool(reach)
    stage2 = None
    used_graphs = graphs is not None
    if not args.no_stage2 and rank == 0:
        graphs = None
        torch.cuda.empty_cache()
        stage2 = stage2_workload(dev)
    large = None
    if not args.no_large and rank == 0:
        graphs = None
        torch.cuda.empty_cache()
        large = large_workload(dev)
    stream_res = None
    if args.stream_frames > 0 and rank == 0:
        graphs = None
        torch.cuda.empty_cache()
        stream_res = stream_workload(dev, args.stream_frames, (warm_table, warm_mlp), ntc)
    if rank == 0 and world == 1 and not args.no_cpu:
        per_iter, desc, cores = oracle_sample(scene)
        cpu = {"value": per_iter * ITERS_PER_FRAME, "unit": "s/frame", "cores": cores,
               "kind": "oracle", "sample": desc}
        if not args.no_oracle_configs:
            cpu["other_workloads"] = oracle_configs()

    if rank == 0:
        clocks = clk.summary()
        line = {"metric": METRIC, "value": s_per_frame, "unit": "s/frame", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "mixed: f16 table, %s mlp, f32 raster" % args.mlp if precision == gs3.GS_MLP_BF16 else "f32",
                "data": "synthetic", "config": config_dict(scene, "replicas%d" % world if world > 1 else "single"),
                "train_it_per_s": 1e3 / ms_max,
                "full_frame_s": full_frame_s,
                "raster_fwd_bwd_it_per_s": 1e3 / raster_ms,
                "raster_fwd_bwd_ms": raster_ms,
                "plain_fp32_direct_opt": plain,
                "speedup_vs_plain_per_iter": (plain["ms_per_iter"] / ms_max) if plain else None,
                "equal_psnr": converge,
                "graphs": used_graphs,
                "stages_ms": {k: round(v, 4) for k, v in stages.items()},
                "bin_pairs_per_step": pairs, "composited_pairs": pair_counts,
                "warmup_loss": wl, "warmup_s": t_warm,
                "roofline": roof, "raster_fwd_bwd_roofline": raster_roof, "mlp_roofline": mlp_roof,
                "render_only": render_only, "bin_autotune": tune, "bin_tiles": bin_side,
                "stage2": stage2, "stream": stream_res, "large": large,
                "paper_context": {"s_per_frame": 12.0, "fps_render": 200,
                                  "hardware": "one RTX 3090", "workload": "N3DV, real video",
                                  "note": "context only: other hardware, data and precision"},
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_ms * ITERS_PER_FRAME / 1e3, "unit": "s/frame",
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 4},
                "gpu_launches": int(launches), "tc_timeouts": gs3.gs_tc_timeouts(), "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


def stage2_workload(dev, warm_iters=300):
    """Stage 2 (Section 4.2) on the 500K-Gaussian, 12-view 1280x720 workload
    whose target frame holds an object absent from the previous frame:
    Stage 1 (150 iterations, view-space statistics over its final epoch),
    then 100 timed Stage-2 iterations (spawn, training of the added
    Gaussians, split/prune at every epoch end, host reads of the count
    included).  Returns timings and the PSNR of the training views."""
    import torch
    from paper_2403_01444_gb300 import gs3, scenes
    from paper_2403_01444_gb300.engine import NTC, Rasterizer, Stage1, Stage2, warmup
    scene = scenes.make_scene(4)
    cfg = scene.cfg
    W, H, Vb = cfg.W, cfg.H, cfg.views_per_batch
    nb = cfg.n_cams // Vb
    G = gs3.Gaussians.from_numpy(scene.prev)
    Gt = gs3.Gaussians.from_numpy(scene.target)
    cd = gs3.cameras_to_device(scene.cams)
    bc = [gs3.camera_slice(cd, b * Vb, Vb) for b in range(nb)]
    rt = Rasterizer(Gt.n, Vb, W, H, 1 << 24, dev)
    tg = torch.empty(cfg.n_cams, 3, H, W, device=dev)
    for b in range(nb):
        rt.fit_capacity(Gt, bc[b], margin=1.2)
        tg[b * Vb:(b + 1) * Vb].copy_(rt.img)
    del rt
    batches = [(bc[b], tg[b * Vb:(b + 1) * Vb]) for b in range(nb)]
    rng = np.random.default_rng(11)
    grid = gs3.hashgrid()
    table = rng.uniform(-1e-4, 1e-4, size=(gs3.ntc_hashgrid_entries(grid), 2)).astype(np.float32)
    Ws = [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
    ntc = NTC(table, Ws, grid, gs3.GS_MLP_BF16, dev)
    warmup(ntc, G, iters=warm_iters)
    st1 = Stage1(G, ntc, Vb, W, H, capacity=1 << 20)
    st1.raster.fit_capacity(G, bc[0], *st1.transform(), margin=2.0)
    track = None
    for it in range(ITERS_PER_FRAME):
        if it == ITERS_PER_FRAME - nb:
            track = st1.track_viewspace(True)
        st1.step(*batches[it % nb])
    st1.track_viewspace(False)
    st1.raster.check()
    mt, qt = [x.clone() for x in st1.transform()]

    def psnr_views(gs, mean=None, quat=None):
        r = Rasterizer(gs.n, Vb, W, H, 1 << 22, dev)
        se = 0.0
        for b in range(nb):
            r.fit_capacity(gs, bc[b], mean, quat, margin=1.2)
            se += float(((r.img - tg[b * Vb:(b + 1) * Vb]) ** 2).sum())
        return -10 * math.log10(se / tg.numel())

    p1 = psnr_views(G, mt, qt)
    st2 = Stage2(G, Vb, W, H, capacity=300_000, pair_capacity=1 << 24)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    spawned = st2.begin(mt, qt, *track)
    st2.run(batches, iters=100)
    e1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    ms = e0.elapsed_time(e1)
    p2 = psnr_views(st2.view())
    added_final = st2.n_add
    del st2
    torch.cuda.empty_cache()
    # the random-spawn ablation (Section 5.3): as many added Gaussians, around
    # fixed ones drawn at random, same training and quantity control
    st_r = Stage2(G, Vb, W, H, capacity=300_000, pair_capacity=1 << 24, seed=5)
    st_r.begin(mt, qt, *track, random_count=spawned)
    st_r.run(batches, iters=100)
    p_rand, n_rand = psnr_views(st_r.view()), st_r.n_add
    return {"workload": "stage2 500K Gaussians SH3 + emerging object of %d, 12 cams 1280x720, "
                        "4 views/launch, 100 it" % (scene.target.n - scene.prev.n),
            "ms_total": ms, "ms_per_iter": ms / 100, "wall_s": wall, "spawned": spawned,
            "added_final": added_final, "psnr_train_views_stage1": p1, "psnr_train_views_stage2": p2,
            "random_spawn_ablation": {"psnr_train_views": p_rand, "added_final": n_rand}}


def large_workload(dev, iters=20):
    """The 1M-Gaussian workload: all 16 views of 1920x1080 rendered in one
    launch per Stage-1 iteration, the whole iteration (cache, projection,
    binning, compositing, loss, reverse, Adam) replayed as one CUDA graph,
    mixed precision; iters timed iterations after the capture."""
    import torch
    from paper_2403_01444_gb300 import gs3, scenes
    from paper_2403_01444_gb300.engine import NTC, Rasterizer, Stage1, warmup
    scene = scenes.make_scene(5)
    cfg = scene.cfg
    W, H, V = cfg.W, cfg.H, cfg.views_per_batch
    G = gs3.Gaussians.from_numpy(scene.prev)
    Gt = gs3.Gaussians.from_numpy(scene.target)
    cd = gs3.cameras_to_device(scene.cams)
    rt = Rasterizer(Gt.n, V, W, H, 1 << 24, dev)
    rt.fit_capacity(Gt, cd, margin=1.2)
    tg = rt.img.clone()
    del rt
    torch.cuda.empty_cache()
    rng = np.random.default_rng(13)
    grid = gs3.hashgrid()
    table = rng.uniform(-1e-4, 1e-4, size=(gs3.ntc_hashgrid_entries(grid), 2)).astype(np.float32)
    Ws = [w.astype(np.float32) for w in scenes.random_mlp([32, 64, 64, 7], rng)]
    ntc = NTC(table, Ws, grid, gs3.GS_MLP_BF16, dev)
    warmup(ntc, G, iters=300)
    st = Stage1(G, ntc, V, W, H, capacity=1 << 24)
    pairs = st.raster.fit_capacity(G, cd, *st.transform(), margin=1.3)
    graph = st.capture([(cd, tg)])[0]
    stream = torch.cuda.current_stream()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(iters):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    st.raster.check()
    ms = e0.elapsed_time(e1) / iters
    return {"workload": "1M Gaussians SH3, 16 views 1920x1080 in one launch per iteration, "
                        "whole iteration one CUDA graph, mixed precision",
            "ms_per_iter": ms, "s_per_frame": ms * ITERS_PER_FRAME / 1e3,
            "bin_pairs_per_iter": int(pairs), "pixels_per_iter": V * W * H}


def stream_workload(dev, n_frames, warm_table_mlp, ntc):
    """The streaming driver on the 250K-Gaussian, 20-view 1352x1014 video:
    n_frames consecutive frames of cumulative rigid+RBF motion, each Stage 1
    (150 iterations, graphs) then Stage 2 (100 iterations) on a second stream
    overlapped with the next frame's Stage 1; targets of each frame rendered
    on the fly (inside the timed loop)."""
    import torch
    from paper_2403_01444_gb300 import gs3, scenes
    from paper_2403_01444_gb300.engine import Rasterizer, Streamer
    cfg, frames, cams, ho = scenes.make_sequence(CFG_INDEX, n_frames)
    W, H, Vb = cfg.W, cfg.H, cfg.views_per_batch
    nb = cfg.n_cams // Vb
    cd = gs3.cameras_to_device(cams)
    hod = gs3.cameras_to_device([ho])
    rt = Rasterizer(frames[0].n, Vb, W, H, 1 << 24, dev)
    rh = Rasterizer(frames[0].n, 1, W, H, 1 << 22, dev)
    out = torch.empty(cfg.n_cams, 3, H, W, device=dev)

    def views(t):
        Gt = gs3.Gaussians.from_numpy(frames[t + 1])
        for b in range(nb):
            rt.fit_capacity(Gt, gs3.camera_slice(cd, b * Vb, Vb), margin=1.2)
            out[b * Vb:(b + 1) * Vb].copy_(rt.img)
        return out

    ho_gt = []
    for t in range(n_frames):
        rh.fit_capacity(gs3.Gaussians.from_numpy(frames[t + 1]), hod, margin=1.2)
        ho_gt.append(rh.img.clone())
    G0 = gs3.Gaussians.from_numpy(frames[0])
    # weights of the motion error: visibility of frame 0's Gaussians in its views
    wvis = visibility(G0, [(gs3.camera_slice(cd, b * Vb, Vb), out[b * Vb:(b + 1) * Vb])
                           for b in range(nb)], W, H, dev)
    mean_gt = lambda t: torch.from_numpy(frames[t + 1].mean).to(dev)
    s = Streamer(G0, ntc, *warm_table_mlp, cd, cfg.n_cams, Vb, W, H, heldout_dev=hod)
    rec = s.run(views, ho_gt, motion_ref=(mean_gt, wvis))
    mean = lambda k: float(np.mean([r[k] for r in rec]))
    return {"workload": "stream: 250K Gaussians SH3, 20 cams 1352x1014, %d frames of cumulative "
                        "rigid+RBF motion; Stage 1 150 it + Stage 2 100 it per frame, Stage 2 "
                        "overlapped with the next frame's Stage 1" % n_frames,
            "frames": n_frames, "wall_s": s.wall_s, "s_per_frame": s.wall_s / n_frames,
            "psnr_heldout_carried": mean("psnr_carried"), "psnr_heldout_stage1": mean("psnr_stage1"),
            "psnr_heldout_stage2": mean("psnr_stage2"), "added_per_frame": mean("added"),
            "motion_err_weighted": mean("motion_err_weighted"),
            "motion_err_if_not_transformed": mean("motion_err_carried_weighted"),
            "storage_bytes_per_frame": mean("storage_bytes"), "per_frame": rec}


PLAIN_LR_SWEEP = (2.4e-3, 1e-3, 5e-4, 2e-4, 1e-4)   # mean rates of the direct path's sweep
PLAIN_QUAT_RATIO = 0.015 / 0.0024                    # rotation : mean rate (Suppl. A proportions)


def visibility(G, batches, W, H, dev):
    """Per Gaussian of the previous frame: sum over the training views and
    pixels of alpha T (its colour gradient under a unit image gradient), the
    weight of its motion error."""
    import torch
    from paper_2403_01444_gb300.engine import Rasterizer
    w = torch.zeros(G.n, device=dev)
    r = None
    for cd, tg in batches:
        if r is None:
            r = Rasterizer(G.n, tg.shape[0], W, H, 1 << 22, dev)
        r.fit_capacity(G, cd, margin=1.2)
        r.backward(G, cd, torch.ones_like(r.img))
        w += r.grads[..., 5].sum(0)
    return w


def equal_psnr(scene, G, Gt, ntc, warm_table, warm_mlp, st, batches, nb, Vb, W, H, ms_ntc, ms_plain,
               dev, iters=ITERS_PER_FRAME, every=5):
    """One frame of each path from the same previous-frame Gaussians, with
    every `every` iterations: PSNR of the held-out view and of the 20 training
    views, and the motion error against the known ground truth (mean
    |mu' - mu_gt| and angle(q', q_gt) of the Gaussians the training views see,
    weighted by visibility).  The plain path runs at each mean rate of
    PLAIN_LR_SWEEP (rotation rate x PLAIN_QUAT_RATIO, the same schedule as the
    cache) and the rate with the best held-out PSNR is compared.  Target = the
    lower of the two paths' best held-out PSNR over the frame; each path's
    time to reach it (within 0.05 dB) = first checkpoint reaching it x its
    measured time per iteration.  Also reported: the same with the lower final
    PSNR as target, and both comparisons on the training views."""
    import torch
    from paper_2403_01444_gb300.engine import DirectOpt, render
    ho = [scene.heldout]
    gt_ho = render(Gt, ho, W, H)
    psnr = lambda a, b: float(-10.0 * math.log10(max(((a - b) ** 2).mean().item(), 1e-20)))
    gt_train = torch.cat([render(Gt, scene.cams[b * Vb:(b + 1) * Vb], W, H) for b in range(nb)])
    w = visibility(G, batches, W, H, dev)
    seen = w > 1.0

    def train_psnr(m, q):
        img = torch.cat([render(G, scene.cams[b * Vb:(b + 1) * Vb], W, H, m, q) for b in range(nb)])
        return psnr(img, gt_train)

    def motion(m, q):
        dm = (m - Gt.mean).norm(dim=1)
        qn = q / q.norm(dim=1, keepdim=True)
        ang = 2 * torch.acos((qn * Gt.quat).sum(1).abs().clamp(max=1.0)) * (180 / math.pi)
        return {"mean_err_weighted": float((dm * w).sum() / w.sum()), "mean_err_seen": float(dm[seen].mean()),
                "angle_deg_weighted": float((ang * w).sum() / w.sum())}

    def point(i, m, q):
        r = {"it": i, "heldout": round(psnr(render(G, ho, W, H, m, q), gt_ho), 3),
             "train": round(train_psnr(m, q), 3)}
        r.update({k: round(v, 6) for k, v in motion(m, q).items()})
        return r

    start = point(0, G.mean, G.quat)
    ntc.reset_to(warm_table, warm_mlp)
    st.reset_state()
    curve_n = [start]
    for i in range(iters):
        st.step(*batches[i % nb])
        if (i + 1) % every == 0:
            curve_n.append(point(i + 1, *st.transform()))
    plain = {}
    for lr in PLAIN_LR_SWEEP:
        do = DirectOpt(G, Vb, W, H, st.raster.capacity, lr_mean=lr, lr_quat=lr * PLAIN_QUAT_RATIO,
                       device=dev)
        c = [start]
        for i in range(iters):
            do.step(*batches[i % nb])
            if (i + 1) % every == 0:
                c.append(point(i + 1, do.mean.p, do.quat.p))
        plain[lr] = c
        del do
    best_lr = max(plain, key=lambda lr: (max(p["heldout"] for p in plain[lr][1:]), -lr))
    curve_d = plain[best_lr]

    def compare(cn, cd, key, best):
        pick = (lambda c: max(p[key] for p in c[1:])) if best else (lambda c: c[-1][key])
        target = min(pick(cn), pick(cd))
        first = lambda c: next(p["it"] for p in c[1:] if p[key] >= target - 0.05)
        it_n, it_d = first(cn), first(cd)
        return {"target_psnr": target, "ntc_iters": it_n, "direct_iters": it_d,
                "ntc_s": it_n * ms_ntc / 1e3, "direct_s": it_d * ms_plain / 1e3,
                "speedup_at_equal_psnr": (it_d * ms_plain) / (it_n * ms_ntc)}

    summ = lambda c: {"final": c[-1], "best_heldout": max(p["heldout"] for p in c[1:]),
                      "best_train": max(p["train"] for p in c[1:])}
    return {"view": "held-out camera (azimuth 7.5, elevation 5)", "checkpoint_every": every,
            "previous_frame": start, "seen_gaussians": int(seen.sum()),
            "motion_weight": "sum over the training views of alpha T (Gaussians with weight > 1 are 'seen')",
            "ntc": dict(summ(curve_n), curve=curve_n),
            "direct": dict(summ(curve_d), lr_mean=best_lr, lr_quat=best_lr * PLAIN_QUAT_RATIO, curve=curve_d),
            "direct_lr_sweep": {("%g" % lr): summ(c) for lr, c in plain.items()},
            "heldout": {"best": compare(curve_n, curve_d, "heldout", True),
                        "final": compare(curve_n, curve_d, "heldout", False)},
            "train_views": {"best": compare(curve_n, curve_d, "train", True),
                            "final": compare(curve_n, curve_d, "train", False)},
            "speedup_at_equal_psnr": compare(curve_n, curve_d, "heldout", True)["speedup_at_equal_psnr"]}


def ctypes_u64():
    import ctypes
    return ctypes.c_uint64


# FP32 operations per (pixel, Gaussian) pair, counted from the compositing
# formulas: the power and alpha of a pair (12), the front-to-back update of
# an added pair (9), and the reverse of an added pair (47: T recovery, colour,
# alpha and conic/mean gradients, behind-colour update).
FLOPS_TESTED, FLOPS_FWD_ADDED, FLOPS_BWD_ADDED = 12, 9, 47


def recorded_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the ncu capture summarised under
    profiles/ (dram__bytes_read.sum + dram__bytes_write.sum), or None when no
    capture is recorded or the kernel's sources changed since it was taken."""
    import glob
    import hashlib
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", kernel + "_traffic_*.md"))):
        fields = {}
        for line in open(path):
            if ":" in line and not line.startswith(("|", "#", " ")):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        if "traffic_bytes_per_launch" not in fields or "sources_sha256" not in fields:
            continue
        h = hashlib.sha256()
        for f in fields.get("sources", "").split():
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest() == fields["sources_sha256"]:
            return int(fields["traffic_bytes_per_launch"])
    return None


def roofline_for(stage, ms, pairs, pair_counts, n, V, W, H, cfg, hbm_gbs, src, sm_mhz, n_sms):
    """Roofline of one launch of the stage's kernels: compositing is bound by
    FP32 arithmetic (FLOPs of the evaluated pairs over the FP32 FMA peak of
    SMs x 128 lanes x 2 FLOPs x SM clock); the other stages by HBM
    (each logically required read or write counted once)."""
    if stage in ("raster_fwd", "raster_bwd"):
        tested, added = (pair_counts[0], pair_counts[1]) if stage == "raster_fwd" else \
            (pair_counts[2], pair_counts[3])
        per_added = FLOPS_FWD_ADDED if stage == "raster_fwd" else FLOPS_BWD_ADDED
        flops = tested * FLOPS_TESTED + added * per_added
        achieved = flops / (ms * 1e-3) / 1e12
        peak = n_sms * 128 * 2 * sm_mhz * 1e6 / 1e12
        return {"bound": "alu", "kernel": stage, "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": recorded_traffic(stage),
                "algorithmic_flops": flops, "pairs_evaluated": tested, "pairs_added": added,
                "ms": ms, "sm_count": n_sms,
                "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 x %.0f MHz (median under load)"
                               % (n_sms, sm_mhz)}
    K = (cfg.sh_deg + 1) ** 2
    px = V * W * H
    per_gauss_params = 12 + 16 + 12 + 4 + 12 * K
    bytes_ = {
        "bin_sort": pairs * (12 + 24 + 8),
        "project": n * per_gauss_params + n * V * 44,
        "project_bwd": n * per_gauss_params + n * V * 32 + n * 28,
        "loss": px * 3 * 4 * 3,
        "ntc_fwd": n * (12 + 16 + 28 + 28 + 64),
        "ntc_bwd": n * (12 + 16 + 28 + 28 + 28 + 64),
        "adam": (1647607 * 2 + 6592) * 30,
    }.get(stage, 0)
    achieved = bytes_ / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": stage, "achieved": achieved, "peak": hbm_gbs,
            "unit": "GB/s", "frac": achieved / hbm_gbs, "traffic": recorded_traffic(stage),
            "algorithmic_bytes": bytes_, "ms": ms, "peak_source": src}



def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
