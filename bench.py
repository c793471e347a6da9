#!/usr/bin/env python
"""Throughput of the TSDF-bounded novel-view render (TSDF-Sampling, arXiv
2311.17878) on GB300, in rays/s, beside the 64 + 32 hierarchical comparator.

Workload (the indoor-room configuration): 8x6x3 m room with 20 boxes and 4
thin plates; 256^3 TSDF (D_T = 4 voxels) fused from 100 synthetic 640x480
depth maps with N(0, 5 mm) noise; SDF network 8x256 (PE L=6, skip at layer 4)
and colour network 4x256 (direction PE L=4), fitted to the scene; one step =
one 640x480 novel view (307200 rays): Alg. 1 bounds + offsets scan + sample
placement + both networks + NeuS compositing, all in the library's kernels.
Fusion runs once before the timed region and is reported separately.

    python bench.py [--steps K] [--warmup W] [--precision bf16|f32]
    python bench.py --impl reference     # the CPU oracle on a bounded sample

One JSON line on stdout (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HIER_LADDER = ((32, 16), (24, 12), (16, 8), (12, 6), (8, 4), (6, 3), (4, 2))
METRIC = "rays/s at PSNR≥oracle−0.1dB, TSDF-bounded vs 96-sample hierarchical, 1 GB300"
UNIT = "rays/s"
WORKLOADS = {
    "view": "room 8x6x3m (20 boxes, 4 plates), 256^3 TSDF from 100x640x480 depth maps, 640x480 novel views",
    "panorama": "room 8x6x3m (20 boxes, 4 plates), 256^3 TSDF from 100x640x480 depth maps, 1024x512 equirect "
                "panoramas from 4 in-room centres (ragged 1-64 samples, fallback 96)",
    "large": "20x20x4m floor (4 rooms, 200 boxes, 40 plates), 512^3 fp16 TSDF from 300x1280x960 depth maps, "
             "batch of 8 2048x1024 equirect panoramas (one panorama per step)",
}
WORKLOAD = WORKLOADS["view"]
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of k_mlp_tc per launch, the mean
# over the 10 timed launches of `bench.py --only-main --no-graph --steps 10 --warmup 3` (room views 0-9,
# network-fused grid, fp16 operands) in one ncu capture; reported only for that
# configuration and while the kernel sources hash to the ones it was captured on
MLP_TC_TRAFFIC = {"sha256": "f9a514cb2bb93e350029ef5ca1fd01644e13714e5f37fd6bb7e165b497660758", "bytes_per_launch": 262874086,
                  "profile": "profiles/k_mlp_tc_room_view_traffic.md"}
# the same for k_ray_bounds (the march of Alg. 1) on the same ten timed views
MARCH_TRAFFIC = {"sha256": "c4307e3a56049f67dc00d5274645fbd858f05161b8c533815f880fbb3a07392b", "bytes_per_launch": 9989350,
                 "profile": "profiles/k_ray_bounds_room_view_traffic.md"}
ALGO_FLOP_PER_SAMPLE = 2.25e6   # SDF fwd + minimal reverse-mode grad + colour, 8x256 / 4x256 networks
# what the tensor-core kernels issue per sample (value + 3 tangent rows through the SDF layers):
# serial, 64-sample tiles in pairs: 4 rows per sample through SDF layers 0-6 and the folded
# output layer's value column (N = 16), one row per sample through the colour layers (M = 128
# over both tiles of a pair; the folded first colour layer with K = 256 + 48); pipelined,
# 32-sample tiles: 4 rows per sample through both networks (M = 128 colour MMAs with 32 live
# rows), the SDF MMAs twice with split operands
EXEC_FLOP_PER_SAMPLE = {"serial": 3.77e6, "pipelined": 5.93e6, "pipelined-split": 9.63e6}
N_VIEWS_TIMED = 10   # views cycled by the timed steps (4 for the panorama workload)
QUALITY_PIXELS = 4096          # seeded pixels spread over every timed view (synth.quality_pixels)
QUALITY_PIXELS_LIVE = 1024     # when the dense reference is rendered during the run (panorama workload)
DENSE_SAMPLES = 1024
DENSE_REF = os.path.join(ROOT, "oracle", "data", "room_view_dense_reference.npz")
# operating points of the quality leg: the paper's own knobs around the timed default (Alg. 1's
# D_s, M and far-test neighbourhood, Sec. 3.4's spacing and cap, the mean-relative count of
# Tab. 2 "full", coarse + fine inside the bound, the recovery pass of Sec. 4.5).  Keys: d_s and
# step in voxels, m (M), nb (neighbourhood radius), n_max, tau (recovery), sampler: "mid"
# (midpoints, counts from the spacing), "rel" (midpoints, counts relative to the mean interval,
# mean n_mean), "cf" (coarse + fine: n_mean coarse relative to the mean, n_fine inverse-CDF)
SWEEP = (
    {"name": "M=2 (Fig. 2)", "m": 2},
    {"name": "M=2 3^3", "m": 2, "nb": 1},
    {"name": "M=4 3^3", "m": 4, "nb": 1},
    {"name": "D_s=2", "d_s": 2.0},
    {"name": "D_s=2 M=2 3^3", "d_s": 2.0, "m": 2, "nb": 1},
    {"name": "D_s=2 M=2 3^3 step 1", "d_s": 2.0, "m": 2, "nb": 1, "step": 1.0},
    {"name": "D_s=3 M=2 3^3 step 1", "d_s": 3.0, "m": 2, "nb": 1, "step": 1.0},
    {"name": "n_max=16", "n_max": 16},
    {"name": "rel n=8", "sampler": "rel", "n_mean": 8.0},
    {"name": "D_s=2 M=2 3^3 rel n=8", "d_s": 2.0, "m": 2, "nb": 1, "sampler": "rel", "n_mean": 8.0},
    {"name": "cf 6+8", "sampler": "cf", "n_mean": 6.0, "n_fine": 8},
    {"name": "D_s=2 M=2 3^3 cf 6+8", "d_s": 2.0, "m": 2, "nb": 1, "sampler": "cf", "n_mean": 6.0, "n_fine": 8},
    {"name": "D_s=2 M=2 3^3 cf 4+4", "d_s": 2.0, "m": 2, "nb": 1, "sampler": "cf", "n_mean": 4.0, "n_fine": 4},
    {"name": "recovery 0.95", "tau": 0.95},
    {"name": "D_s=2 M=2 3^3 recovery 0.95", "d_s": 2.0, "m": 2, "nb": 1, "tau": 0.95},
)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["f16", "bf16", "bf16x2", "f32"], default="f16",
                    help="network operands: f16, bf16, bf16x2 (SDF activations split in two bf16 parts), f32 (SIMT)")
    ap.add_argument("--net-kernel", choices=["auto", "serial", "pipelined"], default="auto",
                    help="tensor-core network kernel; auto: the library's autotuner picks on view 0")
    ap.add_argument("--no-quality", action="store_true")
    ap.add_argument("--no-sweep", dest="sweep", action="store_false", default=True,
                    help="skip the operating-point sweep of the quality leg (D_s, M, neighbourhood, spacing, "
                         "count rule, recovery)")
    ap.add_argument("--grid-source", choices=["network", "analytic"], default="network",
                    help="depth maps the marched grid is fused from (analytic: the exact scene, no network pre-pass)")
    ap.add_argument("--fusion", choices=["projective", "raycast"], default="projective",
                    help="form of Alg. 2 that fuses the network's depth into the marched grid")
    ap.add_argument("--rays", type=int, default=0, help="seeded subset of each view's rays (0: all 307200)")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="view",
                    help="view: 640x480 held-out views; panorama: 1024x512 equirect panoramas")
    ap.add_argument("--graph", dest="graph", action="store_true", default=True,
                    help="replay each view's bounds + render as a captured CUDA graph (the default)")
    ap.add_argument("--no-graph", dest="graph", action="store_false", help="launch each step's kernels eagerly")
    ap.add_argument("--train-pitch", type=float, default=None,
                    help="largest pitch (degrees) of the random training poses (default: the synthetic recipe's)")
    ap.add_argument("--recovery-tau", type=float, default=None,
                    help="recovery pass of Sec. 4.5: re-render rays whose weight sum stays below tau (off by default)")
    ap.add_argument("--quality-only", action="store_true", help="main timing + quality (no e2e / comparator / cpu / "
                                                                   "training legs)")
    ap.add_argument("--only-main", action="store_true", help="time the render path only (no e2e / comparator / "
                                                                  "quality / cpu / training legs): the small profiling case")
    ap.add_argument("--train-only", action="store_true",
                    help="one training step in an NVTX range 'timed' (autograd on the calling thread), on the grid "
                         "fused from the analytic depth maps: the profiling case of the training step")
    ap.add_argument("--train-rays", type=int, default=8192, help="rays of the --train-only step")
    ap.add_argument("--train-chunk", type=int, default=0,
                    help="samples per chunk of the layer-major backward in the --train-only step (0: default)")
    ap.add_argument("--ref-rays", type=int, default=2048, help="rays per reference-arm step")
    ap.add_argument("--ds-vox", type=float, default=1.0, help="D_s of Alg. 1 in voxels (Sec. 4.2 uses 1)")
    ap.add_argument("--m-confirm", type=int, default=None, help="M of Alg. 1 (Sec. 4.2 uses 15)")
    ap.add_argument("--nb-radius", type=int, default=None, help="far-test neighbourhood radius (2: 5^3, Sec. 4.2)")
    ap.add_argument("--step-vox", type=float, default=None, help="sample spacing of Sec. 3.4 in voxels (2)")
    return ap.parse_args()


# ----------------------------------------------------------------------------
class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.path = os.path.join("/tmp", f"tsdfs_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.index)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(5)
            except Exception:
                self.p.kill()
            self.f.close()

    def summary(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(r[0] for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[2][i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": rows[0][1], "reasons": reasons, "samples": len(rows)}


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        if torch.cuda.is_available():
            torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def source_hash(files) -> str:
    """SHA-256 over the library sources a kernel is compiled from."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2311_17878_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


MLP_TC_SOURCES = ("mlp_tc.cu", "tc_common.cuh", "common.cuh")
MARCH_SOURCES = ("bounds.cu", "march.cuh", "common.cuh")


def captured_traffic(t, files, args, prec):
    """A captured per-launch DRAM traffic, or None when this run is not the captured
    configuration or the kernel has changed since."""
    same_run = (args.workload == "view" and args.grid_source == "network" and args.fusion == "projective"
                and prec == "f16" and args.steps % N_VIEWS_TIMED == 0 and not args.rays
                and args.recovery_tau is None)
    if not same_run or t["bytes_per_launch"] is None or t["sha256"] != source_hash(files):
        return None
    return t["bytes_per_launch"]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


# ----------------------------------------------------------------------------
NET_DEPTH_W, NET_DEPTH_H = 320, 240   # resolution of the network-rendered training views


def build_scene(device, mlp, source="network", n_rays=0, workload="view", fusion_form="projective"):
    """Fuse the room's TSDF twice: from the 100 analytic 640x480 depth maps (the
    configuration's fusion workload, timed) and from the network's own rendered
    depth of the same training poses (Sec. 3.2: the TSDF is built from the
    trained model's depth, Eq. 2), rendered with the same-GPU 64+32 sampler.
    The second grid is the one the timed render path marches."""
    import torch
    from paper_2311_17878_gb300 import synth
    from paper_2311_17878_gb300 import tsdfs as T
    wl = synth.room_workload_torch(device=device)
    grid_an = T.Grid(wl.grid, device=device).init()
    depth = wl.views.depth.contiguous()
    K = torch.tensor(wl.views.K, device=device)
    P = torch.tensor(wl.views.c2w, device=device)
    torch.cuda.synchronize()
    fuse_ms = []
    for _ in range(3):
        grid_an.init()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        grid_an.integrate(depth, K, P)
        e1.record()
        torch.cuda.synchronize()
        fuse_ms.append(e0.elapsed_time(e1))
    rays = []
    centres = synth.room_panorama_centres(N_VIEWS_TIMED) if workload == "panorama" else None
    for i in range(N_VIEWS_TIMED):
        o, d = synth.room_heldout_rays(i) if centres is None else synth.room_panorama_rays(center=tuple(centres[i]))
        if n_rays:
            idx = np.sort(synth.sub_sample(len(o), n_rays, seed=50 + i))
            o, d = np.ascontiguousarray(o[idx]), np.ascontiguousarray(d[idx])
        rays.append((torch.tensor(o, device=device), torch.tensor(d, device=device), o, d))
    fusion = {"workload": "100 analytic 640x480 depth maps into 256^3", "ms": min(fuse_ms),
              "voxels_per_s": wl.grid.nx * wl.grid.ny * wl.grid.nz / (min(fuse_ms) / 1e3),
              "voxel_views_per_s": wl.grid.nx * wl.grid.ny * wl.grid.nz * depth.shape[0] / (min(fuse_ms) / 1e3)}
    # Alg. 2 as printed (every pixel's ray marched) on the same maps, timed once after a warm-up
    grid_rc = T.Grid(wl.grid, device=device).init()
    ws_rc = torch.empty(T.tsdfs_raycast_workspace_size(grid_rc), dtype=torch.uint8, device=device)
    grid_rc.integrate_raycast(depth[:2].contiguous(), K[:2].contiguous(), P[:2].contiguous(), ws_rc)
    grid_rc.init()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    grid_rc.integrate_raycast(depth, K, P, ws_rc)
    e1.record()
    torch.cuda.synchronize()
    fusion["raycast_ms"] = e0.elapsed_time(e1)
    fusion["raycast_rays_per_s"] = depth.numel() / (fusion["raycast_ms"] / 1e3)
    del grid_rc
    if source == "analytic":
        mask = grid_an.inside_mask(wl.bounds.nb_radius)
        fusion["grid_for_render"] = "fused from the 100 analytic depth maps"
        return wl, grid_an, grid_an, mask, rays, fusion, depth
    # the network's depth of the training views
    t_net = time.perf_counter()
    c2ws = wl.views.c2w.reshape(-1, 3, 4).astype(np.float64)
    f = 500.0 * NET_DEPTH_W / 640.0
    hier = T.HierRenderer(mlp, NET_DEPTH_W * NET_DEPTH_H, device=device)
    ndepth = torch.empty((len(c2ws), NET_DEPTH_H, NET_DEPTH_W), dtype=torch.float32, device=device)
    bp = wl.bounds
    for i, c2w in enumerate(c2ws):
        o, d = synth.pinhole_rays(c2w, f, f, NET_DEPTH_W / 2.0, NET_DEPTH_H / 2.0, NET_DEPTH_W, NET_DEPTH_H)
        out = hier.render(grid_an, torch.tensor(o, dtype=torch.float32, device=device),
                          torch.tensor(d, dtype=torch.float32, device=device), bp.t_near, bp.t_far)
        ndepth[i] = torch.where(out.wsum > 0.5, out.depth, torch.full_like(out.depth, float("inf"))).reshape(
            NET_DEPTH_H, NET_DEPTH_W)
    Kn = torch.tensor(np.tile(np.array([f, f, NET_DEPTH_W / 2.0, NET_DEPTH_H / 2.0], np.float32), (len(c2ws), 1)),
                      device=device)
    grid = T.Grid(wl.grid, device=device).init()
    if fusion_form == "raycast":
        grid.integrate_raycast(ndepth, Kn, P, ws_rc)
    else:
        grid.integrate(ndepth, Kn, P)
    mask = grid.inside_mask(wl.bounds.nb_radius)
    torch.cuda.synchronize()
    t_net = time.perf_counter() - t_net
    fusion["grid_for_render"] = (f"fused ({fusion_form} form) from the network's depth of the 100 training poses at "
                                 f"{NET_DEPTH_W}x{NET_DEPTH_H} (64+32 sampler, same GPU), setup {t_net:.1f} s")
    return wl, grid, grid_an, mask, rays, fusion, depth


def build_scene_large(device, n_rays=0):
    """The large configuration: 300 analytic 1280x960 depth maps fused into the 512^3
    fp16 grid (timed, three times), 8 panoramas of 2048x1024 from seeded centres."""
    import torch
    from paper_2311_17878_gb300 import synth
    from paper_2311_17878_gb300 import tsdfs as T
    t_gen = time.perf_counter()
    wl = synth.large_workload_torch(device=device)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    grid = T.Grid(wl.grid, device=device).init()
    depth = wl.views.depth.contiguous()
    K = torch.tensor(wl.views.K, device=device)
    P = torch.tensor(wl.views.c2w, device=device)
    fuse_ms = []
    for _ in range(3):
        grid.init()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        grid.integrate(depth, K, P)
        e1.record()
        torch.cuda.synchronize()
        fuse_ms.append(e0.elapsed_time(e1))
    mask = grid.inside_mask(wl.bounds.nb_radius)
    rays = []
    for c in synth.large_panorama_centres(N_VIEWS_TIMED):
        o, d = synth.room_panorama_rays(2048, 1024, center=tuple(c))
        if n_rays:
            idx = np.sort(synth.sub_sample(len(o), n_rays, seed=60 + len(rays)))
            o, d = np.ascontiguousarray(o[idx]), np.ascontiguousarray(d[idx])
        rays.append((torch.tensor(o, device=device), torch.tensor(d, device=device), o, d))
    nvox = wl.grid.nx * wl.grid.ny * wl.grid.nz
    fusion = {"workload": "300 analytic 1280x960 depth maps into 512^3 fp16", "ms": min(fuse_ms),
              "voxels_per_s": nvox / (min(fuse_ms) / 1e3),
              "voxel_views_per_s": nvox * depth.shape[0] / (min(fuse_ms) / 1e3),
              "grid_for_render": f"fused from the analytic depth maps (generated in {t_gen:.1f} s)"}
    return wl, grid, grid, mask, rays, fusion, depth


def run_ours(args, ws, rank, local):
    import torch
    from paper_2311_17878_gb300 import build as B
    from paper_2311_17878_gb300 import synth
    from paper_2311_17878_gb300 import tsdfs as T
    B.build()
    if args.train_pitch is not None:
        synth.TRAIN_PITCH_DEG = args.train_pitch
    dev = f"cuda:{local}"
    spec = synth.scene_mlp("room")
    prec = args.precision
    PREC = {"f16": T.TSDFS_PREC_F16, "bf16": T.TSDFS_PREC_BF16, "bf16x2": T.TSDFS_PREC_BF16X2, "f32": T.TSDFS_PREC_F32}
    mlp = T.Mlp(spec, PREC[prec], device=dev)
    mlp_depth = mlp if prec != "f32" else T.Mlp(spec, T.TSDFS_PREC_F16, device=dev)
    if args.workload == "large":
        wl, grid, grid_an, mask, rays, fusion, depth = build_scene_large(dev, args.rays)
    else:
        wl, grid, grid_an, mask, rays, fusion, depth = build_scene(dev, mlp_depth, args.grid_source, args.rays,
                                                                   args.workload, args.fusion)
    vs = wl.grid.voxel_size
    bp = synth.BoundsParams(**{**wl.bounds.__dict__, "d_s": args.ds_vox * vs})
    if args.m_confirm is not None:
        bp.m_confirm = args.m_confirm
    if args.nb_radius is not None:
        bp.nb_radius = args.nb_radius
    if args.step_vox is not None:
        bp.n_max = max(bp.n_max, int(round(bp.n_max * bp.step / (args.step_vox * vs))))
        bp.step = args.step_vox * vs
    if bp.nb_radius != wl.bounds.nb_radius:
        mask = grid.inside_mask(bp.nb_radius)
    n = rays[0][0].shape[0]
    max_samples = n * max(bp.n_max, bp.n_fallback)
    if args.workload == "large":
        # size the sample workspace from the batch's own counts (n x 96 would be 9.7 GB of records)
        bcount = T.Bounds(n, device=dev)
        tot = 0
        for i in range(N_VIEWS_TIMED):
            bcount.compute(grid, rays[i][0], rays[i][1], bp, mask)
            tot = max(tot, int(bcount.offsets[-1].item()))
        max_samples = tot if args.recovery_tau is None else n * max(bp.n_max, bp.n_fallback)
        del bcount
    bounds = T.Bounds(n, device=dev)
    # the march's launch shape, picked by the library's autotuner on the first view's rays
    tuned = bounds.autotune(grid, rays[0][0], rays[0][1], bp, mask, reps=3)
    rend = T.Renderer(mlp, n, max_samples, device=dev)
    # the network kernel: fixed, or picked by the library's autotuner on view 0's rays
    net_kernel = None
    if prec != "f32":
        if args.net_kernel == "auto":
            bounds.compute(grid, rays[0][0], rays[0][1], bp, mask)
            kk, ms_s, ms_p = rend.autotune(rays[0][0], rays[0][1], bounds, reps=3)
            net_kernel = {"kernel": {1: "serial", 2: "pipelined"}[kk], "autotuned_ms": {"serial": ms_s, "pipelined": ms_p}}
        else:
            kk = {"serial": T.TSDFS_NETKERNEL_SERIAL, "pipelined": T.TSDFS_NETKERNEL_PIPELINED}[args.net_kernel]
            T.tsdfs_set_network_kernel(PREC[prec], kk)
            net_kernel = {"kernel": args.net_kernel, "autotuned_ms": None}
    rec = T.Recovery(mlp, n, bp.n_fallback, device=dev) if args.recovery_tau is not None else None
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 129 MB L2

    def step(i):
        o, d = rays[i % N_VIEWS_TIMED][:2]
        bounds.compute(grid, o, d, bp, mask)
        out = rend.render(o, d, bounds)
        if rec is not None:
            rec.apply(grid, o, d, bp, args.recovery_tau, out, bounds)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    graphs = []
    if args.graph:
        # each view's bounds + render as one CUDA graph (no host synchronisation inside)
        for i in range(N_VIEWS_TIMED):
            step(i)
        torch.cuda.synchronize()
        for i in range(N_VIEWS_TIMED):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                step(i)
            graphs.append(g)
        for i in range(N_VIEWS_TIMED):
            graphs[i].replay()
        torch.cuda.synchronize()

    def timed_step(k):
        if graphs:
            graphs[k % N_VIEWS_TIMED].replay()
        else:
            step(k)

    samples_per_view, fallback_per_view = [], []
    for i in range(N_VIEWS_TIMED):
        bounds.compute(grid, rays[i][0], rays[i][1], bp, mask)
        extra = 0
        if rec is not None:
            out_i = rend.render(rays[i][0], rays[i][1], bounds)
            rec.apply(grid, rays[i][0], rays[i][1], bp, args.recovery_tau, out_i, bounds)
            extra = int(rec.bounds.offsets[-1].item())
        samples_per_view.append(int(bounds.offsets[-1].item()) + extra)
        fallback_per_view.append(round(float((bounds.status == 2).float().mean().item()), 4))
    st = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    T.lib().tsdfs_profile(1)
    barrier(ws)
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")   # lets a profiler select the timed launches
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            evs[k][0].record(st)
            timed_step(k)
            evs[k][1].record(st)
        torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier(ws)
    t_wall = time.perf_counter() - t_wall
    if graphs:
        # graph replays carry no per-kernel events: time the kernels on an eager pass over the same views
        T.lib().tsdfs_profile(0)
        T.lib().tsdfs_profile(1)
        for k in range(args.steps):
            flush.fill_(float(k))
            step(k)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    mlp_name = "mlp_simt" if prec == "f32" else (
        "mlp_pipe" if T.tsdfs_network_kernel(PREC[prec]) == T.TSDFS_NETKERNEL_PIPELINED else "mlp_tc")
    import ctypes as C
    ms_k, n_k = C.c_double(0), C.c_int64(0)
    T.lib().tsdfs_profile_read(mlp_name.encode(), C.byref(ms_k), C.byref(n_k))
    ms_b, n_b = C.c_double(0), C.c_int64(0)
    T.lib().tsdfs_profile_read(b"ray_bounds", C.byref(ms_b), C.byref(n_b))
    ms_all, n_all = C.c_double(0), C.c_int64(0)
    T.lib().tsdfs_profile_read(b"", C.byref(ms_all), C.byref(n_all))
    T.lib().tsdfs_profile(0)
    total_ms = max_over_ranks(sum(step_ms), ws)
    rays_total = n * args.steps * ws
    value = rays_total / (total_ms / 1e3)
    samples_timed = sum(samples_per_view[k % N_VIEWS_TIMED] for k in range(args.steps))
    # dominant kernel roofline (algorithmic FLOPs per launch / mean launch time)
    hbm, bf16_burst, bf16_sus, peak_src = measured_peaks()
    # L2 read bandwidth, measured here: the bound of the march over an L2-resident grid
    l2buf = torch.empty(64 * 1024 * 1024 // 4, dtype=torch.float32, device=dev).fill_(1.0)
    l2_peak = max(T.tsdfs_l2_read_probe(l2buf, reps=20) for _ in range(3))
    del l2buf
    # algorithmic FLOPs of the timed steps over the kernel's time in the same steps (with the
    # recovery pass a step launches the kernel twice, so per-launch means would mislead)
    mlp_ms = ms_k.value / max(args.steps, 1)
    achieved = ALGO_FLOP_PER_SAMPLE * samples_timed / (ms_k.value / 1e3) / 1e12 if ms_k.value > 0 else 0.0
    if prec != "f32":
        roof = {"bound": "tensor", "achieved": achieved, "peak": bf16_burst, "unit": "TFLOP/s",
                "frac": achieved / bf16_burst,
                "traffic": captured_traffic(MLP_TC_TRAFFIC, MLP_TC_SOURCES, args, prec) if mlp_name == "mlp_tc" else None,
                "peak_kind": f"bf16 dense burst ({peak_src}); fp16 dense has the same nominal rate",
                "kernel": mlp_name,
                "executed_tflops": achieved * EXEC_FLOP_PER_SAMPLE[
                    "serial" if mlp_name == "mlp_tc" else ("pipelined-split" if prec == "bf16x2" else "pipelined")]
                / ALGO_FLOP_PER_SAMPLE}
    else:
        fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x 2 flop x max SM clock
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": None,
                "peak_kind": "fp32 FMA, 152 SMs x 128 lanes x 2 x 2.07 GHz", "kernel": "mlp_simt"}
    # the GPU's own bounds of view 0, for the march's roofline line
    bv = T.Bounds(n, device=dev)
    bv.compute(grid, rays[0][0], rays[0][1], bp, mask)
    march_tf, march_status = bv.t_f.cpu().numpy(), bv.status.cpu().numpy()
    del bv
    kernel_share = {"mlp_ms_per_step": mlp_ms, "mlp_launches_per_step": n_k.value / max(args.steps, 1),
                    "all_kernels_ms_per_step": ms_all.value / max(args.steps, 1)}
    main_only = args.only_main
    lean = main_only or args.quality_only
    # end to end through the public API with host buffers
    e2e = None if lean else run_e2e(args, grid, mask, bp, bounds, rend, rays, n, dev, flush)
    # the cpu_baseline leg: the oracle timed on a bounded sample, and its outputs on the quality
    # pixels (the only place outside the reference arm where the bench runs the oracle); the room
    # networks are not fitted to the large floor, so its images have no quality to score
    want_q = not (args.no_quality or main_only or rank != 0 or args.workload == "large")
    cpu = run_cpu_baseline(wl, grid, rays, bp, spec) if (rank == 0 and ws == 1 and not lean) else None
    refs = oracle_references(wl, grid, rays, bp, spec, args.recovery_tau) if want_q else None
    # the hierarchical comparator (K7) and the operating points, timed and scored alike
    hier_r = None if lean else T.HierRenderer(mlp, n, device=dev)
    quality = QualityLeg(refs, args, wl, grid, mask, bounds, rend, rec, mlp, rays, bp, n, dev, flush).run_all(
        hier_r, args.sweep) if (want_q and hier_r is not None) else None
    oracle_best_gate(refs, quality)
    comparator = None
    if quality is not None:
        comparator = {"impl": "hier n_c + n_f (same GPU, same network engine)",
                      "ladder": [{k: h[k] for k in ("name", "rays_s", "ms_per_view", "psnr", "samples_per_ray")}
                                 for h in quality["hier"]]}
    elif hier_r is not None:
        comparator = time_hier_only(hier_r, grid, rays, bp, n, flush)
    del hier_r
    train = None
    if rank == 0 and not lean:
        from paper_2311_17878_gb300 import tsdfs as T
        large = args.workload == "large"
        train = run_train(spec, wl, grid, mask, dev, n_rays=65536 if large else 8192, peak_bf16=bf16_burst)
        if not large:
            # the FP32 SIMT backward on the same step, and the layer-major one at 65 536 rays
            train["simt_backward"] = run_train(spec, wl, grid, mask, dev, n_rays=8192, iters=2,
                                               kind=T.TSDFS_BACKWARD_SIMT)
            train["rays_65536"] = run_train(spec, wl, grid, mask, dev, n_rays=65536, iters=3, peak_bf16=bf16_burst)
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": prec, "data": "synthetic (seeded room scene, fitted networks)",
        "config": {"workload": WORKLOAD, "rays_per_step": n, "views": N_VIEWS_TIMED,
                   "samples_per_step": samples_timed / args.steps,
                   "grid": f"{wl.grid.nx}^3 {wl.grid.dtype} + uint8",
                   "alg1": {"d_s_vox": bp.d_s / vs, "m_confirm": bp.m_confirm, "nb_radius": bp.nb_radius,
                            "step_vox": bp.step / vs, "n_max": bp.n_max, "n_fallback": bp.n_fallback},
                   "fallback_frac_per_view": fallback_per_view,
                   "grid_source": "analytic" if args.workload == "large" else args.grid_source,
                   "fusion_form": args.fusion,
                   "ray_subset": args.rays or None,
                   "cuda_graph": bool(graphs), "train_pitch_deg": synth.TRAIN_PITCH_DEG,
                   "march_launch": {"block": tuned[0], "blocks_per_sm": tuned[1], "autotuned_ms": tuned[2]},
                   "network_kernel": net_kernel,
                   "recovery_tau": args.recovery_tau,
                   "networks": "SDF 8x256 PE6 skip4 + colour 4x256 PE4", "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{ws}, rays independent", "wall_s": t_wall},
        "comparator_equal_psnr": equal_psnr_comparison(quality),
        "pareto": pareto_front(quality),
        "e2e": e2e, "gpu_launches": int(n_all.value), "roofline": roof,
        "roofline_march": dict(march_roofline(wl.grid, rays[0][2], rays[0][3], march_tf, march_status, bp,
                                              ms_b.value / max(n_b.value, 1), hbm, peak_src, l2_peak),
                               traffic=captured_traffic(MARCH_TRAFFIC, MARCH_SOURCES, args, prec))
        if rank == 0 else None,
        "cpu_baseline": cpu, "clocks": clocks, "kernel_time": kernel_share,
        "psnr_gate": None if quality is None else {k: quality[k] for k in (
            "pixels", "psnr_tsdf_gpu", "psnr_tsdf_oracle", "meets_oracle_minus_0p1dB", "psnr_hier96_gpu")},
        "comparator": comparator, "fusion": fusion, "train_step": train,
        "quality": quality,
    }
    return line


def time_hier_only(h, grid, rays, bp, n, flush):
    """The 64 + 32 comparator alone (the large floor has no quality leg): one pass over the
    timed views, L2 flushed before each."""
    import torch
    st = torch.cuda.current_stream()
    h.render(grid, rays[0][0], rays[0][1], bp.t_near, bp.t_far)
    torch.cuda.synchronize()
    ms = []
    for v in range(N_VIEWS_TIMED):
        flush.fill_(float(v))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        h.render(grid, rays[v][0], rays[v][1], bp.t_near, bp.t_far)
        e1.record(st)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return {"impl": "hier 64+32 (same GPU, same network engine)",
            "ladder": [{"name": "hier 64+32", "rays_s": n * len(ms) / (sum(ms) / 1e3), "ms_per_view": float(np.mean(ms)),
                        "psnr": None, "samples_per_ray": 96}]}


def _best_hier(hier, p):
    ok = [h for h in hier if h["psnr"] >= p]
    return max(ok, key=lambda h: h["rays_s"]) if ok else None


def equal_psnr_comparison(q):
    """The target's comparison: the TSDF render (the timed default) against the fastest
    hierarchical configuration (64 + 32 and the smaller ladder) whose PSNR on the quality
    pixels is at least as high, every configuration timed the same way (one pass over the
    timed views, L2 flushed before each view); then the same for each operating point of the
    sweep, and the best of them."""
    if not q:
        return None
    hier, t = q["hier"], q["tsdf"]
    b = _best_hier(hier, t["psnr"])
    out = {"tsdf": {"rays_s": t["rays_s"], "psnr": t["psnr"], "samples_per_ray": t["samples_per_ray"]},
           "hier_at_ge_psnr": None if b is None else {k: b[k] for k in ("name", "rays_s", "psnr")},
           "tsdf_over_hier": t["rays_s"] / b["rays_s"] if b else None}
    best = None
    for c in [t] + q.get("sweep", []):
        bh = _best_hier(hier, c["psnr"])
        # no hierarchical configuration reaches this PSNR: compare with the most accurate one
        ref = bh if bh is not None else max(hier, key=lambda h: h["psnr"])
        r = c["rays_s"] / ref["rays_s"]
        if bh is not None and (best is None or r > best["tsdf_over_hier"]):
            best = {"name": c["name"], "rays_s": c["rays_s"], "psnr": c["psnr"],
                    "samples_per_ray": c["samples_per_ray"], "hier": bh["name"], "hier_rays_s": bh["rays_s"],
                    "hier_psnr": bh["psnr"], "tsdf_over_hier": r}
    if best is not None and q.get("best_operating_point_gate"):
        best["gate"] = q["best_operating_point_gate"]
    out["best_operating_point"] = best
    return out


def pareto_front(q):
    """Every configuration of the quality leg as (rays/s, PSNR), fastest first; `front`
    marks those that no other configuration beats on both."""
    if not q:
        return None
    pts = [dict(kind="tsdf", name=q["tsdf"]["name"], rays_s=q["tsdf"]["rays_s"], psnr=q["tsdf"]["psnr"],
                spr=q["tsdf"]["samples_per_ray"])]
    pts += [dict(kind="tsdf", name=c["name"], rays_s=c["rays_s"], psnr=c["psnr"], spr=c["samples_per_ray"])
            for c in q.get("sweep", [])]
    pts += [dict(kind="hier", name=h["name"], rays_s=h["rays_s"], psnr=h["psnr"], spr=h["samples_per_ray"])
            for h in q["hier"]]
    for p_ in pts:
        p_["front"] = not any(o is not p_ and o["rays_s"] >= p_["rays_s"] and o["psnr"] >= p_["psnr"] and
                              (o["rays_s"] > p_["rays_s"] or o["psnr"] > p_["psnr"]) for o in pts)
    for p_ in pts:
        p_["rays_s"] = round(p_["rays_s"] / 1e6, 3)   # M rays/s
        p_["psnr"] = round(p_["psnr"], 2)
        p_["spr"] = round(p_["spr"], 1)
    return sorted(pts, key=lambda p_: -p_["rays_s"])


def march_roofline(spec, o, d, t_f, status, bp, ms_per_launch, hbm, peak_src, l2=None):
    """Roofline line of the ray march (Alg. 1, k_ray_bounds): every voxel the walk tests reads
    one 32-bit word (its value in the near phase, its inside-mask word in the far phase), plus
    24 B of ray in and 17 B of bounds out per ray.  A ray's walk covers [t0, t_f] when it is
    BOUNDED and [t0, t_end] when it falls back ([t0, t_end]: the grid-box clip of [t_near,
    t_far]); the voxels it tests are counted as that length times the voxel-boundary crossings
    per unit length, (|d_x| + |d_y| + |d_z|) / voxel size, plus the first voxel.  t_f and the
    status are the GPU's own bounds of the same rays."""
    o, d = np.asarray(o, np.float64), np.asarray(d, np.float64)
    lo = np.asarray(spec.origin, np.float64)
    hi = lo + np.array([spec.nx, spec.ny, spec.nz], np.float64) * spec.voxel_size
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        ta, tb = (lo - o) * inv, (hi - o) * inv
        t0 = np.maximum(np.nanmax(np.minimum(ta, tb), axis=1), bp.t_near)
        t_end = np.minimum(np.nanmin(np.maximum(ta, tb), axis=1), bp.t_far)
    stop = np.where(status == 1, t_f, t_end)
    walked = status != 0
    length = np.where(walked, np.maximum(stop - t0, 0.0), 0.0)
    vox = length * np.abs(d).sum(1) / spec.voxel_size + walked
    bytes_per_ray = 4.0 * float(np.mean(vox)) + 41.0
    achieved = bytes_per_ray * len(o) / (ms_per_launch / 1e3) / 1e9 if ms_per_launch > 0 else 0.0
    grid_bytes = spec.nx * spec.ny * spec.nz * (2 if spec.dtype == "f16" else 4)
    in_l2 = grid_bytes < 100e6   # the grid (and its 1-bit inside mask) stays in the 129 MB L2
    out = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
           "traffic": None, "kernel": "ray_bounds", "voxels_per_ray": float(np.mean(vox)),
           "bytes_per_ray": bytes_per_ray, "ms_per_launch": ms_per_launch,
           "peak_kind": f"HBM copy ({peak_src})"}
    if l2:
        # the march reads an L2-resident grid: its bound is L2 bandwidth (measured in this run)
        out["l2_peak"] = l2
        out["frac_l2"] = achieved / l2
        if in_l2:
            out.update(bound="l2", peak=l2, frac=achieved / l2,
                       peak_kind=f"L2 streaming read measured in this run (tsdfs_l2_read_probe, 64 MB); "
                                 f"grid of {grid_bytes / 1e6:.0f} MB stays in L2; HBM copy {hbm} GB/s ({peak_src})")
    return out


def backward_gemm_flops(spec):
    """Algorithmic FLOPs per sample of the layer-major backward's GEMMs: the forward
    recomputation P = X W^T (value + 3 tangent rows per sample in the SDF network), the
    weight gradients G^T X (as many FLOPs) and the input adjoints G W (all layers but
    the SDF network's first)."""
    sdf = 4 * sum(2 * W.shape[0] * W.shape[1] for W, _ in spec.sdf)
    rgb = sum(2 * W.shape[0] * W.shape[1] for W, _ in spec.rgb)
    fwd = sdf + rgb
    first = 4 * 2 * spec.sdf[0][0].size
    return {"forward": fwd, "weight_grad": fwd, "input_adjoint": fwd - first}


def run_train(spec, wl, grid, mask, dev, n_rays=8192, iters=5, kind=None, peak_bf16=None, nvtx=False):
    """One training step of the networks (FP32): n_rays random rays of the training
    views, bounds, render through the autograd op, L1 colour + 0.1 eikonal on the
    bounded samples, backward (render_rays_backward with the given implementation)."""
    import torch
    from paper_2311_17878_gb300 import synth
    from paper_2311_17878_gb300 import tsdfs as T
    kind = T.TSDFS_BACKWARD_GEMM if kind is None else kind
    old_kind = T.tsdfs_backward_kernel()
    T.tsdfs_set_backward_kernel(kind)
    mlp = T.Mlp(spec, T.TSDFS_PREC_F32, device=dev)
    o, d, vi, px, py = synth.random_rays_from_views(wl.views, n_rays)
    o, d = torch.tensor(o, device=dev), torch.tensor(d, device=dev)
    target = torch.rand((n_rays, 3), device=dev, generator=torch.Generator(device=dev).manual_seed(0))
    b = T.Bounds(n_rays, device=dev)
    ms_cap = n_rays * max(wl.bounds.n_max, wl.bounds.n_fallback)
    sdf_w = mlp.sdf_w.clone().requires_grad_(True)
    rgb_w = mlp.rgb_w.clone().requires_grad_(True)

    def step():
        b.compute(grid, o, d, wl.bounds, mask)
        n_b = torch.clamp((b.n * (b.status == 1)).sum(), min=1)
        rgb, depth, eik = T.RenderFunction.apply(sdf_w, rgb_w, mlp, o, d, b, ms_cap)
        loss = (rgb - target).abs().mean() + 0.1 * eik.sum() / n_b
        sdf_w.grad = None
        rgb_w.grad = None
        loss.backward()
        return loss

    try:
        for _ in range(2):
            step()
        torch.cuda.synchronize()
        if nvtx:
            with torch.autograd.set_multithreading_enabled(False):
                torch.cuda.nvtx.range_push("timed")
                step()
                torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
        import ctypes as C
        T.lib().tsdfs_profile(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(iters):
            loss = step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / iters
        split = {}
        for name in ("mlp_simt", "composite", "train_forward", "train_forward_network", "train_forward_composite",
                     "backward", "backward_forward", "backward_composite", "backward_network", "ray_bounds"):
            t, c = C.c_double(0), C.c_int64(0)
            T.lib().tsdfs_profile_read(name.encode(), C.byref(t), C.byref(c))
            if c.value:
                split[name + "_ms"] = t.value / iters
        T.lib().tsdfs_profile(0)
    finally:
        T.tsdfs_set_backward_kernel(old_kind)
    samples = int(b.offsets[-1].item())
    gemm = kind == T.TSDFS_BACKWARD_GEMM
    out = {"rays": n_rays, "ms_per_step": ms, "rays_per_s": n_rays / (ms / 1e3), "samples": samples,
           "loss": float(loss.item()), "kernel_ms": split,
           "backward": "render_rays_train (layer-major FP32 forward that keeps its activations) + "
                       "render_rays_backward_kept: GEMMs in cuBLAS BF16x9-emulated FP32 on the tensor cores"
           if gemm else "render_rays (FP32 SIMT) + render_rays_backward (FP32 SIMT, tiles of 8 samples)",
           "what": "bounds + render (fp32) + L1 + 0.1 eikonal + backward through both networks"}
    if gemm and "backward_network_ms" in split:
        f = backward_gemm_flops(spec)
        chunk = T.tsdfs_backward_chunk_samples(mlp, ms_cap)
        n_chunks = -(-samples // chunk)
        passes = n_chunks   # the training forward, then every chunk but the last recomputed
        flops = samples * f["weight_grad"] + samples * f["input_adjoint"] + \
            min(samples, chunk * (n_chunks - 1)) * f["forward"] + samples * f["forward"]
        t_net = split.get("train_forward_network_ms", 0.0) + split.get("backward_network_ms", 0.0)
        ach = flops / (t_net / 1e3) / 1e12 if t_net > 0 else None
        peak = peak_bf16 / 9.0 if peak_bf16 else None
        out["roofline"] = {"bound": "tensor", "achieved": ach, "unit": "TFLOP/s",
                           "peak": peak, "frac": (ach / peak) if (ach and peak) else None,
                           "flops_per_sample": f, "chunk_samples": chunk, "chunks": passes,
                           "workspace_bytes": T.tsdfs_backward_workspace_size(mlp, n_rays, ms_cap),
                           "what": "GEMM FLOPs (the training forward, chunks other than the last recomputed, "
                                   "weight gradients, input adjoints) over the time of the forward's and the "
                                   "backward's network phases (element-wise kernels and bias GEMVs included)",
                           "peak_kind": "measured bf16 dense peak / 9 (each FP32 operand as three BF16 parts, nine "
                                        "products per FP32 product)"}
    return out


def run_train_only(args):
    """The profiling case of the training step: two warm-up steps, then one step inside an
    NVTX range named 'timed' with autograd on the calling thread (so the backward's kernels
    fall inside the range), on the room grid fused from the 100 analytic depth maps."""
    import torch
    from paper_2311_17878_gb300 import build, synth
    from paper_2311_17878_gb300 import tsdfs as T
    build.build()
    dev = "cuda"
    wl = synth.room_workload_torch(device=dev)
    grid = T.Grid(wl.grid, device=dev).init()
    grid.integrate(wl.views.depth.contiguous(), torch.tensor(wl.views.K, device=dev),
                   torch.tensor(wl.views.c2w, device=dev))
    mask = grid.inside_mask(wl.bounds.nb_radius)
    T.tsdfs_set_backward_chunk(args.train_chunk)
    try:
        return run_train(synth.scene_mlp("room"), wl, grid, mask, dev, n_rays=args.train_rays, iters=1, nvtx=True)
    finally:
        T.tsdfs_set_backward_chunk(0)


def run_e2e(args, grid, mask, bp, bounds, rend, rays, n, dev, flush):
    """The metric end to end through the public Python API over the C ABI: each step copies
    the view's rays in from pinned host memory, runs bounds + render and copies rgb and depth
    out, between CUDA events on the launching stream; L2 is flushed before each step (outside
    the timed region), as in the device-timed leg."""
    import torch
    st = torch.cuda.current_stream()
    h_o = [torch.tensor(r[2]).pin_memory() for r in rays]
    h_d = [torch.tensor(r[3]).pin_memory() for r in rays]
    d_o = torch.empty_like(rays[0][0])
    d_d = torch.empty_like(rays[0][1])
    h_rgb = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    h_depth = torch.empty(n, dtype=torch.float32).pin_memory()

    def step(k):
        i = k % N_VIEWS_TIMED
        d_o.copy_(h_o[i], non_blocking=True)
        d_d.copy_(h_d[i], non_blocking=True)
        bounds.compute(grid, d_o, d_d, bp, mask)
        out = rend.render(d_o, d_d, bounds)
        h_rgb.copy_(out.rgb, non_blocking=True)
        h_depth.copy_(out.depth, non_blocking=True)

    for k in range(max(2, args.warmup)):
        step(k)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record(st)
        step(k)
        evs[k][1].record(st)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs)
    return {"value": n * args.steps / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": n * 24,
            "d2h_bytes_per_step": n * 16, "ms_per_step": ms / args.steps,
            "api": "tsdfs.py binding over the C ABI (Bounds.compute + Renderer.render), pinned host buffers",
            "l2": "flushed before each step (256 MB write, outside the timed region)"}


def psnr(a, b, peak=1.0):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10.0 * math.log10(peak * peak / mse)


class QualityLeg:
    """Image quality and throughput of every configuration on the same footing: one pass over
    the timed views, each view rendered between CUDA events on the launching stream with L2
    flushed before it, the quality pixels (seeded, spread over all views) gathered after and
    scored against the oracle's dense reference (`refs`, from the cpu_baseline leg)."""

    def __init__(self, refs, args, wl, grid, mask, bounds, rend, rec, mlp, rays, bp, n, dev, flush):
        import torch
        self.refs, self.args, self.wl, self.grid, self.mask = refs, args, wl, grid, mask
        self.bounds, self.rend, self.rec, self.mlp, self.rays, self.bp = bounds, rend, rec, mlp, rays, bp
        self.n, self.dev, self.flush = n, dev, flush
        self.idx_t = [torch.as_tensor(ix, device=dev) for ix in refs["pixels"]]
        self.cuts = np.cumsum([0] + [len(ix) for ix in refs["pixels"]])
        self.dense = refs["dense"]
        self.masks = {bp.nb_radius: mask}

    def mask_for(self, nb):
        if nb not in self.masks:
            self.masks[nb] = self.grid.inside_mask(nb)
        return self.masks[nb]

    def run(self, name, render_view, evals=None, keep=None):
        """render_view(v) -> outputs with rgb / depth / wsum / normal; evals(v) -> network
        evaluations of view v (read after the pass); keep(v, out) saves tensors for later."""
        import torch
        st = torch.cuda.current_stream()
        render_view(0)
        torch.cuda.synchronize()
        ms, rgb, depth, ev = [], [], [], 0
        for v in range(N_VIEWS_TIMED):
            self.flush.fill_(float(v))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            out = render_view(v)
            e1.record(st)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            rgb.append(out.rgb[self.idx_t[v]].cpu().numpy())
            depth.append(out.depth[self.idx_t[v]].cpu().numpy())
            if evals is not None:
                ev += evals(v)
            if keep is not None:
                keep(v, out)
        rgb = np.concatenate(rgb)
        c = self.cuts
        return {"name": name, "rays_s": self.n * N_VIEWS_TIMED / (sum(ms) / 1e3), "ms_per_view": float(np.mean(ms)),
                "psnr": psnr(rgb, self.dense["rgb"]),
                "psnr_per_view": [round(psnr(rgb[c[v]:c[v + 1]], self.dense["rgb"][c[v]:c[v + 1]]), 2)
                                  for v in range(N_VIEWS_TIMED)],
                "ms_per_view_list": [round(m, 3) for m in ms],
                "samples_per_ray": ev / (self.n * N_VIEWS_TIMED) if evals is not None else None,
                "_rgb": rgb, "_depth": np.concatenate(depth)}

    # ---- the timed default -------------------------------------------------
    def tsdf_default(self):
        import torch
        b, rend, rec, kept = self.bounds, self.rend, self.rec, {}

        def render_view(v):
            o, d = self.rays[v][:2]
            b.compute(self.grid, o, d, self.bp, self.mask)
            out = rend.render(o, d, b)
            if rec is not None:
                rec.apply(self.grid, o, d, self.bp, self.args.recovery_tau, out, b)
            return out

        def evals(v):
            e = int(b.offsets[-1].item())
            return e + (int(rec.bounds.offsets[-1].item()) if rec is not None else 0)

        def keep(v, out):
            kept[v] = {"t_n": b.t_n.clone(), "t_f": b.t_f.clone(), "n": b.n.clone(), "status": b.status.clone(),
                       "wsum": out.wsum.clone()}
        r = self.run("default", render_view, evals, keep)
        r["_kept"] = kept
        return r

    # ---- the hierarchical comparator (K7) ------------------------------------
    def hier(self, h):
        import torch
        out, kept = [], {}
        for nc, nf in ((64, 32),) + HIER_LADDER:
            h.n_coarse, h.n_fine = nc, nf

            def render_view(v):
                o, d = self.rays[v][:2]
                return h.render(self.grid, o, d, self.bp.t_near, self.bp.t_far)

            def keep(v, o_):
                if nc == 64:
                    kept[v] = {"depth": o_.depth.clone(), "wsum": o_.wsum.clone()}
            r = self.run(f"hier {nc}+{nf}", render_view, lambda v: self.n * (nc + nf), keep)
            r.update(n_coarse=nc, n_fine=nf, value_evals_per_ray=nc)
            out.append(r)
        h.n_coarse, h.n_fine = 64, 32
        return out, kept

    # ---- one operating point of the sweep --------------------------------------
    def operating_point(self, cfg, pools):
        import torch
        from paper_2311_17878_gb300 import synth
        from paper_2311_17878_gb300 import tsdfs as T
        vs = self.wl.grid.voxel_size
        bp = synth.BoundsParams(**{**self.bp.__dict__, "d_s": cfg.get("d_s", self.bp.d_s / vs) * vs,
                                   "step": cfg.get("step", self.bp.step / vs) * vs,
                                   "m_confirm": cfg.get("m", self.bp.m_confirm),
                                   "nb_radius": cfg.get("nb", self.bp.nb_radius),
                                   "n_max": cfg.get("n_max", self.bp.n_max)})
        if cfg.get("step", None) is not None:
            bp.n_max = max(bp.n_max, int(round(self.bp.n_max * self.bp.step / bp.step)))
        mask = self.mask_for(bp.nb_radius)
        b = pools["bounds"]
        sampler = cfg.get("sampler", "mid")
        tau = cfg.get("tau")
        n = self.n
        if sampler == "mid":
            need = n * max(bp.n_max, bp.n_fallback)
            if pools.get("rend_cap", 0) < need:
                pools["rend"] = T.Renderer(self.mlp, n, need, device=self.dev)
                pools["rend_cap"] = need
            rend = pools["rend"]
        elif sampler == "rel":
            rend = pools["rend"]
            ac = pools["ac"]
        else:
            ac = pools["ac"]
            key = ("cf", cfg["n_fine"])
            if key not in pools:
                pools[key] = T.HierBoundedRenderer(self.mlp, n, cfg["n_fine"], n * 64, device=self.dev)
            hb = pools[key]
        rec = pools["rec"] if tau is not None else None
        n_mean = cfg.get("n_mean", 6.0)
        n_min, n_cap = cfg.get("n_min", 2), cfg.get("n_cap", 64)
        used = {}

        def render_view(v):
            o, d = self.rays[v][:2]
            b.compute(self.grid, o, d, bp, mask)
            bb = b if sampler == "mid" else ac.apply(b, n_mean, n_min, n_cap, 64)
            used["b"] = bb
            out = rend.render(o, d, bb) if sampler != "cf" else hb.render(o, d, bb)
            if rec is not None:
                rec.apply(self.grid, o, d, bp, tau, out, b)
            return out

        def evals(v):
            bb = used["b"]
            e = int(bb.offsets[-1].item())
            if sampler == "cf":
                e += cfg["n_fine"] * int((bb.n > 0).sum().item())
            return e + (int(rec.bounds.offsets[-1].item()) if rec is not None else 0)
        r = self.run(cfg["name"], render_view, evals)
        r["params"] = {k: v for k, v in cfg.items() if k != "name"}
        r["_bp"] = bp
        r["_cfg"] = cfg
        return r

    def diagnostics(self, kept, kept_h):
        """Per view, from the default bounds of every ray and the 64 + 32 comparator's depth as
        the surface t* (rays with its weight sum above 0.5): mean count, histogram of n (share at
        n_max), share of BOUNDED rays whose far phase ran to t_end, t_f - t* and t* - t_n in
        voxels, and the share of BOUNDED rays with t* outside [t_n, t_f] (Tab. 1's failures)."""
        import torch
        vs = self.wl.grid.voxel_size
        g = self.wl.grid
        lo = torch.tensor(g.origin, dtype=torch.float64, device=self.dev)
        hi = lo + torch.tensor([g.nx, g.ny, g.nz], dtype=torch.float64, device=self.dev) * vs
        edges = sorted({e for e in (1, 2, 4, 8, 16, 32, self.bp.n_max - 1, self.bp.n_max) if 1 <= e <= self.bp.n_max})
        out = []
        for v in range(N_VIEWS_TIMED):
            k, kh = kept[v], kept_h[v]
            o = self.rays[v][0].double()
            d = self.rays[v][1].double()
            inv = 1.0 / d
            ta, tb = (lo - o) * inv, (hi - o) * inv
            t_end = torch.clamp(torch.nan_to_num(torch.maximum(ta, tb), nan=float("inf")).amin(1), max=self.bp.t_far)
            st = k["status"]
            bnd = st == 1
            nb = max(int(bnd.sum().item()), 1)
            nn = k["n"][bnd]
            hist, prev = {}, 0
            for e in edges:
                hist[f"{prev + 1}-{e}" if e > prev + 1 else f"{e}"] = round(
                    float(((nn > prev) & (nn <= e)).sum().item()) / nb, 4)
                prev = e
            tn, tf = k["t_n"].double(), k["t_f"].double()
            far_end = bnd & (tf >= t_end - 1e-4)
            hit = bnd & (kh["wsum"] > 0.5)
            ts = kh["depth"].double()
            nh = max(int(hit.sum().item()), 1)
            dfar = ((tf - ts) / vs)[hit]
            dnear = ((ts - tn) / vs)[hit]
            fail = hit & ((ts < tn) | (ts > tf))

            def q(x, p_):
                return round(float(torch.quantile(x.float(), p_).item()), 2) if x.numel() else None
            out.append({"view": v, "samples_per_ray": round(float(k["n"].float().mean().item()), 2),
                        "bounded": round(nb / len(st), 4),
                        "fallback": round(float((st == 2).float().mean().item()), 4),
                        "n_hist_bounded": hist, "far_ran_to_t_end": round(float(far_end.sum().item()) / nb, 4),
                        "t_f_minus_tstar_vox": {"p50": q(dfar, 0.5), "p90": q(dfar, 0.9)},
                        "tstar_minus_t_n_vox": {"p10": q(dnear, 0.1), "p50": q(dnear, 0.5)},
                        "tab1_failed": round(float(fail.sum().item()) / nh, 4),
                        "wsum_below_0p95": round(float((bnd & (k["wsum"] < 0.95)).sum().item()) / nb, 4)})
        return out

    def run_all(self, hier_renderer, sweep_on):
        import torch
        from paper_2311_17878_gb300 import tsdfs as T
        t = self.tsdf_default()
        hier, kept_h = self.hier(hier_renderer)
        diag = self.diagnostics(t["_kept"], kept_h)
        sweep = []
        if sweep_on:
            pools = {"bounds": T.Bounds(self.n, device=self.dev), "ac": T.AdaptiveCounts(self.n, device=self.dev),
                     "rec": T.Recovery(self.mlp, self.n, self.bp.n_fallback, device=self.dev),
                     "rend": self.rend, "rend_cap": self.rend.max_samples}
            for cfg in SWEEP:
                sweep.append(self.operating_point(cfg, pools))
                torch.cuda.synchronize()
            del pools
        # the best operating point of the sweep, whose PSNR gate the cpu_baseline leg computes
        q_tmp = {"hier": hier, "tsdf": t, "sweep": sweep}
        bo = (equal_psnr_comparison(q_tmp) or {}).get("best_operating_point")
        best_cfg = None
        if bo is not None and bo["name"] != "default":
            c = next(c for c in sweep if c["name"] == bo["name"])
            best_cfg = (c["name"], c["psnr"], c["_cfg"], c["_bp"])
        dd = self.dense
        hit = dd["wsum"] > 0.5
        geom = {"depth_mae_m": float(np.mean(np.abs(t["_depth"][hit] - dd["depth"][hit]))) if hit.any() else None}
        r = self.refs
        bnd = (r["status"] == 1) & hit
        failed = bnd & ((dd["depth"] < r["t_n"]) | (dd["depth"] > r["t_f"]))
        err = np.abs(t["_rgb"] - dd["rgb"]).max(1)
        p_or = psnr(r["tsdf_rgb"], dd["rgb"])
        for c in [t] + hier + sweep:
            for k_ in [k_ for k_ in c if k_.startswith("_")]:
                del c[k_]
        t["name"] = "default"
        return {"pixels": int(self.cuts[-1]), "views": N_VIEWS_TIMED,
                "reference": f"oracle FP64 dense {DENSE_SAMPLES} midpoints over [t0, t_end], {r['source']}",
                "psnr_tsdf_gpu": t["psnr"], "psnr_tsdf_oracle": p_or,
                "meets_oracle_minus_0p1dB": bool(t["psnr"] >= p_or - 0.1),
                "psnr_hier96_gpu": hier[0]["psnr"], "tsdf_ge_hier96": bool(t["psnr"] >= hier[0]["psnr"]),
                "best_operating_point_gate": None, "_best_cfg": best_cfg,
                "tsdf": t, "hier": hier, "sweep": sweep, "per_view": diag,
                "tab1_failed_frac_oracle_bounds": float(failed.sum() / max(bnd.sum(), 1)),
                "geometry_tsdf_gpu": geom, "colour_err_p99": float(np.percentile(err, 99)),
                "colour_err_max": float(err.max()), "oracle_s": r["seconds"]}


def run_cpu_baseline(wl, grid, rays, bp, spec, seconds=10.0, chunk=2048):
    """The oracle as it stands, on the host cores: Alg. 1 bounds (C, fp32-exact)
    + FP64 render (torch CPU) of seeded chunks of view-0 rays on the fused grid,
    repeated until about `seconds` of CPU work."""
    import torch
    from oracle import cgrid
    from oracle import render as orr
    from paper_2311_17878_gb300 import synth
    V = grid.V.view(torch.int16).cpu().numpy().view(np.uint16) if grid.V.dtype == torch.float16 else grid.V.cpu().numpy()
    n_view = rays[0][2].shape[0]
    order = synth.sub_sample(n_view, n_view, seed=32)
    net = orr.Net(spec)
    done, t = 0, time.perf_counter()
    while done < n_view and time.perf_counter() - t < seconds:
        idx = order[done:done + chunk]
        o, d = rays[0][2][idx], rays[0][3][idx]
        b = cgrid.ray_bounds(wl.grid, V, o, d, bp, "f32")
        with torch.no_grad():
            orr.render_bounded(net, o, d, b["t_n"].astype(np.float64), b["t_f"].astype(np.float64), b["n"])
        done += len(idx)
    dt = time.perf_counter() - t
    return {"value": done / dt, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
            "sample": f"{done} seeded rays of image 0 of the workload in chunks of {chunk}: C bounds (1 thread) "
                      f"+ torch FP64 render", "seconds": dt}


def oracle_references(wl, grid, rays, bp, spec, tau=None):
    """The rest of the cpu_baseline leg: the oracle's outputs on the quality pixels (seeded,
    spread over every timed view), which the quality leg scores the GPU renders against --
    the dense FP64 reference over [t0, t_end] (stored by oracle/make_quality_reference.py for
    the room views and checked here on a few pixels; rendered in the run otherwise), the
    oracle's fp32 Alg. 1 bounds on the same grid and its TSDF-bounded render (with its own
    recovery pass of Sec. 4.5 when tau is set)."""
    import torch
    from oracle import cgrid
    from oracle import render as orr
    from paper_2311_17878_gb300 import synth
    t_q = time.perf_counter()
    n_rays = rays[0][2].shape[0]
    net = orr.Net(spec)
    dense, source = None, None
    if WORKLOAD == WORKLOADS["view"] and os.path.exists(DENSE_REF):
        from oracle import make_quality_reference as mqr
        z = np.load(DENSE_REF)
        sets = synth.quality_pixels(n_rays, N_VIEWS_TIMED, QUALITY_PIXELS)
        same = (str(z["networks_sha256"]) == mqr.network_digest(spec) and int(z["dense_samples"]) == DENSE_SAMPLES
                and np.array_equal(z["pixel"], np.concatenate(sets)))
        if same:
            # a live check of the stored values on the first pixels of view 0
            _, live = mqr.dense_for_view(0, spec, wl.grid, bp, pixels=8)
            diff = max(float(np.abs(live[k] - z[k][:8]).max()) for k in ("rgb", "depth", "wsum"))
            if diff < 1e-7:
                dense = {k: z[k] for k in ("rgb", "depth", "wsum", "normal")}
                source = f"stored by oracle/make_quality_reference.py, 8 pixels re-rendered here (max diff {diff:.1e})"
    if dense is None:
        sets = synth.quality_pixels(n_rays, N_VIEWS_TIMED, QUALITY_PIXELS_LIVE)
        parts = []
        for v in range(N_VIEWS_TIMED):
            on, dn = rays[v][2][sets[v]], rays[v][3][sets[v]]
            t0, te, _ = cgrid.clip_rays(wl.grid, on, dn, bp.t_near, bp.t_far, "f64")
            dd = orr.dense_reference(net, on, dn, t0, te, n=DENSE_SAMPLES)
            parts.append({k: dd[k].numpy() for k in ("rgb", "depth", "wsum", "normal")})
        dense = {k: np.concatenate([p_[k] for p_ in parts]) for k in parts[0]}
        source = "rendered in this run"
    V = grid.V.view(torch.int16).cpu().numpy().view(np.uint16) if grid.V.dtype == torch.float16 else grid.V.cpu().numpy()
    tn, tf, cnt, st, ort, again = [], [], [], [], [], []
    for v in range(N_VIEWS_TIMED):
        on, dn = rays[v][2][sets[v]], rays[v][3][sets[v]]
        ob = cgrid.ray_bounds(wl.grid, V, on, dn, bp, "f32")
        tn_v, tf_v = ob["t_n"].astype(np.float64), ob["t_f"].astype(np.float64)
        if tau is not None:
            t0f, tef, _ = cgrid.clip_rays(wl.grid, on, dn, bp.t_near, bp.t_far, "f32")
            ro, ag = orr.render_recovered(net, on, dn, tn_v, tf_v, ob["n"], ob["status"], t0f.astype(np.float64),
                                          tef.astype(np.float64), tau, bp.n_fallback)
            ort.append(ro["rgb"].numpy())
            again.append(ag)
        else:
            with torch.no_grad():
                ort.append(orr.render_bounded(net, on, dn, tn_v, tf_v, ob["n"])["rgb"].numpy())
        tn.append(tn_v)
        tf.append(tf_v)
        cnt.append(ob["n"])
        st.append(ob["status"])
    def tsdf_for(cfg, bp_cfg):
        """The oracle's TSDF render of a midpoint operating point of the sweep (Alg. 1 with its
        parameters, counts from its spacing, its recovery pass when it has one) on the quality
        pixels."""
        out = []
        for v in range(N_VIEWS_TIMED):
            on, dn = rays[v][2][sets[v]], rays[v][3][sets[v]]
            ob = cgrid.ray_bounds(wl.grid, V, on, dn, bp_cfg, "f32")
            tn_v, tf_v = ob["t_n"].astype(np.float64), ob["t_f"].astype(np.float64)
            cnt_v = ob["n"]
            with torch.no_grad():
                if cfg.get("tau") is not None:
                    t0f, tef, _ = cgrid.clip_rays(wl.grid, on, dn, bp_cfg.t_near, bp_cfg.t_far, "f32")
                    r, _ = orr.render_recovered(net, on, dn, tn_v, tf_v, cnt_v, ob["status"], t0f.astype(np.float64),
                                                tef.astype(np.float64), cfg["tau"], bp_cfg.n_fallback)
                else:
                    r = orr.render_bounded(net, on, dn, tn_v, tf_v, cnt_v)
            out.append(r["rgb"].numpy())
        return np.concatenate(out)

    return {"pixels": sets, "dense": dense, "source": source, "tsdf_rgb": np.concatenate(ort), "tsdf_for": tsdf_for,
            "t_n": np.concatenate(tn), "t_f": np.concatenate(tf), "n": np.concatenate(cnt),
            "status": np.concatenate(st), "again": np.concatenate(again) if again else None,
            "seconds": time.perf_counter() - t_q}


def oracle_best_gate(refs, quality):
    """The rest of the cpu_baseline leg: the metric's PSNR gate for the best operating point
    of the quality leg's sweep -- the oracle's render of that operating point (Alg. 1 with
    its parameters, counts from its spacing, its recovery pass when it has one) on the
    quality pixels against the GPU's.  Counts relative to the batch mean are not gated (the
    mean is over each view's full ray set, which the oracle does not march)."""
    if quality is None:
        return
    best = quality.pop("_best_cfg", None)
    if best is None:
        return
    name, p_gpu, cfg, bp = best
    gate = {"name": name, "psnr_gpu": p_gpu, "psnr_oracle": None, "meets_oracle_minus_0p1dB": None}
    if cfg.get("sampler", "mid") == "mid":
        p_o = psnr(refs["tsdf_for"](cfg, bp), refs["dense"]["rgb"])
        gate.update(psnr_oracle=p_o, meets_oracle_minus_0p1dB=bool(p_gpu >= p_o - 0.1))
    quality["best_operating_point_gate"] = gate


# ----------------------------------------------------------------------------
def run_reference(args, ws, rank):
    """The CPU oracle as the reference arm: each step renders a bounded sample of
    the same workload (ref_rays seeded rays of a held-out view)."""
    if args.workload == "large":
        return {"impl": "reference", "unavailable": "the oracle's fusion of 300 1280x960 maps into 512^3 runs for "
                                                   "hours on the host cores; the reference arm covers view and panorama"}
    import torch
    if rank != 0:
        return None
    from oracle import cgrid
    from oracle import render as orr
    from paper_2311_17878_gb300 import synth
    t_setup = time.perf_counter()
    wl = synth.room_workload_torch(device="cpu")
    views = synth.Views(wl.views.K, wl.views.c2w, wl.views.depth.numpy(), 640, 480)
    V, _ = cgrid.integrate_projective(wl.grid, views, "f32")
    spec = synth.scene_mlp("room")
    net = orr.Net(spec)
    t_setup = time.perf_counter() - t_setup
    bp = wl.bounds

    def step(k):
        if args.workload == "panorama":
            o, d = synth.room_panorama_rays(center=tuple(synth.room_panorama_centres(N_VIEWS_TIMED)[k % N_VIEWS_TIMED]))
        else:
            o, d = synth.room_heldout_rays(k % N_VIEWS_TIMED)
        idx = synth.sub_sample(len(o), args.ref_rays, seed=40 + k)
        b = cgrid.ray_bounds(wl.grid, V, o[idx], d[idx], bp, "f32")
        with torch.no_grad():
            orr.render_bounded(net, o[idx], d[idx], b["t_n"].astype(np.float64), b["t_f"].astype(np.float64), b["n"])

    for k in range(args.warmup):
        step(k)
    t = time.perf_counter()
    for k in range(args.steps):
        step(k)
    dt = time.perf_counter() - t
    value = args.ref_rays * args.steps / dt
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic (seeded room scene, fitted networks)", "impl": "reference",
            "config": {"workload": WORKLOAD, "rays_per_step": args.ref_rays, "setup_s": t_setup},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": torch.get_num_threads(), "kind": "oracle",
                             "sample": f"{args.ref_rays} seeded rays of one image of the workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    global WORKLOAD, N_VIEWS_TIMED
    args = parse()
    WORKLOAD = WORKLOADS[args.workload]
    N_VIEWS_TIMED = {"panorama": 4, "large": 8}.get(args.workload, 10)
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        ws = int(os.environ.get("WORLD_SIZE", "1"))
        line = run_reference(args, ws, rank)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if args.train_only:
        print(json.dumps(run_train_only(args)), flush=True)
        return
    ws, rank, local = dist_setup()
    line = run_ours(args, ws, rank, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
