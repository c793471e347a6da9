"""Write the dense reference image of the room's quality pixels.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the stored values are
the oracle's own (:func:`oracle.render.dense_reference`, FP64, 1024 midpoint
samples over each ray's grid-box clip [t0, t_end] of [t_near, t_far], no opacity
guard), on the seeded pixel subsets of :func:`synth.quality_pixels` (4096 pixels
over the ten held-out 640x480 room views) with the fitted room networks.  They
depend only on the networks, the rays and the grid box, not on any fused TSDF.

    python -m oracle.make_quality_reference      # writes oracle/data/room_view_dense_reference.npz
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from oracle import cgrid  # noqa: E402
from oracle import render as orr  # noqa: E402
from paper_2311_17878_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "data", "room_view_dense_reference.npz")
N_VIEWS = 10
PIXELS = 4096
DENSE_SAMPLES = 1024


def network_digest(spec) -> str:
    h = hashlib.sha256()
    for part in ("sdf", "rgb"):
        h.update(np.ascontiguousarray(spec.packed(part), np.float32).tobytes())
    return h.hexdigest()


def view_pixels(v):
    """Rays of view v's quality pixels: (pixel indices, origins, directions)."""
    o, d = synth.room_heldout_rays(v)
    idx = synth.quality_pixels(len(o), N_VIEWS, PIXELS)[v]
    return idx, o[idx], d[idx]


def dense_for_view(v, spec, grid, bp, pixels=None):
    idx, o, d = view_pixels(v)
    if pixels is not None:
        idx, o, d = idx[:pixels], o[:pixels], d[:pixels]
    t0, te, _ = cgrid.clip_rays(grid, o, d, bp.t_near, bp.t_far, "f64")
    r = orr.dense_reference(orr.Net(spec), o, d, t0, te, n=DENSE_SAMPLES)
    return idx, {k: r[k].numpy() for k in ("rgb", "depth", "wsum", "normal")}


def main():
    spec = synth.scene_mlp("room")
    wl = synth.room_workload(with_views=False)
    out = {"view": [], "pixel": [], "rgb": [], "depth": [], "wsum": [], "normal": []}
    t = time.perf_counter()
    for v in range(N_VIEWS):
        idx, r = dense_for_view(v, spec, wl.grid, wl.bounds)
        out["view"].append(np.full(len(idx), v, np.int32))
        out["pixel"].append(idx.astype(np.int64))
        for k in ("rgb", "depth", "wsum", "normal"):
            out[k].append(r[k])
        print(f"view {v}: {len(idx)} pixels, {time.perf_counter() - t:.0f} s", flush=True)
    arrs = {k: np.concatenate(v) for k, v in out.items()}
    np.savez_compressed(OUT, **arrs, dense_samples=np.int64(DENSE_SAMPLES),
                        networks_sha256=np.array(network_digest(spec)))
    print(OUT)


if __name__ == "__main__":
    main()
