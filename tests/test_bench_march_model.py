"""The bench's model of the voxels Alg. 1's walk tests per ray (the walk's length times the
voxel-boundary crossings per unit length, plus the first voxel; bench.march_roofline),
checked on the CPU against the oracle's exact walk of the same rays."""
import sys
from pathlib import Path

import numpy as np

from oracle import cgrid
from paper_2311_17878_gb300 import synth

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))
import bench  # noqa: E402


def test_march_voxel_model_tracks_the_oracle_walk():
    wl = synth.tiny_workload()
    V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    b = cgrid.ray_bounds(wl.grid, V, wl.rays_o, wl.rays_d, wl.bounds, "f32")
    r = bench.march_roofline(wl.grid, wl.rays_o, wl.rays_d, b["t_f"], b["status"], wl.bounds, 1.0, 1.0, "test")
    exact = float(np.mean(b["steps"]))
    assert exact > 5
    assert abs(r["voxels_per_ray"] - exact) <= 0.1 * exact
    assert r["bytes_per_ray"] == 4.0 * r["voxels_per_ray"] + 41.0
