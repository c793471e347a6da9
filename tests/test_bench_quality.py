"""Host-side logic of the bench's quality leg (CPU): the equal-PSNR comparison, the
Pareto front, the seeded quality pixels and the stored dense reference, which must be
the oracle's own output on those pixels."""
import os

import numpy as np
import pytest

import bench
from paper_2311_17878_gb300 import synth


def _q():
    hier = [{"name": "hier 64+32", "rays_s": 1.0e6, "psnr": 60.0, "samples_per_ray": 96},
            {"name": "hier 8+4", "rays_s": 9.0e6, "psnr": 40.0, "samples_per_ray": 12},
            {"name": "hier 4+2", "rays_s": 18.0e6, "psnr": 17.0, "samples_per_ray": 6}]
    tsdf = {"name": "default", "rays_s": 8.0e6, "psnr": 35.0, "samples_per_ray": 19.0}
    sweep = [{"name": "a", "rays_s": 12.0e6, "psnr": 42.0, "samples_per_ray": 8.0},
             {"name": "b", "rays_s": 20.0e6, "psnr": 30.0, "samples_per_ray": 4.0},
             {"name": "c", "rays_s": 2.0e6, "psnr": 70.0, "samples_per_ray": 64.0}]
    return {"hier": hier, "tsdf": tsdf, "sweep": sweep}


def test_equal_psnr_comparison_picks_fastest_hier_at_or_above():
    c = bench.equal_psnr_comparison(_q())
    assert c["hier_at_ge_psnr"]["name"] == "hier 8+4"
    assert c["tsdf_over_hier"] == pytest.approx(8.0 / 9.0)
    best = c["best_operating_point"]
    # "a" (42 dB) is compared with 64+32, the only configuration at or above 42 dB (12x); "b"
    # with 8+4 (20/9); "c" has no hierarchical configuration at its PSNR and is not a candidate
    assert best["name"] == "a" and best["hier"] == "hier 64+32"
    assert best["tsdf_over_hier"] == pytest.approx(12.0)


def test_pareto_front_marks_undominated_points():
    pts = bench.pareto_front(_q())
    assert {p["name"] for p in pts if p["front"]} == {"a", "b", "c"}
    by = {p["name"]: p for p in pts}
    assert not by["default"]["front"]          # "a" is faster and better
    assert not by["hier 8+4"]["front"]         # "a" again
    assert by["a"]["front"] and by["b"]["front"] and by["c"]["front"]
    assert not by["hier 64+32"]["front"]       # "c" is faster and better
    assert by["hier 4+2"]["front"] is False    # "b" is faster and better
    assert [p["rays_s"] for p in pts] == sorted([p["rays_s"] for p in pts], reverse=True)


def test_quality_pixels_spread_over_views():
    sets = synth.quality_pixels(307200, 10, 4096)
    assert sum(len(s) for s in sets) == 4096
    assert [len(s) for s in sets] == [410] * 6 + [409] * 4
    for s in sets:
        assert np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < 307200
    assert not np.array_equal(sets[0][:409], sets[1][:409])


@pytest.mark.skipif(not os.path.exists(bench.DENSE_REF), reason="dense reference not written")
def test_stored_dense_reference_is_the_oracle_output():
    """The stored dense reference holds the oracle's FP64 dense render of the quality
    pixels of the current networks: same pixels, same network digest, and a few pixels
    of two views re-rendered here agree."""
    from oracle import make_quality_reference as mqr
    z = np.load(bench.DENSE_REF)
    spec = synth.scene_mlp("room")
    assert str(z["networks_sha256"]) == mqr.network_digest(spec)
    assert int(z["dense_samples"]) == bench.DENSE_SAMPLES
    sets = synth.quality_pixels(640 * 480, mqr.N_VIEWS, mqr.PIXELS)
    assert np.array_equal(z["pixel"], np.concatenate(sets))
    assert np.array_equal(z["view"], np.concatenate([np.full(len(s), v) for v, s in enumerate(sets)]))
    wl = synth.room_workload(with_views=False)
    cuts = np.cumsum([0] + [len(s) for s in sets])
    for v in (0, 7):
        _, live = mqr.dense_for_view(v, spec, wl.grid, wl.bounds, pixels=3)
        for k in ("rgb", "depth", "wsum", "normal"):
            assert np.max(np.abs(live[k] - z[k][cuts[v]:cuts[v] + 3])) < 1e-9, (v, k)
