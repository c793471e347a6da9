"""The bench reports a captured DRAM traffic only for the captured configuration and only
while the kernel's sources are the ones it was captured on."""
import sys
from pathlib import Path
from types import SimpleNamespace

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))
import bench  # noqa: E402


def args(**kw):
    a = dict(workload="view", grid_source="network", fusion="projective", steps=20, rays=0, recovery_tau=None,
             graph=False)
    a.update(kw)
    return SimpleNamespace(**a)


def test_traffic_reported_for_the_captured_run():
    t = {"sha256": bench.source_hash(bench.MLP_TC_SOURCES), "bytes_per_launch": 123}
    assert bench.captured_traffic(t, bench.MLP_TC_SOURCES, args(), "f16") == 123


def test_traffic_null_when_the_kernel_changed():
    t = {"sha256": "0" * 64, "bytes_per_launch": 123}
    assert bench.captured_traffic(t, bench.MLP_TC_SOURCES, args(), "f16") is None


def test_traffic_null_for_other_configurations():
    t = {"sha256": bench.source_hash(bench.MARCH_SOURCES), "bytes_per_launch": 7}
    for kw, prec in [({"workload": "panorama"}, "f16"), ({"grid_source": "analytic"}, "f16"), ({}, "bf16"),
                     ({"steps": 3}, "f16"), ({"rays": 65536}, "f16"), ({"recovery_tau": 0.95}, "f16"),
                     ({"fusion": "raycast"}, "f16")]:
        assert bench.captured_traffic(t, bench.MARCH_SOURCES, args(**kw), prec) is None, kw
    assert bench.captured_traffic(t, bench.MARCH_SOURCES, args(), "f16") == 7
    # graph replay launches the same kernels as the eager steps the capture timed
    assert bench.captured_traffic(t, bench.MARCH_SOURCES, args(graph=True), "f16") == 7

