"""GPU parity of the render path (sample placement, SDF + colour networks,
NeuS opacity, compositing) and of the 64 + 32 hierarchical comparator,
against the FP64 oracle on the same seeded inputs.

Tolerances (FP32 networks): depth 1e-4 relative, colour 2e-3 absolute (the
stated bars); weight sums and normals are checked too."""
import numpy as np
import pytest
import torch

from oracle import cgrid
from oracle import render as orr
from paper_2311_17878_gb300 import build, synth
from paper_2311_17878_gb300 import tsdfs as T

pytestmark = pytest.mark.gpu

DEPTH_REL_F32 = 1e-4
RGB_ABS = 2e-3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    T.lib()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def oracle_bounds_tiny():
    wl = synth.tiny_workload()
    V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    b = cgrid.ray_bounds(wl.grid, V, wl.rays_o, wl.rays_d, wl.bounds, "f32")
    return wl, V, b


def gpu_render(spec, o, d, b, precision=T.TSDFS_PREC_F32, max_samples=None):
    mlp = T.Mlp(spec, precision)
    n = len(o)
    offsets = np.concatenate([[0], np.cumsum(b["n"])]).astype(np.int32)
    total = int(offsets[-1])
    ms = total if max_samples is None else max_samples
    r = T.Renderer(mlp, n, max(ms, 1))
    r.max_samples = ms
    bb = T.Bounds(n)
    bb.t_n.copy_(dev(b["t_n"].astype(np.float32)))
    bb.t_f.copy_(dev(b["t_f"].astype(np.float32)))
    bb.offsets.copy_(dev(offsets))
    bb.status.copy_(dev(b["status"]))
    out = r.render(dev(o), dev(d), bb)
    torch.cuda.synchronize()
    return {k: getattr(out, k).cpu().numpy() for k in ("rgb", "depth", "wsum", "normal", "eik")}


def compare(got, ref, depth_rel=DEPTH_REL_F32, rgb_abs=RGB_ABS):
    assert np.max(np.abs(got["rgb"] - ref["rgb"])) < rgb_abs
    assert np.max(np.abs(got["wsum"] - ref["wsum"])) < rgb_abs
    ok = ref["wsum"] > 1e-3
    assert np.all(np.abs(got["depth"][ok] - ref["depth"][ok]) <= depth_rel * np.abs(ref["depth"][ok]) + 1e-6)
    assert np.max(np.abs(got["normal"][ok] - ref["normal"][ok])) < 1e-2


def oracle_render(spec, o, d, b):
    out = orr.render_bounded(orr.Net(spec), o, d, b["t_n"].astype(np.float64), b["t_f"].astype(np.float64), b["n"])
    return {k: out[k].detach().numpy() for k in ("rgb", "depth", "wsum", "normal")}, out


def test_tiny_render_f32_matches_oracle():
    wl, V, b = oracle_bounds_tiny()
    spec = synth.scene_mlp("tiny")
    got = gpu_render(spec, wl.rays_o, wl.rays_d, b)
    ref, raw = oracle_render(spec, wl.rays_o, wl.rays_d, b)
    compare(got, ref)
    # per-ray eikonal sums of BOUNDED rays
    counts = b["n"]
    eik = raw["eik"].detach().numpy()
    per = np.zeros(len(counts))
    np.add.at(per, np.repeat(np.arange(len(counts)), counts), eik)
    per[b["status"] != 1] = 0
    assert np.allclose(got["eik"], per, rtol=1e-4, atol=1e-5)
    miss = b["status"] == 0
    assert np.all(got["rgb"][miss] == 0) and np.all(got["wsum"][miss] == 0)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0


def test_tiny_render_geometric_init_matches_oracle():
    wl, V, b = oracle_bounds_tiny()
    spec = synth.tiny_mlp()
    got = gpu_render(spec, wl.rays_o, wl.rays_d, b)
    ref, _ = oracle_render(spec, wl.rays_o, wl.rays_d, b)
    compare(got, ref)


def test_room_render_f32_matches_oracle():
    wl = synth.room_workload(with_views=False)
    V = synth.analytic_tsdf_torch(wl.scene, wl.grid, device="cuda").cpu().numpy()
    o, d = synth.room_heldout_rays(0)
    idx = synth.sub_sample(len(o), 384, seed=23)
    o, d = o[idx], d[idx]
    b = cgrid.ray_bounds(wl.grid, V, o, d, wl.bounds, "f32")
    spec = synth.scene_mlp("room")
    got = gpu_render(spec, o, d, b)
    ref, _ = oracle_render(spec, o, d, b)
    compare(got, ref)


def test_sample_overflow_sets_status_and_zeroes():
    wl, V, b = oracle_bounds_tiny()
    spec = synth.tiny_mlp()
    total = int(b["n"].sum())
    got = gpu_render(spec, wl.rays_o, wl.rays_d, b, max_samples=total - 1)
    rc, bits = T.tsdfs_sync_status()
    assert rc == T.TSDFS_E_DEVICE and bits & T.TSDFS_DEV_SAMPLES_OVERFLOW
    assert np.all(got["rgb"] == 0) and np.all(got["wsum"] == 0)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0 and bits == 0


def test_ragged_counts_single_and_large():
    """Rays with 1 sample, the n_max cap, and the 96-sample fallback, mixed."""
    wl, V, b = oracle_bounds_tiny()
    rng = np.random.default_rng(5)
    b = dict(b)
    n = b["n"].copy()
    live = b["status"] != 0
    n[live] = rng.choice([1, 2, 31, 32, 96], live.sum())
    b["n"] = n.astype(np.int32)
    spec = synth.scene_mlp("tiny")
    got = gpu_render(spec, wl.rays_o, wl.rays_d, b)
    ref, _ = oracle_render(spec, wl.rays_o, wl.rays_d, b)
    compare(got, ref)


@pytest.mark.parametrize("n_coarse,n_fine", [(64, 32), (16, 8), (37, 5), (2, 1)])
def test_tiny_hier_f32_matches_oracle(n_coarse, n_fine):
    """The hierarchical comparator at its Tab. 2 counts (64 + 32) and at
    smaller ones, including counts that are no multiple of a tile (37 + 5)
    and the fewest the section weights allow (2 + 1)."""
    wl = synth.tiny_workload()
    spec = synth.scene_mlp("tiny")
    bp = wl.bounds
    t0, te, ok = cgrid.clip_rays(wl.grid, wl.rays_o, wl.rays_d, bp.t_near, bp.t_far, "f32")
    mlp = T.Mlp(spec)
    g = T.Grid(wl.grid, V=torch.zeros(wl.grid.shape_zyx, device="cuda"),
               W=torch.zeros(wl.grid.shape_zyx, dtype=torch.uint8, device="cuda"))
    h = T.HierRenderer(mlp, 4096, n_coarse=n_coarse, n_fine=n_fine)
    out = h.render(g, dev(wl.rays_o), dev(wl.rays_d), bp.t_near, bp.t_far)
    torch.cuda.synchronize()
    got = {k: getattr(out, k).cpu().numpy() for k in ("rgb", "depth", "wsum", "normal")}
    live = np.nonzero(ok)[0]
    ro = orr.render_hier(orr.Net(spec), wl.rays_o[live], wl.rays_d[live], t0[live].astype(np.float64),
                         te[live].astype(np.float64), n_coarse=n_coarse, n_fine=n_fine)
    ref = {k: ro[k].detach().numpy() for k in ("rgb", "depth", "wsum", "normal")}
    sub = {k: v[live] for k, v in got.items()}
    compare(sub, ref)
    assert np.all(got["rgb"][~ok] == 0)


# ------------------------------------------------------------------ BF16 ----
DEPTH_REL_BF16 = 2e-3


def _pad16(x):
    return (x + 15) // 16 * 16


def _plain_packed_bytes(spec):
    """Bytes of the unfolded layers: every layer's weights padded to 16 rows and columns."""
    return sum(2 * _pad16(W.shape[0]) * _pad16(W.shape[1]) for W, _ in list(spec.sdf) + list(spec.rgb))


def test_pack_layout_roundtrip():
    """The unfolded part of the packed bf16 tiles holds every weight once (rounded to
    nearest even) and zeros in the padding: the multiset of its values equals the weights."""
    for spec in (synth.tiny_mlp(), synth.room_mlp()):
        mlp = T.Mlp(spec, T.TSDFS_PREC_BF16)
        torch.cuda.synchronize()
        nb = _plain_packed_bytes(spec)
        packed = mlp.packed[:nb].view(torch.bfloat16).float().cpu().numpy()
        w = np.concatenate([np.concatenate([W.reshape(-1) for W, _ in spec.sdf]),
                            np.concatenate([W.reshape(-1) for W, _ in spec.rgb])]).astype(np.float32)
        nz = np.sort(packed[packed != 0])
        assert np.array_equal(nz, np.sort(w[w != 0]))


def _unpack_chunks(raw, n_rows, k_cols):
    """Inverse of the chunked no-swizzle K-major core-matrix layout of one layer: 64-column
    chunks (the last one narrower), within a chunk 8x8 core matrices, row blocks outermost."""
    out = np.zeros((n_rows, k_cols), np.float64)
    pos = 0
    for c0 in range(0, k_cols, 64):
        kc = min(64, k_cols - c0)
        blk = raw[pos:pos + n_rows * kc].reshape(n_rows // 8, kc // 8, 8, 8)
        out[:, c0:c0 + kc] = blk.transpose(0, 2, 1, 3).reshape(n_rows, kc)
        pos += n_rows * kc
    return out, pos


@pytest.mark.parametrize("precision", [T.TSDFS_PREC_F16, T.TSDFS_PREC_BF16])
def test_folded_layers_match_fp64_product(precision):
    """The serial kernel's folded layers after the unfolded ones: the SDF output's value row,
    and the first colour layer on [h, x~, direction, normal] whose h columns hold
    W_c,feat W_f, against the product in FP64 rounded once (within one unit in the 16-bit
    format's last place); the folded biases b_f,0 and b_c + W_c,feat b_f in FP32 (1e-6)."""
    dt = torch.float16 if precision == T.TSDFS_PREC_F16 else torch.bfloat16
    ulp = 2.0 ** -10 if precision == T.TSDFS_PREC_F16 else 2.0 ** -7
    for spec in (synth.tiny_mlp(), synth.room_mlp()):
        mlp = T.Mlp(spec, precision)
        torch.cuda.synchronize()
        nb = _plain_packed_bytes(spec)
        raw = mlp.packed[nb:].view(dt).float().cpu().numpy().astype(np.float64)
        Wo, bo = [np.asarray(a, np.float64) for a in spec.sdf[-1]]
        Wc, bc = [np.asarray(a, np.float64) for a in spec.rgb[0]]
        kh = Wo.shape[1]
        nfeat = Wo.shape[0] - 1
        kx = Wc.shape[1] - nfeat
        vrow, used = _unpack_chunks(raw, 16, _pad16(kh))
        assert np.all(np.abs(vrow[0, :kh] - Wo[0]) <= ulp * np.abs(Wo[0]) + 1e-7)
        assert not vrow[1:].any()
        nc = _pad16(Wc.shape[0])
        fold, used2 = _unpack_chunks(raw[used:], nc, kh + _pad16(kx))
        ref = np.zeros_like(fold)
        ref[:Wc.shape[0], :kh] = Wc[:, kx:] @ Wo[1:]
        ref[:Wc.shape[0], kh:kh + kx] = Wc[:, :kx]
        assert np.all(np.abs(fold - ref) <= ulp * np.abs(ref) + 1e-7), np.abs(fold - ref).max()
        fb_off = (nb + 2 * (used + used2) + 15) // 16 * 16
        fb = mlp.packed[fb_off:fb_off + 4 * (16 + nc)].view(torch.float32).cpu().numpy().astype(np.float64)
        ref_b = np.zeros(16 + nc)
        ref_b[0] = bo[0]
        ref_b[16:16 + Wc.shape[0]] = bc + Wc[:, kx:] @ bo[1:]
        assert np.allclose(fb, ref_b, rtol=1e-6, atol=1e-7), np.abs(fb - ref_b).max()


def _scene_case(scene):
    if scene == "tiny":
        wl, V, b = oracle_bounds_tiny()
        return wl.rays_o, wl.rays_d, b
    wl = synth.room_workload(with_views=False)
    V = synth.analytic_tsdf_torch(wl.scene, wl.grid, device="cuda").cpu().numpy()
    o, d = synth.room_heldout_rays(0)
    idx = synth.sub_sample(len(o), 512, seed=23)
    o, d = o[idx], d[idx]
    return o, d, cgrid.ray_bounds(wl.grid, V, o, d, wl.bounds, "f32")


def _errors(got, ref):
    ok = ref["wsum"] > 1e-3
    er = np.abs(got["rgb"] - ref["rgb"]).max(1)
    ed = np.abs(got["depth"][ok] - ref["depth"][ok]) / np.abs(ref["depth"][ok])
    return er, ed


def test_render_f16_tile_pairs_several_per_cta_odd_count():
    """The tensor-core kernel runs 64-sample tiles in pairs (the colour layers once for both,
    the first tile parked in the render workspace between the SDF passes).  609 tiles: 305
    pairs, so the CTAs take two or three pairs each and the last pair has one tile; sampled
    rays from the whole range (its first and last live rays among them) against the oracle
    within the 16-bit bars."""
    wl = synth.room_workload(with_views=False)
    V = synth.analytic_tsdf_torch(wl.scene, wl.grid, device="cuda").cpu().numpy()
    o, d = synth.room_heldout_rays(1)
    idx = synth.sub_sample(len(o), 1400, seed=31)
    o, d = o[idx], d[idx]
    b = dict(cgrid.ray_bounds(wl.grid, V, o, d, wl.bounds, "f32"))
    live = np.flatnonzero(b["status"] != 0)
    target = 64 * 608 + 13          # 609 tiles of 64 samples, the last one ragged
    rng = np.random.default_rng(7)
    n = np.zeros(len(o), np.int64)
    n[live] = rng.integers(1, 65, len(live))
    # bring the total to the target one sample at a time over the live rays, within [1, 96]
    diff = target - int(n.sum())
    step = 1 if diff > 0 else -1
    i = 0
    while diff != 0:
        r = live[i % len(live)]
        if 1 <= n[r] + step <= 96:
            n[r] += step
            diff -= step
        i += 1
    assert int(n.sum()) == target
    b["n"] = n.astype(np.int32)
    spec = synth.scene_mlp("room")
    got = gpu_render(spec, o, d, b, precision=T.TSDFS_PREC_F16)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    sel = np.unique(np.concatenate([live[:8], live[-8:], live[synth.sub_sample(len(live), 160, seed=32)]]))
    bs = {k: v[sel] for k, v in b.items()}
    ref, _ = oracle_render(spec, o[sel], d[sel], bs)
    got_s = {k: v[sel] for k, v in got.items()}
    er, ed = _errors(got_s, ref)
    print(f"pairs f16: rgb p99 {np.percentile(er, 99):.2e} max {er.max():.2e}; depth max {ed.max() if len(ed) else 0:.2e}")
    compare(got_s, ref, depth_rel=DEPTH_REL_BF16)


@pytest.mark.parametrize("scene", ["tiny", "room"])
def test_render_f16_operands_match_oracle(scene):
    """tcgen05 path with fp16 operands, fp32 accumulation: within the stated
    16-bit bars element by element (colour 2e-3 absolute, depth 2e-3 relative)."""
    o, d, b = _scene_case(scene)
    spec = synth.scene_mlp(scene)
    got = gpu_render(spec, o, d, b, precision=T.TSDFS_PREC_F16)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    ref, _ = oracle_render(spec, o, d, b)
    er, ed = _errors(got, ref)
    print(f"{scene} f16: rgb p99 {np.percentile(er, 99):.2e} max {er.max():.2e}; depth p99 {np.percentile(ed, 99):.2e} max {ed.max():.2e}")
    compare(got, ref, depth_rel=DEPTH_REL_BF16)


@pytest.mark.parametrize("scene", ["tiny", "room"])
@pytest.mark.xfail(reason="plain BF16 operands keep 8 significant bits (unit roundoff 2^-8 against FP16's "
                          "2^-11); the rounding of the SDF network's activations reaches the bars on the worst "
                          "rays: an FP64 emulation with every operand rounded to BF16 gives room colour p99 "
                          "7.0e-3, max 1.3e-2, depth p99 2.5e-3, max 5.8e-3; TSDFS_PREC_BF16X2 meets the bars",
                   strict=False)
def test_render_bf16_operands_match_oracle(scene):
    """tcgen05 path with plain bf16 operands, at the stated 16-bit bars (colour 2e-3
    absolute, depth 2e-3 relative, every ray)."""
    o, d, b = _scene_case(scene)
    spec = synth.scene_mlp(scene)
    got = gpu_render(spec, o, d, b, precision=T.TSDFS_PREC_BF16)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    ref, _ = oracle_render(spec, o, d, b)
    er, ed = _errors(got, ref)
    print(f"{scene} bf16: rgb p99 {np.percentile(er, 99):.2e} max {er.max():.2e}; depth p99 {np.percentile(ed, 99):.2e} max {ed.max():.2e}")
    compare(got, ref, depth_rel=DEPTH_REL_BF16)


@pytest.mark.parametrize("n_coarse,n_fine", [(64, 32), (24, 9)])
def test_bf16_hier_runs_and_tracks_f32(n_coarse, n_fine):
    wl = synth.tiny_workload()
    spec = synth.scene_mlp("tiny")
    g = T.Grid(wl.grid, V=torch.zeros(wl.grid.shape_zyx, device="cuda"),
               W=torch.zeros(wl.grid.shape_zyx, dtype=torch.uint8, device="cuda"))
    outs = []
    for prec in (T.TSDFS_PREC_F32, T.TSDFS_PREC_BF16, T.TSDFS_PREC_F16):
        h = T.HierRenderer(T.Mlp(spec, prec), 4096, n_coarse=n_coarse, n_fine=n_fine)
        o = h.render(g, dev(wl.rays_o), dev(wl.rays_d), wl.bounds.t_near, wl.bounds.t_far)
        torch.cuda.synchronize()
        outs.append(o.rgb.cpu().numpy())
    # BF16 against FP32: the FP32 colour bar scaled by the unit-roundoff ratio 2^-8 / 2^-11 at
    # the 99th percentile, twice that at the maximum (fewer coarse samples place the fine ones
    # from fewer, so more sensitive, section weights)
    e_bf16 = np.abs(outs[0] - outs[1])
    assert np.percentile(e_bf16, 99) <= 8 * RGB_ABS and e_bf16.max() <= 16 * RGB_ABS
    assert np.max(np.abs(outs[0] - outs[2])) < 5e-3


@pytest.mark.parametrize("precision", [T.TSDFS_PREC_F32, T.TSDFS_PREC_F16])
def test_degenerate_rays_render_matches_oracle(precision):
    """Axis-aligned, diagonal, inside-the-sphere and grazing rays (the bounds
    tests' set), rendered through the bounds the oracle computes."""
    from test_gpu_fusion_bounds import _degenerate_rays
    wl = synth.tiny_workload()
    V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    o, d = _degenerate_rays()
    b = cgrid.ray_bounds(wl.grid, V, o, d, wl.bounds, "f32")
    spec = synth.scene_mlp("tiny")
    got = gpu_render(spec, o, d, b, precision=precision)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    ref, _ = oracle_render(spec, o, d, b)
    if precision == T.TSDFS_PREC_F32:
        compare(got, ref)
    else:
        er, ed = _errors(got, ref)
        assert er.max() < RGB_ABS and (ed.size == 0 or ed.max() < 2e-3)
