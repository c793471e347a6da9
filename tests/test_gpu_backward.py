"""GPU parity of render_rays_backward (parameter gradients through compositing,
the NeuS opacity, both networks and the second-order terms through grad f)
against the oracle's FP64 reverse-mode gradient of the same functional, whose
own correctness is pinned by central differences in the CPU tests."""
import numpy as np
import pytest
import torch

from oracle import cgrid
from oracle import render as orr
from paper_2311_17878_gb300 import build, synth
from paper_2311_17878_gb300 import tsdfs as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    T.lib()


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def case(scene, n_rays, seed):
    if scene == "tiny":
        wl = synth.tiny_workload()
        V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
        o, d = wl.rays_o, wl.rays_d
        b = cgrid.ray_bounds(wl.grid, V, o, d, wl.bounds, "f32")
        live = np.nonzero(b["status"] != 0)[0]
        idx = np.random.default_rng(seed).choice(live, n_rays, replace=False)
    else:
        wl = synth.room_workload(with_views=False)
        V = synth.analytic_tsdf_torch(wl.scene, wl.grid, device="cuda").cpu().numpy()
        o, d = synth.room_heldout_rays(0)
        idx = synth.sub_sample(len(o), n_rays, seed=seed)
        b = cgrid.ray_bounds(wl.grid, V, o[idx], d[idx], wl.bounds, "f32")
        return o[idx], d[idx], b
    b = {k: v[idx] for k, v in b.items()}
    return o[idx], d[idx], b


def oracle_grads(spec, o, d, b, d_rgb, d_depth, d_eik):
    net = orr.Net(spec, requires_grad=True)
    out = orr.render_bounded(net, o, d, b["t_n"].astype(np.float64), b["t_f"].astype(np.float64), b["n"])
    counts = torch.as_tensor(b["n"].astype(np.int64))
    eik_ray = torch.zeros(len(counts), dtype=torch.float64).index_add(
        0, torch.repeat_interleave(torch.arange(len(counts)), counts), out["eik"])
    eik_ray = eik_ray * torch.as_tensor(b["status"] == 1)
    L = (out["rgb"] * torch.as_tensor(d_rgb, dtype=torch.float64)).sum() \
        + (out["depth"] * torch.as_tensor(d_depth, dtype=torch.float64)).sum() \
        + (eik_ray * torch.as_tensor(d_eik, dtype=torch.float64)).sum()
    gs = torch.autograd.grad(L, net.params())
    sdf = np.concatenate([np.concatenate([gs[2 * i].numpy().reshape(-1), gs[2 * i + 1].numpy()]) for i in range(len(spec.sdf))])
    k = 2 * len(spec.sdf)
    rgb = np.concatenate([np.concatenate([gs[k + 2 * i].numpy().reshape(-1), gs[k + 2 * i + 1].numpy()]) for i in range(len(spec.rgb))])
    return sdf, rgb


@pytest.fixture
def restore_backward():
    old = T.tsdfs_backward_kernel()
    yield
    T.tsdfs_set_backward_kernel(old)
    T.tsdfs_set_backward_chunk(0)


def gpu_grads(spec, o, d, b, d_rgb, d_depth, d_eik, kind=T.TSDFS_BACKWARD_GEMM, chunk=0, max_samples=None,
              calls=1):
    """Parameter gradients from render_rays_backward with the given implementation and
    chunk; `calls` calls accumulate into the same buffers."""
    T.tsdfs_set_backward_kernel(kind)
    T.tsdfs_set_backward_chunk(chunk)
    n_rays = len(o)
    mlp = T.Mlp(spec)
    offsets = np.concatenate([[0], np.cumsum(b["n"])]).astype(np.int32)
    total = int(offsets[-1])
    ms = total if max_samples is None else max_samples
    d_sdf = torch.zeros_like(mlp.sdf_w)
    d_rw = torch.zeros_like(mlp.rgb_w)
    ws = torch.empty(max(T.tsdfs_backward_workspace_size(mlp, n_rays, ms), 1), dtype=torch.uint8, device="cuda")
    for _ in range(calls):
        T.render_rays_backward(mlp, dev(o), dev(d), dev(b["t_n"].astype(np.float32)), dev(b["t_f"].astype(np.float32)),
                               dev(offsets), dev(b["status"]), ms, dev(d_rgb), dev(d_depth), dev(d_eik), d_sdf, d_rw, ws)
    torch.cuda.synchronize()
    return d_sdf.cpu().numpy(), d_rw.cpu().numpy()


def seeded_adjoints(n_rays, seed=7):
    rng = np.random.default_rng(seed)
    d_rgb = rng.normal(0, 1, (n_rays, 3)).astype(np.float32)
    d_depth = rng.normal(0, 1, n_rays).astype(np.float32)
    d_eik = np.full(n_rays, 0.1, np.float32)
    return d_rgb, d_depth, d_eik


def rel_err(got, ref):
    return np.abs(got - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("kind", [T.TSDFS_BACKWARD_GEMM, T.TSDFS_BACKWARD_SIMT], ids=["gemm", "simt"])
@pytest.mark.parametrize("scene,n_rays", [("tiny", 96), ("room", 48)])
def test_backward_matches_oracle_gradient(scene, n_rays, kind, restore_backward):
    o, d, b = case(scene, n_rays, seed=41)
    spec = synth.scene_mlp(scene)
    d_rgb, d_depth, d_eik = seeded_adjoints(n_rays)
    got_sdf, got_rgb = gpu_grads(spec, o, d, b, d_rgb, d_depth, d_eik, kind=kind)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    ref_sdf, ref_rgb = oracle_grads(spec, o, d, b, d_rgb, d_depth, d_eik)
    for got, ref, name in [(got_sdf, ref_sdf, "sdf"), (got_rgb, ref_rgb, "rgb")]:
        err = rel_err(got, ref)
        print(f"{scene} kind {kind} d{name}: max |err| / max |grad| = {err:.2e} (max |grad| {np.abs(ref).max():.3e})")
        assert err < 2e-3, name


@pytest.mark.parametrize("scene,n_rays", [("tiny", 96), ("room", 48)])
def test_layer_major_matches_simt_backward(scene, n_rays, restore_backward):
    """The two FP32 implementations differ by rounding order and the BF16x9 emulation
    of the GEMM operands: far inside the oracle bar, layer by layer."""
    o, d, b = case(scene, n_rays, seed=43)
    spec = synth.scene_mlp(scene)
    adj = seeded_adjoints(n_rays, 8)
    g = gpu_grads(spec, o, d, b, *adj, kind=T.TSDFS_BACKWARD_GEMM)
    s = gpu_grads(spec, o, d, b, *adj, kind=T.TSDFS_BACKWARD_SIMT)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    for net, (a, r), layers in [("sdf", (g[0], s[0]), spec.sdf), ("rgb", (g[1], s[1]), spec.rgb)]:
        off = 0
        for l, (W, bv) in enumerate(layers):
            k = W.size + bv.size
            err = rel_err(a[off:off + k], r[off:off + k]) if np.abs(r[off:off + k]).max() > 0 else 0.0
            print(f"{scene} {net} layer {l}: {err:.2e}")
            assert err < 2e-4, (net, l)
            off += k


@pytest.mark.parametrize("scene,n_rays,chunk", [("tiny", 96, 37), ("room", 48, 71)])
def test_chunked_backward_matches_one_chunk(scene, n_rays, chunk, restore_backward):
    """Chunks smaller than the batch (a ragged last chunk; the forward recomputed in pass 2)
    give the single-chunk gradients up to the order of the sums."""
    o, d, b = case(scene, n_rays, seed=44)
    total = int(b["n"].sum())
    assert total > 3 * chunk and total % chunk != 0
    spec = synth.scene_mlp(scene)
    adj = seeded_adjoints(n_rays, 9)
    one = gpu_grads(spec, o, d, b, *adj)
    many = gpu_grads(spec, o, d, b, *adj, chunk=chunk)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    for a, r in zip(many, one):
        assert rel_err(a, r) < 1e-4


def test_gradients_accumulate(restore_backward):
    o, d, b = case("tiny", 64, seed=45)
    spec = synth.scene_mlp("tiny")
    adj = seeded_adjoints(64, 10)
    one = gpu_grads(spec, o, d, b, *adj)
    two = gpu_grads(spec, o, d, b, *adj, calls=2)
    assert np.array_equal(two[0], 2 * one[0]) and np.array_equal(two[1], 2 * one[1])


def test_sample_overflow_sets_status_and_leaves_gradients(restore_backward):
    o, d, b = case("tiny", 64, seed=46)
    spec = synth.scene_mlp("tiny")
    total = int(b["n"].sum())
    got = gpu_grads(spec, o, d, b, *seeded_adjoints(64), max_samples=total - 1)
    rc, bits = T.tsdfs_sync_status()
    assert rc == T.TSDFS_E_DEVICE and bits & T.TSDFS_DEV_SAMPLES_OVERFLOW
    assert not got[0].any() and not got[1].any()
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits


@pytest.mark.parametrize("kind", [T.TSDFS_BACKWARD_GEMM, T.TSDFS_BACKWARD_SIMT], ids=["gemm", "simt"])
def test_rays_without_samples_give_zero_gradients(kind, restore_backward):
    o, d, b = case("tiny", 32, seed=47)
    b = dict(b)
    b["n"] = np.zeros_like(b["n"])
    b["status"] = np.zeros_like(b["status"])
    got = gpu_grads(synth.scene_mlp("tiny"), o, d, b, *seeded_adjoints(32), kind=kind, max_samples=16)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    assert not got[0].any() and not got[1].any()


def _bounds_of(o, b):
    offsets = np.concatenate([[0], np.cumsum(b["n"])]).astype(np.int32)
    bb = T.Bounds(len(o))
    bb.t_n.copy_(dev(b["t_n"].astype(np.float32)))
    bb.t_f.copy_(dev(b["t_f"].astype(np.float32)))
    bb.offsets.copy_(dev(offsets))
    bb.status.copy_(dev(b["status"]))
    return bb, int(offsets[-1])


@pytest.mark.parametrize("precision", [T.TSDFS_PREC_F32, T.TSDFS_PREC_F16])
def test_autograd_function_matches_direct_call(precision):
    """RenderFunction renders from the parameter tensors it is given and returns the
    gradients that a direct render_rays_backward call gives at those tensors."""
    o, d, b = case("tiny", 64, seed=5)
    spec = synth.scene_mlp("tiny")
    mlp = T.Mlp(spec, precision)
    bb, total = _bounds_of(o, b)
    # leaves that differ from the descriptor's own parameters: the render must follow them
    g = torch.Generator(device="cuda").manual_seed(3)
    sdf_w = (mlp.sdf_w * (1.0 + 0.01 * torch.randn(mlp.sdf_w.shape, device="cuda", generator=g))).requires_grad_(True)
    rgb_w = (mlp.rgb_w * (1.0 + 0.01 * torch.randn(mlp.rgb_w.shape, device="cuda", generator=g))).requires_grad_(True)
    ro, rd = dev(o), dev(d)
    rgb, depth, eik = T.RenderFunction.apply(sdf_w, rgb_w, mlp, ro, rd, bb, total)
    # the same render through a descriptor built directly on the leaves' values: the
    # training forward for FP32 networks, render_rays for 16-bit ones
    ref = T.Mlp(spec, precision, sdf_w=sdf_w.detach().clone(), rgb_w=rgb_w.detach().clone())
    if precision == T.TSDFS_PREC_F32:
        out = T.RenderOut(len(o))
        wst = torch.empty(T.tsdfs_train_workspace_size(ref, len(o), total), dtype=torch.uint8, device="cuda")
        T.render_rays_train(ref, ro, rd, bb.t_n, bb.t_f, bb.offsets, bb.status, total, out.rgb, out.depth, out.wsum,
                            out.normal, out.eik, wst)
    else:
        out = T.Renderer(ref, len(o), total).render(ro, rd, bb)
    torch.cuda.synchronize()
    assert torch.equal(rgb, out.rgb) and torch.equal(depth, out.depth)
    own = T.Renderer(mlp, len(o), total).render(ro, rd, bb)
    assert not torch.equal(rgb, own.rgb)
    # seeded output gradients, given to autograd and to a direct call at the same parameters
    g_rgb = torch.randn(rgb.shape, device="cuda", generator=g)
    g_depth = torch.randn(depth.shape, device="cuda", generator=g)
    g_eik = torch.full_like(eik, 0.01)
    torch.autograd.backward((rgb, depth, eik), (g_rgb, g_depth, g_eik))
    m32 = T.Mlp(spec, T.TSDFS_PREC_F32, sdf_w=sdf_w.detach().clone(), rgb_w=rgb_w.detach().clone())
    d_sdf = torch.zeros_like(m32.sdf_w)
    d_rw = torch.zeros_like(m32.rgb_w)
    ws = torch.empty(T.tsdfs_backward_workspace_size(m32, len(o), total), dtype=torch.uint8, device="cuda")
    T.render_rays_backward(m32, ro, rd, bb.t_n, bb.t_f, bb.offsets, bb.status, total, g_rgb, g_depth, g_eik, d_sdf,
                           d_rw, ws)
    torch.cuda.synchronize()
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    assert torch.equal(sdf_w.grad, d_sdf) and torch.equal(rgb_w.grad, d_rw)
    assert sdf_w.grad.abs().sum() > 0 and rgb_w.grad.abs().sum() > 0


def test_optimizer_step_on_the_leaves_changes_the_render():
    o, d, b = case("tiny", 64, seed=6)
    spec = synth.scene_mlp("tiny")
    mlp = T.Mlp(spec)
    bb, total = _bounds_of(o, b)
    sdf_w = mlp.sdf_w.clone().requires_grad_(True)
    rgb_w = mlp.rgb_w.clone().requires_grad_(True)
    opt = torch.optim.SGD([sdf_w, rgb_w], lr=1e-2)
    ro, rd = dev(o), dev(d)
    target = torch.zeros((len(o), 3), device="cuda")
    rgb0, _, _ = T.RenderFunction.apply(sdf_w, rgb_w, mlp, ro, rd, bb, total)
    loss0 = (rgb0 - target).abs().mean()
    loss0.backward()
    opt.step()
    opt.zero_grad()
    rgb1, _, _ = T.RenderFunction.apply(sdf_w, rgb_w, mlp, ro, rd, bb, total)
    loss1 = (rgb1 - target).abs().mean()
    assert not torch.equal(rgb0, rgb1)
    assert loss1.item() < loss0.item()
    # the descriptor's own copy is untouched
    assert torch.equal(mlp.sdf_w, torch.tensor(spec.packed("sdf"), device="cuda"))


def train_call(spec, o, d, b, adj, max_samples=None, chunk=0):
    """render_rays_train then render_rays_backward_kept over one workspace: outputs and gradients."""
    T.tsdfs_set_backward_chunk(chunk)
    n = len(o)
    mlp = T.Mlp(spec)
    bb, total = _bounds_of(o, b)
    ms = total if max_samples is None else max_samples
    out = T.RenderOut(n)
    ws = torch.empty(max(T.tsdfs_train_workspace_size(mlp, n, ms), 1), dtype=torch.uint8, device="cuda")
    ro, rd = dev(o), dev(d)
    T.render_rays_train(mlp, ro, rd, bb.t_n, bb.t_f, bb.offsets, bb.status, ms, out.rgb, out.depth, out.wsum,
                        out.normal, out.eik, ws)
    d_sdf = torch.zeros_like(mlp.sdf_w)
    d_rw = torch.zeros_like(mlp.rgb_w)
    T.render_rays_backward_kept(mlp, ro, rd, bb.t_n, bb.t_f, bb.offsets, bb.status, ms, *[dev(a) for a in adj], d_sdf,
                                d_rw, ws)
    torch.cuda.synchronize()
    fwd = {k: getattr(out, k).cpu().numpy() for k in ("rgb", "depth", "wsum", "normal", "eik")}
    return fwd, (d_sdf.cpu().numpy(), d_rw.cpu().numpy())


@pytest.mark.parametrize("scene,n_rays", [("tiny", 96), ("room", 48)])
def test_train_forward_matches_oracle_and_render(scene, n_rays, restore_backward):
    """The layer-major FP32 forward meets the FP32 render bars against the oracle and agrees
    with the SIMT FP32 render far inside them."""
    from test_gpu_render import DEPTH_REL_F32, compare, gpu_render, oracle_render
    o, d, b = case(scene, n_rays, seed=48)
    spec = synth.scene_mlp(scene)
    fwd, _ = train_call(spec, o, d, b, seeded_adjoints(n_rays))
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    ref, _ = oracle_render(spec, o, d, b)
    compare(fwd, ref, depth_rel=DEPTH_REL_F32)
    simt = gpu_render(spec, o, d, b)
    assert np.max(np.abs(fwd["rgb"] - simt["rgb"])) < 1e-4
    assert np.max(np.abs(fwd["eik"] - simt["eik"])) <= 1e-4 * max(1.0, np.abs(simt["eik"]).max())


@pytest.mark.parametrize("scene,n_rays,chunk", [("tiny", 96, 0), ("room", 48, 0), ("tiny", 96, 37), ("room", 48, 71)])
def test_kept_backward_equals_backward(scene, n_rays, chunk, restore_backward):
    """render_rays_backward_kept after render_rays_train returns exactly the gradients of a
    render_rays_backward call on the same inputs, in one chunk and in several."""
    o, d, b = case(scene, n_rays, seed=49)
    spec = synth.scene_mlp(scene)
    adj = seeded_adjoints(n_rays, 11)
    _, kept = train_call(spec, o, d, b, adj, chunk=chunk)
    direct = gpu_grads(spec, o, d, b, *adj, chunk=chunk)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    assert np.array_equal(kept[0], direct[0]) and np.array_equal(kept[1], direct[1])


def test_train_forward_overflow_zeroes_outputs(restore_backward):
    o, d, b = case("tiny", 64, seed=50)
    total = int(b["n"].sum())
    fwd, grads = train_call(synth.scene_mlp("tiny"), o, d, b, seeded_adjoints(64), max_samples=total - 1)
    rc, bits = T.tsdfs_sync_status()
    assert rc == T.TSDFS_E_DEVICE and bits & T.TSDFS_DEV_SAMPLES_OVERFLOW
    assert not fwd["rgb"].any() and not fwd["wsum"].any()
    assert not grads[0].any() and not grads[1].any()


def test_nonfinite_parameter_flagged(restore_backward):
    """The layer-major GEMMs assume finite operands: a NaN or an infinity planted in the
    parameters is reported as TSDFS_DEV_NONFINITE, and the context stays usable."""
    o, d, b = case("tiny", 32, seed=51)
    spec = synth.scene_mlp("tiny")
    adj = seeded_adjoints(32, 12)
    for bad in (float("nan"), float("inf")):
        mlp = T.Mlp(spec)
        mlp.sdf_w[7] = bad
        bb, total = _bounds_of(o, b)
        d_sdf = torch.zeros_like(mlp.sdf_w)
        d_rw = torch.zeros_like(mlp.rgb_w)
        ws = torch.empty(T.tsdfs_backward_workspace_size(mlp, len(o), total), dtype=torch.uint8, device="cuda")
        T.render_rays_backward(mlp, dev(o), dev(d), bb.t_n, bb.t_f, bb.offsets, bb.status, total,
                               *[dev(a) for a in adj], d_sdf, d_rw, ws)
        rc, bits = T.tsdfs_sync_status()
        assert rc == T.TSDFS_E_DEVICE and bits & T.TSDFS_DEV_NONFINITE
    good = gpu_grads(spec, o, d, b, *adj)
    rc, bits = T.tsdfs_sync_status()
    assert rc == 0, bits
    assert np.isfinite(good[0]).all() and np.abs(good[0]).max() > 0
