"""Device-side failure reporting without faults: non-finite network parameters
are detected by tsdfs_check_mlp and by packing, and reported through the
status word; the context stays usable afterwards."""
import numpy as np
import pytest
import torch

from paper_2311_17878_gb300 import build, synth
from paper_2311_17878_gb300 import tsdfs as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    T.lib()
    T.tsdfs_sync_status()


def test_clean_parameters_report_nothing():
    mlp = T.Mlp(synth.scene_mlp("room"), T.TSDFS_PREC_F16)
    T.tsdfs_check_mlp(mlp)
    rc, bits = T.tsdfs_sync_status()
    assert rc == T.TSDFS_OK and bits == 0


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_non_finite_parameter_is_reported(bad):
    mlp = T.Mlp(synth.scene_mlp("room"), T.TSDFS_PREC_F32)
    mlp.sdf_w[12345] = bad
    T.tsdfs_check_mlp(mlp)
    rc, bits = T.tsdfs_sync_status()
    assert rc == T.TSDFS_E_DEVICE and bits & T.TSDFS_DEV_NONFINITE
    # packing the same values reports it too; the status word was cleared by the read
    mlp16 = T.Mlp(synth.scene_mlp("room"), T.TSDFS_PREC_F16)
    torch.cuda.synchronize()
    T.tsdfs_sync_status()
    mlp16.rgb_w[7] = bad
    T.tsdfs_pack_mlp(mlp16, mlp16.packed)
    rc, bits = T.tsdfs_sync_status()
    assert rc == T.TSDFS_E_DEVICE and bits & T.TSDFS_DEV_NONFINITE
    # the context still works
    x = torch.ones(4, device="cuda") * 2
    assert float(x.sum().item()) == 8.0


# ---------------------------------------------------------------------------
# failure paths of the kernels, made to run out without a fault
# ---------------------------------------------------------------------------
@pytest.fixture
def limits():
    yield T.tsdfs_set_test_limits
    T.tsdfs_set_test_limits(0, 0, -1)
    T.tsdfs_sync_status()


def _room_case():
    from test_gpu_render import _scene_case
    return _scene_case("room")


@pytest.mark.parametrize("precision,kernel", [(T.TSDFS_PREC_F16, T.TSDFS_NETKERNEL_SERIAL),
                                              (T.TSDFS_PREC_F16, T.TSDFS_NETKERNEL_PIPELINED),
                                              (T.TSDFS_PREC_BF16X2, T.TSDFS_NETKERNEL_PIPELINED)])
def test_network_wait_runs_out_and_context_recovers(limits, precision, kernel):
    """A weight chunk that is never copied: the MMA issuer's bounded wait for it runs
    out, the kernel reports TSDFS_DEV_TIMEOUT and returns, compositing writes zeros;
    with the limits lifted the next call on the same context matches the oracle."""
    from test_gpu_render import DEPTH_REL_BF16, compare, gpu_render, oracle_render
    o, d, b = _room_case()
    spec = synth.scene_mlp("room")
    old = T.tsdfs_network_kernel(precision)
    T.tsdfs_set_network_kernel(precision, kernel)
    try:
        limits(1 << 14, 0, 5)
        got = gpu_render(spec, o, d, b, precision=precision)
        rc, bits = T.tsdfs_sync_status()
        assert rc == T.TSDFS_E_DEVICE and bits & T.TSDFS_DEV_TIMEOUT, bits
        assert np.all(got["rgb"] == 0) and np.all(got["wsum"] == 0) and np.all(got["depth"] == 0)
        limits(0, 0, -1)
        got = gpu_render(spec, o, d, b, precision=precision)
        rc, bits = T.tsdfs_sync_status()
        assert rc == T.TSDFS_OK and bits == 0
    finally:
        T.tsdfs_set_network_kernel(precision, old)
    ref, _ = oracle_render(spec, o, d, b)
    compare(got, ref, depth_rel=DEPTH_REL_BF16)


def test_value_kernel_wait_runs_out(limits):
    """The comparator's coarse pass (the value-only tensor-core kernel) the same way."""
    wl = synth.tiny_workload()
    spec = synth.scene_mlp("tiny")
    g = T.Grid(wl.grid, V=torch.zeros(wl.grid.shape_zyx, device="cuda"),
               W=torch.zeros(wl.grid.shape_zyx, dtype=torch.uint8, device="cuda"))
    h = T.HierRenderer(T.Mlp(spec, T.TSDFS_PREC_F16), 4096)
    o, d = torch.tensor(wl.rays_o).cuda(), torch.tensor(wl.rays_d).cuda()
    limits(1 << 14, 0, 1)
    h.render(g, o, d, wl.bounds.t_near, wl.bounds.t_far)
    rc, bits = T.tsdfs_sync_status()
    assert rc == T.TSDFS_E_DEVICE and bits & T.TSDFS_DEV_TIMEOUT, bits
    limits(0, 0, -1)
    out = h.render(g, o, d, wl.bounds.t_near, wl.bounds.t_far)
    rc, bits = T.tsdfs_sync_status()
    assert rc == T.TSDFS_OK and bits == 0
    assert float(out.wsum.max()) > 0.5


def test_march_step_cap_reports_and_recovers(limits):
    """A voxel walk cut short after a few steps: TSDFS_DEV_MARCH_CAP, the cut rays fall
    back to their whole grid-box clip (near phase) or keep t_f = t_end (far phase);
    without the cap the bounds are bit-exact against the oracle again."""
    from oracle import cgrid
    wl = synth.tiny_workload()
    V, _ = cgrid.integrate_projective(wl.grid, wl.views, "f32")
    ref = cgrid.ray_bounds(wl.grid, V, wl.rays_o, wl.rays_d, wl.bounds, "f32")
    t0, te, ok = cgrid.clip_rays(wl.grid, wl.rays_o, wl.rays_d, wl.bounds.t_near, wl.bounds.t_far, "f32")
    g = T.Grid(wl.grid, V=torch.tensor(V).cuda(), W=torch.ones(wl.grid.shape_zyx, dtype=torch.uint8, device="cuda"))
    o, d = torch.tensor(wl.rays_o).cuda(), torch.tensor(wl.rays_d).cuda()
    b = T.Bounds(len(o))
    limits(0, 4, -1)
    b.compute(g, o, d, wl.bounds)
    rc, bits = T.tsdfs_sync_status()
    assert rc == T.TSDFS_E_DEVICE and bits & T.TSDFS_DEV_MARCH_CAP, bits
    st, tn, tf = b.status.cpu().numpy(), b.t_n.cpu().numpy(), b.t_f.cpu().numpy()
    cut = (ref["status"] == 1) & (st == 2)
    assert cut.sum() > 0
    assert np.array_equal(tn[cut], t0[cut]) and np.array_equal(tf[cut], te[cut])
    kept = (ref["status"] == 1) & (st == 1)
    assert np.array_equal(tn[kept], ref["t_n"][kept])
    assert np.all((tf[kept] == ref["t_f"][kept]) | (tf[kept] == te[kept]))
    limits(0, 0, -1)
    b.compute(g, o, d, wl.bounds)
    rc, bits = T.tsdfs_sync_status()
    assert rc == T.TSDFS_OK and bits == 0
    assert np.array_equal(b.status.cpu().numpy(), ref["status"])
    assert np.array_equal(b.t_n.cpu().numpy().view(np.uint32), ref["t_n"].view(np.uint32))
    assert np.array_equal(b.t_f.cpu().numpy().view(np.uint32), ref["t_f"].view(np.uint32))
    assert np.array_equal(b.n.cpu().numpy(), ref["n"])
