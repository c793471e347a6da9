"""tsdf_ray_bounds_noalloc: the ray-bounds entry point for callers that cannot
allocate device memory (no workspace argument; the library's own fixed device
scratch holds the offsets scan's partial sums).

Its results must equal tsdf_ray_bounds' (bit for bit, like every bounds test)
on two calls in a row, which share and reuse that scratch; a batch above the
stated maximum is refused.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

from paper_2311_17878_gb300 import build, synth
from paper_2311_17878_gb300 import tsdfs as T

pytestmark = pytest.mark.gpu

FIELDS = ("t_n", "t_f", "n", "offsets", "t_zero", "status")


def _grid_and_rays():
    wl = synth.room_workload(with_views=False)
    V = synth.analytic_tsdf_torch(wl.scene, wl.grid, device="cuda")
    g = T.Grid(wl.grid, V=V, W=torch.zeros(V.shape, dtype=torch.uint8, device="cuda"))
    return wl, g


def _noalloc(g, o, d, bp, mask):
    n = o.shape[0]
    out = T.Bounds(n)
    T.tsdf_ray_bounds_noalloc(g, mask, o, d, T.bounds_params(bp), out.t_n, out.t_f, out.n, out.offsets, out.t_zero,
                              out.status)
    return out


def _same(a, b):
    for k in FIELDS:
        x, y = getattr(a, k).cpu().numpy(), getattr(b, k).cpu().numpy()
        if x.dtype == np.float32:
            x, y = x.view(np.uint32), y.view(np.uint32)
        assert np.array_equal(x, y), k


def test_noalloc_bounds_match_workspace_bounds_twice():
    build.build()
    wl, g = _grid_and_rays()
    bp = wl.bounds
    mask = g.inside_mask(bp.nb_radius)
    for call, (o, d) in enumerate([synth.room_heldout_rays(2), synth.room_panorama_rays()]):
        o, d = torch.tensor(o).cuda(), torch.tensor(d).cuda()
        ref = T.Bounds(o.shape[0]).compute(g, o, d, bp, mask)
        got = _noalloc(g, o, d, bp, mask if call == 0 else None)
        torch.cuda.synchronize()
        _same(got, ref)
        assert int(got.offsets[-1].item()) > 0
    rc, bits = T.tsdfs_sync_status()
    assert rc == T.TSDFS_OK and bits == 0


def test_noalloc_refuses_batches_above_its_scratch():
    build.build()
    wl, g = _grid_and_rays()
    big = T.tsdf_ray_bounds_noalloc_max_rays() + 1
    e = torch.empty((1, 3), device="cuda")
    with pytest.raises(T.TsdfsError) as err:
        T.lib().tsdf_ray_bounds_noalloc  # resolves the symbol
        T._check(T.lib().tsdf_ray_bounds_noalloc(
            T.C.byref(g.c), None, T._p(e), T._p(e), T.C.c_int64(big), T.C.byref(T.bounds_params(wl.bounds)),
            T._p(e), T._p(e), T._p(e), T._p(e), None, T._p(e), T._stream()))
    assert err.value.code == T.TSDFS_E_INVALID
    assert "at most" in str(err.value)
