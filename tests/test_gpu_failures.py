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
