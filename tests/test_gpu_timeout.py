"""The timeout path of the bounded device waits, on the GPU: a wait that
nothing completes gives up after its bound (about a second), the handle's
flag reports DC_ERR_TIMEOUT on the host, and the context stays usable."""
import numpy as np
import pytest
import torch

from paper_2410_14900_gb300 import api
from paper_2410_14900_gb300 import _lib as L

from cases import circle64, phantom_projections, rel_l2

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_is_reported():
    case = circle64()
    geom = api.Geometry(case.desc, case.P, case.vdl)
    g = torch.as_tensor(phantom_projections(case).astype(np.float32), device="cuda")
    before = api.reconstruct(geom, g)
    api.dc_sync_status(geom)
    Lh = L.load()
    assert Lh.dc_debug_wait_timeout(geom.handle, None) == L.DC_OK
    with pytest.raises(L.DCError) as err:
        api.dc_sync_status(geom)
    assert err.value.code == L.DC_ERR_TIMEOUT
    # the flag is cleared once reported, and the context keeps working
    after = api.reconstruct(geom, g)
    api.dc_sync_status(geom)
    torch.cuda.synchronize()
    assert rel_l2(after.double().cpu().numpy(), before.double().cpu().numpy()) == 0.0
