"""The allocation-free atmospheric-light entry point (for callers that cannot
call cudaMalloc, e.g. a plug-in whose host owns all device memory) gives the
same A and index as the workspace entry point, on two calls in a row.  Named
to be collected last."""
import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_08793_gb300 import _native as N
    from paper_2506_08793_gb300 import api

    # sizes beyond the maximum are rejected before any GPU work
    assert N.dh_atmospheric_light_noalloc(1, 1, 1 << 15, 1 << 15, 1, 1, None) == N.DH_EINVAL
    # two calls in a row on different images: stale scratch would show
    for seed, H, W in ((1000, 256, 256), (2000, 1080, 1920), (4, 301, 517)):
        I = torch.from_numpy(scenes.hazy_scene(seed, H, W)["I"]).cuda()
        dc = api.dark_channel(I, 15)
        A_ref, idx_ref, _ = api.atmospheric_light(I, dc, 1)
        A = torch.full((3,), float("nan"), device="cuda")
        idx = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        rc = N.dh_atmospheric_light_noalloc(I, dc, H, W, 1, A, idx, torch.cuda.current_stream())
        assert rc == N.DH_OK, N.dh_strerror(rc)
        torch.cuda.synchronize()
        assert torch.equal(idx, idx_ref)
        assert np.array_equal(A.cpu().numpy(), A_ref.cpu().numpy())  # bit-exact, as the selection is
