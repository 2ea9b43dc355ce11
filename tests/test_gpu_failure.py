"""Failure detection without a GPU fault: a device wait that nothing completes
gives up after its bound and reports DH_ETIMEOUT to the host; the context stays
usable afterwards (a normal call succeeds)."""
import time

import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_08793_gb300 import _native

    _native.lib()
    return _native


def test_bounded_wait_reports_timeout_and_context_survives(N):
    t0 = time.perf_counter()
    assert N.dh_selftest_bounded_wait(2_000_000) == N.DH_ETIMEOUT  # about 1 ms of SM clocks
    assert time.perf_counter() - t0 < 5.0
    assert N.dh_selftest_bounded_wait(0) == N.DH_EINVAL
    from paper_2506_08793_gb300 import api

    out = api.dehaze(torch.from_numpy(scenes.hazy_scene(5, 48, 64)["I"]).cuda(), api.params("stable"))
    assert out["report"].status == N.DH_OK
    assert np.isfinite(out["u"].cpu().numpy()).all()
