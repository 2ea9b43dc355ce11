"""The autotuner times every usable sweep variant and its choice is used by
later calls; every variant computes the same iterates (to a few ulps)."""
import json

import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_08793_gb300 import _native, api as a

    _native.lib()
    return a


def test_tune_records_best_and_is_used(api, tmp_path):
    from paper_2506_08793_gb300 import _native as N

    H, W = 200, 384
    I = torch.from_numpy(scenes.hazy_scene(71, H, W)["I"]).cuda()
    r = api.tune(I, api.params("stable"), iters=10)
    assert r["best"] >= 1 and len(r["us_per_iter"]) == N.dh_sweep_variants() - 1
    assert all(v > 0 for v in r["us_per_iter"].values())
    assert r["us_per_iter"][r["best"]] == min(r["us_per_iter"].values())
    assert N.dh_tune_get(H, W, 0) == r["best"]
    # the tuned variant gives the default variant's result (to a few ulps)
    a = api.dehaze(I, api.params("stable"))
    b = api.dehaze(I, api.params("stable", sweep_variant=1))
    assert abs(a["report"].n_iter - b["report"].n_iter) <= 1
    if a["report"].n_iter == b["report"].n_iter:
        assert torch.allclose(a["u"], b["u"], rtol=1e-6, atol=1e-6)
    path = tmp_path / "tune.json"
    api.save_tuning(str(path), [(H, W)])
    assert json.load(open(path))["variants"][f"{H}x{W}"] == r["best"]
    assert N.dh_tune_set(H, W, 0, 0) == 0 and N.dh_tune_get(H, W, 0) == 0
    assert api.load_tuning(str(path)) == 1 and N.dh_tune_get(H, W, 0) == r["best"]


def test_unaligned_width_only_generic_variants(api):
    H, W = 50, 70
    I = torch.from_numpy(scenes.hazy_scene(72, H, W)["I"]).cuda()
    r = api.tune(I, api.params("stable"), iters=5)
    assert len(r["us_per_iter"]) == 3  # the three gather-based variants
