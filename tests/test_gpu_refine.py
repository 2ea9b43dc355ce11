"""The front-end refinements (multiscale dark channel, guided-filter
refinement of t) through the C ABI against the FP64 oracle: t_d, t, lambda and
Phi to float32 rounding on ragged shapes and every radius regime (window
larger than the image included), and the whole method with both refinements
converging to the oracle's fixed point."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("H,W", [(40, 52), (97, 130), (16, 16), (1, 40), (33, 7)])
@pytest.mark.parametrize("scales,r", [(3, 0), (1, 4), (3, 8), (1, 24), (3, 1)])
def test_refined_transmission_matches_oracle(api, orc, H, W, scales, r):
    I = scenes.hazy_scene(500 + H * W + r, H, W)["I"]
    op = orc.params(**dict(orc.STABLE, dc_scales=scales, gf_radius=r, gf_eps=1e-3))
    dc = orc.dark_channel(I, 15, None)
    A, _, _ = orc.atmospheric_light(I, dc, 1)
    otd = orc.dark_channel_ms(I, 15, scales, A)
    ot, olam, oPhi = orc.transmission(I, A, otd, op)
    p = api.params("stable", dc_scales=scales, gf_radius=r, gf_eps=1e-3)
    td, t, lam, Phi = api.transmission(dev(I), dev(A.astype(np.float32)), p)
    assert np.max(np.abs(host(td) - otd)) <= 6e-8  # the FP64 mean rounded once
    assert np.max(np.abs(host(t) - ot)) <= 2e-7
    assert np.max(np.abs(host(lam) - olam) / olam) <= 2e-6
    assert np.max(np.abs(host(Phi) - oPhi) / np.maximum(1.0, np.abs(oPhi))) <= 4e-6


def test_whole_method_with_refinements(api, orc):
    H, W = 64, 96
    I = scenes.hazy_scene(601, H, W)["I"]
    op = orc.params(**dict(orc.STABLE, dc_scales=3, gf_radius=8, gf_eps=1e-3))
    want = orc.dehaze(I, op, 5000, 1e-4)
    out = api.dehaze(dev(I), api.params("stable", dc_scales=3, gf_radius=8, gf_eps=1e-3))
    rep = out["report"]
    assert rep.status == 0 and rep.a_index == want["a_index"]
    assert abs(rep.n_iter - want["n"]) <= 1
    assert np.max(np.abs(host(out["u"]) - want["u"])) <= 1e-4
    # the refinement changes the result (it is not a no-op)
    plain = api.dehaze(dev(I), api.params("stable"))
    assert np.max(np.abs(host(plain["t"]) - host(out["t"]))) > 1e-3


def test_batch_with_refinements_matches_single(api):
    p = api.params("stable", dc_scales=3, gf_radius=6)
    sizes = [(48, 64), (37, 52)]
    imgs = [dev(scenes.hazy_scene(610 + k, H, W)["I"]) for k, (H, W) in enumerate(sizes)]
    res = api.dehaze_batch(imgs, p)
    for I, r in zip(imgs, res):
        one = api.dehaze(I, p)
        assert r["report"].n_iter == one["report"].n_iter
        assert np.max(np.abs(host(r["u"]) - host(one["u"])) / np.maximum(1.0, np.abs(host(one["u"])))) <= 1e-6
