"""What the learned warm start gains: a network trained on solver-generated
pairs (by the library's own forward / backward kernels) starts the plain
fixed-point iteration closer to its fixed point, so held-out images reach the
same residual in fewer iterations than from u0 = Phi (the method without it)
and than from the analytic guess u0 = Phi / lambda, with the same accuracy."""
import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def trained():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_08793_gb300 import _native, warmstart as WS

    _native.lib()
    data = WS.make_dataset(96, 128, 128, seed0=5_000_000)
    net = WS.WarmStartNet(32, seed=1)
    log = net.train(data, steps=400, batch=8, lr=1e-3, lr_end=5e-5, log_every=100)
    return WS, net, log


def test_training_loss_falls(trained):
    _, _, log = trained
    assert log[-1][1] < 0.5 * log[0][1], log


def test_warm_start_saves_iterations(trained):
    WS, net, _ = trained
    e = WS.evaluate(net, range(6_000_000, 6_000_006), 128, 128, repeats=1)
    s = e["summary"]
    assert s["net"]["mean_iter"] < 0.8 * s["cold"]["mean_iter"], s
    assert s["net"]["mean_iter"] < s["analytic"]["mean_iter"], s
    for r in e["images"]:
        assert r["net"]["rho"] <= 1e-4 and r["cold"]["rho"] <= 1e-4


def test_warm_start_accuracy_against_oracle(trained, orc):
    """Same residual, same accuracy against the FP64 fixed point as the cold start."""
    from paper_2506_08793_gb300 import api

    WS, net, _ = trained
    H, W = 64, 96
    I = scenes.hazy_scene(6_200_000, H, W)["I"]
    r = orc.dehaze(I, orc.params(**orc.STABLE), 20000, 1e-9)
    Id = torch.from_numpy(I).cuda()
    cold = api.dehaze(Id, api.params("stable"))
    wd = WS.WarmDehazer(net, H, W)
    rep = wd(Id)
    assert rep.status == 0 and max(rep.rho) <= 1e-4
    torch.cuda.synchronize()
    e_cold = np.max(np.abs(cold["u"].cpu().numpy() - r["u"]))
    e_warm = np.max(np.abs(wd.dz.u.cpu().numpy() - r["u"]))
    assert e_warm <= 2 * e_cold + 2e-4, (e_warm, e_cold)
    assert np.array_equal(wd.dz.A.cpu().numpy(), r["A"].astype(np.float32))


WARM_SHAPES = [(64, 128), (56, 96), (48, 136), (128, 128)]


def test_warm_batch_matches_single_image_warm_start(trained):
    """dh_dehaze_batch_warm: per image the same front end and network u0 as
    dh_dehaze_warm, then the batched loop; every image ends where the
    single-image warm solve ends (n within one, u to float32 rounding)."""
    from paper_2506_08793_gb300 import api

    WS, net, _ = trained
    imgs = [torch.from_numpy(scenes.hazy_scene(6_300_000 + k, H, W)["I"]).cuda()
            for k, (H, W) in enumerate(WARM_SHAPES)]
    b = api.BatchDehazer(WARM_SHAPES, api.params("stable"), net=net)
    reps = b(imgs)
    for k, ((H, W), I, r, o) in enumerate(zip(WARM_SHAPES, imgs, reps, b.out)):
        wd = WS.WarmDehazer(net, H, W)
        one = wd(I)
        assert r.status == 0 and max(r.rho) <= 1e-4, k
        assert r.a_index == one.a_index and torch.equal(o["A"], wd.dz.A) and torch.equal(o["t"], wd.dz.t), k
        assert abs(r.n_iter - one.n_iter) <= 1, (k, r.n_iter, one.n_iter)
        if r.n_iter == one.n_iter:
            assert torch.allclose(o["u"], wd.dz.u, rtol=1e-6, atol=1e-6), k
        assert torch.equal(torch.clamp(o["u"], 0, 1), o["J"])


def test_warm_batch_groups_of_one_shape(trained):
    """Images of one shape share a network forward (1080p: two a forward, so
    three 1080p images make a group of two and one of one; three 64x128
    images interleaved with other shapes make one group of three).  Every
    image still ends where its single-image warm solve ends."""
    from paper_2506_08793_gb300 import api

    WS, net, _ = trained
    shapes = [(1080, 1920), (64, 128), (1080, 1920), (56, 96), (64, 128), (1080, 1920), (64, 128)]
    imgs = [torch.from_numpy(scenes.hazy_scene(6_500_000 + k, H, W)["I"]).cuda() for k, (H, W) in enumerate(shapes)]
    b = api.BatchDehazer(shapes, api.params("stable"), net=net)
    reps = b(imgs)
    for k, ((H, W), I, r, o) in enumerate(zip(shapes, imgs, reps, b.out)):
        wd = WS.WarmDehazer(net, H, W)
        one = wd(I)
        assert r.status == 0 and max(r.rho) <= 1e-4, k
        assert abs(r.n_iter - one.n_iter) <= 1, (k, r.n_iter, one.n_iter)
        if r.n_iter == one.n_iter:
            assert torch.allclose(o["u"], wd.dz.u, rtol=1e-6, atol=1e-6), k
        del wd


@pytest.mark.parametrize("storage", [0, 3, 4])  # DH_STORE_F32, DH_STORE_BF16_F32, DH_STORE_F16_F32
def test_warm_batch_reaches_tolerance_with_cold_accuracy(trained, orc, storage):
    """The warm-started batched form (network u0, then the batched loop in
    float32 or a switched 16-bit -> float32 storage) reaches 1e-4 on every
    image, as close to the FP64 fixed point as the cold float32 batch, and the
    float32 form takes fewer iterations than the cold batch."""
    from paper_2506_08793_gb300 import api

    WS, net, _ = trained
    shapes = WARM_SHAPES[:3]
    Is = [scenes.hazy_scene(6_400_000 + k, H, W)["I"] for k, (H, W) in enumerate(shapes)]
    imgs = [torch.from_numpy(I).cuda() for I in Is]
    cold = api.dehaze_batch(imgs, api.params("stable"))
    wb = api.BatchDehazer(shapes, api.params("stable", storage=storage), net=net)
    reps = wb(imgs)
    op = orc.params(**orc.STABLE)
    for k, I in enumerate(Is):
        assert reps[k].status == 0 and max(reps[k].rho) <= 1e-4, k
        ustar = orc.dehaze(I, op, 20000, 1e-9)["u"]
        e_cold = np.max(np.abs(cold[k]["u"].cpu().numpy() - ustar))
        e_warm = np.max(np.abs(wb.out[k]["u"].cpu().numpy() - ustar))
        assert e_warm <= 2 * e_cold + 2e-4, (k, e_warm, e_cold)
    if storage == 0:
        assert sum(r.n_iter for r in reps) < 0.8 * sum(c["report"].n_iter for c in cold)
