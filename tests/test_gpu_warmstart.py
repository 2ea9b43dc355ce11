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
