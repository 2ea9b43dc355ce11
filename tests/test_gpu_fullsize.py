"""Accuracy at the workload sizes, through the C ABI, against FP64 oracle
values stored in tests/golden/ by tests/golden/make_fixed_points.py (the
oracle alone wrote them; see that script):

  - the 1920x1080 scene (seed 2000) solved to 1e-4: the same stopping n (within
    one) and A, and, after exactly the oracle's n updates, u and J within the
    float32 tolerance 1e-4 at 16384 sampled pixels;
  - the 3840x2160 scene (seed 2001) after 64 updates, at 16384 sampled pixels;
  - every fourth image of the 64-image uneven batch (all four photo sizes)
    after exactly its oracle n, at 4096 sampled pixels each."""
import os

import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = 1e-4


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_08793_gb300 import _native, api as a

    _native.lib()
    return a


def gold(name):
    return dict(np.load(os.path.join(GOLDEN, name)))


def at(t, ys, xs):
    torch.cuda.synchronize()
    return t[:, torch.from_numpy(ys).cuda(), torch.from_numpy(xs).cuda()].double().cpu().numpy()


def test_1080p_converged_against_oracle(api):
    g = gold("fp_1080p_seed2000.npz")
    H, W, seed, n = int(g["H"]), int(g["W"]), int(g["seed"]), int(g["n"])
    I = torch.from_numpy(scenes.hazy_scene(seed, H, W)["I"]).cuda()
    free = api.dehaze(I, api.params("stable"))
    assert free["report"].status == 0
    assert abs(free["report"].n_iter - n) <= 1, (free["report"].n_iter, n)
    assert free["report"].a_index == int(g["a_index"])
    assert np.array_equal(free["A"].cpu().numpy(), g["A"].astype(np.float32))
    fixed = api.dehaze(I, api.params("stable", tol=0.0, max_iter=n))
    assert fixed["report"].n_iter == n
    u = at(fixed["u"], g["ys"], g["xs"])
    J = at(fixed["J"], g["ys"], g["xs"])
    err_u = np.max(np.abs(u - g["u"]))
    assert err_u <= TOL, err_u
    assert np.max(np.abs(J - np.clip(g["u"], 0.0, 1.0))) <= TOL


def test_4k_64_updates_against_oracle(api):
    g = gold("fp_4k_seed2001_n64.npz")
    H, W, seed, n = int(g["H"]), int(g["W"]), int(g["seed"]), int(g["n"])
    I = torch.from_numpy(scenes.hazy_scene(seed, H, W)["I"]).cuda()
    out = api.dehaze(I, api.params("stable", tol=0.0, max_iter=n))
    assert out["report"].n_iter == n and out["report"].a_index == int(g["a_index"])
    u = at(out["u"], g["ys"], g["xs"])
    err = np.max(np.abs(u - g["u"]))
    assert err <= TOL, err
    # the residual the library reports is the oracle's to float32 summation accuracy
    assert np.allclose(out["report"].rho, g["rho"], rtol=1e-4)


def test_batch_images_converged_against_oracle(api):
    g = gold("fp_batch64_subset.npz")
    for i, k in enumerate(g["k"]):
        H, W, n1 = int(g["H"][i]), int(g["W"][i]), int(g["n1"][i])
        I = torch.from_numpy(scenes.hazy_scene(3000 + int(k), H, W)["I"]).cuda()
        out = api.dehaze(I, api.params("stable", tol=0.0, max_iter=n1))
        assert out["report"].n_iter == n1
        u = at(out["u"], g["ys"][i], g["xs"][i])
        err = np.max(np.abs(u - g["u1"][i]))
        assert err <= TOL, (int(k), W, H, err)
