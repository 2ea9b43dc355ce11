"""The largest image the library accepts (H * W = 2^28 pixels, W = 32768, the
per-dimension maximum): every index and byte offset of the front end and the
sweep stays in range.  Checked on sampled pixels (corners, last rows and
columns included) against the oracle on crops, after two fixed-point steps.
One size past the limit is rejected before any work."""
import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

H, W = 8192, 32768


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_08793_gb300 import _native, api as a

    _native.lib()
    return a


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def test_maximum_size(api, orc):
    from paper_2506_08793_gb300 import _native as N

    assert N.dh_workspace_bytes(H, W + 1, api.params("stable")) == 0  # past the per-dimension limit
    assert N.dh_workspace_bytes(H + 1, W, api.params("stable")) == 0  # past the pixel limit
    tile = scenes.hazy_scene(4242, 2048, 2048)["I"]
    I = np.tile(tile, (1, H // 2048, W // 2048))
    Id = torch.from_numpy(I).cuda()
    n = 2
    out = api.dehaze(Id, api.params("stable", tol=0.0, max_iter=n))
    rep = out["report"]
    assert rep.status == N.DH_WNOCONV and rep.n_iter == n
    A = host(out["A"]).astype(np.float64)
    idx = rep.a_index
    assert 0 <= idx < H * W and np.array_equal(A.astype(np.float32), I[:, idx // W, idx % W])
    ug = host(out["u"])
    op = orc.params(**orc.STABLE)
    rng = np.random.default_rng(7)
    ys = np.r_[rng.integers(0, H, 10), [0, H - 1, 0, H - 1, H // 2]]
    xs = np.r_[rng.integers(0, W, 10), [0, W - 1, W - 1, 0, W - 1]]
    rad = 2 * n + 2
    for y, x in zip(ys, xs):
        # the oracle's front end and n steps on a crop wide enough for the
        # 15x15 windows and the dependency cone (2 pixels per step)
        y0, y1, x0, x1 = max(0, y - rad), min(H, y + rad + 1), max(0, x - rad), min(W, x + rad + 1)
        Y0, Y1, X0, X1 = max(0, y0 - 7), min(H, y1 + 7), max(0, x0 - 7), min(W, x1 + 7)
        td = orc.dark_channel(I[:, Y0:Y1, X0:X1], 15, A)[y0 - Y0: y1 - Y0, x0 - X0: x1 - X0]
        _, lam, Phi = orc.transmission(I[:, y0:y1, x0:x1], A, td, op)
        Phi32, lam32 = Phi.astype(np.float32), lam.astype(np.float32)
        uc, _, _ = orc.solve(Phi32.astype(np.float64), Phi32, lam32, op, n, 0.0)
        assert np.max(np.abs(uc[:, y - y0, x - x0] - ug[:, y, x])) <= 2e-5, (y, x)
    del out, Id
    torch.cuda.empty_cache()
