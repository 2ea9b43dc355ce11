"""Each tensor-core convolution family run 20 times in one process: the
outputs must be bit-identical from run to run and within the element-wise
bf16 tolerance of the FP64 oracle (oracle/unet.py).  The shapes cover the
three kernels behind dh_conv3x3_forward: the shallow-layer halo kernel (TMA
and cp.async staging, including a grid in which every CTA has one tile), the
general kernel with cp.async staging, and the TMA-fed general kernel, at
small ragged sizes and at the sizes of the 1080p network's layers.  A race
between the staging of a tile and the MMAs that read it shows up as a run
that differs from the others."""
import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RUNS = 20


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_08793_gb300 import _native

    _native.lib()
    return _native


def rnd(seed, *shape, lo=-1.0, hi=1.0):
    return scenes.uniform(seed, 93, int(np.prod(shape)), lo, hi).reshape(shape)


def oracle_rows(x, w, b, relu, rows):
    """The oracle's output rows [r0, r1) of every image, from input rows
    r0 - 1 .. r1 (zero padding outside the image)."""
    from oracle import unet as U

    r0, r1 = rows
    H = x.shape[1]
    a, z = max(r0 - 1, 0), min(r1 + 1, H)
    y = U.conv3x3(x[:, a:z], w, b)[:, r0 - a:r0 - a + (r1 - r0)]
    return np.maximum(y, 0) if relu else y


@pytest.mark.parametrize("n,H,W,C,ldx,Cout,relu,bands", [
    # shallow-layer kernel, cp.async staging: one tile per CTA (the grid is the tile count)
    (1, 5, 129, 64, 64, 64, 1, None),
    (1, 3, 200, 96, 96, 32, 1, None),
    # shallow-layer kernel at 1080p: cp.async (96 -> 32) and TMA (32 -> 32) staging
    (1, 1080, 1920, 96, 96, 32, 1, ((0, 24), (530, 560), (1060, 1080))),
    (1, 1080, 1920, 32, 32, 32, 1, ((0, 24), (530, 560), (1060, 1080))),
    # general kernel, cp.async staging (rows too short for the TMA-fed one)
    (1, 12, 8, 96, 96, 96, 1, None),
    (1, 67, 50, 128, 128, 256, 0, None),
    # TMA-fed general kernel: a ragged row and the 1080p network's deepest layer
    (1, 2, 230, 192, 192, 64, 1, None),
    (1, 135, 240, 256, 256, 256, 1, ((0, 8), (60, 70), (127, 135))),
])
def test_conv_repeatable_and_exact(N, n, H, W, C, ldx, Cout, relu, bands):
    x = rnd(11 + C, n, H, W, ldx)
    w = rnd(12 + C, Cout, 3, 3, C, lo=-0.3, hi=0.3)
    b = rnd(13 + Cout, Cout)
    xb = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16)
    wb = torch.from_numpy(w.astype(np.float32)).to(torch.bfloat16)
    xd, wd = xb.cuda(), wb.cuda()
    bd = torch.from_numpy(b.astype(np.float32)).cuda()
    ys = []
    for _ in range(RUNS):
        y = torch.full((n, H, W, Cout), float("nan"), dtype=torch.bfloat16, device="cuda")
        assert N.dh_conv3x3_forward(xd, ldx, C, n, H, W, wd, bd, Cout, relu, y, Cout) == 0
        ys.append(y)
    torch.cuda.synchronize()
    first = ys[0]
    for k, y in enumerate(ys[1:], 1):
        assert torch.equal(y.view(torch.int16), first.view(torch.int16)), f"run {k} differs from run 0"
    got = first.float().cpu().numpy()
    xo = xb.float().numpy()[..., :C].astype(np.float64)
    wo = wb.float().numpy().astype(np.float64)
    for rows in bands or ((0, H),):
        want = oracle_rows(xo, wo, b, relu, rows)
        g = got[:, rows[0]:rows[1]]
        tol = 2.0 ** -8 * np.abs(want) + 1e-3 * np.abs(want).max()
        bad = np.abs(g - want) > tol
        assert not bad.any(), (rows, int(bad.sum()), np.argwhere(bad)[:5])
