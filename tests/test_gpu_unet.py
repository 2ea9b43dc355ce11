"""Warm-start network kernels (bf16 tensor-core convolutions, whole-network
forward / backward, Adam) against the FP64 oracle in oracle/unet.py, through
the C ABI."""
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


def rnd(seed, *shape, lo=-1.0, hi=1.0):
    return scenes.uniform(seed, 93, int(np.prod(shape)), lo, hi).reshape(shape)


def bf(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)


def host(t):
    torch.cuda.synchronize()
    return t.float().cpu().numpy()


@pytest.mark.parametrize("n,H,W,C,ldx,Cout,relu", [(2, 7, 13, 16, 16, 32, 1), (1, 9, 20, 32, 48, 64, 0),
                                                   (1, 12, 8, 96, 96, 96, 1), (3, 5, 5, 64, 64, 128, 0),
                                                   # the shallow-layer (halo) kernel: every channel pair,
                                                   # row segments of 128 pixels with ragged ends
                                                   (1, 3, 200, 96, 96, 32, 1), (2, 4, 130, 32, 32, 32, 0),
                                                   (1, 5, 129, 64, 64, 64, 1), (1, 6, 140, 64, 80, 32, 0),
                                                   (1, 4, 257, 32, 32, 96, 1), (1, 2, 128, 16, 16, 32, 1),
                                                   (2, 3, 64, 32, 40, 64, 0),
                                                   # the TMA-fed general kernel (rows of >= 96 pixels):
                                                   # ragged segments, C < 32 and C % 32 != 0, pitch != C,
                                                   # every N tile
                                                   (1, 3, 128, 64, 64, 128, 1), (2, 2, 100, 48, 48, 64, 0),
                                                   (1, 2, 230, 192, 192, 64, 1), (1, 2, 256, 384, 384, 128, 1),
                                                   (2, 3, 128, 16, 16, 64, 1), (1, 2, 120, 32, 40, 256, 0),
                                                   (1, 3, 97, 96, 96, 192, 1), (1, 2, 128, 128, 128, 96, 0),
                                                   (1, 2, 112, 64, 64, 48, 1)])
def test_conv_forward(N, n, H, W, C, ldx, Cout, relu):
    from oracle import unet as U

    x = rnd(1 + C, n, H, W, ldx)
    w = rnd(2 + C, Cout, 3, 3, C, lo=-0.3, hi=0.3)
    b = rnd(3 + C, Cout)
    xb, wb = bf(x), bf(w)
    want = U.conv3x3(xb.float().numpy()[..., :C].astype(np.float64), wb.float().numpy().astype(np.float64), b)
    if relu:
        want = np.maximum(want, 0)
    y = torch.zeros((n, H, W, Cout + 8), dtype=torch.bfloat16, device="cuda")
    rc = N.dh_conv3x3_forward(xb.cuda(), ldx, C, n, H, W, wb.cuda(), torch.from_numpy(b.astype(np.float32)).cuda(),
                              Cout, relu, y, Cout + 8)
    assert rc == 0
    got = host(y)[..., :Cout]
    assert np.all(np.abs(got - want) <= 2.0 ** -8 * np.abs(want) + 1e-3 * np.abs(want).max())
    assert np.all(host(y)[..., Cout:] == 0)


@pytest.mark.parametrize("n,H,W,C,ldx,Cout,lddy", [
    (2, 7, 13, 16, 16, 32, 32), (1, 30, 41, 64, 64, 32, 32), (2, 16, 16, 96, 96, 64, 64),
    # the tensor-core kernel (C >= 96 or Cout >= 128) and the mma.sync one:
    # channel pitches wider than C (skip concatenations), rows that end inside a
    # 32-pixel segment, two output-channel tiles, two input-channel tiles,
    # several pixel splits
    (1, 9, 40, 48, 96, 16, 48), (1, 34, 70, 128, 128, 128, 128), (1, 9, 40, 384, 384, 256, 256),
    (2, 64, 96, 32, 96, 32, 32), (1, 5, 3, 192, 192, 64, 64), (1, 9, 40, 96, 144, 32, 48)])
def test_conv_weight_gradient(N, n, H, W, C, ldx, Cout, lddy):
    from oracle import unet as U

    x = bf(rnd(5 + C, n, H, W, ldx))
    dy = bf(rnd(6 + C, n, H, W, lddy))
    _, gw, gb = U.conv3x3_backward(x.float().numpy()[..., :C].astype(np.float64), np.zeros((Cout, 3, 3, C)),
                                   dy.float().numpy()[..., :Cout].astype(np.float64))
    dw = torch.zeros(Cout * 9 * C, device="cuda")
    db = torch.zeros(Cout, device="cuda")
    scratch = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
    rc = N.dh_conv3x3_backward_weights(x.cuda(), ldx, C, dy.cuda(), lddy, Cout, n, H, W, dw, db, scratch,
                                       scratch.numel())
    assert rc == 0
    assert np.max(np.abs(host(dw).reshape(gw.shape) - gw)) <= 1e-4 * np.abs(gw).max()
    assert np.max(np.abs(host(db) - gb)) <= 1e-3 * max(1.0, np.abs(gb).max())


def _net_inputs(n, H, W, seed):
    I = np.stack([scenes.hazy_scene(seed + k, H, W)["I"] for k in range(n)])
    t = rnd(seed, n, H, W, lo=0.1, hi=1.0)
    A = rnd(seed + 1, n, 3, lo=0.8, hi=1.0)
    tgt = rnd(seed + 2, n, 3, H, W, lo=0.0, hi=1.0)
    Phi = rnd(seed + 3, n, 3, H, W, lo=0.0, hi=1.5)
    return (I.astype(np.float32), t.astype(np.float32), A.astype(np.float32), tgt.astype(np.float32),
            Phi.astype(np.float32))


def test_network_forward_backward_against_oracle(N):
    """The whole network, element by element, against the oracle network
    with bf16 storage (oracle/unet.py, q = bf16: the same rounding points as
    the library, FP64 arithmetic in between).  What remains is the order of
    the float32 sums, which can move a stored value to the neighbouring bf16
    value (one ulp, at most 2^-7 relative) now and then; so each output or
    gradient element is held to a few bf16 ulps of the sum of the absolute
    values of the terms it adds up (its scale).  In the backward pass such
    moves add up along the chain of rounded gradient maps between the loss
    and a layer (the head's input gradient, each data gradient, each
    upsampling adjoint and skip + pooled sum): a layer whose gradient map went
    through s rounding stages is held to 2 + s ulps of its scale.  A ReLU
    decision within such rounding of zero could go either way and pass or stop
    a whole gradient value, so the test's network keeps every pre-activation
    at least 2^-4 of its scale away from zero (checked on the oracle side):
    half of each layer's channels have bias +0.5, half -0.5, and the weights
    are uniform in +-1 / (9 C_in), so both ReLU paths are exercised."""
    from oracle import unet as U

    base, n, H, W = 16, 2, 16, 24
    I, t, A, tgt, Phi = _net_inputs(n, H, W, 40)
    npar = N.dh_unet_param_count(base)
    assert npar == U.param_count(base)
    host_params = np.zeros(npar)
    o = 0
    for k, (cin, cout) in enumerate(U.convs(base)):
        nw = cout * 9 * cin
        host_params[o:o + nw] = rnd(100 + k, nw, lo=-1.0, hi=1.0) / (9 * cin)
        host_params[o + nw:o + nw + cout] = np.where(np.arange(cout) % 2 == 0, 0.5, -0.5)
        o += nw + cout
    # a head of ordinary size, so that the network's part of y is not negligible next to Phi
    host_params[o:] = rnd(41, 3 * base + 3, lo=-0.3, hi=0.3)
    params = torch.from_numpy(host_params.astype(np.float32)).cuda()
    ws = torch.empty(N.dh_unet_workspace_bytes(base, n, H, W, 1), dtype=torch.uint8, device="cuda")
    d = {k: torch.from_numpy(v).cuda() for k, v in dict(I=I, t=t, A=A, tgt=tgt, Phi=Phi).items()}
    y = torch.empty((n, 3, H, W), device="cuda")
    assert N.dh_unet_forward(params, base, d["I"], d["t"], d["A"], d["Phi"], n, H, W, y, ws, ws.numel()) == 0
    P = host(params).astype(np.float64)
    yo, c = U.forward(P, base, I, t, A, Phi, q=U.bf16)
    assert min(c["margin"]) >= 2.0 ** -4, c["margin"]  # no ReLU decision near zero
    ulp = 2.0 ** -7
    dy = np.abs(host(y) - yo)
    bad = dy > 2 * ulp * c["y_scale"] + 1e-6
    assert not bad.any(), (int(bad.sum()), float((dy / (c["y_scale"] + 1e-30)).max()))
    grads = torch.empty(npar, device="cuda")
    loss = torch.empty(1, device="cuda")
    assert N.dh_unet_backward(params, base, d["I"], d["t"], d["A"], d["Phi"], d["tgt"], n, H, W, grads, loss, ws,
                              ws.numel()) == 0
    lo, go, so = U.loss_and_grads(P, base, I, t, A, Phi, tgt, q=U.bf16, scales=True)
    assert abs(host(loss)[0] - lo) <= 1e-3 * lo
    g = host(grads).astype(np.float64)
    # rounding stages of the gradient map each convolution's weight gradient sums
    # (counted along oracle/unet.py loss_and_grads, from the loss down)
    stages = {13: 1, 12: 2, 11: 4, 10: 5, 9: 7, 8: 8, 7: 10, 6: 11, 5: 13, 4: 14, 3: 16, 2: 17, 1: 19, 0: 20}
    o = 0
    for k, (cin, cout) in enumerate(U.convs(base)):
        for size in (cout * 9 * cin, cout):
            a, b, sc = g[o:o + size], go[o:o + size], so[o:o + size]
            o += size
            err = np.abs(a - b)
            bad = err > (2 + stages[k]) * ulp * sc + 1e-6 * max(sc.max(), 1e-30)
            assert not bad.any(), (k, size, int(bad.sum()), float((err / (sc + 1e-30)).max()))
    a, b, sc = g[o:], go[o:], so[o:]  # the head: no rounded gradient map before it
    assert np.all(np.abs(a - b) <= 2 * ulp * sc + 1e-6 * sc.max())


def test_adam_training_reduces_loss(N):
    base, n, H, W = 16, 2, 32, 32
    I, t, A, _, Phi = _net_inputs(n, H, W, 60)
    tgt = (Phi + 0.5 * I - 0.3 * t[:, None]).astype(np.float32)  # a target the inputs determine
    d = {k: torch.from_numpy(v).cuda() for k, v in dict(I=I, t=t, A=A, tgt=tgt, Phi=Phi).items()}
    npar = N.dh_unet_param_count(base)
    params = torch.empty(npar, device="cuda")
    N.dh_unet_init(params, base, 3)
    grads, m, v = torch.empty(npar, device="cuda"), torch.zeros(npar, device="cuda"), torch.zeros(npar, device="cuda")
    loss = torch.empty(1, device="cuda")
    ws = torch.empty(N.dh_unet_workspace_bytes(base, n, H, W, 1), dtype=torch.uint8, device="cuda")
    losses = []
    for step in range(1, 61):
        assert N.dh_unet_backward(params, base, d["I"], d["t"], d["A"], d["Phi"], d["tgt"], n, H, W, grads, loss,
                                  ws, ws.numel()) == 0
        losses.append(float(host(loss)[0]))
        assert N.dh_unet_adam(params, grads, m, v, npar, 1e-3, 0.9, 0.999, 1e-8, step) == 0
    assert np.isfinite(losses).all() and losses[-1] < 0.2 * losses[0], losses[::10]
