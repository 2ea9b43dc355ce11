"""Pins of the network oracle (oracle/unet.py): the convolution, pooling and
upsampling against brute-force loops, the hand-written backward against
central differences and as the transpose of the forward."""
import numpy as np

from oracle import unet as U
from paper_2506_08793_gb300 import scenes


def rnd(seed, *shape, lo=-1.0, hi=1.0):
    return scenes.uniform(seed, 91, int(np.prod(shape)), lo, hi).reshape(shape)


def test_conv3x3_brute_force():
    x = rnd(1, 2, 5, 6, 3)
    w = rnd(2, 4, 3, 3, 3)
    b = rnd(3, 4)
    y = U.conv3x3(x, w, b)
    for n in range(2):
        for i in range(5):
            for j in range(6):
                for co in range(4):
                    s = b[co]
                    for dy in range(3):
                        for dx in range(3):
                            ii, jj = i + dy - 1, j + dx - 1
                            if 0 <= ii < 5 and 0 <= jj < 6:
                                s += np.dot(x[n, ii, jj], w[co, dy, dx])
                    assert abs(y[n, i, j, co] - s) < 1e-12


def test_pool_and_upsample_brute_force_and_adjoints():
    """2x2 average pooling and nearest upsampling against loops, and each
    backward as the transpose of its forward (<f(x), g> = <x, f'(g)>)."""
    x = rnd(4, 2, 6, 8, 3)
    p = U.pool(x)
    for n in range(2):
        for i in range(3):
            for j in range(4):
                want = (x[n, 2 * i, 2 * j] + x[n, 2 * i + 1, 2 * j] + x[n, 2 * i, 2 * j + 1]
                        + x[n, 2 * i + 1, 2 * j + 1]) / 4.0
                assert np.allclose(p[n, i, j], want, rtol=0, atol=1e-15)
    z = rnd(5, 2, 3, 4, 3)
    u = U.up(z)
    for i in range(6):
        for j in range(8):
            assert np.array_equal(u[:, i, j], z[:, i // 2, j // 2])
    gp = rnd(6, *p.shape)
    assert abs(np.sum(p * gp) - np.sum(x * U.pool_backward(gp, x.shape))) < 1e-12
    gu = rnd(7, *u.shape)
    assert abs(np.sum(u * gu) - np.sum(z * U.up_backward(gu))) < 1e-12


def test_conv_backward_finite_differences():
    x = rnd(4, 1, 4, 5, 3)
    w = rnd(5, 2, 3, 3, 3)
    b = rnd(6, 2)
    g = rnd(7, 1, 4, 5, 2)
    gx, gw, gb = U.conv3x3_backward(x, w, g)
    f = lambda x_, w_, b_: float(np.sum(g * U.conv3x3(x_, w_, b_)))
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 3, 4, 2), (0, 1, 2, 1)]:
        e = np.zeros_like(x); e[idx] = h
        assert abs((f(x + e, w, b) - f(x - e, w, b)) / (2 * h) - gx[idx]) < 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 1, 2), (1, 1, 1, 1)]:
        e = np.zeros_like(w); e[idx] = h
        assert abs((f(x, w + e, b) - f(x, w - e, b)) / (2 * h) - gw[idx]) < 1e-6
    assert np.allclose(gb, g.sum(axis=(0, 1, 2)))


def test_network_gradient_finite_differences():
    """The whole network's loss gradient (base 8 keeps it small) against
    central differences on a sample of parameters of every layer."""
    b, N, H, W = 8, 1, 8, 8
    rng = np.random.default_rng(0)
    params = rng.normal(0, 0.3, U.param_count(b))
    I = rng.uniform(0, 1, (N, 3, H, W))
    t = rng.uniform(0.1, 1, (N, H, W))
    A = rng.uniform(0.8, 1, (N, 3))
    tgt = rng.normal(0, 1, (N, 3, H, W))
    Phi = rng.normal(0, 1, (N, 3, H, W))
    loss, g = U.loss_and_grads(params, b, I, t, A, Phi, tgt)
    h = 1e-6
    idx = np.unique(np.linspace(0, params.size - 1, 60).astype(int))
    for i in idx:
        e = np.zeros_like(params); e[i] = h
        lp, _ = U.loss_and_grads(params + e, b, I, t, A, Phi, tgt)
        lm, _ = U.loss_and_grads(params - e, b, I, t, A, Phi, tgt)
        num = (lp - lm) / (2 * h)
        assert abs(num - g[i]) <= 1e-4 * max(1.0, abs(num)), (i, num, g[i])


def test_bf16_rounding_matches_torch():
    """The oracle's bfloat16 rounding (float32 first, nearest even) against
    torch's float32 -> bfloat16 conversion, exact ties and signs included."""
    import torch

    rng = np.random.default_rng(3)
    f = (rng.normal(0, 1, 4000) * np.exp2(rng.integers(-30, 30, 4000))).astype(np.float32)
    ties = f.view(np.uint32) & np.uint32(0xFFFF0000) | np.uint32(0x8000)  # halfway between two bf16 values
    vals = np.concatenate([f, ties.view(np.float32), np.float32([0.0, -0.0, 1.0, -3.5, 65504.0])])
    want = torch.from_numpy(vals).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(U.bf16(vals.astype(np.float64)), want)


def test_gradient_scales_bound_the_gradients():
    """The per-element scale (sum of |terms|) bounds |gradient| (triangle
    inequality), in the exact and in the bf16 network."""
    b, N, H, W = 8, 1, 8, 8
    rng = np.random.default_rng(1)
    params = rng.normal(0, 0.3, U.param_count(b))
    I = rng.uniform(0, 1, (N, 3, H, W))
    t = rng.uniform(0.1, 1, (N, H, W))
    A = rng.uniform(0.8, 1, (N, 3))
    tgt = rng.normal(0, 1, (N, 3, H, W))
    Phi = rng.normal(0, 1, (N, 3, H, W))
    for q in (None, U.bf16):
        _, g, s = U.loss_and_grads(params, b, I, t, A, Phi, tgt, q=q, scales=True)
        assert g.shape == s.shape and np.all(np.abs(g) <= s * (1 + 1e-12) + 1e-300)
    y, c = U.forward(params, b, I, t, A, Phi, q=U.bf16)
    assert np.all(np.abs(y - Phi - (c["d1"] @ U.unpack(params, b)[2].T + U.unpack(params, b)[3]).transpose(0, 3, 1, 2))
                  <= 1e-12 * (1 + c["y_scale"]))


def test_relu_margin():
    """forward() reports, per convolution, the smallest |pre-activation| over
    the sum of |terms| of the pre-activation: 1 for a single positive term,
    and 0 when a unit sits exactly at zero."""
    b = 8
    params = np.zeros(U.param_count(b))
    N, H, W = 1, 8, 8
    I = np.full((N, 3, H, W), 0.5)
    t = np.full((N, H, W), 0.5)
    A = np.full((N, 3), 0.9)
    Phi = np.full((N, 3, H, W), 0.2)
    _, c = U.forward(params, b, I, t, A, Phi)
    assert all(m == 0.0 for m in c["margin"])  # zero weights and biases: every unit at zero
    o = 0
    for cin, cout in U.convs(b):
        o += cout * 9 * cin
        params[o:o + cout] = 1.0  # biases only: every pre-activation is its bias
        o += cout
    _, c = U.forward(params, b, I, t, A, Phi)
    assert all(m == 1.0 for m in c["margin"])
