"""FP64 CPU oracle of the warm-start U-Net (TEST INFRASTRUCTURE ONLY).

The same network as the CUDA library's: 14 3x3 convolutions (zero padding,
bias, ReLU) in a 4-level U-Net with 2x2 average pooling, nearest 2x
upsampling and skip concatenation (upsampled channels first), then a 1x1
head to 3 channels, with an MSE loss.  Plain numpy in float64 on NHWC
arrays; a convolution is an explicit sum over the 9 taps of matrix products
(numpy's matmul is the only library step).  The backward pass is written out
by hand; tests/test_oracle_unet.py pins it to central finite differences and
the convolution to a brute-force loop.

Parameters come as one flat float vector in the library's layout: for each
convolution k, weights [cout][3][3][cin] then bias [cout]; then the head
weights [3][base] and bias [3].
"""
from __future__ import annotations

import numpy as np


def convs(b: int):
    """(cin, cout) of the 14 convolutions, in order."""
    return [(16, b), (b, b), (b, 2 * b), (2 * b, 2 * b), (2 * b, 4 * b), (4 * b, 4 * b), (4 * b, 8 * b),
            (8 * b, 8 * b), (12 * b, 4 * b), (4 * b, 4 * b), (6 * b, 2 * b), (2 * b, 2 * b), (3 * b, b), (b, b)]


def unpack(params: np.ndarray, b: int):
    ws, bs, o = [], [], 0
    for cin, cout in convs(b):
        n = cout * 9 * cin
        ws.append(params[o:o + n].reshape(cout, 3, 3, cin))
        o += n
        bs.append(params[o:o + cout])
        o += cout
    hw = params[o:o + 3 * b].reshape(3, b)
    o += 3 * b
    hb = params[o:o + 3]
    o += 3
    assert o == params.size
    return ws, bs, hw, hb


def param_count(b: int) -> int:
    return sum(cout * 9 * cin + cout for cin, cout in convs(b)) + 3 * b + 3


def pack_input(I, t, A, Phi):
    """(N,3,H,W), (N,H,W), (N,3), (N,3,H,W) -> NHWC with channels I, t, A,
    Phi, zeros (16)."""
    N, _, H, W = I.shape
    x = np.zeros((N, H, W, 16))
    x[..., 0:3] = np.moveaxis(I, 1, -1)
    x[..., 3] = t
    x[..., 4:7] = A[:, None, None, :]
    x[..., 7:10] = np.moveaxis(Phi, 1, -1)
    return x


def conv3x3(x, w, b):
    """y[n,i,j,co] = b[co] + sum_{dy,dx,ci} x[n,i+dy-1,j+dx-1,ci] w[co,dy,dx,ci]."""
    N, H, W, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((N, H, W, w.shape[0])) + b
    for dy in range(3):
        for dx in range(3):
            y += xp[:, dy:dy + H, dx:dx + W, :] @ w[:, dy, dx, :].T
    return y


def conv3x3_backward(x, w, g):
    """Gradients of sum(g * conv3x3(x, w, b)) w.r.t. x, w, b."""
    N, H, W, C = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    gx = np.zeros((N, H + 2, W + 2, C))
    gw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            gw[:, dy, dx, :] = np.einsum("nhwo,nhwc->oc", g, xp[:, dy:dy + H, dx:dx + W, :])
            gx[:, dy:dy + H, dx:dx + W, :] += g @ w[:, dy, dx, :]
    return gx[:, 1:H + 1, 1:W + 1, :], gw, g.sum(axis=(0, 1, 2))


def relu(x):
    return np.maximum(x, 0.0)


def bf16(x):
    """x rounded to float32, then to bfloat16, both to nearest even, returned
    as float64: the storage format of the network's weights and activations
    (BF16 weights and activations with FP32 accumulation)."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def pool(x):
    N, H, W, C = x.shape
    return x.reshape(N, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_backward(g, shape):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_backward(g):
    N, H, W, C = g.shape
    return g.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def forward(params, b, I, t, A, Phi, q=None):
    """Returns (y (N,3,H,W) = lambda*u* prediction = Phi + head, cache).

    q: None for the exact network, or a rounding function (bf16) applied
    where the network stores a value: the packed input, the convolution
    weights, every convolution output (after bias and ReLU) and every pooled
    map; the head accumulates without rounding."""
    r = q or (lambda v: v)
    ws, bs, hw, hb = unpack(np.asarray(params, np.float64), b)
    ws = [r(w) for w in ws]
    c = {"ws": ws}
    Phi = np.asarray(Phi, np.float64)
    x0 = r(pack_input(np.asarray(I, np.float64), np.asarray(t, np.float64), np.asarray(A, np.float64), Phi))
    c["x0"] = x0

    c["margin"] = [None] * 14

    def conv(x, k):
        pre = conv3x3(x, ws[k], bs[k])
        # how far the ReLU decisions are from zero, relative to the sum of the
        # absolute values of each pre-activation's terms (smallest over units)
        sc = conv3x3(np.abs(x), np.abs(ws[k]), np.abs(bs[k]))
        c["margin"][k] = float(np.min(np.where(sc > 0, np.abs(pre) / np.where(sc > 0, sc, 1.0), 0.0)))
        return r(relu(pre))

    a1 = conv(x0, 0); c["a1"] = a1
    e1 = conv(a1, 1); c["e1"] = e1
    p1 = r(pool(e1)); c["p1"] = p1
    a2 = conv(p1, 2); c["a2"] = a2
    e2 = conv(a2, 3); c["e2"] = e2
    p2 = r(pool(e2)); c["p2"] = p2
    a3 = conv(p2, 4); c["a3"] = a3
    e3 = conv(a3, 5); c["e3"] = e3
    p3 = r(pool(e3)); c["p3"] = p3
    a4 = conv(p3, 6); c["a4"] = a4
    e4 = conv(a4, 7); c["e4"] = e4
    cat3 = np.concatenate([up(e4), e3], axis=-1); c["cat3"] = cat3
    d3a = conv(cat3, 8); c["d3a"] = d3a
    d3 = conv(d3a, 9); c["d3"] = d3
    cat2 = np.concatenate([up(d3), e2], axis=-1); c["cat2"] = cat2
    d2a = conv(cat2, 10); c["d2a"] = d2a
    d2 = conv(d2a, 11); c["d2"] = d2
    cat1 = np.concatenate([up(d2), e1], axis=-1); c["cat1"] = cat1
    d1a = conv(cat1, 12); c["d1a"] = d1a
    d1 = conv(d1a, 13); c["d1"] = d1
    y = d1 @ hw.T + hb  # (N,H,W,3)
    c["y_scale"] = np.moveaxis(np.abs(d1) @ np.abs(hw).T + np.abs(hb), -1, 1)  # sum of |terms| of the head
    return np.moveaxis(y, -1, 1) + Phi, c


def loss_and_grads(params, b, I, t, A, Phi, target, q=None, scales=False):
    """MSE loss mean((y - target)^2) and its gradient w.r.t. params.

    q: as in forward(); it also rounds every stored gradient map (the head's
    input gradient, each data gradient, the upsampling adjoints and the
    skip + pooled gradient sums).  scales: also return, in the parameters'
    layout, the sum of the absolute values of the terms each gradient element
    sums (the natural scale of its rounding error)."""
    r = q or (lambda v: v)
    params = np.asarray(params, np.float64)
    _, _, hw, hb = unpack(params, b)
    y, c = forward(params, b, I, t, A, Phi, q)
    ws = c["ws"]
    d = y - np.asarray(target, np.float64)
    loss = float(np.mean(d * d))
    gy = np.moveaxis(2.0 * d / d.size, 1, -1)  # NHWC
    gws = [None] * 14
    gbs = [None] * 14
    sws = [None] * 14
    sbs = [None] * 14
    ghw = np.einsum("nhwo,nhwc->oc", gy, c["d1"])
    ghb = gy.sum(axis=(0, 1, 2))
    shw = np.einsum("nhwo,nhwc->oc", np.abs(gy), np.abs(c["d1"]))
    shb = np.abs(gy).sum(axis=(0, 1, 2))
    g = r(gy @ hw)

    def conv_back(k, x, g_out, y_out):
        g_pre = g_out * (y_out > 0)
        gx, gws[k], gbs[k] = conv3x3_backward(x, ws[k], g_pre)
        if scales:
            _, sws[k], sbs[k] = conv3x3_backward(np.abs(x), ws[k], np.abs(g_pre))
        return r(gx)

    B = b
    g = conv_back(13, c["d1a"], g, c["d1"])
    g = conv_back(12, c["cat1"], g, c["d1a"])
    g_d2, g_e1 = r(up_backward(g[..., :2 * B])), g[..., 2 * B:]
    g = conv_back(11, c["d2a"], g_d2, c["d2"])
    g = conv_back(10, c["cat2"], g, c["d2a"])
    g_d3, g_e2 = r(up_backward(g[..., :4 * B])), g[..., 4 * B:]
    g = conv_back(9, c["d3a"], g_d3, c["d3"])
    g = conv_back(8, c["cat3"], g, c["d3a"])
    g_e4, g_e3 = r(up_backward(g[..., :8 * B])), g[..., 8 * B:]
    g = conv_back(7, c["a4"], g_e4, c["e4"])
    g_p3 = conv_back(6, c["p3"], g, c["a4"])
    g = conv_back(5, c["a3"], r(g_e3 + pool_backward(g_p3, c["e3"].shape)), c["e3"])
    g_p2 = conv_back(4, c["p2"], g, c["a3"])
    g = conv_back(3, c["a2"], r(g_e2 + pool_backward(g_p2, c["e2"].shape)), c["e2"])
    g_p1 = conv_back(2, c["p1"], g, c["a2"])
    g = conv_back(1, c["a1"], r(g_e1 + pool_backward(g_p1, c["e1"].shape)), c["e1"])
    conv_back(0, c["x0"], g, c["a1"])
    parts, sparts = [], []
    for k in range(14):
        parts += [gws[k].ravel(), gbs[k].ravel()]
        if scales:
            sparts += [sws[k].ravel(), sbs[k].ravel()]
    parts += [ghw.ravel(), ghb.ravel()]
    sparts += [shw.ravel(), shb.ravel()]
    if scales:
        return loss, np.concatenate(parts), np.concatenate(sparts)
    return loss, np.concatenate(parts)
