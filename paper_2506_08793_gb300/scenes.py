"""Seeded synthetic hazy scenes (input data only).

This module is the single source of inputs for the CUDA path, the FP64 CPU
oracle, the tests and the benchmark.  It synthesises a clear scene J, a depth
map d, a scattering coefficient beta and an atmospheric light A, and applies the
forward scattering model of Sec. II-A, I = J*t + A*(1 - t) with
t = exp(-beta*d), to produce the hazy input I.  It holds none of the dehazing
method's own arithmetic (dark channel, atmospheric-light selection,
transmission, lambda(t), Phi, the diffusion/Gaussian operator or the
fixed-point iteration).

Randomness is counter based: every value is a pure function of
(seed, stream, counter) through the SplitMix64 output mix (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so a
scene is reproducible bit for bit on any host regardless of numpy's own RNG.

Recipe (stand-in for the paper's unnamed real-world hazy photographs):
  * J: an affine colour ramp background plus 8..40 convex polygons (regular
    polygons under a random rotation and anisotropic scale), each filled with
    its own affine colour ramp in [0, 0.9]^3 (later polygons paint over
    earlier ones), plus Gaussian texture noise of sigma in [0.01, 0.02];
    clipped to [0, 1].
  * d: a coarse random grid (5x5 .. 9x9) upsampled with Keys' cubic
    convolution (a = -0.5) and rescaled to [0.1, 2.0].
  * beta ~ U[0.5, 1.5]; t = exp(-beta*d); A ~ U[0.8, 1.0]^3.
  * I = J*t + A*(1 - t), computed in float64, stored as float32 planar 3xHxW.
"""
from __future__ import annotations

import numpy as np

_M64 = (1 << 64) - 1
_GOLD = 0x9E3779B97F4A7C15


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> int:
    k = ((seed & _M64) * _GOLD + (stream & _M64) * 0xD1B54A32D192ED03 + 0x632BE59BD9B4E019) & _M64
    return int(_mix64(np.array([k], dtype=np.uint64))[0])


def uniform(seed: int, stream: int, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """n float64 values in [lo, hi) for (seed, stream), counters 0..n-1."""
    key = np.uint64(_key(seed, stream))
    with np.errstate(over="ignore"):
        ctr = np.arange(n, dtype=np.uint64) * np.uint64(_GOLD) + key
    bits = _mix64(ctr) >> np.uint64(11)
    return lo + (hi - lo) * (bits.astype(np.float64) * (1.0 / 9007199254740992.0))


def normal(seed: int, stream: int, n: int) -> np.ndarray:
    """n standard normal float64 values (Box-Muller on two uniform streams)."""
    u1 = uniform(seed, stream, n)
    u2 = uniform(seed, stream + 0x5151, n)
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


def _keys_cubic_matrix(n_out: int, n_in: int) -> np.ndarray:
    """Interpolation matrix (n_out x n_in) of Keys' cubic convolution, a=-0.5,
    sampling n_in grid nodes spread over [0, n_out-1] with edge clamping."""
    a = -0.5
    pos = np.linspace(0.0, n_in - 1.0, n_out) if n_out > 1 else np.zeros(1)
    base = np.floor(pos).astype(np.int64)
    M = np.zeros((n_out, n_in))
    for off in (-1, 0, 1, 2):
        idx = base + off
        s = np.abs(pos - idx)
        w = np.where(
            s <= 1.0,
            (a + 2) * s**3 - (a + 3) * s**2 + 1,
            np.where(s < 2.0, a * s**3 - 5 * a * s**2 + 8 * a * s - 4 * a, 0.0),
        )
        np.add.at(M, (np.arange(n_out), np.clip(idx, 0, n_in - 1)), w)
    return M


def _smooth_field(seed: int, stream: int, H: int, W: int, gh: int, gw: int) -> np.ndarray:
    g = uniform(seed, stream, gh * gw).reshape(gh, gw)
    return _keys_cubic_matrix(H, gh) @ g @ _keys_cubic_matrix(W, gw).T


def _ramp(seed, stream, H, W, y0, x0, y1, x1, cx, cy, scale):
    """Affine colour ramp (3, h, w) over the window [y0:y1, x0:x1]."""
    p = uniform(seed, stream, 9)
    base = 0.05 + 0.8 * p[0:3]
    gx = (p[3:6] - 0.5) * 0.6
    gy = (p[6:9] - 0.5) * 0.6
    ys = (np.arange(y0, y1)[:, None] - cy) / scale
    xs = (np.arange(x0, x1)[None, :] - cx) / scale
    c = base[:, None, None] + gx[:, None, None] * xs[None] + gy[:, None, None] * ys[None]
    return np.clip(c, 0.0, 0.9)


def clear_scene(seed: int, H: int, W: int) -> np.ndarray:
    """Clear image J, float64 (3, H, W) in [0, 1]."""
    J = _ramp(seed, 1, H, W, 0, 0, H, W, W / 2.0, H / 2.0, max(H, W))
    n_poly = 8 + int(uniform(seed, 2, 1)[0] * 33)
    m = float(min(H, W))
    for p in range(n_poly):
        q = uniform(seed, 100 + p, 8)
        cx, cy = q[0] * W, q[1] * H
        r = (0.05 + 0.25 * q[2]) * m + 1.0
        k = 3 + int(q[3] * 6)
        rot = 2 * np.pi * q[4]
        sx, sy = 0.6 + 0.8 * q[5], 0.6 + 0.8 * q[6]
        ang = rot + 2 * np.pi * np.arange(k) / k
        vx = cx + r * sx * np.cos(ang) * np.cos(rot) - r * sy * np.sin(ang) * np.sin(rot)
        vy = cy + r * sx * np.cos(ang) * np.sin(rot) + r * sy * np.sin(ang) * np.cos(rot)
        x0, x1 = max(0, int(np.floor(vx.min()))), min(W, int(np.ceil(vx.max())) + 1)
        y0, y1 = max(0, int(np.floor(vy.min()))), min(H, int(np.ceil(vy.max())) + 1)
        if x0 >= x1 or y0 >= y1:
            continue
        X = np.arange(x0, x1, dtype=np.float64)[None, :] + 0.5
        Y = np.arange(y0, y1, dtype=np.float64)[:, None] + 0.5
        inside = np.ones((y1 - y0, x1 - x0), dtype=bool)
        # A linear map of a counter-clockwise regular polygon stays convex;
        # the orientation is that of the map's determinant (sx*sy > 0).
        for e in range(k):
            ax, ay = vx[e], vy[e]
            bx, by = vx[(e + 1) % k], vy[(e + 1) % k]
            inside &= (bx - ax) * (Y - ay) - (by - ay) * (X - ax) >= 0.0
        if not inside.any():
            continue
        col = _ramp(seed, 200 + p, H, W, y0, x0, y1, x1, cx, cy, r)
        J[:, y0:y1, x0:x1] = np.where(inside[None], col, J[:, y0:y1, x0:x1])
    sig = 0.01 + 0.01 * uniform(seed, 3, 1)[0]
    J = J + sig * normal(seed, 4, 3 * H * W).reshape(3, H, W)
    return np.clip(J, 0.0, 1.0)


def depth_map(seed: int, H: int, W: int) -> np.ndarray:
    q = uniform(seed, 5, 2)
    gh, gw = 5 + int(q[0] * 5), 5 + int(q[1] * 5)
    d = _smooth_field(seed, 6, H, W, gh, gw)
    lo, hi = d.min(), d.max()
    d = (d - lo) / (hi - lo) if hi > lo else np.zeros_like(d)
    return 0.1 + 1.9 * d


def hazy_scene(seed: int, H: int, W: int) -> dict:
    """Hazy scene following the module recipe.

    Returns a dict with I (float32, 3xHxW, C-contiguous), J (float64),
    t_true (float64 HxW), A_true (float64 [3]), d, beta.
    """
    if H < 1 or W < 1:
        raise ValueError("H and W must be positive")
    J = clear_scene(seed, H, W)
    d = depth_map(seed, H, W)
    q = uniform(seed, 7, 4)
    beta = 0.5 + q[0]
    A = 0.8 + 0.2 * q[1:4]
    t = np.exp(-beta * d)
    I = J * t[None] + A[:, None, None] * (1.0 - t[None])
    return dict(I=np.ascontiguousarray(I.astype(np.float32)), J=J, t_true=t, A_true=A, d=d, beta=beta)


def prior_scene(seed: int, H: int, W: int, sky_rows: int) -> dict:
    """A scene built so that the dark channel prior holds exactly.

    * J <= 0.75 < A componentwise, and one colour channel of J is 0 at every
      pixel of the lattice (y % 8 == 0, x % 8 == 0), so every 15x15 window,
      clipped at the border, contains a pixel with a zero channel.
    * Rows [0, sky_rows) are sky: t = 0 there, so I = A exactly.
    * Below the sky the depth is piecewise constant on vertical bands of
      width 32, so t is constant inside each band.
    Returns the same keys as hazy_scene plus 'band_w'.
    """
    J = 0.75 * clear_scene(seed, H, W)
    zc = (np.floor(uniform(seed, 8, H * W) * 3).astype(np.int64)).reshape(H, W)
    yy, xx = np.mgrid[0:H, 0:W]
    lattice = (yy % 8 == 0) & (xx % 8 == 0)
    for c in range(3):
        J[c][lattice & (zc == c)] = 0.0
    band_w = 32
    nb = (W + band_w - 1) // band_w
    t_band = 0.15 + 0.8 * uniform(seed, 9, nb)
    t = np.repeat(t_band, band_w)[:W][None, :].repeat(H, axis=0)
    t[:sky_rows, :] = 0.0
    q = uniform(seed, 7, 4)
    A = 0.8 + 0.2 * q[1:4]
    I = J * t[None] + A[:, None, None] * (1.0 - t[None])
    return dict(I=np.ascontiguousarray(I.astype(np.float32)), J=J, t_true=t, A_true=A,
                d=None, beta=None, band_w=band_w)


def batch_sizes(seed: int, n: int, sizes=((480, 640), (720, 1280), (1080, 1920), (1200, 1600))):
    """n (H, W) pairs drawn uniformly from `sizes`."""
    u = uniform(seed, 10, n)
    return [sizes[min(len(sizes) - 1, int(v * len(sizes)))] for v in u]
