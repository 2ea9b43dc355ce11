"""Pins of the oracle's front-end refinements named by the Sec. IV-E ablation:
the guided filter (He, Sun and Tang's box-filter form) and the multiscale dark
channel.  CPU only; every expected value comes from scipy.ndimage or from a
closed form, none from the CUDA path."""
import numpy as np
import pytest
import scipy.ndimage as ndi

from paper_2506_08793_gb300 import scenes


def rnd(seed, *shape):
    n = int(np.prod(shape))
    return scenes.uniform(seed, 91, n, 0.0, 1.0).reshape(shape)


def box_mean_scipy(v, r):
    """Mean over the (2r+1)^2 window clipped to the image, from scipy's
    zero-padded uniform filter divided by the same filter of ones."""
    k = 2 * r + 1
    return ndi.uniform_filter(v, k, mode="constant") / ndi.uniform_filter(np.ones_like(v), k, mode="constant")


def guided_scipy(g, p, r, eps):
    mg, mp = box_mean_scipy(g, r), box_mean_scipy(p, r)
    a = (box_mean_scipy(g * p, r) - mg * mp) / (box_mean_scipy(g * g, r) - mg * mg + eps)
    b = mp - a * mg
    return box_mean_scipy(a, r) * g + box_mean_scipy(b, r)


@pytest.mark.parametrize("H,W", [(9, 13), (20, 7), (1, 10), (16, 16)])
@pytest.mark.parametrize("r", [1, 2, 4])
@pytest.mark.parametrize("eps", [1e-3, 1e-1])
def test_guided_filter_is_the_box_filter_composition(orc, H, W, r, eps):
    g, p = rnd(H * W + r, H, W), rnd(H * W + r + 1, H, W)
    got = orc.guided_filter(g, p, r, eps)
    want = guided_scipy(g, p, r, eps)
    assert np.max(np.abs(got - want)) <= 1e-11


def test_guided_filter_constant_input_is_kept(orc):
    g = rnd(3, 12, 15)
    p = np.full_like(g, 0.37)
    assert np.max(np.abs(orc.guided_filter(g, p, 3, 1e-3) - 0.37)) <= 1e-13


def test_guided_filter_large_eps_is_double_box_mean(orc):
    """a -> 0, b -> mean(p): q -> mean(mean(p))."""
    g, p = rnd(4, 11, 14), rnd(5, 11, 14)
    got = orc.guided_filter(g, p, 2, 1e12)
    want = box_mean_scipy(box_mean_scipy(p, 2), 2)
    assert np.max(np.abs(got - want)) <= 1e-10


def test_guided_filter_reproduces_a_linear_function_of_the_guide(orc):
    """p = 2 g + 0.3 with eps -> 0: a = 2, b = 0.3 in every window, q = p."""
    g = rnd(6, 10, 12)
    p = 2.0 * g + 0.3
    assert np.max(np.abs(orc.guided_filter(g, p, 2, 1e-14) - p)) <= 1e-8


def test_multiscale_dark_channel_is_mean_of_min_filters(orc):
    I = scenes.hazy_scene(77, 40, 52)["I"]
    A = np.array([0.9, 0.85, 0.95])
    assert orc.scale_patches(15, 3) == [7, 15, 31]
    want = 0.0
    for q in (7, 15, 31):
        n = (I.astype(np.float32) / A.astype(np.float32)[:, None, None]).min(axis=0)
        want = want + ndi.minimum_filter(n.astype(np.float64), size=q, mode="nearest")
    want = want / 3.0
    got = orc.dark_channel_ms(I, 15, 3, A)
    assert np.max(np.abs(got - want)) <= 1e-7  # float32 quotients (R4), mean in float64
    assert np.array_equal(orc.dark_channel_ms(I, 15, 1, A), orc.dark_channel(I, 15, A))


def test_transmission_refined_by_the_guided_filter(orc):
    """or_transmission with gf_radius > 0 = the guided filter (gray guide)
    applied to t = 1 - omega td, then lambda and Phi from the refined t."""
    I = scenes.hazy_scene(78, 24, 30)["I"]
    p = orc.params(**dict(orc.PAPER, gf_radius=3, gf_eps=1e-3))
    dc = orc.dark_channel(I, 15, None)
    A, _, _ = orc.atmospheric_light(I, dc, 1)
    td = orc.dark_channel(I, 15, A)
    t, lam, Phi = orc.transmission(I, A, td, p)
    I64 = I.astype(np.float64)
    g = ((I64[0] + I64[1]) + I64[2]) / 3.0
    t_want = guided_scipy(g, 1.0 - 0.95 * td, 3, 1e-3)
    assert np.max(np.abs(t - t_want)) <= 1e-12
    assert np.allclose(lam, 0.5 * np.exp(-3.0 * (1.0 - t_want)), rtol=1e-13, atol=0)
    Phi_want = (I64 - A[:, None, None] * (1.0 - t_want)) / np.maximum(t_want, 0.1)
    assert np.max(np.abs(Phi - Phi_want)) <= 1e-12
