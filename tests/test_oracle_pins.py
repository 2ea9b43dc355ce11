"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test checks one oracle function against something the paper or the
mathematics fixes: library routines the paper names (scipy.ndimage), closed
forms derived by hand, brute force, invariants of the discretisation, and the
exact recovery of the scattering model on scenes where the dark channel prior
holds.  No expected value here comes from the CUDA path.
"""
import json
import os

import numpy as np
import pytest
import scipy.ndimage as ndi

from paper_2506_08793_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rnd(seed, *shape, lo=0.0, hi=1.0):
    n = int(np.prod(shape))
    return scenes.uniform(seed, 77, n, lo, hi).reshape(shape)


# ------------------------------------------------------------ constants

def test_paper_constants_match_presets(orc):
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    P = orc.PAPER
    for k in ("patch", "omega", "eps", "sigma", "lambda0", "beta", "tau"):
        assert P[k] == g[k]["value"], k
    assert 2 * P["radius"] + 1 == g["gauss_size"]["value"]
    # the stable preset changes eps only
    diff = {k for k in P if orc.STABLE[k] != P[k]}
    assert diff == {"eps"}


# ------------------------------------------------------------ dark channel

@pytest.mark.parametrize("H,W", [(1, 1), (1, 9), (9, 1), (15, 15), (16, 17), (40, 33), (7, 64)])
def test_dark_channel_is_min_filter(orc, H, W):
    """Sec. II-D: min over channels of a 15x15 min filter, window clipped at
    the border == scipy minimum_filter with 'nearest' padding."""
    I = rnd(H * 100 + W, 3, H, W).astype(np.float32)
    got = orc.dark_channel(I, 15, None)
    want = ndi.minimum_filter(I.min(axis=0).astype(np.float64), size=15, mode="nearest")
    assert np.array_equal(got, want)
    A = np.array([0.9, 0.7, 0.95])
    got = orc.dark_channel(I, 15, A)
    want = np.min([ndi.minimum_filter(I[c].astype(np.float64) / A[c], size=15, mode="nearest")
                   for c in range(3)], axis=0)
    assert np.array_equal(got, want)


def test_dark_channel_brute_force_small_patch(orc):
    I = rnd(5, 3, 6, 7).astype(np.float32)
    got = orc.dark_channel(I, 3, None)
    for y in range(6):
        for x in range(7):
            ys, xs = slice(max(0, y - 1), y + 2), slice(max(0, x - 1), x + 2)
            assert got[y, x] == I[:, ys, xs].min()


def test_normalised_quotient_rounds_like_fp32_division(orc):
    """R4: rounding the FP64 quotient of two floats to FP32 equals the FP32
    IEEE quotient (53 >= 2*24+2), so the normalised dark channel is exact."""
    I = rnd(9, 3, 20, 20).astype(np.float32)
    A = np.array([0.83, 0.91, 0.977], np.float32)
    got = orc.dark_channel(I, 15, A.astype(np.float64)).astype(np.float32)
    q = I / A[:, None, None]  # float32 division
    want = np.min([ndi.minimum_filter(q[c], size=15, mode="nearest") for c in range(3)], axis=0)
    assert np.array_equal(got, want)


# ------------------------------------------------------------ atmospheric light

def _lexsort_A(I, dc, permille):
    N = dc.size
    k = max(1, N * permille // 1000)
    order = np.lexsort((np.arange(N), -dc.ravel()))[:k]
    s = (I[0].ravel()[order].astype(np.float64) + I[1].ravel()[order]) + I[2].ravel()[order]
    best = order[np.lexsort((order, -s))[0]]
    return best


@pytest.mark.parametrize("H,W,levels", [(1, 1, 0), (31, 37, 0), (64, 64, 4), (100, 30, 2), (50, 50, 1)])
def test_atmospheric_light_matches_sorted_selection(orc, H, W, levels):
    I = rnd(H + 7 * W, 3, H, W)
    if levels:  # many exact ties in both keys
        I = np.floor(I * levels) / levels
    I = I.astype(np.float32)
    dc = orc.dark_channel(I, 15, None)
    A, idx, clamped = orc.atmospheric_light(I, dc, 1)
    best = _lexsort_A(I, dc, 1)
    assert idx == best
    if not clamped:
        assert np.array_equal(A, I.reshape(3, -1)[:, best].astype(np.float64))


def test_atmospheric_light_clamps_nonpositive(orc):
    I = np.zeros((3, 8, 8), np.float32)
    dc = orc.dark_channel(I, 15, None)
    A, idx, clamped = orc.atmospheric_light(I, dc, 1)
    assert clamped and idx == 0 and np.all(A == 1e-6)


# ------------------------------------------------------------ prior-holding scenes

def test_scattering_model_recovered_where_prior_holds(orc):
    """Sec. II-A/II-D: on a scene where every window has a zero channel, J < A
    and a sky band has t = 0, the method recovers A exactly, t = 1-w+w*t_true
    inside constant-depth bands, and with w = 1, Phi = J there."""
    H, W, sky = 96, 128, 24
    s = scenes.prior_scene(11, H, W, sky)
    I = s["I"]
    p = orc.params(**orc.STABLE)
    dc = orc.dark_channel(I, p.patch, None)
    A, idx, clamped = orc.atmospheric_light(I, dc, p.topk_permille)
    assert not clamped
    assert np.array_equal(A, s["A_true"].astype(np.float32).astype(np.float64))
    td = orc.dark_channel(I, p.patch, A)
    t, lam, Phi = orc.transmission(I, A, td, p)
    bw = s["band_w"]
    mask = np.zeros((H, W), bool)
    for x0 in range(0, W, bw):
        mask[sky + 7: H, x0 + 7: min(W, x0 + bw) - 7] = True
    tt = s["t_true"]
    assert np.max(np.abs(t[mask] - (1 - 0.95 + 0.95 * tt[mask]))) < 1e-6
    assert np.max(np.abs(t[: sky - 7] - 0.05)) < 1e-12
    p1 = orc.params(**dict(orc.STABLE, omega=1.0))
    t1, _, Phi1 = orc.transmission(I, A, td, p1)
    assert np.max(np.abs(t1[mask] - tt[mask])) < 1e-6
    err = np.abs(Phi1[:, mask] - s["J"][:, mask])
    assert err.max() < 2e-5


# ------------------------------------------------------------ constant image closed form

@pytest.mark.parametrize("c", [0.3, 0.6, 0.9])
def test_constant_image_closed_form(orc, c):
    """I = c: A = c, t = 1-w = 0.05, lambda = l0 exp(-3*0.95), Phi = 0.05c/t0,
    div = 0, G(u) = u, so u^n = u* + (1-tau*l)^n (Phi-u*), u* = Phi/l and
    rho_n = (1-tau*l)^n (1-l): 1583 iterations to 1e-4 for any eps."""
    H, W = 12, 10
    I = np.full((3, H, W), c, np.float32)
    cf = float(np.float32(c))
    for preset in (orc.PAPER, orc.STABLE):
        p = orc.params(**preset)
        r = orc.dehaze(I, p, 5000, 1e-4)
        assert np.all(r["A"] == cf)
        assert np.allclose(r["t"], 0.05, atol=1e-15, rtol=0)
        lam = 0.5 * np.exp(-3.0 * 0.95)
        assert np.allclose(r["lam"], lam, rtol=1e-14, atol=0)
        assert np.allclose(r["Phi"], 0.05 * cf / 0.1, rtol=1e-13, atol=0)
        q = 1.0 - 0.2 * lam
        n = np.arange(r["n"] + 1)
        assert np.allclose(r["rho"], ((q ** n) * (1 - lam))[:, None], rtol=1e-9, atol=0)
        assert r["n"] == int(np.ceil(np.log(1e-4 / (1 - lam)) / np.log(q))) == 1583
        Phi0 = 0.05 * cf / 0.1
        ustar = Phi0 / lam
        assert np.allclose(r["u"], ustar + q ** r["n"] * (Phi0 - ustar), rtol=1e-10, atol=0)


# ------------------------------------------------------------ Gaussian term

def test_gauss_weights_are_scipy_truncated_kernel(orc):
    """App. A-B-2: 5x5, sigma = 2 (scipy gaussian_filter, truncate = 1)."""
    d = np.zeros(11)
    d[5] = 1.0
    want = ndi.gaussian_filter1d(d, 2.0, truncate=1.0)[3:8]
    assert np.allclose(orc.gauss_weights(2.0, 2), want, rtol=1e-15, atol=1e-16)
    assert abs(orc.gauss_weights(2.0, 2).sum() - 1.0) < 1e-15


@pytest.mark.parametrize("H,W", [(1, 1), (2, 3), (5, 9), (33, 20)])
def test_gauss_is_scipy_gaussian_filter(orc, H, W):
    u = rnd(H * W + 3, H, W, lo=-3, hi=5)
    want = ndi.gaussian_filter(u, 2.0, truncate=1.0, mode="reflect")
    assert np.allclose(orc.gauss(u), want, rtol=0, atol=1e-13)


# ------------------------------------------------------------ diffusion term

@pytest.mark.parametrize("H,W", [(2, 2), (7, 11), (30, 25)])
def test_div_linear_limit_is_laplacian(orc, H, W):
    """eps -> inf: D -> 1/eps, so eps*div(D grad u) -> 5-point Laplacian with
    the reflecting (zero-flux) boundary (scipy.ndimage.laplace, 'reflect')."""
    u = rnd(H + W, H, W, lo=-1, hi=1)
    eps = 1e9
    got = eps * orc.div(u, eps)
    want = ndi.laplace(u, mode="reflect")
    assert np.allclose(got, want, rtol=0, atol=1e-7)


@pytest.mark.parametrize("eps", [1e-3, 1.0])
def test_div_step_closed_form(orc, eps):
    """u = 1 for i >= m (columns), 0 otherwise: only the face between m-1 and
    m carries flux 1/(1+eps); its transpose exercises the y-faces."""
    H, W, m = 6, 9, 4
    u = np.zeros((H, W))
    u[:, m:] = 1.0
    want = np.zeros((H, W))
    want[:, m - 1] = 1.0 / (1.0 + eps)
    want[:, m] = -1.0 / (1.0 + eps)
    assert np.allclose(orc.div(u, eps), want, rtol=1e-15, atol=1e-15)
    assert np.allclose(orc.div(u.T.copy(), eps), want.T, rtol=1e-15, atol=1e-15)


def test_div_tangential_difference_at_left_cell(orc):
    """App. A-B-1: D on the x-face (i+1/2, j) takes the y-difference of cell i.
    For u(i, j) = i*j this gives, at interior cells,
    div = (j+i)/(r(i,j)+e) - j/(r(i-1,j)+e) - i/(r(i,j-1)+e), r(a,b) = sqrt(a^2+b^2)."""
    H, W, e = 9, 11, 0.25
    jj, ii = np.mgrid[0:H, 0:W].astype(np.float64)
    u = ii * jj
    got = orc.div(u, e)
    r = lambda a, b: np.sqrt(a * a + b * b)
    want = (jj + ii) / (r(ii, jj) + e) - jj / (r(ii - 1, jj) + e) - ii / (r(ii, jj - 1) + e)
    inner = (slice(1, H - 1), slice(1, W - 1))
    assert np.allclose(got[inner], want[inner], rtol=1e-13, atol=1e-13)


def test_div_conserves_and_is_transpose_equivariant(orc):
    u = rnd(3, 23, 31, lo=-2, hi=2)
    d = orc.div(u, 1e-3)
    assert abs(d.sum()) < 1e-9 * np.abs(d).sum()
    assert np.allclose(orc.div(u.T.copy(), 1e-3), d.T, rtol=0, atol=1e-12)


def test_F_composition(orc):
    """F = div - lambda*G + Phi: with eps huge the diffusion vanishes and F is
    -lambda*gaussian_filter(u) + Phi from scipy."""
    H, W = 13, 17
    u = rnd(1, 3, H, W, lo=-1, hi=3)
    Phi = rnd(2, 3, H, W)
    lam = rnd(3, H, W, lo=0.02, hi=0.5)
    p = orc.params(eps=1e12)
    got = orc.F(u, Phi, lam, p)
    want = np.stack([-lam * ndi.gaussian_filter(u[c], 2.0, truncate=1.0, mode="reflect") + Phi[c]
                     for c in range(3)])
    assert np.allclose(got, want, rtol=0, atol=1e-10)


# ------------------------------------------------------------ fixed-point solver

def _small_problem(orc, seed, H, W, preset):
    s = scenes.hazy_scene(seed, H, W)
    p = orc.params(**preset)
    I = s["I"]
    dc = orc.dark_channel(I, p.patch, None)
    A, _, _ = orc.atmospheric_light(I, dc, p.topk_permille)
    td = orc.dark_channel(I, p.patch, A)
    t, lam, Phi = orc.transmission(I, A, td, p)
    return I, p, lam, Phi


def test_fixed_point_is_newton_root(orc):
    """App. A-A: the iteration's limit solves F(u) = 0 (dense Newton, FP64)."""
    I, p, lam, Phi = _small_problem(orc, 21, 8, 9, orc.STABLE)
    u, n, rho = orc.solve(Phi, Phi, lam, p, 200000, 1e-13)
    assert rho[-1].max() <= 1e-13
    v = Phi.copy()
    m = v.size
    for _ in range(30):
        f = orc.F(v, Phi, lam, p).ravel()
        if np.abs(f).max() < 1e-13:
            break
        Jm = np.empty((m, m))
        h = 1e-6
        for k in range(m):
            e = np.zeros(m)
            e[k] = h
            Jm[:, k] = (orc.F(v + e.reshape(v.shape), Phi, lam, p).ravel()
                        - orc.F(v - e.reshape(v.shape), Phi, lam, p).ravel()) / (2 * h)
        v = v - np.linalg.solve(Jm, f).reshape(v.shape)
    assert np.abs(orc.F(v, Phi, lam, p)).max() < 1e-11
    assert np.abs(u - v).max() < 1e-9


def test_linear_limit_root_and_instability(orc):
    """eps = 1e6: D = 1/eps to 1e-12 relative, so F(u) = Lap(u)/eps - lambda G(u)
    + Phi is linear.  Its root, from operator matrices built by applying scipy's
    reflecting laplace and gaussian_filter to unit vectors and a dense solve,
    zeroes the oracle's F.  The explicit iteration does not reach it: the
    truncated Gaussian's symbol is negative near 1.94 rad (Sec. III-C's
    coercivity claim fails), and without diffusion to damp those modes
    u + tau F amplifies them by 1 + tau lambda |g| per step."""
    I, p, lam, Phi = _small_problem(orc, 24, 7, 9, orc.STABLE)
    eps = 1e6
    p.eps = eps
    H, W = lam.shape
    m = H * W
    Lap = np.empty((m, m))
    Gm = np.empty((m, m))
    for k in range(m):
        e = np.zeros(m)
        e[k] = 1.0
        e = e.reshape(H, W)
        Lap[:, k] = ndi.laplace(e, mode="reflect").ravel()
        Gm[:, k] = ndi.gaussian_filter(e, 2.0, mode="reflect", truncate=1.0).ravel()
    A = -Lap / eps + lam.ravel()[:, None] * Gm
    want = np.stack([np.linalg.solve(A, Phi[c].ravel()).reshape(H, W) for c in range(3)])
    # (lambda G is nearly singular where the symbol crosses zero and D deviates
    # from 1/eps by |grad u|/eps: the root holds to ~1e-6 of |Phi|)
    f = orc.F(want, Phi, lam, p)
    assert np.abs(f).max() <= 1e-5 * np.abs(Phi).max()
    # the explicit iteration drifts away from it
    _, n, rho = orc.solve(Phi, Phi, lam, p, 6000, 0.0)
    r = rho.max(axis=1)
    assert n == 6000 and r[-1] > 10 * r.min()


def test_uniqueness_from_different_initial_guesses(orc):
    """Sec. III-D claims a unique solution; the stable preset reaches the same
    u from u0 = Phi, 0, I and a random field."""
    I, p, lam, Phi = _small_problem(orc, 22, 24, 20, orc.STABLE)
    starts = [Phi, np.zeros_like(Phi), I.astype(np.float64), 5 * rnd(4, *Phi.shape)]
    us = [orc.solve(u0, Phi, lam, p, 100000, 1e-11)[0] for u0 in starts]
    for u in us[1:]:
        assert np.abs(u - us[0]).max() < 1e-7


def test_stable_residual_is_monotone_and_resume_exact(orc):
    I, p, lam, Phi = _small_problem(orc, 23, 40, 48, orc.STABLE)
    u, n, rho = orc.solve(Phi, Phi, lam, p, 5000, 1e-4)
    assert rho[-1].max() <= 1e-4 < rho[-2].max()
    assert np.all(np.diff(rho.max(axis=1)) < 0)
    # resume: n = n1 + n2 reproduces u bit for bit
    u1, n1, _ = orc.solve(Phi, Phi, lam, p, 37, 0.0)
    u2, n2, _ = orc.solve(u1, Phi, lam, p, n - 37, 0.0)
    u3, _, _ = orc.solve(Phi, Phi, lam, p, n, 0.0)
    assert n1 == 37 and n2 == n - 37
    assert np.array_equal(u2, u3) and np.array_equal(u3, u)


def test_paper_preset_violates_step_condition(orc):
    """R1: with eps = 1e-3 and tau = 0.2 the explicit scheme breaks the step
    bound of App. A-A (tau < 2/(8/eps + lambda*M)); the residual does not
    decrease monotonically."""
    assert 0.2 > 2.0 / (8.0 / 1e-3 + 0.5)
    assert 0.2 < 2.0 / (8.0 / 1.0 + 0.5)
    I, p, lam, Phi = _small_problem(orc, 24, 32, 32, orc.PAPER)
    _, n, rho = orc.solve(Phi, Phi, lam, p, 200, 1e-4)
    r = rho.max(axis=1)
    assert n == 200 and np.any(np.diff(r) > 0) and r[-1] > 1e-2


# ------------------------------------------------------------ boundary option and ablations

@pytest.mark.parametrize("H,W", [(3, 4), (17, 11)])
def test_dirichlet_boundary_is_zero_padding(orc, H, W):
    """u = 0 outside the image (H^1_0, Sec. III): the Gaussian is scipy's with
    zero padding and eps*div tends to the zero-padded 5-point Laplacian."""
    u = rnd(H * W + 5, H, W, lo=-2, hi=3)
    want = ndi.gaussian_filter(u, 2.0, truncate=1.0, mode="constant", cval=0.0)
    assert np.allclose(orc.gauss(u, boundary=1), want, rtol=0, atol=1e-13)
    eps = 1e9
    want = ndi.laplace(u, mode="constant", cval=0.0)
    assert np.allclose(eps * orc.div(u, eps, boundary=1), want, rtol=0, atol=1e-6)


def test_no_edge_ablation_is_linear_diffusion(orc):
    """D == 1 (w/o edge-preserving term): div(grad u) is the 5-point Laplacian."""
    u = rnd(8, 19, 23, lo=-1, hi=1)
    assert np.allclose(orc.div(u, 1e-3, no_edge=True), ndi.laplace(u, mode="reflect"), rtol=0, atol=1e-13)


def test_lambda_ablations(orc):
    I = scenes.hazy_scene(12, 20, 30)["I"]
    dc = orc.dark_channel(I, 15, None)
    A, _, _ = orc.atmospheric_light(I, dc, 1)
    td = orc.dark_channel(I, 15, A)
    _, lam, Phi = orc.transmission(I, A, td, orc.params(variant=1))
    assert np.all(lam == 0.5)
    _, lam0, Phi0 = orc.transmission(I, A, td, orc.params(variant=4))
    assert np.all(lam0 == 0.0) and np.array_equal(Phi, Phi0)
