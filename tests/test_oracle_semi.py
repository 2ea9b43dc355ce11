"""Pins of the semi-implicit (lagged-diffusivity) oracle, CPU only.

The frozen operator is tied to the pinned divergence (A u = u/s - div(D(u)
grad u)), its algebra to symmetry and definiteness, the iteration to a closed
form, and its fixed point to the explicit scheme's (stable preset) and to
F(u) = 0 through the pinned or_F (the paper's eps, where the explicit scheme
cannot converge)."""
import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

S = 2.0  # semi-implicit step s


@pytest.fixture(scope="module")
def semi(orc):
    from oracle import semi as m

    return m


def scene_problem(orc, seed, H, W, preset="stable", boundary=0):
    I = scenes.hazy_scene(seed, H, W)["I"]
    p = orc.params(**dict(orc.PAPER if preset == "paper" else orc.STABLE, boundary=boundary))
    dc = orc.dark_channel(I, 15, None)
    A, _, _ = orc.atmospheric_light(I, dc, 1)
    td = orc.dark_channel(I, 15, A)
    _, lam, Phi = orc.transmission(I, A, td, p)
    return p, Phi, lam


@pytest.mark.parametrize("H,W", [(7, 9), (1, 5), (6, 1), (12, 10)])
@pytest.mark.parametrize("boundary", [0, 1])
@pytest.mark.parametrize("eps,no_edge", [(1e-3, False), (1.0, False), (1.0, True)])
def test_frozen_operator_applied_to_u_is_minus_div(orc, semi, H, W, boundary, eps, no_edge):
    u = np.random.default_rng(H * 100 + W).normal(size=(H, W))
    Dx, Dy = orc.faces(u, eps, boundary, no_edge)
    A = semi.matrix(Dx, Dy, S, boundary)
    got = A @ u.ravel()
    want = u.ravel() / S - orc.div(u, eps, boundary, no_edge).ravel()
    assert np.max(np.abs(got - want)) <= 1e-9 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("boundary", [0, 1])
def test_matrix_symmetric_positive_definite(orc, semi, boundary):
    u = np.random.default_rng(5).random((9, 11))
    Dx, Dy = orc.faces(u, 1e-3, boundary)
    A = semi.matrix(Dx, Dy, S, boundary).toarray()
    assert np.array_equal(A, A.T)
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= (1.0 / S) * (1 - 1e-9)  # L is positive semidefinite
    if boundary == 1:
        assert ev.min() > (1.0 / S) * (1 + 1e-6)  # Dirichlet: L is definite


def test_no_edge_matrix_is_scaled_laplacian(orc, semi):
    """D == 1: I/s + L is I/s plus the reflecting 5-point graph Laplacian."""
    H, W = 4, 5
    Dx, Dy = orc.faces(np.zeros((H, W)), 1.0, 0, True)
    A = semi.matrix(Dx, Dy, S, 0).toarray()
    deg = np.zeros((H, W))
    deg[:, :-1] += 1
    deg[:, 1:] += 1
    deg[:-1, :] += 1
    deg[1:, :] += 1
    assert np.array_equal(np.diag(A), 1.0 / S + deg.ravel())
    assert np.array_equal(A.sum(axis=1), np.full(H * W, 1.0 / S))


def test_constant_image_closed_form(orc, semi):
    """Constant Phi^c and lambda: D grad u = 0 and G(u) = u on constants, so
    u^n = Phi/lam + (1 - s lam)^n (u^0 - Phi/lam) and
    rho_n = |1 - s lam|^n |1 - lam| from u^0 = Phi."""
    H, W, lam0 = 6, 7, 0.3
    p = orc.params(**orc.PAPER)
    phi = np.array([0.2, 0.5, 0.9])
    Phi = np.broadcast_to(phi[:, None, None], (3, H, W)).copy()
    lam = np.full((H, W), lam0)
    tol = 1e-6
    u, n, rho = semi.solve(Phi, Phi, lam, p, S, 500, tol)
    q = abs(1 - S * lam0)
    n_want = int(np.ceil(np.log(tol / abs(1 - lam0)) / np.log(q)))
    assert n == n_want
    # (the sparse solves carry D = 1/eps = 1000 on every face: the rounding of
    # u is ~1e-13, which is what rho's small values are differences of)
    assert np.allclose(rho[:, 0], q ** np.arange(n + 1) * abs(1 - lam0), rtol=1e-6, atol=1e-11)
    u_want = phi / lam0 + (1 - S * lam0) ** n * (phi - phi / lam0)
    assert np.allclose(u[:, 0, 0], u_want, rtol=1e-12)


@pytest.mark.parametrize("boundary", [0, 1])
def test_fixed_point_equals_explicit_scheme(orc, semi, boundary):
    p, Phi, lam = scene_problem(orc, 4242, 10, 12, "stable", boundary)
    ue, ne, _ = orc.solve(Phi, Phi, lam, p, 20000, 1e-11)
    us, ns, _ = semi.solve(Phi, Phi, lam, p, S, 2000, 1e-11)
    assert ne < 20000 and ns < 2000
    assert ns < ne / 5  # the semi-implicit scheme takes far fewer steps
    assert np.max(np.abs(us - ue)) <= 1e-8


def test_paper_eps_converges_to_F_zero(orc, semi):
    """eps = 1e-3 (the paper's constant): the semi-implicit scheme reaches
    ||F(u)|| / ||Phi|| <= 1e-8, F evaluated by the pinned or_F; two starting
    points give the same fixed point."""
    p, Phi, lam = scene_problem(orc, 4343, 12, 14, "paper")
    u1, n1, rho = semi.solve(Phi, Phi, lam, p, S, 3000, 1e-8)
    assert n1 < 3000
    f = orc.F(u1, Phi, lam, p)
    assert np.sqrt((f.reshape(3, -1) ** 2).sum(1) / (Phi.reshape(3, -1) ** 2).sum(1)).max() <= 1e-8
    u2, n2, _ = semi.solve(np.zeros_like(Phi), Phi, lam, p, S, 3000, 1e-8)
    assert n2 < 3000
    assert np.max(np.abs(u1 - u2)) <= 1e-5
