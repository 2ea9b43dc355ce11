"""The multi-iteration sweep (one cooperative launch runs up to 64 fixed-point
iterations, separated by in-kernel grid barriers) against the single-iteration
TMA kernel and the FP64 oracle: same iterates, same stopping n, same residual
history, stop rule honoured in the middle of a launch, several launches per
solve, host-queued launches, resume, Dirichlet boundary."""
import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MULTI = (25, 26, 27, 28)  # multi-iteration variants of dh_params.sweep_variant
SINGLE = 1                # the single-iteration TMA kernel with the default tiling
ITERS_PER_LAUNCH = 64


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_08793_gb300 import _native, api as a

    _native.lib()
    return a


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def problem(orc, seed, H, W, boundary=0):
    I = scenes.hazy_scene(seed, H, W)["I"]
    op = orc.params(**dict(orc.STABLE, boundary=boundary))
    dc = orc.dark_channel(I, 15, None)
    A, _, _ = orc.atmospheric_light(I, dc, 1)
    td = orc.dark_channel(I, 15, A)
    _, lam, Phi = orc.transmission(I, A, td, op)
    return op, Phi.astype(np.float32), lam.astype(np.float32)


def run(api, Phi, lam, variant, **kw):
    u = dev(Phi.copy())
    rep, hist = api.fixed_point(u, dev(Phi), dev(lam), api.params("stable", sweep_variant=variant, **kw),
                                history=True)
    return rep, host(u), host(hist)


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


@pytest.mark.parametrize("H,W", [(64, 128), (100, 260), (45, 132), (1, 200), (300, 516)])
def test_fixed_steps_match_single_iteration_kernel(api, orc, H, W):
    _, Phi, lam = problem(orc, 7000 + H, H, W)
    ref, uref, href = run(api, Phi, lam, SINGLE, tol=0.0, max_iter=150)  # 151 sweeps: 3 launches
    assert ref.n_iter == 150
    for v in MULTI:
        rep, u, hist = run(api, Phi, lam, v, tol=0.0, max_iter=150)
        assert rep.n_iter == 150 and rep.status == 2, v  # DH_WNOCONV at max_iter
        assert rel(u, uref) <= 1e-6, v
        assert rel(hist, href) <= 1e-5, v


def test_stop_rule_inside_a_launch(api, orc):
    """The stop rule fires mid-launch: the returned iterate is u^n (not a
    later one of the same launch) and equals the oracle's fixed point."""
    H, W = 96, 256
    op, Phi, lam = problem(orc, 7101, H, W)
    ref, uref, _ = run(api, Phi, lam, SINGLE, tol=1e-3, max_iter=2000)
    assert ref.status == 0 and ref.n_iter % ITERS_PER_LAUNCH != ITERS_PER_LAUNCH - 1
    uo, no, _ = orc.solve(Phi.astype(np.float64), Phi.astype(np.float64), lam.astype(np.float64), op, 2000, 1e-3)
    for v in MULTI:
        rep, u, _ = run(api, Phi, lam, v, tol=1e-3, max_iter=2000)
        assert rep.status == 0 and rep.n_iter == ref.n_iter, v
        assert rel(u, uref) <= 1e-6, v
        assert abs(rep.n_iter - no) <= 1
        assert np.max(np.abs(u - uo)) <= 1e-4


def test_max_iter_on_a_launch_boundary(api, orc):
    _, Phi, lam = problem(orc, 7202, 64, 128)
    for m in (0, 1, ITERS_PER_LAUNCH - 1, ITERS_PER_LAUNCH, ITERS_PER_LAUNCH + 1, 2 * ITERS_PER_LAUNCH - 1):
        ref, uref, _ = run(api, Phi, lam, SINGLE, tol=0.0, max_iter=m)
        rep, u, _ = run(api, Phi, lam, MULTI[0], tol=0.0, max_iter=m)
        assert rep.n_iter == ref.n_iter == m
        assert rel(u, uref) <= 1e-6, m


def test_deferred_decisions_return_the_exact_iterate(api, orc):
    """The multi-iteration float32 sweep decides on u^n one iteration late
    (three iterate buffers): stopping at n must still return u^n itself.  With
    the same split of rows over warps as the single-iteration kernel (variant
    25: 8 rows a warp, like variant 1) the iterate, the residual history and
    the stopping n are bit-identical, at and around launch boundaries and for
    a residual stop in the middle of a launch."""
    _, Phi, lam = problem(orc, 7252, 72, 136)
    for kw in [dict(tol=0.0, max_iter=m) for m in (0, 1, 2, 62, 63, 64, 65, 126, 127, 128)] + [
            dict(tol=1e-3, max_iter=2000), dict(tol=1e-3, max_iter=2000, use_graph=0)]:
        ref, uref, href = run(api, Phi, lam, SINGLE, **kw)
        rep, u, hist = run(api, Phi, lam, 25, **kw)
        assert rep.n_iter == ref.n_iter and rep.status == ref.status, kw
        assert np.array_equal(u, uref), kw
        n = rep.n_iter
        assert np.array_equal(hist[: n + 1], href[: n + 1]), kw
        assert np.allclose(rep.rho, ref.rho, rtol=0, atol=0), kw


def test_host_queued_launches_equal_graph_loop(api, orc):
    _, Phi, lam = problem(orc, 7303, 80, 200)
    a, ua, ha = run(api, Phi, lam, MULTI[1], tol=1e-3, max_iter=700)
    b, ub, hb = run(api, Phi, lam, MULTI[1], tol=1e-3, max_iter=700, use_graph=0)
    assert a.n_iter == b.n_iter and a.status == b.status == 0
    assert np.array_equal(ua, ub)
    assert np.array_equal(ha[: a.n_iter + 1], hb[: a.n_iter + 1])


def test_deterministic_and_resumable(api, orc):
    _, Phi, lam = problem(orc, 7404, 72, 136)
    outs = [run(api, Phi, lam, MULTI[0], tol=0.0, max_iter=100)[1] for _ in range(2)]
    assert np.array_equal(outs[0], outs[1])
    u = dev(Phi.copy())
    api.fixed_point(u, dev(Phi), dev(lam), api.params("stable", sweep_variant=MULTI[0], tol=0.0, max_iter=30))
    api.fixed_point(u, dev(Phi), dev(lam), api.params("stable", sweep_variant=MULTI[0], tol=0.0, max_iter=70))
    assert np.array_equal(host(u), outs[0])


def test_dirichlet_boundary(api, orc):
    op, Phi, lam = problem(orc, 7505, 61, 84, boundary=1)
    rep, u, _ = run(api, Phi, lam, MULTI[0], tol=0.0, max_iter=3, boundary=1)
    uo, n, _ = orc.solve(Phi.astype(np.float64), Phi.astype(np.float64), lam.astype(np.float64), op, 3, 0.0)
    assert rep.n_iter == n == 3
    assert np.max(np.abs(u - uo)) <= 1e-5


def test_launch_count_reported(api, orc):
    _, Phi, lam = problem(orc, 7606, 64, 128)
    rep, _, _ = run(api, Phi, lam, MULTI[0], tol=0.0, max_iter=200)
    sweeps = rep.n_iter + 1
    # ||Phi||^2 (2) + descriptor (1) + output (1) + the loop's launches
    assert rep.launches == 4 + (sweeps + ITERS_PER_LAUNCH - 1) // ITERS_PER_LAUNCH
