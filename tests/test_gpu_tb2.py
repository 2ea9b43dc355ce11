"""The two-iterations-per-load sweep (temporal blocking, sweep variants 31 and
32) against the one-iteration TMA kernel and the FP64 oracle: the same
iterates and residual history, the stop rule honoured when u^{n+1} of a
two-iteration step is the answer (the switch to single iterations), every
max_iter parity, ragged tile edges (widths that end anywhere in a 120-column
tile, heights anywhere in a tile), both boundaries, host-queued launches,
resume, and the launch count."""
import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TB2 = (31, 32)  # 120 x 16 and 120 x 24 output tiles
SINGLE = 1


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


def problem(orc, seed, H, W, boundary=0, variant=0):
    I = scenes.hazy_scene(seed, H, W)["I"]
    op = orc.params(**dict(orc.STABLE, boundary=boundary, variant=variant))
    dc = orc.dark_channel(I, 15, None)
    A, _, _ = orc.atmospheric_light(I, dc, 1)
    td = orc.dark_channel(I, 15, A)
    _, lam, Phi = orc.transmission(I, A, td, op)
    return op, Phi.astype(np.float32), lam.astype(np.float32)


def run(api, Phi, lam, v, **kw):
    u = dev(Phi.copy())
    rep, hist = api.fixed_point(u, dev(Phi), dev(lam), api.params("stable", sweep_variant=v, **kw), history=True)
    return rep, host(u), host(hist)


def rel(a, b):
    return float(np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))))


@pytest.mark.parametrize("H,W", [(64, 128), (100, 260), (45, 132), (1, 200), (300, 516), (37, 124), (50, 248),
                                 (17, 4), (2, 240), (130, 364)])
def test_fixed_steps_match_single_iteration_kernel(api, orc, H, W):
    _, Phi, lam = problem(orc, 8000 + H + W, H, W)
    for m in (40, 41):  # even and odd: the odd one ends with a single iteration
        ref, uref, href = run(api, Phi, lam, SINGLE, tol=0.0, max_iter=m)
        assert ref.n_iter == m
        for v in TB2:
            rep, u, hist = run(api, Phi, lam, v, tol=0.0, max_iter=m)
            assert rep.n_iter == m and rep.status == 2, (v, m)
            assert rel(u, uref) <= 1e-6, (v, m)
            assert rel(hist[: m + 1], href[: m + 1]) <= 1e-5, (v, m)


@pytest.mark.parametrize("H,W", [(40, 36), (61, 84), (64, 128)])
@pytest.mark.parametrize("boundary,variant", [(0, 0), (1, 0), (0, 2), (1, 2), (0, 1)])
def test_two_steps_match_oracle(api, orc, H, W, boundary, variant):
    op, Phi, lam = problem(orc, 8100 + H, H, W, boundary, variant)
    for v in TB2:
        rep, u, _ = run(api, Phi, lam, v, tol=0.0, max_iter=2, boundary=boundary, variant=variant)
        uo, n, _ = orc.solve(Phi.astype(np.float64), Phi.astype(np.float64), lam.astype(np.float64), op, 2, 0.0)
        assert rep.n_iter == n == 2
        assert np.max(np.abs(u - uo)) <= 1e-5, v


@pytest.mark.parametrize("tol", [1e-3, 3e-4, 1e-4])
def test_stop_rule(api, orc, tol):
    """Whatever the parity of the stopping n, the returned iterate and n are
    the one-iteration kernel's."""
    _, Phi, lam = problem(orc, 8202, 96, 256)
    ref, uref, _ = run(api, Phi, lam, SINGLE, tol=tol, max_iter=3000)
    assert ref.status == 0
    for v in TB2:
        rep, u, _ = run(api, Phi, lam, v, tol=tol, max_iter=3000)
        assert rep.status == 0 and abs(rep.n_iter - ref.n_iter) <= 1, v
        if rep.n_iter == ref.n_iter:
            assert rel(u, uref) <= 1e-6, v
        assert max(rep.rho) <= tol


def test_max_iter_values(api, orc):
    _, Phi, lam = problem(orc, 8303, 48, 136)
    for m in (0, 1, 2, 3, 62, 63, 64, 65, 127, 128, 129):
        ref, uref, _ = run(api, Phi, lam, SINGLE, tol=0.0, max_iter=m)
        rep, u, _ = run(api, Phi, lam, TB2[0], tol=0.0, max_iter=m)
        assert rep.n_iter == ref.n_iter == m
        assert rel(u, uref) <= 1e-6, m


def test_host_queued_equals_graph(api, orc):
    _, Phi, lam = problem(orc, 8404, 80, 200)
    a, ua, ha = run(api, Phi, lam, TB2[1], tol=1e-3, max_iter=900)
    b, ub, hb = run(api, Phi, lam, TB2[1], tol=1e-3, max_iter=900, use_graph=0)
    assert a.n_iter == b.n_iter and a.status == b.status == 0
    assert np.array_equal(ua, ub)
    assert np.array_equal(ha[: a.n_iter + 1], hb[: a.n_iter + 1])


def test_deterministic_and_resumable(api, orc):
    _, Phi, lam = problem(orc, 8505, 72, 248)
    outs = [run(api, Phi, lam, TB2[0], tol=0.0, max_iter=100)[1] for _ in range(2)]
    assert np.array_equal(outs[0], outs[1])
    u = dev(Phi.copy())
    api.fixed_point(u, dev(Phi), dev(lam), api.params("stable", sweep_variant=TB2[0], tol=0.0, max_iter=30))
    api.fixed_point(u, dev(Phi), dev(lam), api.params("stable", sweep_variant=TB2[0], tol=0.0, max_iter=70))
    assert rel(host(u), outs[0]) <= 1e-6


def test_converged_matches_oracle(api, orc):
    op, Phi, lam = problem(orc, 8606, 64, 120)
    rep, u, _ = run(api, Phi, lam, TB2[0], tol=1e-4, max_iter=5000)
    uo, no, _ = orc.solve(Phi.astype(np.float64), Phi.astype(np.float64), lam.astype(np.float64), op, 5000, 1e-4)
    assert rep.status == 0 and abs(rep.n_iter - no) <= 1
    assert np.max(np.abs(u - uo)) <= 1e-4


def test_launch_count(api, orc):
    _, Phi, lam = problem(orc, 8707, 64, 128)
    rep, _, _ = run(api, Phi, lam, TB2[0], tol=0.0, max_iter=300)
    # ||Phi||^2 (2) + descriptor (1) + output (1) + sweep launches: 64 loop steps each,
    # two iterations per step while n + 1 < max_iter
    loop_steps = 300 // 2 + 1
    assert rep.launches == 4 + (loop_steps + 63) // 64


def test_tb_depth_parameter_selects_the_sweep(api, orc):
    """tb_depth = 2 asks for two iterations per tile load (the 120 x 16
    variant), tb_depth = 1 for one (the library default) whatever was tuned."""
    _, Phi, lam = problem(orc, 8808, 64, 128)
    two = run(api, Phi, lam, 0, tol=0.0, max_iter=21, tb_depth=2)
    ref2 = run(api, Phi, lam, TB2[0], tol=0.0, max_iter=21)
    assert np.array_equal(two[1], ref2[1])
    one = run(api, Phi, lam, 0, tol=0.0, max_iter=21, tb_depth=1)
    ref1 = run(api, Phi, lam, 26, tol=0.0, max_iter=21)  # the default variant's configuration
    assert rel(one[1], ref1[1]) <= 1e-6 and one[0].n_iter == 21
