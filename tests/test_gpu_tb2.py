"""The temporally blocked sweeps (K iterations per tile load: K = 2, tuner
variants 31 and 32; K = 3, variants 36 and 37; K = 4, variant 38) against the
one-iteration TMA kernel and the FP64 oracle: the same iterates and residual
history, the stop rule honoured when some u^{n+l}, 0 < l < K, of a K-iteration
step is the answer (the switch to single iterations), every max_iter residue,
ragged tile edges (widths that end anywhere in a 120-, 112- or 104-column
tile, heights anywhere in a tile), both boundaries and the ablations,
host-queued launches, resume, and the launch count."""
import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TB2 = (31, 32)  # 120 x 16 and 120 x 24 output tiles
TBK = TB2 + (36, 37, 38)  # and depth 3 (112 x 16, 112 x 24), depth 4 (104 x 16)
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
    for m in (40, 41, 42, 43):  # every residue mod 2, 3 and 4: the last steps switch to single iterations
        ref, uref, href = run(api, Phi, lam, SINGLE, tol=0.0, max_iter=m)
        assert ref.n_iter == m
        for v in TBK:
            rep, u, hist = run(api, Phi, lam, v, tol=0.0, max_iter=m)
            assert rep.n_iter == m and rep.status == 2, (v, m)
            assert rel(u, uref) <= 1e-6, (v, m)
            assert rel(hist[: m + 1], href[: m + 1]) <= 1e-5, (v, m)


@pytest.mark.parametrize("H,W", [(40, 36), (61, 84), (64, 128)])
@pytest.mark.parametrize("boundary,variant", [(0, 0), (1, 0), (0, 2), (1, 2), (0, 1)])
def test_two_steps_match_oracle(api, orc, H, W, boundary, variant):
    op, Phi, lam = problem(orc, 8100 + H, H, W, boundary, variant)
    for v, m in ((31, 2), (32, 2), (36, 3), (37, 3), (38, 4)):  # one full K-iteration step each
        rep, u, _ = run(api, Phi, lam, v, tol=0.0, max_iter=m, boundary=boundary, variant=variant)
        uo, n, _ = orc.solve(Phi.astype(np.float64), Phi.astype(np.float64), lam.astype(np.float64), op, m, 0.0)
        assert rep.n_iter == n == m
        assert np.max(np.abs(u - uo)) <= 1e-5, v


@pytest.mark.parametrize("tol", [1e-3, 3e-4, 1e-4])
def test_stop_rule(api, orc, tol):
    """Whatever the parity of the stopping n, the returned iterate and n are
    the one-iteration kernel's."""
    _, Phi, lam = problem(orc, 8202, 96, 256)
    ref, uref, _ = run(api, Phi, lam, SINGLE, tol=tol, max_iter=3000)
    assert ref.status == 0
    for v in TBK:
        rep, u, _ = run(api, Phi, lam, v, tol=tol, max_iter=3000)
        assert rep.status == 0 and abs(rep.n_iter - ref.n_iter) <= 1, v
        if rep.n_iter == ref.n_iter:
            assert rel(u, uref) <= 1e-6, v
        assert max(rep.rho) <= tol


def test_max_iter_values(api, orc):
    _, Phi, lam = problem(orc, 8303, 48, 136)
    for m in (0, 1, 2, 3, 4, 5, 62, 63, 64, 65, 127, 128, 129, 130, 191, 192, 193, 194, 255, 256, 257):
        ref, uref, _ = run(api, Phi, lam, SINGLE, tol=0.0, max_iter=m)
        for v in (31, 36, 38):
            rep, u, _ = run(api, Phi, lam, v, tol=0.0, max_iter=m)
            assert rep.n_iter == ref.n_iter == m, (v, m)
            assert rel(u, uref) <= 1e-6, (v, m)


@pytest.mark.parametrize("v", [32, 37])
def test_host_queued_equals_graph(api, orc, v):
    _, Phi, lam = problem(orc, 8404, 80, 200)
    a, ua, ha = run(api, Phi, lam, v, tol=1e-3, max_iter=900)
    b, ub, hb = run(api, Phi, lam, v, tol=1e-3, max_iter=900, use_graph=0)
    assert a.n_iter == b.n_iter and a.status == b.status == 0
    assert np.array_equal(ua, ub)
    assert np.array_equal(ha[: a.n_iter + 1], hb[: a.n_iter + 1])


@pytest.mark.parametrize("v", [31, 36, 38])
def test_deterministic_and_resumable(api, orc, v):
    _, Phi, lam = problem(orc, 8505, 72, 248)
    outs = [run(api, Phi, lam, v, tol=0.0, max_iter=100)[1] for _ in range(2)]
    assert np.array_equal(outs[0], outs[1])
    u = dev(Phi.copy())
    api.fixed_point(u, dev(Phi), dev(lam), api.params("stable", sweep_variant=v, tol=0.0, max_iter=30))
    api.fixed_point(u, dev(Phi), dev(lam), api.params("stable", sweep_variant=v, tol=0.0, max_iter=70))
    assert rel(host(u), outs[0]) <= 1e-6


@pytest.mark.parametrize("v", [31, 36, 38])
def test_converged_matches_oracle(api, orc, v):
    op, Phi, lam = problem(orc, 8606, 64, 120)
    rep, u, _ = run(api, Phi, lam, v, tol=1e-4, max_iter=5000)
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
    """tb_depth = K (2, 3, 4) asks for K iterations per tile load (the 120 x
    16, 112 x 16 and 104 x 16 variants), tb_depth = 1 for one (the library
    default) whatever was tuned."""
    _, Phi, lam = problem(orc, 8808, 64, 128)
    for depth, v in ((2, 31), (3, 36), (4, 38)):
        got = run(api, Phi, lam, 0, tol=0.0, max_iter=21, tb_depth=depth)
        ref = run(api, Phi, lam, v, tol=0.0, max_iter=21)
        assert np.array_equal(got[1], ref[1]), depth
    one = run(api, Phi, lam, 0, tol=0.0, max_iter=21, tb_depth=1)
    ref1 = run(api, Phi, lam, 26, tol=0.0, max_iter=21)  # the default variant's configuration
    assert rel(one[1], ref1[1]) <= 1e-6 and one[0].n_iter == 21
