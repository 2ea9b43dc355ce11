"""16-bit iterate storage (bf16 / f16 u, float32 Phi, lambda and arithmetic)
and the switched schedules that finish in float32, through the C ABI."""
import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def problem(orc, seed, H, W):
    I = scenes.hazy_scene(seed, H, W)["I"]
    op = orc.params(**orc.STABLE)
    dc = orc.dark_channel(I, 15, None)
    A, _, _ = orc.atmospheric_light(I, dc, 1)
    td = orc.dark_channel(I, 15, A)
    _, lam, Phi = orc.transmission(I, A, td, op)
    return op, Phi.astype(np.float32), lam.astype(np.float32)


def round16(x, kind):
    t = torch.from_numpy(np.ascontiguousarray(x, np.float32))
    return (t.to(torch.bfloat16) if kind == "bf16" else t.to(torch.float16)).float().numpy()


# half an ulp relative of each 16-bit format (round to nearest)
HALF_ULP = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}
STORE = {"bf16": 1, "f16": 2, "bf16_f32": 3, "f16_f32": 4}


@pytest.mark.parametrize("kind", ["bf16", "f16"])
@pytest.mark.parametrize("H,W", [(64, 128), (61, 83), (40, 36), (130, 264)])
def test_one_step_16bit(api, orc, kind, H, W):
    """One update from a u^0 that is exact in the 16-bit format: the GPU's
    u^1 is the oracle's u^1 rounded to 16 bits (plus float32 noise)."""
    op, Phi, lam = problem(orc, 5 + H + W, H, W)
    u0 = round16(Phi, kind)
    u = dev(u0.copy())
    rep, _ = api.fixed_point(u, dev(Phi), dev(lam),
                             api.params("stable", tol=0.0, max_iter=1, storage=STORE[kind]))
    assert rep.n_iter == 1
    ou, _, _ = orc.solve(u0.astype(np.float64), Phi, lam, op, 1, 0.0)
    err = np.abs(host(u) - ou)
    assert np.all(err <= HALF_ULP[kind] * np.abs(ou) * 1.001 + 1e-5)


@pytest.mark.parametrize("kind", ["bf16", "f16"])
def test_pure_16bit_stalls_above_tolerance(api, orc, kind):
    """Stored in 16 bits the iterate cannot reach 1e-4 (u is O(10), so the
    storage quantum dominates tau*F near the fixed point): the run ends at
    max_iter with a finite residual above tol."""
    op, Phi, lam = problem(orc, 8, 96, 128)
    u = dev(Phi.copy())
    rep, hist = api.fixed_point(u, dev(Phi), dev(lam),
                                api.params("stable", max_iter=1500, storage=STORE[kind]), history=True)
    assert rep.status == 2 and rep.n_iter == 1500
    assert np.all(np.isfinite(rep.rho)) and max(rep.rho) > 1e-4


@pytest.mark.parametrize("kind", ["bf16_f32", "f16_f32"])
@pytest.mark.parametrize("H,W", [(96, 128), (61, 83)])
def test_switched_schedule_reaches_tolerance(api, orc, kind, H, W):
    """16-bit storage until the residual stalls, then float32 to 1e-4: the
    result is as close to the FP64 fixed point as the float32 path's."""
    op, Phi, lam = problem(orc, 9 + H, H, W)
    ustar, _, _ = orc.solve(Phi.astype(np.float64), Phi, lam, op, 20000, 1e-9)
    outs = {}
    for name, st in (("f32", 0), (kind, STORE[kind])):
        u = dev(Phi.copy())
        rep, hist = api.fixed_point(u, dev(Phi), dev(lam), api.params("stable", storage=st), history=True)
        assert rep.status == 0 and max(rep.rho) <= 1e-4
        outs[name] = (host(u), rep.n_iter)
    err32 = np.max(np.abs(outs["f32"][0] - ustar))
    errsw = np.max(np.abs(outs[kind][0] - ustar))
    assert errsw <= 2 * err32 + 2e-4, (errsw, err32)


def test_switched_dehaze_whole_method(api, orc):
    I = scenes.hazy_scene(1000, 256, 256)["I"]
    out32 = api.dehaze(dev(I), api.params("stable"))
    outbf = api.dehaze(dev(I), api.params("stable", storage=3))
    assert outbf["report"].status == 0 and max(outbf["report"].rho) <= 1e-4
    assert torch.equal(out32["A"], outbf["A"]) and torch.equal(out32["t"], outbf["t"])
    r = orc.dehaze(I, orc.params(**orc.STABLE), 20000, 1e-9)
    e32 = np.max(np.abs(host(out32["u"]) - r["u"]))
    ebf = np.max(np.abs(host(outbf["u"]) - r["u"]))
    assert ebf <= 2 * e32 + 2e-4
