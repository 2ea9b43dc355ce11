"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every entry point include/dehaze.h declares, and rejects bad
arguments before touching the device."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2506_08793_gb300 import _native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dehaze.h")


@pytest.fixture(scope="module")
def L():
    return N.lib()


def header_symbols():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(dh_\w+)\s*\(", txt, flags=re.M))


def test_exports_every_declared_symbol(L):
    decl = header_symbols()
    assert decl == set(N.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", N.SO], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (dh_\w+)", out))
    assert decl <= exported, decl - exported
    for s in decl:
        assert hasattr(L, s)


def test_struct_sizes_match_header():
    # dh_params: 21 4-byte fields; dh_report: 2 ints, 6 floats, long long, 2 floats, int (+pad)
    assert ctypes.sizeof(N.DhParams) == 84
    assert ctypes.sizeof(N.DhReport) == 56


def test_defaults_are_the_paper_constants():
    p = N.dh_params_default(N.DH_PRESET_PAPER)
    assert (p.patch, p.radius, p.topk_permille) == (15, 2, 1)
    for k, v in dict(omega=0.95, eps=1e-3, sigma=2.0, lambda0=0.5, beta=3.0, tau=0.2, t0=0.1).items():
        assert getattr(p, k) == pytest.approx(v, rel=1e-7), k
    s = N.dh_params_default(N.DH_PRESET_STABLE)
    assert s.eps == 1.0
    assert {k for k, _ in p._fields_ if getattr(p, k) != getattr(s, k)} == {"eps"}
    with pytest.raises(ValueError):
        N.dh_params_default(7)
    assert N.dh_version() == 1


def test_strerror_covers_codes():
    for c in (0, 1, 2, -1, -2, -3, -4, -5):
        assert N.dh_strerror(c) != "unknown status"
    assert N.dh_strerror(99) == "unknown status"


def test_workspace_bytes():
    p = N.dh_params_default(N.DH_PRESET_STABLE)
    b = N.dh_workspace_bytes(1080, 1920, p)
    n = 1080 * 1920
    # per pixel: dark channel, lambda, Phi (3) and two float32 iterate buffers (3 each)
    assert b >= 4 * (11 * n) and b < 4 * (11 * n) + (1 << 22)
    # a batched solve keeps no third iterate buffer (its sweep decides at once)
    fake = 1 << 20
    img = N.dh_image(fake, 1080, 1920, None, fake, fake, fake, fake)
    bb = N.dh_batch_workspace_bytes(1, [img], p)
    assert 4 * (8 * n) <= bb < b - 4 * (3 * n) + (1 << 22)
    assert N.dh_workspace_bytes(0, 5, p) == 0
    assert N.dh_workspace_bytes(5, 40000, p) == 0
    assert N.dh_workspace_bytes(4, 4, p.replace(patch=4)) == 0
    assert N.dh_workspace_bytes(4, 4, p.replace(radius=3)) == 0
    assert N.dh_workspace_bytes(4, 4, p.replace(eps=0.0)) == 0
    assert N.dh_workspace_bytes(4, 4, p.replace(boundary=2)) == 0
    assert N.dh_workspace_bytes(4, 4, None) > 0


def test_invalid_arguments_rejected_on_host():
    p = N.dh_params_default(N.DH_PRESET_STABLE)
    fake = 1 << 20  # never dereferenced: every call below fails validation first
    assert N.dh_dark_channel(fake, 8, 8, 4, None, fake) == N.DH_EINVAL
    assert N.dh_dark_channel(None, 8, 8, 15, None, fake) == N.DH_EINVAL
    assert N.dh_dark_channel(fake, 0, 8, 15, None, fake) == N.DH_EINVAL
    assert N.dh_transmission(fake, fake, 8, 8, p.replace(omega=2.0), None, fake, fake, fake) == N.DH_EINVAL
    assert N.dh_fixed_point(fake, fake, fake, 8, 8, p, None, None, 0) == N.DH_EWORKSPACE
    assert N.dh_fixed_point(fake, fake, fake, 8, 8, p, None, fake + 8, 1 << 30) == N.DH_EWORKSPACE
    assert N.dh_fixed_point(fake, fake, fake, 8, 8, p.replace(max_iter=-1), None, fake, 1 << 30) == N.DH_EINVAL
    assert N.dh_dehaze(fake, 8, 8, p, None, fake, fake, fake, fake, fake, 16) == N.DH_EWORKSPACE
    assert N.dh_dehaze(fake, 8, 8, p.replace(storage=9), None, fake, fake, fake, fake, fake, 1 << 30) == N.DH_EINVAL
    assert N.dh_atmospheric_light(fake, fake, 8, 8, 0, fake, None, fake, 1 << 30) == N.DH_EINVAL
    img = N.dh_image(fake, 8, 8, None, fake, fake, fake, fake)
    assert N.dh_batch_workspace_bytes(1, [img], p) > 0
    assert N.dh_batch_workspace_bytes(1, [N.dh_image(fake, 0, 8, None, fake, fake, fake, fake)], p) == 0
    assert N.dh_dehaze_batch(1, [img], p, None, 0) == N.DH_EWORKSPACE
    assert N.dh_dehaze_batch(1, [N.dh_image(None, 8, 8, None, fake, fake, fake, fake)], p, fake, 1 << 30) == N.DH_EINVAL
    assert N.dh_dehaze_batch(1, [img], p.replace(storage=9), fake, 1 << 30) == N.DH_EINVAL
    assert N.dh_sweep_variants() >= 2
    assert N.dh_workspace_bytes(4, 4, p.replace(sweep_variant=N.dh_sweep_variants())) == 0
    assert N.dh_tune(fake, fake, fake, 8, 8, p, 0, fake, 1 << 30) == N.DH_EINVAL
    assert N.dh_tune_set(8, 8, 0, 999) == N.DH_EINVAL


def test_batch_net_workspace_groups_by_shape():
    """dh_dehaze_batch_warm runs one network forward per group of same-shape
    images (up to about 4.2 million pixels a group): its workspace is the
    largest group's gathered inputs (I and Phi 3HW, t HW floats, A 3 floats per
    image, none for a group of one) plus that group's network workspace."""
    fake = 1 << 20

    def img(H, W):
        return N.dh_image(fake, H, W, None, fake, fake, fake, fake)

    def gathered(n, H, W):
        al = lambda b: (b + 255) // 256 * 256
        return 2 * al(n * 3 * H * W * 4) + al(n * H * W * 4) + al(n * 12) if n > 1 else 0

    def net(n, H, W):
        return N.dh_unet_workspace_bytes(32, n, H, W, 0)

    a, b = (64, 128), (56, 96)
    assert N.dh_batch_net_workspace_bytes(32, 1, [img(*a)]) == net(1, *a)
    assert N.dh_batch_net_workspace_bytes(32, 2, [img(*a), img(*b)]) == max(net(1, *a), net(1, *b))
    assert N.dh_batch_net_workspace_bytes(32, 5, [img(*a), img(*b), img(*a), img(*b), img(*a)]) == max(
        gathered(3, *a) + net(3, *a), gathered(2, *b) + net(2, *b))
    # 1080p: two images a group, so a third image adds nothing
    hd = (1080, 1920)
    two = N.dh_batch_net_workspace_bytes(32, 2, [img(*hd)] * 2)
    assert two == gathered(2, *hd) + net(2, *hd)
    assert N.dh_batch_net_workspace_bytes(32, 3, [img(*hd)] * 3) == two
    # 64 images a group at most
    tiny = (16, 16)
    assert N.dh_batch_net_workspace_bytes(32, 70, [img(*tiny)] * 70) == gathered(64, *tiny) + net(64, *tiny)
    assert N.dh_batch_net_workspace_bytes(32, 1, [img(60, 100)]) == 0  # sides not multiples of 8
    assert N.dh_batch_net_workspace_bytes(24, 1, [img(*a)]) == 0  # no such network


def test_semi_implicit_arguments_rejected_on_host():
    p = N.dh_params_default(N.DH_PRESET_PAPER)
    fake = 1 << 20  # never dereferenced
    b = N.dh_semi_implicit_workspace_bytes(64, 96)
    assert b >= 4 * 3 * 64 * 96 * 6 and b < 4 * 3 * 64 * 96 * 9 + (1 << 20)
    assert N.dh_semi_implicit_workspace_bytes(0, 96) == 0
    args = (fake, None, fake, fake, 64, 96)
    assert N.dh_semi_implicit(*args, p, 0.0, 16, None, None, fake, b) == N.DH_EINVAL
    assert N.dh_semi_implicit(*args, p, float("nan"), 16, None, None, fake, b) == N.DH_EINVAL
    assert N.dh_semi_implicit(*args, p, 2.0, 0, None, None, fake, b) == N.DH_EINVAL
    assert N.dh_semi_implicit(*args, p.replace(storage=1), 2.0, 16, None, None, fake, b) == N.DH_EINVAL
    assert N.dh_semi_implicit(*args, p.replace(eps=0.0), 2.0, 16, None, None, fake, b) == N.DH_EINVAL
    assert N.dh_semi_implicit(*args, p, 2.0, 16, None, None, fake, b - 1) == N.DH_EWORKSPACE
    assert N.dh_semi_implicit(*args, p, 2.0, 16, None, None, fake + 8, b) == N.DH_EWORKSPACE
    assert N.dh_semi_implicit(None, None, fake, fake, 64, 96, p, 2.0, 16, None, None, fake, b) == N.DH_EINVAL


def test_refinement_parameters_validated_on_host():
    p = N.dh_params_default(N.DH_PRESET_STABLE)
    fake = 1 << 20  # never dereferenced
    assert N.dh_workspace_bytes(64, 64, p.replace(dc_scales=2)) == 0
    assert N.dh_workspace_bytes(64, 64, p.replace(dc_scales=3, patch=17)) == 0
    assert N.dh_workspace_bytes(64, 64, p.replace(gf_radius=25)) == 0
    assert N.dh_workspace_bytes(64, 64, p.replace(gf_radius=4, gf_eps=0.0)) == 0
    plain = N.dh_workspace_bytes(64, 64, p)
    assert N.dh_workspace_bytes(64, 64, p.replace(dc_scales=3, gf_radius=4)) > plain
    # the workspace-free call cannot hold the refinements' scratch
    assert N.dh_transmission(fake, fake, 8, 8, p.replace(gf_radius=4), None, fake, fake, fake) == N.DH_EINVAL
    assert N.dh_transmission_ws(fake, fake, 8, 8, p.replace(gf_radius=4), None, fake, fake, fake, None, 0) == \
        N.DH_EWORKSPACE
