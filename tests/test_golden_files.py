"""The stored FP64 oracle values in tests/golden/ (written by
tests/golden/make_fixed_points.py, which calls only oracle/): their sample
positions regenerate from the counter-based generator, their iteration counts
and residuals are those of the stop rule, and the 1080p file's atmospheric
light is what the oracle's front end gives for that scene today."""
import importlib.util
import os

import numpy as np
import pytest

from paper_2506_08793_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def maker():
    spec = importlib.util.spec_from_file_location("make_fixed_points", os.path.join(GOLDEN, "make_fixed_points.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_1080p_file(orc):
    g = dict(np.load(os.path.join(GOLDEN, "fp_1080p_seed2000.npz")))
    H, W, seed = int(g["H"]), int(g["W"]), int(g["seed"])
    assert (H, W, seed) == (1080, 1920, 2000) and float(g["tol"]) == 1e-4
    ys, xs = maker().sample_positions(seed, H, W, 16384)
    assert np.array_equal(ys, g["ys"]) and np.array_equal(xs, g["xs"])
    assert g["u"].shape == (3, 16384) and np.isfinite(g["u"]).all()
    assert np.max(g["rho"]) <= 1e-4 and 500 < int(g["n"]) < 2000
    I = scenes.hazy_scene(seed, H, W)["I"]
    op = orc.params(**orc.STABLE)
    A, idx, _ = orc.atmospheric_light(I, orc.dark_channel(I, op.patch, None), op.topk_permille)
    assert idx == int(g["a_index"]) and np.array_equal(A, g["A"])


def test_4k_file():
    g = dict(np.load(os.path.join(GOLDEN, "fp_4k_seed2001_n64.npz")))
    H, W, seed = int(g["H"]), int(g["W"]), int(g["seed"])
    assert (H, W, seed, int(g["n"])) == (2160, 3840, 2001, 64)
    ys, xs = maker().sample_positions(seed, H, W, 16384)
    assert np.array_equal(ys, g["ys"]) and np.array_equal(xs, g["xs"])
    assert g["u"].shape == (3, 16384) and np.isfinite(g["u"]).all()


def test_batch_file():
    g = dict(np.load(os.path.join(GOLDEN, "fp_batch64_subset.npz")))
    sizes = scenes.batch_sizes(3000, 64)
    assert list(g["k"]) == list(range(0, 64, 4))
    m = maker()
    for i, k in enumerate(g["k"]):
        H, W = sizes[int(k)]
        assert (int(g["H"][i]), int(g["W"][i])) == (H, W)
        ys, xs = m.sample_positions(3000 + int(k), H, W, 4096)
        assert np.array_equal(ys, g["ys"][i]) and np.array_equal(xs, g["xs"][i])
        assert np.max(g["rho1"][i]) <= 1e-4 and np.max(g["rho2"][i]) <= 1e-5
        assert int(g["n2"][i]) > int(g["n1"][i]) > 0
        # continuing from the tol-1e-4 stop moves u by less than the solution's size
        assert np.max(np.abs(g["u2"][i] - g["u1"][i])) < 0.1 * np.max(np.abs(g["u1"][i]))


@pytest.mark.parametrize("name", ["fp_1080p_seed2000.npz", "fp_4k_seed2001_n64.npz", "fp_batch64_subset.npz"])
def test_files_are_small(name):
    assert os.path.getsize(os.path.join(GOLDEN, name)) < 4 << 20
