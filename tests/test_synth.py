"""The seeded input generators shared by both sides (host only): each is
deterministic in its seed and draws the distribution and block structure its
docstring states (the input recipe of the workloads)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402


@pytest.mark.parametrize("kind", ["gaussian", "laplace", "uniform"])
def test_iid_deterministic_and_seed_sensitive(kind):
    a = synth.iid(kind, (64, 48), 5, np.float32)
    b = synth.iid(kind, (64, 48), 5, np.float32)
    c = synth.iid(kind, (64, 48), 6, np.float32)
    assert a.dtype == np.float32 and a.shape == (64, 48)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_iid_moments():
    n = (512, 512)
    g = synth.gaussian(n, 1)
    lp = synth.laplace(n, 2)
    u = synth.uniform(n, 3)
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1.0) < 0.02
    assert abs(lp.mean()) < 0.01 and abs(lp.var() - 2.0) < 0.05          # 2 b^2, b = 1
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.var() - 1.0 / 3.0) < 0.01


def test_int_uniform_range():
    x = synth.int_uniform((200, 200), 4, 127)
    assert np.all(x == np.rint(x)) and x.min() == -127 and x.max() == 127


def test_blockwise_range_uniform_block_maxima():
    L = 32
    x = synth.blockwise_range_uniform((128, 96), 7, L, emin=4, emax=2048)
    for i in range(0, 128, L):
        for j in range(0, 96, L):
            m = np.abs(x[i:i + L, j:j + L]).max()
            assert 0.9 * 4 <= m <= 2048          # |u| max near 1 over 1024 draws


def test_blockwise_crest_blocks_differ_in_shape():
    L = 64
    x = synth.blockwise_crest((256, 256), 8, L)
    crest = []
    for i in range(0, 256, L):
        for j in range(0, 256, L):
            b = x[i:i + L, j:j + L]
            crest.append(np.abs(b).max() / np.sqrt((b * b).mean()))
    assert min(crest) < 2.0 < 4.0 < max(crest)   # uniform blocks ~1.7, k = 11 blocks far larger


def test_eigenface_pixels_mean_removed_integers():
    x = synth.eigenface_pixels(300, 40, 9, np.float64)
    assert np.allclose(x.mean(axis=1), 0.0, atol=1e-9)
    # removing a row's mean shifts it: integer steps and a span of at most 255 remain
    assert np.all(x.max(axis=1) - x.min(axis=1) <= 255)
    d = x - x[:, :1]
    assert np.allclose(d, np.rint(d))


def test_faces_2dpca_shape_and_range():
    f = synth.faces_2dpca(3, 4, 32, 7)
    assert f.shape == (3, 4, 32, 32)
    assert f.min() >= 0 and f.max() <= 255 and np.all(f == np.rint(f))


def test_sample_tiles_distinct_in_range():
    t = synth.sample_tiles(32, 32, 10, seed=1)
    assert len(set(t)) == 10
    assert all(0 <= i < 32 and 0 <= j < 32 for i, j in t)
    assert t == synth.sample_tiles(32, 32, 10, seed=1)
