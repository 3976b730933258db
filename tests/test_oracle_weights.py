"""Pins for the per-column integration weights of irregular geometries (Voronoi areas).

The weights multiply the kernel's columns (the integration points x_R).  A one-hot weight
must reduce the MDC to the single-column convolution, a uniform weight to a plain scaling,
and the Voronoi areas of any point set must tile the survey square.
"""
import numpy as np

import synth
from oracle import mdc


def rand(nt=32, nf=9, nr=4, ns=5, nv=2, seed=0):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((nf, nr, ns)) + 1j * rng.standard_normal((nf, nr, ns))
    x = rng.standard_normal((nt, ns, nv))
    return G, x


def test_one_hot_weight_keeps_only_that_column():
    G, x = rand()
    for j in range(G.shape[2]):
        w = np.zeros(G.shape[2])
        w[j] = 1.0
        y = mdc.forward(mdc.weighted_kernel(G, w), x, 0.004, 1.0)
        y1 = mdc.forward(G[:, :, j:j + 1], x[:, j:j + 1], 0.004, 1.0)
        assert np.allclose(y, y1, rtol=0, atol=1e-12 * np.abs(y1).max())
    # a row weight instead (a transposed reading) would not reduce to one column
    w = np.zeros(G.shape[2]); w[0] = 1.0
    wrong = mdc.forward(G * np.eye(G.shape[1], 1)[None, :, :], x, 0.004, 1.0)
    assert not np.allclose(wrong, mdc.forward(mdc.weighted_kernel(G, w), x, 0.004, 1.0))


def test_uniform_weight_is_the_scalar_areal_weight():
    G, x = rand(seed=2)
    y = mdc.forward(mdc.weighted_kernel(G, np.full(G.shape[2], 400.0)), x, 0.004, 1.0)
    assert np.allclose(y, mdc.forward(G, x, 0.004, 400.0), rtol=1e-13, atol=0)


def test_voronoi_areas_tile_the_square_and_match_a_regular_grid():
    xy = synth.grid_xy(9)
    lo, hi = -0.5 * synth.GRID_DX, synth.GRID_DX * 8.5
    a = synth.voronoi_areas(xy, lo, hi, res=720)
    assert abs(a.sum() - (hi - lo) ** 2) <= 1e-9 * (hi - lo) ** 2
    assert np.allclose(a, synth.GRID_DX ** 2, rtol=0.03)
    idx = synth.irregular_subset(9, 0.5, seed=1)
    b = synth.voronoi_areas(xy[idx], lo, hi, res=720)
    assert abs(b.sum() - (hi - lo) ** 2) <= 1e-9 * (hi - lo) ** 2 and b.min() > 0
