"""Pins of the oracle's gridder (Section 6: each visibility convolved with a
compact gridding convolution function, zero beyond r_max; reading R18: a radial
function given as a table, linearly interpolated).

Independent of the oracle's scatter loop: a dense numpy gather over every
(pixel, visibility) pair with numpy's own interpolation, exact counts for a
top-hat function, translation, linearity and conjugation invariants, the
grid's edge rule, and the sum over pixels of a smooth function against its
continuous integral.
"""
import numpy as np
import pytest

import oracle


def kaiser_bessel(n_tab, beta=8.0):
    r = np.linspace(0.0, 1.0, n_tab)
    return np.i0(beta * np.sqrt(np.clip(1.0 - r * r, 0.0, None))) / np.i0(beta)


def dense_gather(n_pix, r_max, gcf, xy, vis):
    """Every pixel against every visibility (numpy broadcasting, np.interp)."""
    vis = vis.reshape(len(xy), -1)
    inside = (xy[:, 0] >= 0) & (xy[:, 0] < n_pix) & (xy[:, 1] >= 0) & (xy[:, 1] < n_pix)
    py, px = np.mgrid[0:n_pix, 0:n_pix]
    d = np.hypot(px[..., None] - xy[:, 0], py[..., None] - xy[:, 1])          # [y][x][vis]
    w = np.where((d < r_max) & inside, np.interp(d, np.linspace(0, r_max, len(gcf)), gcf), 0.0)
    return np.einsum("yxi,ip->pyx", w, vis)


def case(n_pix=40, n_vis=60, n_pol=2, seed=1):
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-2.0, n_pix + 2.0, size=(n_vis, 2))
    vis = rng.normal(size=(n_vis, n_pol)) + 1j * rng.normal(size=(n_vis, n_pol))
    return xy, vis


@pytest.mark.parametrize("r_max", [2.5, 6.0])
def test_grid_equals_dense_gather(r_max):
    xy, vis = case()
    gcf = kaiser_bessel(33)
    G = oracle.grid(40, r_max, gcf, xy, vis)
    np.testing.assert_allclose(G, dense_gather(40, r_max, gcf, xy, vis), rtol=0, atol=1e-12)


def test_top_hat_counts_visibilities_in_range():
    xy, _ = case(n_vis=80, n_pol=1, seed=2)
    G = oracle.grid(40, 4.0, np.ones(5), xy, np.ones((80, 1)))
    inside = (xy[:, 0] >= 0) & (xy[:, 0] < 40) & (xy[:, 1] >= 0) & (xy[:, 1] < 40)
    count = np.zeros((40, 40))
    for (x, y), ok in zip(xy, inside):
        if ok:
            for py in range(40):
                for px in range(40):
                    count[py, px] += (px - x) ** 2 + (py - y) ** 2 < 16.0
    np.testing.assert_array_equal(G[0].real, count)
    assert np.all(G[0].imag == 0)


def test_translation_linearity_and_conjugation():
    rng = np.random.default_rng(3)
    xy = rng.uniform(10.0, 25.0, size=(30, 2))
    v1 = rng.normal(size=(30, 1)) + 1j * rng.normal(size=(30, 1))
    v2 = rng.normal(size=(30, 1)) + 1j * rng.normal(size=(30, 1))
    gcf = kaiser_bessel(17)
    G1 = oracle.grid(48, 5.0, gcf, xy, v1)
    shifted = oracle.grid(48, 5.0, gcf, xy + np.array([3.0, -2.0]), v1)
    np.testing.assert_allclose(shifted[:, :-2, 3:], G1[:, 2:, :-3], rtol=0, atol=1e-13)
    a, b = 0.3 - 1.2j, 2.0 + 0.5j
    np.testing.assert_allclose(oracle.grid(48, 5.0, gcf, xy, a * v1 + b * v2),
                               a * G1 + b * oracle.grid(48, 5.0, gcf, xy, v2), rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.grid(48, 5.0, gcf, xy, np.conj(v1)), np.conj(G1), rtol=0, atol=0)


def test_edge_rule():
    gcf = np.ones(3)
    out = oracle.grid(16, 3.0, gcf, np.array([[-0.5, 8.0]]), np.ones((1, 1)))
    assert np.all(out == 0)                      # outside the grid: not gridded
    inn = oracle.grid(16, 3.0, gcf, np.array([[15.99, 8.0]]), np.ones((1, 1)))
    assert inn[0, 8, 15] == 1 and inn[0, 8, 13] == 1 and inn[0, 8, 12] == 0


def test_pixel_sum_approximates_the_integral():
    """Sum over pixel centres of a smooth radial function ~ its integral
    int f(r) 2 pi r dr (the midpoint rule on the unit pixel lattice)."""
    rm = 12.0
    gcf = kaiser_bessel(2049, beta=6.0)
    r = np.linspace(0.0, rm, 200001)
    f = np.interp(r, np.linspace(0, rm, len(gcf)), gcf)
    integral = np.sum(0.5 * (f[1:] * r[1:] + f[:-1] * r[:-1]) * np.diff(r)) * 2 * np.pi
    rng = np.random.default_rng(4)
    for x, y in rng.uniform(20.0, 21.0, size=(3, 2)):
        G = oracle.grid(48, rm, gcf, np.array([[x, y]]), np.ones((1, 1)))
        assert abs(G.real.sum() - integral) <= 1e-3 * integral
