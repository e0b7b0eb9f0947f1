"""Pins for the post-processing oracle (Eq. 24-27): cases whose result
follows from the definitions by hand."""
import numpy as np
import pytest

from oracle import fem, postprocess as pp


def test_projection_keeps_constants_and_weights():
    g = fem.Grid(7, 5)
    ns = pp.nodal_projection(g, np.full(g.n_elems, 3.25), 1.5)
    np.testing.assert_allclose(ns, 3.25, rtol=0, atol=1e-15)
    # an interior node with r = 1: only the four elements sharing it, each at
    # distance sqrt(2)/2, equal weights -> the plain mean
    s = np.arange(g.n_elems, dtype=float)
    ns = pp.nodal_projection(g, s, 1.0)
    i, j = 3, 2
    elems = [(i - 1) + 7 * (j - 1), i + 7 * (j - 1), (i - 1) + 7 * j, i + 7 * j]
    assert abs(ns[i + 8 * j] - s[elems].mean()) < 1e-12


def test_shape_functions_interpolate_corners():
    for dim in (2, 3):
        N = pp.lattice_shape_values(dim)
        assert N.shape == (5 ** dim, 2 ** dim)
        np.testing.assert_allclose(N.sum(axis=1), 1.0, atol=1e-15)
        corner_rows = [r for r in range(N.shape[0]) if np.isclose(N[r].max(), 1.0)]
        assert len(corner_rows) == 2 ** dim


@pytest.mark.parametrize("frac,expected", [(0.1, 0.8), (0.3, 0.6), (0.6, 0.4), (0.9, 0.2)])
def test_linear_field_gives_exact_lattice_shares(frac, expected):
    """ns = x: the element spanning [2, 3] with level 2 + frac keeps the
    lattice columns x = 2 + m/4 > level (bilinear interpolation of a linear
    field is exact), so ev is their share; elements right of it are solid,
    left of it void."""
    g = fem.Grid(6, 3)
    x = np.tile(np.arange(7, dtype=float), 4)
    rho = pp.densities(g, x, 2.0 + frac)
    rho = rho.reshape(3, 6)
    np.testing.assert_array_equal(rho[:, :2], 0.0)
    np.testing.assert_array_equal(rho[:, 3:], 1.0)
    np.testing.assert_allclose(rho[:, 2], expected)


def test_level_keeps_the_volume_and_is_tight():
    rng = np.random.default_rng(3)
    g = fem.Grid(12, 10)
    ns = pp.nodal_projection(g, rng.random(g.n_elems), 1.5)
    vf = 0.45
    level, rho = pp.level_for_volume(g, ns, vf)
    assert rho.mean() <= vf
    # a slightly lower level already exceeds the volume fraction
    below = pp.densities(g, ns, level - 1e-9 * (abs(level) + 1)).mean()
    assert below > vf or below == rho.mean()
    # densities are shares of the 25 lattice points
    np.testing.assert_allclose(rho * 25, np.round(rho * 25), atol=1e-12)
