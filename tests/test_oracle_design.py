"""Pins for the oracle's filter, sensitivities and OC update (Eq. 5-11)."""
import numpy as np
import pytest

from oracle import design, fem, solvers


@pytest.mark.parametrize("dims,r", [((7, 5, 0), 1.5), ((5, 4, 3), 1.5), ((9, 8, 0), 3.0)])
def test_filter_preserves_constants_and_is_adjoint(dims, r):
    g = fem.Grid(*dims)
    H, Hs = design.filter_matrix(g, r)
    np.testing.assert_allclose(design.filter_forward(H, Hs, np.full(g.n_elems, 0.37)), 0.37,
                               rtol=1e-15)
    rng = np.random.default_rng(10)
    x, y = rng.standard_normal((2, g.n_elems))
    lhs = design.filter_forward(H, Hs, x) @ y
    rhs = x @ design.filter_transpose(H, Hs, y)
    assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + 1)
    Hd = H.toarray()
    np.testing.assert_allclose(Hd, Hd.T, atol=0)


def test_filter_weights_rmin_1p5():
    """r = 1.5: centroid distances 0, 1, sqrt2 are inside (weights 1.5, 0.5,
    1.5 - sqrt2); sqrt3 and 2 are outside; 9 / 19 neighbours in 2D / 3D."""
    for dims, count in (((5, 5, 0), 9), ((5, 5, 5), 19)):
        g = fem.Grid(*dims)
        H, _ = design.filter_matrix(g, 1.5)
        centre = g.n_elems // 2
        row = H.getrow(centre).toarray().reshape(-1)
        nz = row[row != 0]
        assert nz.size == count
        assert set(np.round(nz, 12)) == {1.5, 0.5, round(1.5 - np.sqrt(2), 12)}
        cen = g.element_centroids()
        d = np.linalg.norm(cen - cen[centre], axis=1)
        np.testing.assert_allclose(row, np.maximum(0.0, 1.5 - d), atol=1e-15)


def test_filter_boundary_normalisation():
    """A corner element of a 2D grid has itself, two edge neighbours and
    one diagonal neighbour in range."""
    g = fem.Grid(4, 4, 0)
    H, Hs = design.filter_matrix(g, 1.5)
    assert abs(Hs[0] - (1.5 + 2 * 0.5 + (1.5 - np.sqrt(2)))) < 1e-15


def _compliance(g, H, Hs, rho, fixed, q):
    rho_phys = design.filter_forward(H, Hs, rho)
    A = fem.system_matrix(g, rho_phys, fixed)
    return q @ solvers.exact_solve(A, q)


@pytest.mark.parametrize("dims", [(8, 6, 0), (4, 4, 3)])
def test_sensitivities_match_finite_differences(dims):
    g = fem.Grid(*dims)
    H, Hs = design.filter_matrix(g, 1.5)
    rng = np.random.default_rng(11)
    rho = rng.uniform(0.2, 0.9, g.n_elems)
    fixed = np.zeros(g.n_nodes, np.uint8)
    fixed[0] = fixed[g.NX] = 1
    q = np.where(fixed != 0, 0.0, 0.01)
    rho_phys = design.filter_forward(H, Hs, rho)
    t = solvers.exact_solve(fem.system_matrix(g, rho_phys, fixed), q)
    dc, dv = design.sensitivities(g, H, Hs, rho_phys, t)
    h = 1e-5
    for e in rng.choice(g.n_elems, 6, replace=False):
        rp, rm = rho.copy(), rho.copy()
        rp[e] += h
        rm[e] -= h
        fd = (_compliance(g, H, Hs, rp, fixed, q) - _compliance(g, H, Hs, rm, fixed, q)) / (2 * h)
        assert abs(fd - dc[e]) < 1e-6 * abs(dc).max()
    assert np.all(dc <= 0.0)
    # dv is the gradient of mean(F rho): it sums to one and matches F^T(1/n)
    assert abs(dv.sum() - 1.0) < 1e-14
    x = rng.standard_normal(g.n_elems)
    assert abs(dv @ x - design.filter_forward(H, Hs, x).mean()) < 1e-14


@pytest.mark.parametrize("dims", [(10, 8, 0), (5, 4, 4)])
def test_oc_keeps_volume_and_limits(dims):
    g = fem.Grid(*dims)
    H, Hs = design.filter_matrix(g, 1.5)
    rng = np.random.default_rng(12)
    rho = rng.uniform(0.1, 0.7, g.n_elems)
    dc = -rng.uniform(0.0, 2.0, g.n_elems)
    _, dv = design.sensitivities(g, H, Hs, rho, np.zeros(g.n_nodes))
    vol = 0.4
    rn, lam = design.oc_update(rho, dc, dv, vol, move=0.2)
    assert abs(design.filter_forward(H, Hs, rn).mean() - vol) < 1e-12
    assert np.all(rn >= np.maximum(0, rho - 0.2) - 1e-15)
    assert np.all(rn <= np.minimum(1, rho + 0.2) + 1e-15)
    # the unclamped elements follow rho * sqrt(-dc / (lambda dv))
    raw = rho * np.sqrt(-dc / (lam * dv))
    inside = (raw > rho - 0.2 + 1e-9) & (raw < rho + 0.2 - 1e-9) & (raw < 1 - 1e-9) & (raw > 1e-9)
    np.testing.assert_allclose(rn[inside], raw[inside], rtol=1e-14)


def test_filter_radius_schedule_eq22_23():
    """Eq. 22-23: r starts at alpha L, shrinks geometrically by eta per cycle
    and reaches r_min after lp cycles; the recursion with max() equals the
    closed form max(r_min, (alpha L) eta^k)."""
    import math
    rmin, alpha, L, lp = 3.0, 1.4 / 50, 480.0, 250
    r0 = alpha * L
    eta = math.exp((math.log(rmin) - math.log(r0)) / lp)
    assert abs(eta ** lp * r0 - rmin) < 1e-12
    prev = r0
    for k in range(1, 301):
        r = design.filter_radius(k, rmin, alpha, L, lp)
        assert r <= prev + 1e-15 and r >= rmin
        assert abs(r - max(rmin, r0 * eta ** k)) < 1e-11 * r0
        prev = r
    assert abs(design.filter_radius(lp, rmin, alpha, L, lp) - rmin) < 1e-11
    assert design.filter_radius(lp + 1, rmin, alpha, L, lp) == rmin
    assert design.filter_radius(300, rmin, alpha, L, lp) == rmin
    # nothing to shrink: alpha L below r_min
    assert design.filter_radius(5, 3.0, 0.01, 100.0, 10) == 3.0
