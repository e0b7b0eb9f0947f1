"""The oracle's optimisation loop (Section 3.1, Figure 5) on small grids."""
import numpy as np

from oracle import design, loop
from paper_2210_00947_gb300 import workloads


def _settings(**kw):
    base = dict(nx=24, ny=24, nz=0, volfrac=0.4, iters=12, n_on=3, nl=3, eps2=1e-10)
    base.update(kw)
    return loop.LoopSettings(**base)


def test_loop_descends_and_keeps_volume():
    s = _settings()
    fixed = workloads.heat_sink_mask(s.nx, s.ny)
    q = workloads.nodal_load(fixed)
    rho, t, hist = loop.optimise(s, fixed, q, np.full(s.nx * s.ny, 0.4))
    c = [h["compliance"] for h in hist]
    assert c[-1] < 0.5 * c[0]
    an = loop.Analysis(s, fixed, q)
    assert abs(design.filter_forward(an.H, an.Hs, rho).mean() - 0.4) < 1e-11
    assert all(h["mgcg"] for h in hist[: s.n_on - 1])


def test_rejecting_every_mgar_reproduces_mgcg():
    """eps1 = 0 rejects every reanalysis, so the loop equals pure MGCG."""
    fixed = workloads.heat_sink_mask(16, 16)
    q = workloads.nodal_load(fixed)
    rho0 = np.full(256, 0.4)
    r1, t1, h1 = loop.optimise(_settings(nx=16, ny=16, iters=6, eps1=0.0), fixed, q, rho0)
    r2, t2, h2 = loop.optimise(_settings(nx=16, ny=16, iters=6, use_mgar=False), fixed, q, rho0)
    np.testing.assert_allclose(r1, r2, rtol=0, atol=0)
    assert all(h["mgcg"] for h in h1)


def test_accepted_reanalysis_is_close():
    s = _settings(nx=32, ny=32, iters=20, n_on=8, eps1=0.5, basis_guess="zero")
    fixed = workloads.heat_sink_mask(s.nx, s.ny)
    q = workloads.nodal_load(fixed)
    rho, t, hist = loop.optimise(s, fixed, q, np.full(s.nx * s.ny, 0.4))
    acc = [h for h in hist if h["accepted"]]
    assert len(acc) > 0
    assert all(h["res"] <= 0.5 for h in acc)


def test_continuous_filter_schedule_in_the_loop():
    """With the continuous filter (Eq. 22-23) cycle k filters with radius
    r^(k): the filter the loop holds after cycle k is the filter of that
    radius, and once the radius has reached r_min the loop equals the plain
    filter's loop started from the same design."""
    s = _settings(nx=20, ny=20, iters=5, n_on=6, filter_alpha=0.2, filter_lp=3)
    fixed = workloads.heat_sink_mask(s.nx, s.ny)
    q = workloads.nodal_load(fixed)
    an = loop.Analysis(s, fixed, q)
    rho = np.full(s.nx * s.ny, 0.4)
    t = np.zeros(an.grid.n_nodes)
    radii = []
    for k in range(1, s.iters + 1):
        rho, t, _ = an.cycle(k, rho, t)
        radii.append(an.r)
        H, Hs = design.filter_matrix(an.grid, an.r)
        assert abs(H - an.H).max() == 0.0
    assert radii[0] < 4.0 and radii[0] > radii[1] > 1.5
    assert radii[2] == radii[3] == radii[4] == 1.5 or abs(radii[2] - 1.5) < 1e-12
    # from the cycle after r reached r_min on, the plain loop continues identically
    plain = loop.Analysis(_settings(nx=20, ny=20, iters=5, n_on=6), fixed, q)
    r_a, t_a, _ = an.cycle(6, rho, t)
    r_b, t_b, _ = plain.cycle(6, rho, t)
    np.testing.assert_array_equal(r_a, r_b)
