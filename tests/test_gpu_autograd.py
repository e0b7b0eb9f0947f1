"""The compliance autograd function: its gradient is the oracle's
sensitivity (Eq. 9-11) and matches central finite differences of the
compliance it returns."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import design, fem, solvers  # noqa: E402
from paper_2210_00947_gb300 import autograd, mgar, workloads  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _problem(nx, ny, nz):
    fixed = workloads.heat_sink_mask(nx, ny, nz)
    q = workloads.nodal_load(fixed)
    ne = workloads.num_elements(nx, ny, nz)
    rho = workloads.random_density(ne, 0.2, 0.9, seed=11)
    return fixed, q, rho


@pytest.mark.parametrize("dims,nl", [((40, 32, 0), 3), ((12, 10, 8), 3)])
def test_gradient_is_the_oracle_sensitivity(dims, nl):
    nx, ny, nz = dims
    fixed, q, rho = _problem(nx, ny, nz)
    p = mgar.default_params(nx=nx, ny=ny, nz=nz, nl=nl, eps2=1e-12, cg_max=500)
    comp = autograd.Compliance(p, fixed, q)
    r = torch.tensor(rho, device=DEV, requires_grad=True)
    c = comp(r)
    c.backward()
    g = fem.Grid(nx, ny, nz)
    H, Hs = design.filter_matrix(g, p.rmin)
    rho_phys = design.filter_forward(H, Hs, rho)
    A = fem.system_matrix(g, rho_phys, fixed)
    t = solvers.exact_solve(A, q)
    dc, _ = design.sensitivities(g, H, Hs, rho_phys, t, p.k0, p.kmin, p.penal)
    assert abs(c.item() - q @ t) / (q @ t) < 1e-10
    np.testing.assert_allclose(r.grad.cpu().numpy(), dc, rtol=1e-8, atol=1e-10 * np.abs(dc).max())
    comp.close()


def test_gradient_matches_finite_differences():
    nx, ny = 24, 24
    fixed, q, rho = _problem(nx, ny, 0)
    p = mgar.default_params(nx=nx, ny=ny, nz=0, nl=3, eps2=1e-13, cg_max=500)
    comp = autograd.Compliance(p, fixed, q)
    r = torch.tensor(rho, device=DEV, requires_grad=True)
    c = comp(r)
    c.backward()
    grad = r.grad.cpu().numpy()
    rng = np.random.default_rng(5)
    h = 1e-5
    for _ in range(3):
        v = rng.standard_normal(rho.size)
        cp = comp(torch.tensor(rho + h * v, device=DEV)).item()
        cm = comp(torch.tensor(rho - h * v, device=DEV)).item()
        fd = (cp - cm) / (2 * h)
        assert abs(fd - grad @ v) < 1e-6 * abs(grad @ v)
    comp.close()


def test_set_load_solves_for_another_right_hand_side():
    """mgar_set_load replaces q for the next solves; setting the original
    load back restores the original solution."""
    nx, ny, nz = 20, 18, 16
    fixed, q, rho = _problem(nx, ny, nz)
    p = mgar.default_params(nx=nx, ny=ny, nz=nz, nl=3, eps2=1e-11, cg_max=500,
                            precision=mgar.MGAR_MIXED)
    g = fem.Grid(nx, ny, nz)
    H, Hs = design.filter_matrix(g, p.rmin)
    A = fem.system_matrix(g, design.filter_forward(H, Hs, rho), fixed)
    q2 = np.random.default_rng(3).uniform(-1.0, 1.0, g.n_nodes)
    q2[fixed != 0] = 7.0  # ignored: fixed rows are eliminated
    q2_free = np.where(fixed != 0, 0.0, q2)
    with mgar.Solver(p, fixed, q) as s:
        s.set_density(torch.tensor(rho, device=DEV))
        for load, ref in ((q2, q2_free), (q, q)):
            s.set_load(torch.tensor(load, device=DEV))
            T = torch.zeros(g.n_nodes, dtype=torch.float64, device=DEV)
            it, rr, ok = s.solve_mgcg(T)
            assert ok
            t = T.cpu().numpy()
            t_ex = solvers.exact_solve(A, ref)
            assert np.linalg.norm(t - t_ex) / np.linalg.norm(t_ex) < 1e-8
            assert abs(s.sensitivity(T) - ref @ t) <= 1e-12 * abs(ref @ t) + 1e-300


# The differentiation workload at full size: 256^3 H8 elements (16,974,593
# nodes), i.i.d. densities U[0.05, 1] from SplitMix64(2210), the centred sink
# patch of the 128^3 workload, mixed path.
C5 = "heat3d_256"


@pytest.fixture(scope="module")
def c5_gradient():
    w = workloads.WORKLOADS[C5]
    fixed, q = w.fixed(), w.q()
    rho = workloads.random_density(w.n_elems, 0.05, 1.0, seed=2210)
    p = mgar.params_for(w, precision=mgar.MGAR_MIXED, eps2=1e-11, cg_max=500)
    comp = autograd.Compliance(p, fixed, q)
    r = torch.tensor(rho, device=DEV, requires_grad=True)
    c = comp(r)
    c.backward()
    yield dict(w=w, fixed=fixed, q=q, rho=rho, comp=comp, c=c.item(),
               grad=r.grad.detach().clone())
    comp.close()


def test_c5_gradient_against_central_difference_solves(c5_gradient):
    """dc/drho_j on 32 random elements against central finite differences
    (h = 1e-4) in which each compliance change comes from a difference solve
    (K + dK) dt = -dK t, c(rho + h e_j) - c(rho) = q^T dt, so the change is
    resolved to the solve's tolerance instead of cancelling in two
    compliances of 17 M nodes."""
    d = c5_gradient
    w, s, T = d["w"], d["comp"].solver, d["comp"].T
    rho = torch.tensor(d["rho"], device=DEV)
    q_d = torch.tensor(d["q"], device=DEV)
    s.set_density(rho)
    y0 = torch.empty_like(T)
    s.apply_K(T, y0)
    y1 = torch.empty_like(T)
    dt = torch.empty_like(T)
    h = 1e-4
    elems = np.random.default_rng(2210).choice(w.n_elems, 32, replace=False)
    grad = d["grad"].cpu().numpy()
    try:
        for e in elems:
            dcs = []
            for sign in (1.0, -1.0):
                rp = rho.clone()
                rp[int(e)] += sign * h
                s.set_density(rp)
                s.apply_K(T, y1)
                s.set_load(y0 - y1)  # -dK t
                dt.zero_()
                it, rr, ok = s.solve_mgcg(dt)
                assert ok
                dcs.append(float(torch.dot(q_d, dt)))
            fd = (dcs[0] - dcs[1]) / (2 * h)
            # both sides carry the solves' errors at the scale of the whole
            # field (eps2 of ||q||), so the bar is relative plus a part of
            # the largest gradient: elements near the sink, with gradients
            # five orders below the largest, are resolved to ~1e-5 of
            # their own size
            assert abs(fd - grad[e]) <= 1e-6 * abs(grad[e]) + 1e-9 * np.abs(grad).max(), \
                (int(e), fd, grad[e])
    finally:
        s.set_load(q_d)
        s.set_density(rho)


def test_c5_gradient_on_a_crop_against_the_oracle(c5_gradient):
    """The oracle's gradient (Eq. 9-11 with an exact solve) on the 32^3 crop
    x < 32, 112 <= y, z < 144 of the same random field, with the 128^3
    workload's boundary conditions on the crop (centred sink patch on its
    x = 0 face, nodal load 0.01), against the autograd gradient of the mixed
    path on that crop."""
    d = c5_gradient
    w = d["w"]
    R = d["rho"].reshape(w.nz, w.ny, w.nx)
    crop = np.ascontiguousarray(R[112:144, 112:144, 0:32]).reshape(-1)
    n = 32
    fixed = workloads.heat_sink_mask(n, n, n)
    q = workloads.nodal_load(fixed)
    p = mgar.default_params(nx=n, ny=n, nz=n, nl=4, eps2=1e-11, cg_max=500,
                            precision=mgar.MGAR_MIXED)
    comp = autograd.Compliance(p, fixed, q)
    r = torch.tensor(crop, device=DEV, requires_grad=True)
    c = comp(r)
    c.backward()
    g = fem.Grid(n, n, n)
    H, Hs = design.filter_matrix(g, p.rmin)
    rho_phys = design.filter_forward(H, Hs, crop)
    t = solvers.exact_solve(fem.system_matrix(g, rho_phys, fixed), q)
    dc, _ = design.sensitivities(g, H, Hs, rho_phys, t, p.k0, p.kmin, p.penal)
    # the mixed path's solution carries its df64 accuracy floor (true residual
    # near 1e-10 of ||q||), which bounds compliance and gradient agreement
    assert abs(c.item() - q @ t) / (q @ t) < 1e-8
    np.testing.assert_allclose(r.grad.cpu().numpy(), dc, rtol=1e-6, atol=1e-8 * np.abs(dc).max())
    comp.close()
