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
