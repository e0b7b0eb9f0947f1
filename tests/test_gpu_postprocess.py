"""The boundary post-processing (Eq. 24-27) on the GPU against the oracle,
on designs taken from a few optimisation cycles."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import design, fem, loop, postprocess as pp  # noqa: E402
from paper_2210_00947_gb300 import mgar, workloads  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("dims,nl", [((40, 32, 0), 3), ((12, 10, 8), 3)])
def test_postprocess_matches_oracle(dims, nl):
    nx, ny, nz = dims
    vf = 0.4
    fixed = workloads.heat_sink_mask(nx, ny, nz)
    q = workloads.nodal_load(fixed)
    ne = workloads.num_elements(nx, ny, nz)
    s = loop.LoopSettings(nx=nx, ny=ny, nz=nz, volfrac=vf, iters=6, n_on=7, nl=nl, eps2=1e-12)
    rho, t, _ = loop.optimise(s, fixed, q, np.full(ne, vf))
    g = fem.Grid(nx, ny, nz)
    H, Hs = design.filter_matrix(g, s.rmin)
    rho_phys = design.filter_forward(H, Hs, rho)
    A = fem.system_matrix(g, rho_phys, fixed)
    from oracle import solvers
    t = solvers.exact_solve(A, q)  # the temperatures of the final design
    rho_o, ns_o, level_o = pp.postprocess(g, rho_phys, t, vf, s.rmin)

    p = mgar.default_params(nx=nx, ny=ny, nz=nz, nl=nl)
    with mgar.Solver(p, fixed, q) as sv:
        out = torch.empty(ne, dtype=torch.float64, device=DEV)
        level, vol = sv.postprocess(torch.tensor(rho, device=DEV), torch.tensor(t, device=DEV),
                                    vf, out)
        rho_g = out.cpu().numpy()
    assert abs(level - level_o) <= 1e-9 * abs(level_o)
    assert vol <= vf and abs(vol - rho_g.mean()) < 1e-12
    # the bisection ends on a step of the volume, i.e. at the value of some
    # lattice point (a node's value is shared by up to 2^d elements): elements
    # whose interpolated values come within 1e-9 of the level may round
    # either way; every other element is identical
    nodes = g.element_nodes()
    N = pp.lattice_shape_values(g.dim)
    vals = ns_o[nodes] @ N.T
    ambiguous = np.any(np.abs(vals - level_o) <= 1e-9 * abs(level_o), axis=1)
    assert ambiguous.sum() <= 2 ** (g.dim + 1)
    np.testing.assert_array_equal(rho_g[~ambiguous], rho_o[~ambiguous])
    assert 0.2 < np.mean((rho_g == 0) | (rho_g == 1))  # mostly crisp
