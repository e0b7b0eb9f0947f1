"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Sizes span several thread blocks with ragged tails (odd element counts,
grids whose coarsening truncates an axis).  Tolerances: FP64 kernels agree
with the oracle to rounding (relative 1e-12 for single operator
applications; 1e-10 for anything that goes through the coarsest direct solve,
whose rounding is amplified by the condition number of the coarsest Galerkin
operator (up to ~1e4 with a 1e-3..1 conductivity contrast), and for solves
run to eps2 = 1e-13, the bar set for T and compliance); the mixed path to
1e-6 relative in compliance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import design, fem, multigrid as mg, solvers  # noqa: E402
from paper_2210_00947_gb300 import mgar, workloads  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def dev(a):
    return torch.tensor(np.asarray(a, dtype=np.float64), device=DEV)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def assert_elementwise(got, ref, rel):
    """Element by element |got - ref| <= rel * max|ref|: an absolute bar scaled
    to the field (temperatures and V-cycle outputs pass through zero, so a
    per-element relative bar would be meaningless there)."""
    np.testing.assert_allclose(got, ref, rtol=0, atol=rel * np.abs(ref).max())


def make_problem(dims, seed=0, rho_lo=0.05, mask="random"):
    nx, ny, nz = dims
    g = fem.Grid(nx, ny, nz)
    rng = np.random.default_rng(seed)
    rho = rng.uniform(rho_lo, 1.0, g.n_elems)
    if mask == "random":
        fixed = (rng.uniform(size=g.n_nodes) < 0.05).astype(np.uint8)
        fixed[0] = 1
    else:
        fixed = workloads.heat_sink_mask(nx, ny, nz)
    q = workloads.nodal_load(fixed)
    return g, rho, fixed, q


def solver_for(dims, fixed, q, **kw):
    nx, ny, nz = dims
    p = mgar.default_params(nx=nx, ny=ny, nz=nz, **kw)
    return mgar.Solver(p, fixed, q)


DIMS_2D = [(37, 23, 0), (64, 48, 0)]
DIMS_3D = [(13, 11, 9), (16, 16, 12)]


@pytest.mark.parametrize("dims,r", [((37, 23, 0), 1.5), ((40, 33, 0), 2.5), ((13, 11, 9), 1.5),
                                    ((12, 10, 8), 2.2)])
def test_filter_matches_oracle(dims, r):
    g, rho, fixed, q = make_problem(dims)
    H, Hs = design.filter_matrix(g, r)
    with solver_for(dims, fixed, q, rmin=r, nl=2) as s:
        x = np.random.default_rng(1).standard_normal(g.n_elems)
        out = torch.empty(g.n_elems, dtype=torch.float64, device=DEV)
        s.filter(dev(x), out)
        np.testing.assert_allclose(host(out), design.filter_forward(H, Hs, x), rtol=1e-13, atol=1e-15)
        s.filter(dev(x), out, transpose=True)
        np.testing.assert_allclose(host(out), design.filter_transpose(H, Hs, x), rtol=1e-13,
                                   atol=1e-15)


@pytest.mark.parametrize("dims", DIMS_2D + DIMS_3D)
def test_apply_K_matches_oracle(dims):
    g, rho, fixed, q = make_problem(dims)
    A = fem.system_matrix(g, rho, fixed)
    with solver_for(dims, fixed, q, nl=2) as s:
        s.set_density(dev(rho), physical=True)
        x = np.random.default_rng(2).standard_normal(g.n_nodes)
        y = torch.empty(g.n_nodes, dtype=torch.float64, device=DEV)
        s.apply_K(dev(x), y)
        ref = A @ x
        np.testing.assert_allclose(host(y), ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("dims,nl", [((37, 23, 0), 3), ((64, 48, 0), 4), ((100, 100, 0), 4),
                                     ((13, 11, 9), 3), ((16, 16, 12), 3), ((20, 18, 16), 4)])
@pytest.mark.parametrize("zero_guess", [True, False])
def test_vcycle_matches_oracle(dims, nl, zero_guess):
    g, rho, fixed, q = make_problem(dims, mask="sink")
    A = fem.system_matrix(g, rho, fixed)
    dims_e = dims[:2] if dims[2] == 0 else dims
    levels = mg.build_hierarchy(A, fixed, dims_e, nl)
    rng = np.random.default_rng(3)
    b = rng.standard_normal(g.n_nodes)
    b[fixed != 0] = 0.0
    x0 = np.zeros(g.n_nodes) if zero_guess else rng.standard_normal(g.n_nodes)
    if not zero_guess:
        x0[fixed != 0] = 0.0
    ref = mg.vcycle(levels, b, x0.copy())
    with solver_for(dims, fixed, q, nl=nl) as s:
        s.set_density(dev(rho), physical=True)
        s.build_hierarchy()
        x = dev(x0)
        s.vcycle(dev(b), x)
        assert relerr(host(x), ref) < 1e-10
        assert_elementwise(host(x), ref, 1e-10)


# The mixed path's FP32 V-cycle (tiled finest-level passes, the restriction
# that leaves each coarse level's zero-guess sweep, the coarse residual, the
# column interpolation; the small levels as separate launches, or in one
# cluster launch on request) against the oracle's FP64 V-cycle on the same
# hierarchy.  FP32 storage and arithmetic bound the agreement (the operands
# carry 2^-24 and each stencil row cancels its 21-27 terms down to the
# residual); the bar is 1e-4.  (42, 42, 21) selects the 43 x 5 tiles and
# coarsens z oddly.  The coarsest factor and inverse: band widths below 32
# take the windowed kernels (all but the last three cases; (16, 16, 12) at
# nl 3 is width 31), (10, 10, 8) and (60, 20, 0) at nl 2 (widths 43 and 32)
# the shared-memory df64 kernels, (42, 42, 21) the global-memory FP64 ones.
@pytest.mark.parametrize("dims,nl", [((37, 23, 0), 3), ((100, 100, 0), 4), ((13, 11, 9), 3),
                                     ((20, 18, 16), 4), ((16, 16, 12), 3), ((10, 10, 8), 2),
                                     ((60, 20, 0), 2), ((42, 42, 21), 3)])
@pytest.mark.parametrize("zero_guess", [True, False])
@pytest.mark.parametrize("cluster", [False, True])
def test_mixed_vcycle_matches_oracle(dims, nl, zero_guess, cluster, monkeypatch):
    if cluster:
        monkeypatch.setenv("MGAR_CLUSTER_BOTTOM", "1")
    g, rho, fixed, q = make_problem(dims, mask="sink")
    A = fem.system_matrix(g, rho, fixed)
    dims_e = dims[:2] if dims[2] == 0 else dims
    levels = mg.build_hierarchy(A, fixed, dims_e, nl)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(g.n_nodes)
    b[fixed != 0] = 0.0
    x0 = np.zeros(g.n_nodes) if zero_guess else rng.standard_normal(g.n_nodes)
    if not zero_guess:
        x0[fixed != 0] = 0.0
    ref = mg.vcycle(levels, b, x0.copy())
    with solver_for(dims, fixed, q, nl=nl, precision=mgar.MGAR_MIXED) as s:
        s.set_density(dev(rho), physical=True)
        s.build_hierarchy()
        x = dev(x0)
        s.vcycle(dev(b), x)
        assert relerr(host(x), ref) < 1e-4
        assert_elementwise(host(x), ref, 5e-4)


@pytest.mark.parametrize("dims,nl", [((37, 23, 0), 3), ((100, 100, 0), 4), ((13, 11, 9), 3),
                                     ((16, 16, 12), 3)])
def test_mgcg_matches_oracle(dims, nl):
    g, rho, fixed, q = make_problem(dims, mask="sink")
    A = fem.system_matrix(g, rho, fixed)
    dims_e = dims[:2] if dims[2] == 0 else dims
    levels = mg.build_hierarchy(A, fixed, dims_e, nl)
    t_ref, it_ref, _ = solvers.mgcg(A, q, np.zeros(g.n_nodes), levels, eps2=1e-13, cg_max=500)
    with solver_for(dims, fixed, q, nl=nl, eps2=1e-13, cg_max=500) as s:
        s.set_density(dev(rho), physical=True)
        T = torch.zeros(g.n_nodes, dtype=torch.float64, device=DEV)
        it, rr, ok = s.solve_mgcg(T)
        assert ok and rr <= 1e-13
        t = host(T)
        assert relerr(t, t_ref) < 1e-10
        assert_elementwise(t, t_ref, 1e-10)
        assert abs(q @ t - q @ t_ref) / abs(q @ t_ref) < 1e-10
        assert abs(it - it_ref) <= 1
        # and against the definition: the exact solve
        assert relerr(t, solvers.exact_solve(A, q)) < 1e-10


def test_mgcg_iteration_cap_and_warm_start():
    dims = (40, 40, 0)
    g, rho, fixed, q = make_problem(dims, mask="sink")
    with solver_for(dims, fixed, q, nl=3, eps2=1e-30, cg_max=3) as s:
        s.set_density(dev(rho), physical=True)
        T = torch.zeros(g.n_nodes, dtype=torch.float64, device=DEV)
        it, rr, ok = s.solve_mgcg(T)
        assert it == 3 and not ok
    A = fem.system_matrix(g, rho, fixed)
    t_ex = solvers.exact_solve(A, q)
    with solver_for(dims, fixed, q, nl=3, eps2=1e-8) as s:
        s.set_density(dev(rho), physical=True)
        T = dev(t_ex)
        it, rr, ok = s.solve_mgcg(T)
        assert it == 0 and ok


def _mgar_case(dims, nl, seed=5):
    g, rho, fixed, q = make_problem(dims, seed=seed, rho_lo=0.1, mask="sink")
    rng = np.random.default_rng(seed + 1)
    rho0 = np.clip(rho + rng.uniform(-0.15, 0.15, g.n_elems), 0.0, 1.0)
    return g, rho, rho0, fixed, q


@pytest.mark.parametrize("dims,nl", [((37, 23, 0), 3), ((100, 100, 0), 4), ((13, 11, 9), 3)])
@pytest.mark.parametrize("m,guess", [(2, "previous"), (3, "previous"), (2, "zero"), (4, "zero")])
def test_mgar_matches_oracle(dims, nl, m, guess):
    g, rho, rho0, fixed, q = _mgar_case(dims, nl)
    dims_e = dims[:2] if dims[2] == 0 else dims
    A = fem.system_matrix(g, rho, fixed)
    A0 = fem.system_matrix(g, rho0, fixed)
    levels0 = mg.build_hierarchy(A0, fixed, dims_e, nl)
    t0 = solvers.exact_solve(A0, q)
    t_ref, res_ref = solvers.mgar(A, A0, levels0, q, t0, m=m, basis_guess=guess)
    bg = mgar.MGAR_GUESS_PREVIOUS if guess == "previous" else mgar.MGAR_GUESS_ZERO
    with solver_for(dims, fixed, q, nl=nl, m=m, basis_guess=bg, eps1=0.5) as s:
        s.set_density(dev(rho0), physical=True)
        s.build_hierarchy()
        s.set_density(dev(rho), physical=True)
        T = torch.empty(g.n_nodes, dtype=torch.float64, device=DEV)
        res, acc = s.solve_mgar(dev(t0), T)
        assert relerr(host(T), t_ref) < 1e-10
        assert_elementwise(host(T), t_ref, 1e-10)
        assert abs(res - res_ref) < 1e-10 * max(1.0, res_ref)
        assert acc == (res_ref <= 0.5)


@pytest.mark.parametrize("dims", [(37, 23, 0), (13, 11, 9)])
def test_sensitivity_matches_oracle(dims):
    g, rho, fixed, q = make_problem(dims, mask="sink")
    H, Hs = design.filter_matrix(g, 1.5)
    rho_phys = design.filter_forward(H, Hs, rho)
    t = solvers.exact_solve(fem.system_matrix(g, rho_phys, fixed), q)
    dc_ref, dv_ref = design.sensitivities(g, H, Hs, rho_phys, t)
    with solver_for(dims, fixed, q, nl=2) as s:
        s.set_density(dev(rho), physical=False)
        dc = torch.empty(g.n_elems, dtype=torch.float64, device=DEV)
        dv = torch.empty(g.n_elems, dtype=torch.float64, device=DEV)
        c = s.sensitivity(dev(t), dc, dv)
        assert abs(c - q @ t) / abs(q @ t) < 1e-13
        # Rounding of t_e^T k0 t_e is ~ eps |t_e|^2 ||k0|| (cancellation when
        # the temperatures are large and their differences small); scaled by
        # Eq. 10's factor and carried through the filter transpose it bounds
        # the per-element difference.
        te = t[g.element_nodes()]
        bound = 16 * 2.2e-16 * (3.0 * (1 - 1e-3)) * rho_phys ** 2 * (te * te).sum(axis=1)
        atol = 10 * design.filter_transpose(H, Hs, bound)
        got = host(dc)
        assert np.all(np.abs(got - dc_ref) <= atol + 1e-13 * np.abs(dc_ref))
        assert relerr(got, dc_ref) < 1e-10
        np.testing.assert_allclose(host(dv), dv_ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("dims,r", [((37, 23, 0), 1.5), ((13, 11, 9), 1.5), ((12, 10, 8), 2.2)])
def test_mixed_filter_and_sensitivity_match_oracle(dims, r):
    """Mixed path: filter + SIMP (Eq. 4, 6) and the sensitivities (Eq. 9-11)
    run in double-float pairs (2^-46 relative per operation).  The filter
    sums have terms of one sign; the element energy is a sum of squared
    pair differences.  Rounding t to a pair moves a difference by up to
    2^-47 |t|, which bounds the energy error as eps |t_e|^2 does in FP64."""
    g, rho, fixed, q = make_problem(dims, mask="sink")
    H, Hs = design.filter_matrix(g, r)
    rho_phys = design.filter_forward(H, Hs, rho)
    t = solvers.exact_solve(fem.system_matrix(g, rho_phys, fixed), q)
    dc_ref, _ = design.sensitivities(g, H, Hs, rho_phys, t)
    with solver_for(dims, fixed, q, rmin=r, nl=2, precision=mgar.MGAR_MIXED) as s:
        s.set_density(dev(rho), physical=False)
        dc = torch.empty(g.n_elems, dtype=torch.float64, device=DEV)
        s.sensitivity(dev(t), dc, None)
        te = t[g.element_nodes()]
        eps_df = 2.0 ** -46
        bound = 16 * eps_df * (3.0 * (1 - 1e-3)) * rho_phys ** 2 * (te * te).sum(axis=1)
        atol = 10 * design.filter_transpose(H, Hs, bound)
        got = host(dc)
        assert np.all(np.abs(got - dc_ref) <= atol + 1e-12 * np.abs(dc_ref))
        assert relerr(got, dc_ref) < 1e-9


@pytest.mark.parametrize("dims", [(37, 23, 0), (13, 11, 9), (100, 100, 0)])
def test_oc_matches_oracle(dims):
    g, rho, fixed, q = make_problem(dims, mask="sink")
    rng = np.random.default_rng(9)
    dc = -rng.uniform(0.0, 5.0, g.n_elems) * 10.0 ** rng.uniform(-3, 3, g.n_elems)
    H, Hs = design.filter_matrix(g, 1.5)
    dv = design.filter_transpose(H, Hs, np.full(g.n_elems, 1.0 / g.n_elems))
    ref, lam_ref = design.oc_update(rho, dc, dv, 0.4, 0.2)
    with solver_for(dims, fixed, q, nl=2) as s:
        r = dev(rho)
        lam, change = s.oc_update(r, dev(dc), 0.4, 0.2)
        out = host(r)
        assert abs(lam - lam_ref) / lam_ref < 1e-12
        np.testing.assert_allclose(out, ref, rtol=1e-11, atol=1e-12)
        assert abs(change - np.max(np.abs(ref - rho))) < 1e-11
        assert abs(dv @ out - 0.4) < 1e-11


def test_oc_unreachable_volume_matches_oracle():
    """Volume out of reach of the move limits: the bracket collapses to its
    end (lambda -> 1e-40, every element at its upper move limit)."""
    dims = (30, 20, 0)
    g, rho, fixed, q = make_problem(dims, mask="sink")
    rho = np.full(g.n_elems, 0.1)
    dc = -np.random.default_rng(10).uniform(0.1, 1.0, g.n_elems)
    H, Hs = design.filter_matrix(g, 1.5)
    dv = design.filter_transpose(H, Hs, np.full(g.n_elems, 1.0 / g.n_elems))
    ref, lam_ref = design.oc_update(rho, dc, dv, 0.5, 0.2)
    with solver_for(dims, fixed, q, nl=2) as s:
        r = dev(rho)
        lam, change = s.oc_update(r, dev(dc), 0.5, 0.2)
        np.testing.assert_allclose(host(r), ref, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(host(r), 0.3, rtol=1e-12)
        assert lam < 1e-30 and lam_ref < 1e-30


@pytest.mark.parametrize("dims", [(128, 96, 0), (40, 36, 30)])
def test_oc_large_matches_oracle(dims):
    g, rho, fixed, q = make_problem(dims, mask="sink", seed=11)
    rng = np.random.default_rng(12)
    dc = -(10.0 ** rng.uniform(-4, 2, g.n_elems))
    H, Hs = design.filter_matrix(g, 1.5)
    dv = design.filter_transpose(H, Hs, np.full(g.n_elems, 1.0 / g.n_elems))
    ref, lam_ref = design.oc_update(rho, dc, dv, 0.35, 0.2)
    with solver_for(dims, fixed, q, nl=3) as s:
        r = dev(rho)
        lam, change = s.oc_update(r, dev(dc), 0.35, 0.2)
        assert abs(lam - lam_ref) / lam_ref < 1e-12
        np.testing.assert_allclose(host(r), ref, rtol=1e-11, atol=1e-12)


# (42, 42, 21): 43-node planes select the 43 x 5 FP32 tile and the 43 x 11
# df64 tile (one tile column, ragged rows), and 22 planes leave a ragged run
# of the four-plane unrolled z march.  (42, 42, 21) and (32, 32, 20) at
# eps2 = 1e-11 lie below the accuracy floor of the FP32 iterations: without
# the restart on drift and the hand-over to the df64 CG the first stalled
# near 5e-10 and the second diverged.
@pytest.mark.parametrize("dims,nl,cg", [((64, 48, 0), 4, "df64"), ((100, 100, 0), 4, "df64"),
                                        ((16, 16, 12), 3, "ru"), ((20, 18, 16), 4, "ru"),
                                        ((16, 16, 12), 3, "df64"), ((20, 18, 16), 4, "df64"),
                                        ((42, 42, 21), 3, "ru"), ((42, 42, 21), 3, "df64"),
                                        ((32, 32, 20), 3, "ru")])
def test_mixed_mgcg_matches_exact_solve(dims, nl, cg, monkeypatch):
    """Mixed path with the FP32 V-cycle as preconditioner: on 2D grids (and
    on 3D grids with MGAR_DF64_CG=1) a df64 CG, on 3D grids by default FP32
    CG iterations with reliable df64 updates.  The preconditioner and the
    precision of the Krylov vectors only change the iteration count.
    Double-float vectors carry ~48 bits, so the true residual bottoms out
    near 2^-46 ||A|| ||T|| / ||q|| (a few 1e-10 here); the bars are set from
    that floor, two orders below the 1e-8 the workloads use."""
    if cg == "df64":
        monkeypatch.setenv("MGAR_DF64_CG", "1")
    g, rho, fixed, q = make_problem(dims, mask="sink")
    A = fem.system_matrix(g, rho, fixed)
    t_ex = solvers.exact_solve(A, q)
    with solver_for(dims, fixed, q, nl=nl, eps2=1e-11, cg_max=500, precision=mgar.MGAR_MIXED) as s:
        s.set_density(dev(rho), physical=True)
        T = torch.zeros(g.n_nodes, dtype=torch.float64, device=DEV)
        it, rr, ok = s.solve_mgcg(T)
        assert ok and rr <= 1e-11
        t = host(T)
        # the true residual, evaluated by the oracle
        assert np.linalg.norm(q - A @ t) / np.linalg.norm(q) < 2e-9
        assert relerr(t, t_ex) < 1e-7
        assert_elementwise(t, t_ex, 1e-7)
        assert abs(q @ t - q @ t_ex) / abs(q @ t_ex) < 1e-8


@pytest.mark.parametrize("dims,nl", [((100, 100, 0), 4), ((13, 11, 9), 3)])
@pytest.mark.parametrize("guess", ["previous", "zero"])
def test_mixed_mgar_compliance_matches_oracle(dims, nl, guess):
    """Mixed MGAR: FP32 basis V-cycles, FP64 Gram-Schmidt and reduced solve;
    the reduced solution's compliance within 1e-6 of the oracle's."""
    g, rho, rho0, fixed, q = _mgar_case(dims, nl)
    dims_e = dims[:2] if dims[2] == 0 else dims
    A = fem.system_matrix(g, rho, fixed)
    A0 = fem.system_matrix(g, rho0, fixed)
    levels0 = mg.build_hierarchy(A0, fixed, dims_e, nl)
    t0 = solvers.exact_solve(A0, q)
    t_ref, res_ref = solvers.mgar(A, A0, levels0, q, t0, m=2, basis_guess=guess)
    bg = mgar.MGAR_GUESS_PREVIOUS if guess == "previous" else mgar.MGAR_GUESS_ZERO
    with solver_for(dims, fixed, q, nl=nl, m=2, basis_guess=bg, precision=mgar.MGAR_MIXED) as s:
        s.set_density(dev(rho0), physical=True)
        s.build_hierarchy()
        s.set_density(dev(rho), physical=True)
        T = torch.empty(g.n_nodes, dtype=torch.float64, device=DEV)
        res, acc = s.solve_mgar(dev(t0), T)
        t = host(T)
        assert abs(q @ t - q @ t_ref) / abs(q @ t_ref) < 1e-6
        assert abs(res - res_ref) < 1e-4 * max(1.0, res_ref)


# The benchmark's tile shapes: 129-node planes select the 43 x 5 FP32 tiles
# (three tile columns) of the V-cycle and the 43 x 11 df64 tile of the MGAR
# projection's products; 17 planes leave a ragged run of the unrolled z
# march.  The oracle's reference temperatures t0 come from its own MGCG (an
# exact solve of 283,985 unknowns is out of reach); both sides take the same
# t0 as r_1.
@pytest.mark.parametrize("guess", ["previous", "zero"])
def test_mixed_mgar_at_benchmark_tiles(guess):
    dims, nl = (128, 128, 16), 4
    g, rho, rho0, fixed, q = _mgar_case(dims, nl)
    A = fem.system_matrix(g, rho, fixed)
    A0 = fem.system_matrix(g, rho0, fixed)
    levels0 = mg.build_hierarchy(A0, fixed, dims, nl)
    t0, _, rr0 = solvers.mgcg(A0, q, np.zeros(g.n_nodes), levels0, eps2=1e-10, cg_max=200)
    assert rr0 <= 1e-10
    t_ref, res_ref = solvers.mgar(A, A0, levels0, q, t0, m=2, basis_guess=guess)
    bg = mgar.MGAR_GUESS_PREVIOUS if guess == "previous" else mgar.MGAR_GUESS_ZERO
    with solver_for(dims, fixed, q, nl=nl, m=2, basis_guess=bg, precision=mgar.MGAR_MIXED) as s:
        s.set_density(dev(rho0), physical=True)
        s.build_hierarchy()
        s.set_density(dev(rho), physical=True)
        T = torch.empty(g.n_nodes, dtype=torch.float64, device=DEV)
        res, acc = s.solve_mgar(dev(t0), T)
        t = host(T)
        assert abs(q @ t - q @ t_ref) / abs(q @ t_ref) < 1e-6
        assert abs(res - res_ref) < 1e-4 * max(1.0, res_ref)
        assert_elementwise(t, t_ref, 1e-5)
