"""Pins for the oracle's MGCG and MGAR solvers (Eq. 12-21, 28)."""
import numpy as np
import pytest

from oracle import fem, multigrid as mg, solvers


def _setup(dims, seed=7, nfix=3):
    nx, ny = dims[0], dims[1]
    nz = dims[2] if len(dims) == 3 else 0
    g = fem.Grid(nx, ny, nz)
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.05, 1.0, g.n_elems)
    fixed = np.zeros(g.n_nodes, np.uint8)
    fixed[: g.NX * nfix: g.NX] = 1
    q = np.where(fixed != 0, 0.0, 0.01)
    return g, rho, fixed, q


def dense_brute_force(g, rho, fixed, q):
    """Brute force: element loops into a dense matrix, fixed unknowns
    removed, numpy dense solve."""
    ke = fem.element_conductivity(g.dim)
    K = np.zeros((g.n_nodes, g.n_nodes))
    en = g.element_nodes()
    k = 1e-3 + (1 - 1e-3) * rho ** 3
    for e in range(g.n_elems):
        for a in range(g.nen):
            for b in range(g.nen):
                K[en[e, a], en[e, b]] += k[e] * ke[a, b]
    free = np.flatnonzero(fixed == 0)
    t = np.zeros(g.n_nodes)
    t[free] = np.linalg.solve(K[np.ix_(free, free)], q[free])
    return t


@pytest.mark.parametrize("dims,nl", [((4, 4), 2), ((8, 8), 3), ((4, 4, 4), 2), ((9, 5), 3)])
def test_mgcg_matches_dense_solve(dims, nl):
    g, rho, fixed, q = _setup(dims)
    A = fem.system_matrix(g, rho, fixed)
    levels = mg.build_hierarchy(A, fixed, dims, nl)
    t, it, rr = solvers.mgcg(A, q, np.zeros(g.n_nodes), levels, eps2=1e-14, cg_max=500)
    t_ref = dense_brute_force(g, rho, fixed, q)
    assert rr <= 1e-14
    np.testing.assert_allclose(t, t_ref, rtol=1e-11, atol=1e-12 * np.abs(t_ref).max())
    np.testing.assert_allclose(q @ t, q @ t_ref, rtol=1e-12)
    assert q @ t > 0.0


def test_mgcg_warm_start_and_iteration_cap():
    g, rho, fixed, q = _setup((16, 16))
    A = fem.system_matrix(g, rho, fixed)
    levels = mg.build_hierarchy(A, fixed, (16, 16), 3)
    t_ex = solvers.exact_solve(A, q)
    t, it, rr = solvers.mgcg(A, q, t_ex, levels, eps2=1e-8)
    assert it == 0
    t, it, rr = solvers.mgcg(A, q, np.zeros(g.n_nodes), levels, eps2=1e-30, cg_max=3)
    assert it == 3 and rr > 1e-30


def _mgar_setup(dims=(16, 12), nl=3, seed=8):
    g, rho, fixed, q = _setup(dims, seed)
    rng = np.random.default_rng(seed + 1)
    rho0 = np.clip(rho + rng.uniform(-0.1, 0.1, g.n_elems), 0.0, 1.0)
    A = fem.system_matrix(g, rho, fixed)
    A0 = fem.system_matrix(g, rho0, fixed)
    levels0 = mg.build_hierarchy(A0, fixed, dims, nl)
    t0 = solvers.exact_solve(A0, q)
    return g, A, A0, levels0, q, t0


def test_mgar_one_vector_closed_form():
    g, A, A0, levels0, q, t0 = _mgar_setup()
    t, res = solvers.mgar(A, A0, levels0, q, t0, m=1)
    expect = (t0 @ q) / (t0 @ (A @ t0)) * t0
    np.testing.assert_allclose(t, expect, rtol=1e-12, atol=1e-14 * np.abs(expect).max())
    assert abs(res - np.linalg.norm(A @ expect - q) / np.linalg.norm(q)) < 1e-12


def test_mgar_exact_when_unchanged():
    """K = K0 and t0 the exact solution: the reduced solve returns t0."""
    g, A, A0, levels0, q, t0 = _mgar_setup()
    t, res = solvers.mgar(A0, A0, levels0, q, t0, m=2)
    np.testing.assert_allclose(t, t0, rtol=1e-10, atol=1e-12 * np.abs(t0).max())
    assert res < 1e-10


@pytest.mark.parametrize("guess", ["previous", "zero"])
@pytest.mark.parametrize("m", [2, 3])
def test_mgar_galerkin_identities(guess, m):
    g, A, A0, levels0, q, t0 = _mgar_setup()
    t, res = solvers.mgar(A, A0, levels0, q, t0, m=m, basis_guess=guess)
    # energy identity of the Galerkin projection, and compliance from below
    assert abs(q @ t - t @ (A @ t)) < 1e-12 * abs(q @ t)
    c_exact = q @ solvers.exact_solve(A, q)
    assert q @ t <= c_exact * (1 + 1e-13)
    # PCA (SVD, Eq. 18) and Gram-Schmidt span the same space
    t_svd, res_svd = solvers.mgar(A, A0, levels0, q, t0, m=m, basis_guess=guess,
                                  orthonormalise="svd")
    np.testing.assert_allclose(t, t_svd, rtol=1e-10, atol=1e-12 * np.abs(t).max())
    assert abs(res - res_svd) < 1e-10


def test_mgar_basis_follows_eq17():
    """With initial guess r_1 the V-cycle gives r_2 = r_1 - M0 K r_1 (since
    K0 r_1 + dK r_1 = K r_1); with zero guess r_2 = -M0 dK r_1."""
    g, A, A0, levels0, q, t0 = _mgar_setup()
    R = solvers.mgar_basis(A, A0, levels0, t0, 2, basis_guess="previous")
    M = lambda v: mg.vcycle(levels0, v, np.zeros_like(v))
    np.testing.assert_allclose(R[:, 1], t0 - M(A @ t0), atol=1e-11 * np.abs(t0).max())
    R = solvers.mgar_basis(A, A0, levels0, t0, 2, basis_guess="zero")
    np.testing.assert_allclose(R[:, 1], -M(A @ t0 - A0 @ t0), atol=1e-11 * np.abs(t0).max())


def test_reduced_residual_orthogonal_to_basis():
    g, A, A0, levels0, q, t0 = _mgar_setup()
    R = solvers.mgar_basis(A, A0, levels0, t0, 3)
    Rt = solvers.gram_schmidt(R)
    np.testing.assert_allclose(Rt.T @ Rt, np.eye(Rt.shape[1]), atol=1e-14)
    t, res, y = solvers.reduced_solve(A, q, Rt)
    assert np.abs(Rt.T @ (A @ t - q)).max() < 1e-12 * np.linalg.norm(q)


def test_gram_schmidt_drops_dependent_vectors():
    rng = np.random.default_rng(9)
    a = rng.standard_normal(50)
    b = rng.standard_normal(50)
    Q = solvers.gram_schmidt(np.stack([a, b, 2 * a - 3 * b], axis=1))
    assert Q.shape[1] == 2
