"""Pins for the oracle's multigrid (Section 2.2, Table 1)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, multigrid as mg

from test_oracle_fem import kron_sum


@pytest.mark.parametrize("dims", [(8, 6), (7, 5), (5, 4, 3), (6, 3, 4)])
def test_prolongation_reproduces_linear_fields(dims):
    """Bilinear/trilinear interpolation is exact for affine functions."""
    P, cdims = mg.prolongation(dims)
    fine_nodes = [np.arange(n + 1, dtype=float) for n in dims]
    coarse_nodes = [np.minimum(2 * np.arange(c + 1), n).astype(float) for c, n in zip(cdims, dims)]
    coef = [0.3, -1.7, 2.2][:len(dims)]

    def field(axes):
        grids = np.meshgrid(*axes[::-1], indexing="ij")[::-1]  # x fastest
        return (1.25 + sum(c * g for c, g in zip(coef, grids))).reshape(-1)

    np.testing.assert_allclose(P @ field(coarse_nodes), field(fine_nodes), atol=1e-12)
    # each fine node's weights sum to one, and coarse nodes are injected
    np.testing.assert_allclose(np.asarray(P.sum(axis=1)).reshape(-1), 1.0, atol=1e-15)


def coarse_positions(positions):
    """Node positions of the next coarser grid: every other node, keeping
    the last one (ceil coarsening)."""
    n = len(positions) - 1
    return positions[np.minimum(2 * np.arange(mg.coarse_count(n) + 1), n)]


def fe_matrix_on_mesh(X):
    """Conductivity matrix (rho = 1) assembled directly on the tensor mesh
    with node positions X[d] per axis; box element matrices from 1D
    Kronecker sums."""
    import itertools
    dim = len(X)
    NN = [len(x) for x in X]
    n = int(np.prod(NN))
    K = np.zeros((n, n))
    for e in itertools.product(*[range(m - 1) for m in NN]):
        h = [X[d][e[d] + 1] - X[d][e[d]] for d in range(dim)]
        ke = kron_sum(dim, h)
        nodes = []
        for a in range(2 ** dim):
            idx, stride = 0, 1
            for d in range(dim):
                idx += (e[d] + ((a >> d) & 1)) * stride
                stride *= NN[d]
            nodes.append(idx)
        K[np.ix_(nodes, nodes)] += ke
    return K


@pytest.mark.parametrize("dims", [(8, 6), (7, 5), (4, 4, 4), (5, 3, 4), (6, 10, 4)])
def test_galerkin_operator_equals_coarse_fe_matrix(dims):
    """Nested FE spaces: P^T K_h P equals the conductivity matrix assembled
    on the coarse mesh itself (non-uniform where an odd axis was halved).
    P interpolates in each level's own node-index coordinates, which is
    geometric interpolation while the finer level is uniform; the second
    level is checked when the first coarsening truncated nothing."""
    g = fem.Grid(*(list(dims) + ([0] if len(dims) == 2 else [])))
    K = fem.assemble(g, np.ones(g.n_elems))
    no_fixed = np.zeros(g.n_nodes, np.uint8)
    X1 = [coarse_positions(np.arange(n + 1, dtype=float)) for n in dims]
    levels = mg.build_hierarchy(K, no_fixed, dims, 2)
    np.testing.assert_allclose(levels[1].A.toarray(), fe_matrix_on_mesh(X1), atol=1e-13)
    if all(n % 2 == 0 for n in dims):
        X2 = [coarse_positions(x) for x in X1]
        cd = tuple(mg.coarse_count(n) for n in dims)
        P1, _ = mg.prolongation(cd)
        A2 = (P1.T @ levels[1].A @ P1).toarray()
        np.testing.assert_allclose(A2, fe_matrix_on_mesh(X2), atol=1e-12)


def _problem(dims, seed=3):
    nx, ny = dims[0], dims[1]
    nz = dims[2] if len(dims) == 3 else 0
    g = fem.Grid(nx, ny, nz)
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.05, 1.0, g.n_elems)
    fixed = np.zeros(g.n_nodes, np.uint8)
    fixed[: g.NX * 2: g.NX] = 1  # two nodes on x = 0
    A = fem.system_matrix(g, rho, fixed)
    return g, A, fixed


@pytest.mark.parametrize("dims,nl", [((16, 12), 3), ((9, 7), 3), ((6, 6, 4), 3)])
def test_vcycle_is_symmetric_and_affine(dims, nl):
    g, A, fixed = _problem(dims)
    levels = mg.build_hierarchy(A, fixed, dims, nl)
    rng = np.random.default_rng(4)
    a, b = rng.standard_normal((2, g.n_nodes))
    Ma = mg.vcycle(levels, a, np.zeros_like(a))
    Mb = mg.vcycle(levels, b, np.zeros_like(b))
    assert abs(Ma @ b - a @ Mb) < 1e-12 * np.linalg.norm(Ma) * np.linalg.norm(b)
    # one V-cycle from an initial guess x0 equals x0 + M (b - A x0)
    x0 = rng.standard_normal(g.n_nodes)
    lhs = mg.vcycle(levels, b, x0)
    rhs = x0 + mg.vcycle(levels, b - A @ x0, np.zeros_like(b))
    np.testing.assert_allclose(lhs, rhs, atol=1e-11 * np.linalg.norm(lhs))


@pytest.mark.parametrize("dims,nl", [((16, 16), 4), ((8, 8, 8), 3)])
def test_vcycle_contracts_error(dims, nl):
    g, A, fixed = _problem(dims)
    levels = mg.build_hierarchy(A, fixed, dims, nl)
    rng = np.random.default_rng(5)
    x_true = rng.standard_normal(g.n_nodes)
    x_true[fixed != 0] = 0
    b = A @ x_true
    x = np.zeros(g.n_nodes)
    e0 = np.sqrt((x - x_true) @ (A @ (x - x_true)))
    for _ in range(3):
        x = mg.vcycle(levels, b, x)
    e3 = np.sqrt((x - x_true) @ (A @ (x - x_true)))
    assert e3 < 0.5 * e0


def test_single_level_is_direct_solve():
    g, A, fixed = _problem((6, 5))
    levels = mg.build_hierarchy(A, fixed, (6, 5), 1)
    b = np.random.default_rng(6).standard_normal(g.n_nodes)
    x = mg.vcycle(levels, b, np.zeros_like(b))
    np.testing.assert_allclose(A @ x, b, atol=1e-11)


def test_coarse_operators_spd_with_dirichlet():
    g, A, fixed = _problem((12, 10, 6))
    levels = mg.build_hierarchy(A, fixed, (12, 10, 6), 3)
    for L in levels:
        Ad = L.A.toarray()
        np.testing.assert_allclose(Ad, Ad.T, atol=1e-14)
        assert np.linalg.eigvalsh(Ad)[0] > 0.0
    # fixed fine nodes receive no coarse correction
    P0 = levels[0].P.toarray()
    assert np.all(P0[fixed != 0] == 0.0)


@pytest.mark.parametrize("dim,lo,hi,at_lo", [(2, 0.75, 1.5, (0.5, 0.0)),
                                              (3, 0.5, 1.5, (1.0, 1.0, 1.0))])
def test_default_smoother_weight_damps_oscillatory_modes(dim, lo, hi, at_lo):
    """The reading omega = 0.9: on a periodic unit-conductivity grid the
    Fourier modes with some |theta_d| >= pi/2 are eigenvectors of D^-1 A with
    eigenvalues in [lo, hi] (checked here by applying the assembled interior
    stencil of the oracle's element matrix to sampled modes), so one damped
    Jacobi sweep with the default weight multiplies each by at most
    max(|1 - omega lo|, |1 - omega hi|) < 0.6."""
    import inspect
    omega = inspect.signature(mg.vcycle).parameters["omega"].default
    assert omega == 0.9
    k0 = kron_sum(dim)  # element matrix built from 1D matrices, not the oracle's
    stencil = {}
    for a in range(2 ** dim):
        for b in range(2 ** dim):
            off = tuple(((b >> d) & 1) - ((a >> d) & 1) for d in range(dim))
            stencil[off] = stencil.get(off, 0.0) + k0[a, b]
    diag = stencil[(0,) * dim]
    rng = np.random.default_rng(0)
    thetas = rng.uniform(-np.pi, np.pi, (4000, dim))
    thetas[:, 0] = np.where(np.abs(thetas[:, 0]) < np.pi / 2, np.pi, thetas[:, 0])
    lam = np.array([sum(v * np.cos(np.dot(o, t)) for o, v in stencil.items()) / diag
                    for t in thetas])
    assert lam.min() >= lo - 1e-12 and lam.max() <= hi + 1e-12
    # the extremes are reached: hi at theta = (pi, 0, ...), lo at at_lo * pi
    for t, want in ((np.pi * np.eye(dim)[0], hi), (np.pi * np.array(at_lo), lo)):
        v = sum(c * np.cos(np.dot(o, t)) for o, c in stencil.items()) / diag
        assert abs(v - want) < 1e-12
    assert max(abs(1 - omega * lo), abs(1 - omega * hi)) < 0.6
