"""Pins for the oracle's FE discretisation (Eq. 2-4).

Each check compares the oracle with something other than itself: closed
forms of the unit element matrices built from 1D matrices, their spectra,
structural invariants of the assembled matrix, and the textbook 1D solution
that linear elements reproduce exactly at the nodes."""
import numpy as np
import pytest

from oracle import fem, solvers, multigrid
from paper_2210_00947_gb300 import workloads

K1 = np.array([[1.0, -1.0], [-1.0, 1.0]])        # 1D unit stiffness
M1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])  # 1D unit mass


def kron_sum(dim, h=None):
    """Element matrix of a box element from 1D matrices: sum over axes d of
    (K1/h_d on axis d) x (M1*h_e on the other axes); axis 0 is x (fastest)."""
    h = np.ones(dim) if h is None else np.asarray(h, float)
    total = 0
    for d in range(dim):
        mats = [K1 / h[e] if e == d else M1 * h[e] for e in range(dim)]
        M = mats[0]
        for e in range(1, dim):
            M = np.kron(mats[e], M)
        total = total + M
    return total


def test_q4_closed_form():
    k = fem.element_conductivity(2)
    # local order (0,0),(1,0),(0,1),(1,1): self 4/6, edge -1/6, opposite -2/6
    expect = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    np.testing.assert_allclose(k, expect, atol=1e-15)


def test_h8_closed_form():
    k = fem.element_conductivity(3)
    for a in range(8):
        for b in range(8):
            diff = bin(a ^ b).count("1")
            expect = {0: 4 / 12, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[diff]
            assert abs(k[a, b] - expect) < 1e-15


@pytest.mark.parametrize("dim,eigs", [(2, [0, 2 / 3, 1, 1]),
                                      (3, [0, 1 / 6, 1 / 3, 1 / 3, 1 / 3, 0.5, 0.5, 0.5])])
def test_element_spectrum(dim, eigs):
    w = np.linalg.eigvalsh(fem.element_conductivity(dim))
    np.testing.assert_allclose(np.sort(w), np.sort(eigs), atol=1e-14)


@pytest.mark.parametrize("dim,h", [(2, (2.0, 1.0)), (3, (2.0, 1.0, 2.0)), (3, (1.0, 1.0, 1.0))])
def test_box_element_matches_kronecker(dim, h):
    np.testing.assert_allclose(fem.element_conductivity(dim, h), kron_sum(dim, h), atol=1e-14)


@pytest.mark.parametrize("dims", [(5, 4, 0), (3, 4, 2)])
def test_assembled_invariants(dims):
    g = fem.Grid(*dims)
    rng = np.random.default_rng(1)
    kv = fem.simp(rng.uniform(0.05, 1.0, g.n_elems), 1.0, 1e-3, 3.0)
    K = fem.assemble(g, kv).toarray()
    np.testing.assert_allclose(K, K.T, atol=1e-15)
    np.testing.assert_allclose(K.sum(axis=1), 0.0, atol=1e-14)
    w = np.linalg.eigvalsh(K)
    assert w[0] > -1e-13 and abs(w[0]) < 1e-12 and w[1] > 1e-8  # one-dimensional kernel (constants)
    fixed = np.zeros(g.n_nodes, np.uint8)
    fixed[0] = 1
    A = fem.apply_dirichlet(fem.assemble(g, kv), fixed).toarray()
    assert np.linalg.eigvalsh(A)[0] > 0.0


def test_simp_endpoints():
    k = fem.simp(np.array([0.0, 1.0, 0.5]), 1.0, 1e-3, 3.0)
    np.testing.assert_allclose(k, [1e-3, 1.0, 1e-3 + (1 - 1e-3) * 0.125])


@pytest.mark.parametrize("dims", [(12, 3, 0), (8, 2, 2)])
def test_one_dimensional_exact_solution(dims):
    """rho = 1, T = 0 on the whole x = 0 face, uniform source Q: linear FE
    is nodally exact for -T'' = Q, T(0) = 0, T'(L) = 0: T = Q (L x - x^2/2)."""
    nx, ny, nz = dims
    g = fem.Grid(nx, ny, nz)
    idx = np.arange(g.n_nodes)
    x = idx % g.NX
    fixed = (x == 0).astype(np.uint8)
    Q = 0.37
    q = workloads.volumetric_load(nx, ny, nz, Q, fixed)
    A = fem.system_matrix(g, np.ones(g.n_elems), fixed)
    expect = Q * (nx * x - 0.5 * x * x)
    np.testing.assert_allclose(solvers.exact_solve(A, q), expect, rtol=1e-12, atol=1e-12)
    dims_e = (nx, ny) if nz == 0 else (nx, ny, nz)
    levels = multigrid.build_hierarchy(A, fixed, dims_e, 2)
    t, it, rr = solvers.mgcg(A, q, np.zeros(g.n_nodes), levels, eps2=1e-14, cg_max=200)
    np.testing.assert_allclose(t, expect, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("dims", [(7, 5, 0), (4, 3, 5)])
def test_node_by_node_matches_assembly(dims):
    g = fem.Grid(*dims)
    rng = np.random.default_rng(2)
    kv = fem.simp(rng.uniform(0.0, 1.0, g.n_elems), 1.0, 1e-3, 3.0)
    fixed = (rng.uniform(size=g.n_nodes) < 0.1).astype(np.uint8)
    A = fem.apply_dirichlet(fem.assemble(g, kv), fixed)
    x = rng.standard_normal(g.n_nodes)
    nodes = np.arange(g.n_nodes)
    np.testing.assert_allclose(fem.apply_node(g, kv, fixed, x, nodes), A @ x, atol=1e-13)


# ------------------------------------------------- the vectorised operator
# apply_structured is the checker of the full-size residual test; it is pinned
# here to the assembled matrix, to a brute-force element loop over the
# Kronecker-built element matrix, and to the textbook solution it must map to
# the load.
@pytest.mark.parametrize("dims", [(7, 5, 0), (13, 1, 0), (4, 3, 5), (5, 2, 3), (1, 1, 1)])
def test_structured_matches_assembly(dims):
    g = fem.Grid(*dims)
    rng = np.random.default_rng(3)
    kv = fem.simp(rng.uniform(0.0, 1.0, g.n_elems), 1.0, 1e-3, 3.0)
    fixed = (rng.uniform(size=g.n_nodes) < 0.15).astype(np.uint8)
    A = fem.apply_dirichlet(fem.assemble(g, kv), fixed)
    x = rng.standard_normal(g.n_nodes)
    np.testing.assert_allclose(fem.apply_structured(g, kv, fixed, x), A @ x, atol=1e-13)


@pytest.mark.parametrize("dims", [(4, 3, 0), (3, 2, 2)])
def test_structured_matches_element_loop(dims):
    """y_i = x_i on fixed nodes, else sum over elements e and local pairs (a, b)
    with node_a(e) = i and node_b(e) free of k_e k0_ab x_b."""
    g = fem.Grid(*dims)
    dim = 2 if dims[2] == 0 else 3
    k0 = kron_sum(dim)
    rng = np.random.default_rng(4)
    kv = rng.uniform(0.01, 2.0, g.n_elems)
    fixed = (rng.uniform(size=g.n_nodes) < 0.2).astype(np.uint8)
    x = rng.standard_normal(g.n_nodes)
    y = np.zeros(g.n_nodes)
    nz = max(dims[2], 1)
    for ek in range(nz):
        for ej in range(dims[1]):
            for ei in range(dims[0]):
                e = ei + dims[0] * (ej + dims[1] * ek)
                nodes = [(ei + (a & 1)) + g.NX * ((ej + ((a >> 1) & 1)) + g.NY * (ek + ((a >> 2) & 1)))
                         for a in range(2 ** dim)]
                for a, na in enumerate(nodes):
                    for b, nb in enumerate(nodes):
                        if not fixed[na] and not fixed[nb]:
                            y[na] += kv[e] * k0[a, b] * x[nb]
    y[fixed == 1] = x[fixed == 1]
    np.testing.assert_allclose(fem.apply_structured(g, kv, fixed, x), y, atol=1e-13)


@pytest.mark.parametrize("dims", [(12, 3, 0), (8, 2, 2)])
def test_structured_maps_exact_solution_to_load(dims):
    """With rho = 1 and T = 0 on the x = 0 face, A applied to the nodally exact
    T = Q (L x - x^2/2) returns the consistent load (zero on fixed nodes)."""
    nx, ny, nz = dims
    g = fem.Grid(nx, ny, nz)
    x = np.arange(g.n_nodes) % g.NX
    fixed = (x == 0).astype(np.uint8)
    Q = 0.37
    q = workloads.volumetric_load(nx, ny, nz, Q, fixed)
    t = Q * (nx * x - 0.5 * x * x)
    np.testing.assert_allclose(fem.apply_structured(g, np.ones(g.n_elems), fixed, t), q,
                               rtol=1e-12, atol=1e-12)
