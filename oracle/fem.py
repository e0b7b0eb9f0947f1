"""Finite-element discretisation of steady conduction (oracle).

Eq. 2-3: the isotropic steady heat equation discretised by the Galerkin
method on a structured grid of unit bilinear (Q4, 2D) or trilinear (H8, 3D)
elements gives K t = q.  Eq. 4: each element's conductivity is the SIMP
interpolation k_e = kmin + (k0 - kmin) * rho_e^p.

The element matrix is not printed in the paper; here it is the plain
definition k0_ab = integral over the element of grad N_a . grad N_b, taken by
2-point Gauss quadrature per axis (exact for these polynomials).

Numbering: nodes and elements x-fastest; local node a of an element has bits
(a & 1, (a >> 1) & 1, (a >> 2) & 1) = offsets along x, y, z.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp


class Grid:
    """Structured grid of nx x ny (x nz) unit elements; nz = 0 means 2D."""

    def __init__(self, nx: int, ny: int, nz: int = 0):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.dim = 2 if self.nz == 0 else 3
        self.NX, self.NY = self.nx + 1, self.ny + 1
        self.NZ = self.nz + 1 if self.dim == 3 else 1
        self.n_nodes = self.NX * self.NY * self.NZ
        self.n_elems = self.nx * self.ny * (self.nz if self.dim == 3 else 1)
        self.nen = 2 ** self.dim  # nodes per element

    def node_index(self, i, j, k=0):
        return i + self.NX * (j + self.NY * k)

    def element_nodes(self) -> np.ndarray:
        """(n_elems, 2^dim) global node numbers in local order."""
        ez = np.arange(self.nz if self.dim == 3 else 1)
        ey = np.arange(self.ny)
        ex = np.arange(self.nx)
        EZ, EY, EX = np.meshgrid(ez, ey, ex, indexing="ij")
        EX, EY, EZ = EX.reshape(-1), EY.reshape(-1), EZ.reshape(-1)
        cols = []
        for a in range(self.nen):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            cols.append(self.node_index(EX + ax, EY + ay, EZ + az))
        return np.stack(cols, axis=1)

    def element_centroids(self) -> np.ndarray:
        ez = np.arange(self.nz if self.dim == 3 else 1) + 0.5
        ey = np.arange(self.ny) + 0.5
        ex = np.arange(self.nx) + 0.5
        EZ, EY, EX = np.meshgrid(ez, ey, ex, indexing="ij")
        if self.dim == 2:
            return np.stack([EX.reshape(-1), EY.reshape(-1)], axis=1)
        return np.stack([EX.reshape(-1), EY.reshape(-1), EZ.reshape(-1)], axis=1)


def element_conductivity(dim: int, h=None) -> np.ndarray:
    """k0_ab = int grad N_a . grad N_b over a box element of sides h (unit
    conductivity), by 2x2(x2) Gauss quadrature on the reference cube."""
    h = np.ones(dim) if h is None else np.asarray(h, dtype=np.float64)
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])  # Gauss points on [0,1]
    nen = 2 ** dim
    k = np.zeros((nen, nen))
    for pt in itertools.product(g, repeat=dim):
        # physical gradient of N_a = prod_d (bit ? s_d : 1 - s_d), s = x / h
        grads = np.zeros((nen, dim))
        for a in range(nen):
            bits = [(a >> d) & 1 for d in range(dim)]
            for d in range(dim):
                val = 1.0 / h[d] * (1.0 if bits[d] else -1.0)
                for e in range(dim):
                    if e != d:
                        val *= pt[e] if bits[e] else 1.0 - pt[e]
                grads[a, d] = val
        weight = np.prod(h) / 2 ** dim  # each Gauss weight is 1/2 per axis on [0,1]
        k += weight * grads @ grads.T
    return k


def simp(rho_phys: np.ndarray, k0: float, kmin: float, penal: float) -> np.ndarray:
    """Eq. 4: k = kmin + (k0 - kmin) * rho^p."""
    return kmin + (k0 - kmin) * rho_phys ** penal


def assemble(grid: Grid, kvals: np.ndarray) -> sp.csr_matrix:
    """K = sum_e k_e A_e^T k0 A_e (Eq. 3), assembled as CSR."""
    ke = element_conductivity(grid.dim)
    en = grid.element_nodes()
    nen = grid.nen
    rows = np.repeat(en, nen, axis=1).reshape(-1)
    cols = np.tile(en, (1, nen)).reshape(-1)
    vals = (kvals[:, None, None] * ke[None, :, :]).reshape(-1)
    K = sp.coo_matrix((vals, (rows, cols)), shape=(grid.n_nodes, grid.n_nodes)).tocsr()
    K.sum_duplicates()
    return K


def apply_dirichlet(K: sp.csr_matrix, fixed: np.ndarray) -> sp.csr_matrix:
    """A = Z K Z + (I - Z), Z = diag(free): fixed rows/columns replaced by
    identity rows (T = 0 imposed by elimination)."""
    free = (np.asarray(fixed) == 0).astype(np.float64)
    Z = sp.diags(free)
    return (Z @ K @ Z + sp.diags(1.0 - free)).tocsr()


def system_matrix(grid: Grid, rho_phys: np.ndarray, fixed: np.ndarray, k0=1.0, kmin=1e-3,
                  penal=3.0) -> sp.csr_matrix:
    """The Dirichlet-reduced conductivity matrix A(rho~) of K(rho~) t = q."""
    return apply_dirichlet(assemble(grid, simp(rho_phys, k0, kmin, penal)), fixed)


def apply_node(grid: Grid, kvals: np.ndarray, fixed: np.ndarray, x: np.ndarray, nodes) -> np.ndarray:
    """(A x)_i for selected nodes i, computed node by node from the element
    definition (sum over the elements touching i).  For checking sampled
    outputs on grids too large to assemble quickly."""
    ke = element_conductivity(grid.dim)
    out = np.zeros(len(nodes))
    fixed = np.asarray(fixed)
    for t, node in enumerate(nodes):
        node = int(node)
        if fixed[node]:
            out[t] = x[node]
            continue
        i = node % grid.NX
        j = (node // grid.NX) % grid.NY
        k = node // (grid.NX * grid.NY)
        acc = 0.0
        for off in itertools.product((-1, 0), repeat=grid.dim):
            ei, ej = i + off[0], j + off[1]
            ek = k + off[2] if grid.dim == 3 else 0
            if not (0 <= ei < grid.nx and 0 <= ej < grid.ny):
                continue
            if grid.dim == 3 and not (0 <= ek < grid.nz):
                continue
            e = ei + grid.nx * (ej + grid.ny * ek)
            a = (i - ei) + 2 * (j - ej) + (4 * (k - ek) if grid.dim == 3 else 0)
            for b in range(grid.nen):
                nb = grid.node_index(ei + (b & 1), ej + ((b >> 1) & 1),
                                     ek + ((b >> 2) & 1) if grid.dim == 3 else 0)
                if fixed[nb]:
                    continue
                acc += kvals[e] * ke[a, b] * x[nb]
        out[t] = acc
    return out


def apply_structured(grid: Grid, kvals: np.ndarray, fixed: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = A x with A = Z K Z + (I - Z), summed element by element over the
    local node pairs (a, b): y[node_a(e)] += k_e k0[a, b] x[node_b(e)].
    Same definition as assemble + apply_dirichlet, vectorised over elements
    so it stays usable on grids of millions of nodes."""
    ke = element_conductivity(grid.dim)
    free = (np.asarray(fixed) == 0)
    xf = np.where(free, x, 0.0)
    shape = (grid.NZ, grid.NY, grid.NX)
    X = xf.reshape(shape)
    Y = np.zeros(shape)
    nz = grid.nz if grid.dim == 3 else 1
    K = kvals.reshape(nz, grid.ny, grid.nx)

    def sl(a):
        ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
        zs = slice(az, az + nz) if grid.dim == 3 else slice(0, 1)
        return (zs, slice(ay, ay + grid.ny), slice(ax, ax + grid.nx))

    for a in range(grid.nen):
        acc = np.zeros_like(K)
        for b in range(grid.nen):
            if ke[a, b] != 0.0:
                acc += ke[a, b] * X[sl(b)]
        Y[sl(a)] += K * acc
    y = Y.reshape(-1)
    return np.where(free, y, x)
