"""Projection-based boundary post-processing (oracle), Section 2.3,
Eq. 24-27, run once after the optimisation loop.

Test infrastructure: only tests/, the smoke check and the benchmark's CPU
legs use this module.

Steps, in the paper's order:
  1. element sensitivities of the final design, s_e = -df/drho~_e (Eq. 10);
  2. projection onto the nodes "analogous to the density filter":
     ns_i = sum_e w_ie s_e / sum_e w_ie, w_ie = max(0, r - |x_i - c_e|);
  3. Eq. 24: an element is solid when all its nodes have ns > ns_level, void
     when all have ns < ns_level, and otherwise gets the intermediate density
     ev of Eq. 27: the element is discretised again by a lattice of points
     (the original nodes included), ns is interpolated to them with the
     bilinear / trilinear shape functions of Eq. 25-26, and ev is the share
     of lattice points with ns > ns_level;
  4. ns_level by bisection so that the mean density matches the volume
     fraction (the volume is non-increasing in ns_level).
Readings (the paper is silent): s_e is the magnitude of the physical-element
sensitivity; the projection radius is the filter radius r_min; the lattice
has S + 1 = 5 points per axis (local coordinates -1, -1/2, 0, 1/2, 1); the
bisection keeps the volume at or below the volume fraction and stops when
the bracket no longer shrinks.
"""
from __future__ import annotations

import itertools

import numpy as np

from .design import sensitivity_physical
from .fem import Grid

LATTICE = 4  # S: lattice intervals per axis in Eq. 25-27


def element_signal(grid: Grid, rho_phys, t, k0=1.0, kmin=1e-3, penal=3.0) -> np.ndarray:
    """s_e = -df/drho~_e (Eq. 10)."""
    return -sensitivity_physical(grid, rho_phys, t, k0, kmin, penal)


def nodal_projection(grid: Grid, s, r: float) -> np.ndarray:
    """ns_i = sum_e w_ie s_e / sum_e w_ie, w_ie = max(0, r - |x_i - c_e|),
    x_i the node position, c_e the element centroid (unit elements)."""
    dim = grid.dim
    ne_dims = (grid.nx, grid.ny) if dim == 2 else (grid.nx, grid.ny, grid.nz)
    nn_dims = tuple(n + 1 for n in ne_dims)
    s_arr = np.asarray(s, dtype=np.float64).reshape(ne_dims[::-1])
    num = np.zeros(nn_dims[::-1])
    den = np.zeros(nn_dims[::-1])
    reach = int(np.ceil(r + 0.5))
    # element e = node i + offset o (o: -reach..reach-1 per axis) has its
    # centroid at x_i + o + 1/2
    for off in itertools.product(range(-reach, reach), repeat=dim):
        d = np.sqrt(sum((o + 0.5) ** 2 for o in off))
        w = r - d
        if w <= 0.0:
            continue
        # nodes i with 0 <= i + o < ne along every axis
        node_sl, elem_sl = [], []
        for o, n in zip(off, ne_dims):
            lo = max(0, -o)
            hi = min(n + 1, n - o)
            node_sl.append(slice(lo, hi))
            elem_sl.append(slice(lo + o, hi + o))
        ns = tuple(node_sl[::-1])
        es = tuple(elem_sl[::-1])
        num[ns] += w * s_arr[es]
        den[ns] += w
    return (num / den).reshape(-1)


def lattice_shape_values(dim: int, S: int = LATTICE) -> np.ndarray:
    """(points, 2^dim) values of the shape functions of Eq. 26 (and their
    3D counterpart) at the (S+1)^dim lattice points of one element."""
    pts = np.linspace(-1.0, 1.0, S + 1)
    rows = []
    for p in itertools.product(pts, repeat=dim):  # p = (xi, eta[, zeta])
        vals = []
        for a in range(2 ** dim):
            loc = [2 * ((a >> b) & 1) - 1 for b in range(dim)]
            v = 1.0
            for pc, lc in zip(p, loc):
                v *= (1.0 + pc * lc)
            vals.append(v / 2 ** dim)
        rows.append(vals)
    return np.array(rows)


def densities(grid: Grid, ns, level: float, S: int = LATTICE) -> np.ndarray:
    """Eq. 24 with ev from Eq. 25-27."""
    nodes = grid.element_nodes()
    v = np.asarray(ns)[nodes]  # (E, 2^dim)
    rho = np.zeros(grid.n_elems)
    above = v > level
    below = v < level
    rho[above.all(axis=1)] = 1.0
    mixed = ~(above.all(axis=1) | below.all(axis=1))
    if mixed.any():
        N = lattice_shape_values(grid.dim, S)  # (P, 2^dim)
        vals = v[mixed] @ N.T  # (M, P), Eq. 25
        rho[mixed] = (vals > level).sum(axis=1) / N.shape[0]  # Eq. 27
    return rho


def level_for_volume(grid: Grid, ns, volfrac: float, S: int = LATTICE, max_steps: int = 200):
    """Bisection on ns_level: the bracket [lo, hi] keeps mean(rho(lo)) >
    volfrac >= mean(rho(hi)); returns (hi, rho(hi))."""
    lo, hi = float(np.min(ns)), float(np.max(ns))
    lo = lo - (abs(lo) + 1.0) * 1e-12  # everything solid below the smallest value
    for _ in range(max_steps):
        mid = 0.5 * (lo + hi)
        if not (lo < mid < hi):
            break
        if densities(grid, ns, mid, S).mean() > volfrac:
            lo = mid
        else:
            hi = mid
    return hi, densities(grid, ns, hi, S)


def postprocess(grid: Grid, rho_phys, t, volfrac: float, r: float, k0=1.0, kmin=1e-3,
                penal=3.0):
    """The whole post-processing: returns (rho_pp, ns, level)."""
    s = element_signal(grid, rho_phys, t, k0, kmin, penal)
    ns = nodal_projection(grid, s, r)
    level, rho = level_for_volume(grid, ns, volfrac)
    return rho, ns, level
