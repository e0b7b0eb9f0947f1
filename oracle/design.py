"""Density filter, compliance, sensitivities and the OC update (oracle).

Eq. 6-8: rho~_e = sum_i w_ei rho_i / sum_i w_ei over elements whose
centroid lies within r of e's centroid, with the cone weight
w_ei = max(0, r - ||c_i - c_e||); element volumes are equal and cancel.
Reading: only in-domain neighbours enter both sums.

Eq. 5: compliance f = t^T K t, which equals q^T t at equilibrium.
Eq. 10: df/drho~_e = -p (k0 - kmin) rho~_e^(p-1) t_e^T k0_e t_e.
Eq. 9, 11: df/drho_j = sum_e df/drho~_e * w_ej / sum_i w_ei.

The optimality-criteria update is not in the paper (it only names the
classical SIMP framework); this is the usual OC rule: rho_new =
clamp(rho * sqrt(-dc / (lambda dv)), rho - move, rho + move, [0, 1]) with
lambda found by bisection so that the mean filtered density equals volfrac.
Reading of the volume constraint g_v of Eq. 5: mean(rho~) = volfrac, whose
gradient is dv = F^T (1 / n_elems).  The bisection runs on [1e-40, 1e40]
with geometric midpoints until (hi - lo) / (hi + lo) <= 1e-13 or 200 steps.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.sparse as sp

from .fem import Grid, element_conductivity


def filter_matrix(grid: Grid, r: float) -> tuple[sp.csr_matrix, np.ndarray]:
    """H (n_elems x n_elems) with H_ei = max(0, r - dist(c_e, c_i)) and its
    row sums Hs."""
    dims = (grid.nx, grid.ny) if grid.dim == 2 else (grid.nx, grid.ny, grid.nz)
    reach = int(np.ceil(r))
    shape = dims[::-1]  # array order (z, y, x)
    ids = np.arange(grid.n_elems).reshape(shape)
    rows, cols, vals = [], [], []
    for off in itertools.product(range(-reach, reach + 1), repeat=grid.dim):
        w = r - np.sqrt(float(sum(o * o for o in off)))
        if w <= 0.0:
            continue
        # offsets are (dx, dy[, dz]); array axes are reversed
        src = [slice(max(0, -o), n - max(0, o)) for o, n in zip(off, dims)][::-1]
        dst = [slice(max(0, o), n + min(0, o)) for o, n in zip(off, dims)][::-1]
        a = ids[tuple(src)].reshape(-1)
        b = ids[tuple(dst)].reshape(-1)
        rows.append(a)
        cols.append(b)
        vals.append(np.full(a.shape[0], w))
    H = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(grid.n_elems, grid.n_elems))
    Hs = np.asarray(H.sum(axis=1)).reshape(-1)
    return H, Hs


def filter_radius(k: int, rmin: float, alpha: float, L: float, lp: int) -> float:
    """Filter radius of design cycle k (1-based) under the continuous
    schedule, Eq. 22-23: r^(k) = max(r_min, eta r^(k-1)) from r^(0) = alpha L,
    eta = exp((ln r_min - ln(alpha L)) / lp), so that r reaches r_min after lp
    cycles.  Reading: the recursion is applied from the first cycle on; when
    alpha L <= r_min there is nothing to shrink and r = r_min throughout."""
    r0 = alpha * L
    if not (r0 > rmin) or lp <= 0:
        return rmin
    eta = math.exp((math.log(rmin) - math.log(r0)) / lp)
    r = r0
    for _ in range(k):
        r = max(rmin, eta * r)
    return r


def filter_forward(H, Hs, x):
    """Eq. 6."""
    return (H @ x) / Hs


def filter_transpose(H, Hs, y):
    """Chain rule of Eq. 9 with Eq. 11: (F^T y)_j = sum_e H_ej y_e / Hs_e."""
    return H.T @ (y / Hs)


def compliance(q, t) -> float:
    """Eq. 5 at equilibrium: f = q^T t."""
    return float(q @ t)


def element_energy(grid: Grid, t: np.ndarray) -> np.ndarray:
    """t_e^T k0 t_e per element."""
    ke = element_conductivity(grid.dim)
    te = t[grid.element_nodes()]
    return np.einsum("ea,ab,eb->e", te, ke, te)


def sensitivity_physical(grid: Grid, rho_phys, t, k0=1.0, kmin=1e-3, penal=3.0):
    """Eq. 10: df/drho~_e."""
    return -penal * (k0 - kmin) * rho_phys ** (penal - 1.0) * element_energy(grid, t)


def sensitivities(grid: Grid, H, Hs, rho_phys, t, k0=1.0, kmin=1e-3, penal=3.0):
    """Design sensitivities of compliance and of the mean filtered density:
    (dc, dv) = (F^T df/drho~, F^T 1/n_elems)."""
    dct = sensitivity_physical(grid, rho_phys, t, k0, kmin, penal)
    dc = filter_transpose(H, Hs, dct)
    dv = filter_transpose(H, Hs, np.full(grid.n_elems, 1.0 / grid.n_elems))
    return dc, dv


def oc_update(rho, dc, dv, volfrac, move=0.2, lo=1e-40, hi=1e40, tol=1e-13, max_steps=200):
    """OC update with bisection on lambda.  Returns (rho_new, lambda)."""
    rho = np.asarray(rho, dtype=np.float64)
    ratio = np.maximum(-dc, 0.0) / dv
    lower = np.maximum(0.0, rho - move)
    upper = np.minimum(1.0, rho + move)
    lam = np.sqrt(lo * hi)
    for _ in range(max_steps):
        lam = np.sqrt(lo * hi)
        rho_new = np.clip(rho * np.sqrt(ratio / lam), lower, upper)
        if dv @ rho_new > volfrac:
            lo = lam
        else:
            hi = lam
        if (hi - lo) / (hi + lo) <= tol:
            break
    lam = np.sqrt(lo * hi)
    rho_new = np.clip(rho * np.sqrt(ratio / lam), lower, upper)
    return rho_new, lam
