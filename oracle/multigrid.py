"""Geometric multigrid V-cycle (oracle), Section 2.2 and Table 1.

Table 1 gives one V-cycle x <- MG(A, b, x, P): pre-smooth, residual
restricted by P^T, coarse correction A^c x^c = res, interpolation
x <- x + P x^c, post-smooth; the smoother is damped Jacobi
x <- x + omega D^-1 (b - A x).  With more than two levels the coarse
correction is itself one V-cycle (zero initial guess) on the next level, and
the coarsest level is solved directly.

Readings where the paper is silent:
  * P is bilinear / trilinear interpolation between the node positions of
    the fine grid and of a grid with half as many elements per axis (rounded
    up, so an odd axis ends with one coarse element spanning one fine
    element, whose nodes are injected); R = P^T unscaled, as in Table 1.
    Positions are each level's own node indices, so on a level coarsened
    from a truncated one the interpolation is algebraic rather than
    geometric (the Galerkin product stays exact either way).
  * Dirichlet nodes: the finest transfer uses P0 = Z P (fixed fine nodes
    receive no correction), so every coarse operator is the Galerkin
    product A_{l+1} = P_l^T A_l P_l with no boundary conditions of its own.
  * omega = 0.9, one pre- and one post-sweep (parameters).  On the
    oscillatory modes the Jacobi-scaled symbol of the unit-conductivity
    stencil spans [0.75, 1.5] for Q4 and [0.5, 1.5] for H8, so the weights
    that best damp those modes are 2 / (0.75 + 1.5) = 0.89 and 1.0; 0.9 is
    taken for both.
  * the coarsest level is solved by a dense Cholesky factorisation.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def coarse_count(n: int) -> int:
    """Elements along an axis on the next coarser grid: ceil(n / 2)."""
    return (n + 1) // 2


def prolongation_1d(nf: int) -> sp.csr_matrix:
    """(nf+1) x (nc+1) linear interpolation from coarse node positions
    X_I = min(2I, nf) to fine node positions i = 0..nf."""
    nc = coarse_count(nf)
    X = np.minimum(2 * np.arange(nc + 1), nf).astype(np.float64)
    rows, cols, vals = [], [], []
    for i in range(nf + 1):
        J = np.searchsorted(X, i, side="right") - 1
        J = min(J, nc - 1)
        x0, x1 = X[J], X[J + 1]
        w1 = (i - x0) / (x1 - x0)
        for col, w in ((J, 1.0 - w1), (J + 1, w1)):
            if w != 0.0:
                rows.append(i)
                cols.append(col)
                vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf + 1, nc + 1))


def prolongation(dims) -> tuple[sp.csr_matrix, tuple]:
    """Tensor-product interpolation for an element grid `dims` = (nx, ny[, nz]),
    returning P and the coarse element dims.  Node vectors are x-fastest, so
    P = Pz (x) Py (x) Px."""
    Ps = [prolongation_1d(n) for n in dims]
    P = Ps[0]
    for Pd in Ps[1:]:
        P = sp.kron(Pd, P, format="csr")
    return P.tocsr(), tuple(coarse_count(n) for n in dims)


@dataclasses.dataclass
class Level:
    A: sp.csr_matrix          # operator on this level
    dinv: np.ndarray          # 1 / diag(A)
    P: sp.csr_matrix | None   # prolongation to this level from the next coarser one
    chol: tuple | None = None  # Cholesky factor on the coarsest level


def build_hierarchy(A0: sp.csr_matrix, fixed: np.ndarray, dims, nl: int) -> list[Level]:
    """Levels 0..nl-1: A_0 is the Dirichlet-reduced fine matrix; A_{l+1} =
    P_l^T A_l P_l with P_0 = Z P(dims) and P_l = P(coarse dims) for l >= 1."""
    free = (np.asarray(fixed) == 0).astype(np.float64)
    levels = []
    A = A0.tocsr()
    dims = tuple(dims)
    for l in range(nl):
        if l == nl - 1:
            levels.append(Level(A=A, dinv=1.0 / A.diagonal(), P=None,
                                chol=sla.cho_factor(A.toarray(), lower=True)))
            break
        P, cdims = prolongation(dims)
        if l == 0:
            P = (sp.diags(free) @ P).tocsr()
        levels.append(Level(A=A, dinv=1.0 / A.diagonal(), P=P))
        A = (P.T @ A @ P).tocsr()
        dims = cdims
    return levels


def jacobi(A, dinv, b, x, omega, sweeps):
    """Damped Jacobi x <- x + omega D^-1 (b - A x), `sweeps` times."""
    for _ in range(sweeps):
        x = x + omega * dinv * (b - A @ x)
    return x


def vcycle(levels: list[Level], b: np.ndarray, x: np.ndarray, omega=0.9, nu_pre=1, nu_post=1,
           level: int = 0) -> np.ndarray:
    """One V-cycle x <- MG(A_l, b, x, P) (Table 1), recursive over levels."""
    L = levels[level]
    if L.chol is not None:
        return sla.cho_solve(L.chol, b)
    x = jacobi(L.A, L.dinv, b, x, omega, nu_pre)               # 1: pre-smooth
    res = L.P.T @ (b - L.A @ x)                                # 2: restricted residual
    xc = vcycle(levels, res, np.zeros(res.shape[0]), omega,    # 3: coarse correction
                nu_pre, nu_post, level + 1)
    x = x + L.P @ xc                                           # 4: interpolation
    return jacobi(L.A, L.dinv, b, x, omega, nu_post)           # 5: post-smooth
