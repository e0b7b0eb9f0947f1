"""Solvers of K(rho~) t = q (oracle): exact, MGCG and MGAR.

MGCG (Section 1, Section 3.2): conjugate gradients preconditioned by one
multigrid V-cycle, stopped when the solution accuracy drops below eps2 or
after cg_max iterations.  Reading of "solution accuracy": the relative norm
||r||_2 / ||q||_2 of the recursively updated CG residual.

MGAR (Section 2.2, Eq. 12-21, and Eq. 28):
  r_1 = t_0 (the previous design cycle's temperatures),
  r_i <- MG(K0, -dK r_{i-1}, r_{i-1}, P)   (Eq. 17, one V-cycle on the
          hierarchy of the last factorised matrix K0, initial guess r_{i-1}),
  R~  = orthonormal basis of span(R)       (Eq. 18; Gram-Schmidt here),
  (R~^T K R~) y = R~^T q,  t~ = R~ y       (Eq. 19-21),
  Res = ||K R~ y - q|| / ||q||             (Eq. 28).
Readings: dK = A(rho~) - A(rho~_0) with both Dirichlet-reduced; the
orthonormalisation is modified Gram-Schmidt applied twice, dropping a vector
whose norm falls below 1e-12 ||r_1||; the zero-initial-guess form of Eq. 17
is available as `basis_guess="zero"`.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from . import multigrid as mg


def exact_solve(A, b) -> np.ndarray:
    """The plain definition: t = A^{-1} b by sparse LU."""
    return spla.spsolve(A.tocsc(), b)


def mgcg(A, b, x0, levels, eps2=1e-8, cg_max=200, omega=0.9, nu_pre=1, nu_post=1):
    """Preconditioned CG with z = V-cycle(r) (zero initial guess).
    Returns (x, iterations, relres)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(x), 0, 0.0
    r = b - A @ x
    relres = np.linalg.norm(r) / bnorm
    if relres <= eps2:
        return x, 0, relres
    z = mg.vcycle(levels, r, np.zeros_like(r), omega, nu_pre, nu_post)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < cg_max:
        Ap = A @ p
        alpha = rz / (p @ Ap)
        x = x + alpha * p
        r = r - alpha * Ap
        it += 1
        relres = np.linalg.norm(r) / bnorm
        if relres <= eps2:
            break
        z = mg.vcycle(levels, r, np.zeros_like(r), omega, nu_pre, nu_post)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, relres


def gram_schmidt(R: np.ndarray, drop_tol=1e-12) -> np.ndarray:
    """Orthonormal basis of the columns of R: modified Gram-Schmidt, each
    vector orthogonalised twice against the accepted ones; a vector whose
    norm falls below drop_tol * ||R[:, 0]|| is dropped."""
    ref = np.linalg.norm(R[:, 0])
    Q = []
    for i in range(R.shape[1]):
        v = R[:, i].copy()
        for _ in range(2):
            for q in Q:
                v = v - (q @ v) * q
        nv = np.linalg.norm(v)
        if nv > drop_tol * ref and nv > 0.0:
            Q.append(v / nv)
    return np.stack(Q, axis=1)


def orthonormal_basis_svd(R: np.ndarray, drop_tol=1e-12) -> np.ndarray:
    """Eq. 18 as printed: R = R~ Sigma V^T, keeping left singular vectors
    whose singular value exceeds drop_tol * sigma_max."""
    U, s, _ = np.linalg.svd(R, full_matrices=False)
    return U[:, s > drop_tol * s[0]]


def mgar_basis(A, A0, levels0, t0, m, omega=0.9, nu_pre=1, nu_post=1, basis_guess="previous"):
    """Eq. 17: r_1 = t_0; r_i = one V-cycle on K0 with right-hand side
    -dK r_{i-1} and initial guess r_{i-1} (or zero)."""
    R = [np.array(t0, dtype=np.float64, copy=True)]
    for _ in range(1, m):
        prev = R[-1]
        b = -(A @ prev - A0 @ prev)
        guess = prev.copy() if basis_guess == "previous" else np.zeros_like(prev)
        R.append(mg.vcycle(levels0, b, guess, omega, nu_pre, nu_post))
    return np.stack(R, axis=1)


def reduced_solve(A, q, Rt):
    """Eq. 19-21 and Eq. 28: y from (R~^T A R~) y = R~^T q by Cholesky,
    t~ = R~ y, Res = ||A R~ y - q|| / ||q||."""
    W = A @ Rt
    KR = Rt.T @ W
    qR = Rt.T @ q
    y = sla.cho_solve(sla.cho_factor(KR, lower=True), qR)
    t = Rt @ y
    res = np.linalg.norm(W @ y - q) / np.linalg.norm(q)
    return t, res, y


def mgar(A, A0, levels0, q, t0, m=2, omega=0.9, nu_pre=1, nu_post=1, basis_guess="previous",
         orthonormalise="gs"):
    """One MGAR reanalysis.  Returns (t~, Res)."""
    R = mgar_basis(A, A0, levels0, t0, m, omega, nu_pre, nu_post, basis_guess)
    Rt = gram_schmidt(R) if orthonormalise == "gs" else orthonormal_basis_svd(R)
    t, res, _ = reduced_solve(A, q, Rt)
    return t, res
