"""The MGAR-based optimisation loop (oracle), Section 3.1 / Figure 5.

Per design cycle k = 1..iters:
  rho~ = F rho                                       (Eq. 6-8)
  if k < N_on or no factorised matrix yet:            (Section 3.1)
      t = MGCG(K(rho~), q, t_prev); K0 <- K(rho~)    (hierarchy rebuilt)
  else:
      t~, Res = MGAR(K0 hierarchy, K(rho~), t_prev)  (Eq. 17-21, 28)
      if Res <= eps1: t = t~
      else: t = MGCG(K(rho~), q, t_prev); K0 <- K(rho~)
  f = q^T t; (dc, dv) = sensitivities                 (Eq. 5, 9-11)
  rho = OC(rho, dc, dv)                               (not in the paper)
Reading: t_prev starts at zero; MGCG always starts from t_prev.  With the
continuous filter (Eq. 22-23) the filter of cycle k has radius r^(k).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import design, fem, multigrid, solvers


@dataclasses.dataclass
class LoopSettings:
    nx: int
    ny: int
    nz: int
    volfrac: float
    iters: int
    n_on: int
    nl: int
    k0: float = 1.0
    kmin: float = 1e-3
    penal: float = 3.0
    rmin: float = 1.5
    move: float = 0.2
    eps1: float = 0.5
    eps2: float = 1e-8
    cg_max: int = 200
    m: int = 2
    omega: float = 0.9
    nu_pre: int = 1
    nu_post: int = 1
    basis_guess: str = "previous"
    use_mgar: bool = True
    # continuous filter radius (Eq. 22-23): off when filter_alpha is 0;
    # L defaults to the longest side in elements
    filter_alpha: float = 0.0
    filter_lp: int = 0
    filter_L: float = 0.0


class Analysis:
    """State that persists across design cycles: the filter, and the
    factorised matrix K0 with its multigrid hierarchy."""

    def __init__(self, s: LoopSettings, fixed, q):
        self.s = s
        self.grid = fem.Grid(s.nx, s.ny, s.nz)
        self.fixed = np.asarray(fixed)
        self.q = np.asarray(q, dtype=np.float64)
        self.r = s.rmin
        self.H, self.Hs = design.filter_matrix(self.grid, self.r)
        self.A0 = None
        self.levels0 = None
        self.dims = (s.nx, s.ny) if s.nz == 0 else (s.nx, s.ny, s.nz)

    def system(self, rho_phys):
        s = self.s
        return fem.system_matrix(self.grid, rho_phys, self.fixed, s.k0, s.kmin, s.penal)

    def run_mgcg(self, A, t_prev):
        s = self.s
        levels = multigrid.build_hierarchy(A, self.fixed, self.dims, s.nl)
        t, it, relres = solvers.mgcg(A, self.q, t_prev, levels, s.eps2, s.cg_max, s.omega,
                                     s.nu_pre, s.nu_post)
        self.A0, self.levels0 = A, levels
        return t, it, relres

    def cycle(self, k, rho, t_prev):
        """One design cycle; returns (rho_new, t, info)."""
        s = self.s
        if s.filter_alpha > 0.0:
            L = s.filter_L or float(max(s.nx, s.ny, s.nz))
            r = design.filter_radius(k, s.rmin, s.filter_alpha, L, s.filter_lp)
            if r != self.r:
                self.r = r
                self.H, self.Hs = design.filter_matrix(self.grid, r)
        rho_phys = design.filter_forward(self.H, self.Hs, rho)
        A = self.system(rho_phys)
        info = dict(cycle=k, mgcg=False, accepted=False, res=float("nan"), cg_iters=0,
                    compliance_mgar=float("nan"))
        if (not s.use_mgar) or k < s.n_on or self.levels0 is None:
            t, it, relres = self.run_mgcg(A, t_prev)
            info.update(mgcg=True, cg_iters=it, relres=relres)
        else:
            t, res = solvers.mgar(A, self.A0, self.levels0, self.q, t_prev, s.m, s.omega,
                                  s.nu_pre, s.nu_post, s.basis_guess)
            info["res"] = res
            info["compliance_mgar"] = design.compliance(self.q, t)
            if res <= s.eps1:
                info["accepted"] = True
            else:
                t, it, relres = self.run_mgcg(A, t_prev)
                info.update(mgcg=True, cg_iters=it, relres=relres)
        info["compliance"] = design.compliance(self.q, t)
        dc, dv = design.sensitivities(self.grid, self.H, self.Hs, rho_phys, t, s.k0, s.kmin,
                                      s.penal)
        rho_new, lam = design.oc_update(rho, dc, dv, s.volfrac, s.move)
        info["lambda"] = lam
        info["change"] = float(np.max(np.abs(rho_new - rho)))
        return rho_new, t, info


def optimise(s: LoopSettings, fixed, q, rho0, callback=None):
    """Run s.iters design cycles from rho0; returns (rho, t, history)."""
    an = Analysis(s, fixed, q)
    rho = np.array(rho0, dtype=np.float64, copy=True)
    t = np.zeros(an.grid.n_nodes)
    history = []
    for k in range(1, s.iters + 1):
        t0 = time.perf_counter()
        rho, t, info = an.cycle(k, rho, t)
        info["seconds"] = time.perf_counter() - t0
        history.append(info)
        if callback is not None:
            callback(k, rho, t, info)
    return rho, t, history
