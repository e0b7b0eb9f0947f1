"""Whole design cycles (filter, MGCG/MGAR, sensitivities, OC) on the GPU
against the oracle's loop, fed the same inputs each cycle (stepwise)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import design, loop  # noqa: E402
from paper_2210_00947_gb300 import mgar, workloads  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def run_stepwise(nx, ny, nz, nl, iters, n_on, precision, eps1=0.5, eps2=1e-12, guess="previous",
                 volfrac=0.4, filter_alpha=0.0, filter_lp=0, omega=0.9):
    """Feed the GPU the oracle's design and temperatures every cycle and
    record both cycles.  When the two decide MGCG/MGAR differently (Res within
    rounding of eps1), the GPU's reference K0 is set back to the oracle's
    (the physical density of the oracle's last MGCG cycle, hierarchy
    rebuilt), so the cycles after it are compared on the same K0; the entry
    of such a cycle is marked synced = False."""
    fixed = workloads.heat_sink_mask(nx, ny, nz)
    q = workloads.nodal_load(fixed)
    nel = workloads.num_elements(nx, ny, nz)
    s = loop.LoopSettings(nx=nx, ny=ny, nz=nz, volfrac=volfrac, iters=iters, n_on=n_on, nl=nl,
                          eps1=eps1, eps2=eps2, basis_guess=guess, filter_alpha=filter_alpha,
                          filter_lp=filter_lp, omega=omega)
    an = loop.Analysis(s, fixed, q)
    bg = mgar.MGAR_GUESS_PREVIOUS if guess == "previous" else mgar.MGAR_GUESS_ZERO
    p = mgar.default_params(nx=nx, ny=ny, nz=nz, nl=nl, eps1=eps1, eps2=eps2, n_on=n_on,
                            volfrac=volfrac, move=0.2, precision=precision, basis_guess=bg,
                            filter_alpha=filter_alpha, filter_lp=filter_lp, omega=omega)
    out = []
    with mgar.Solver(p, fixed, q) as solver:
        rho = np.full(nel, volfrac)
        t = np.zeros(an.grid.n_nodes)
        rho_g = torch.empty(nel, dtype=torch.float64, device=DEV)
        T_g = torch.empty(an.grid.n_nodes, dtype=torch.float64, device=DEV)
        k0_phys = None
        for k in range(1, iters + 1):
            rho_g.copy_(torch.from_numpy(rho))
            T_g.copy_(torch.from_numpy(t))
            g = solver.step(rho_g, T_g, k)
            rho_n, t_n, o = an.cycle(k, rho, t)
            if o["mgcg"]:  # the oracle's K0 is now K(F rho) with this cycle's filter
                k0_phys = design.filter_forward(an.H, an.Hs, rho)
            torch.cuda.synchronize()
            synced = g["used_mgcg"] == o["mgcg"]
            out.append((k, g, o, rho_g.cpu().numpy(), rho_n, T_g.cpu().numpy(), t_n, synced))
            if not synced:
                solver.set_density(torch.from_numpy(k0_phys).to(DEV), physical=True)
                solver.build_hierarchy()
            rho, t = rho_n, t_n
    return out


def counts(out):
    """(cycles compared with the same decision, accepted MGAR cycles among them)."""
    same = [e for e in out if e[7]]
    return len(same), sum(1 for e in same if e[2]["accepted"])


def test_fp64_loop_2d_heat2d_100():
    out = run_stepwise(100, 100, 0, nl=4, iters=24, n_on=13, precision=mgar.MGAR_FP64)
    assert len(out) == 24
    for k, g, o, rg, ro, tg, to, synced in out:
        assert g["used_mgcg"] == o["mgcg"]
        assert abs(g["compliance"] - o["compliance"]) / o["compliance"] < 1e-9, k
        if o["res"] == o["res"]:
            assert abs(g["res"] - o["res"]) < 1e-9 * max(1, o["res"]), k
            assert abs(g["compliance_mgar"] - o["compliance_mgar"]) < 1e-9 * o["compliance_mgar"], k
        assert np.max(np.abs(rg - ro)) < 1e-8, k


def test_fp64_loop_zero_guess_accepts():
    out = run_stepwise(64, 64, 0, nl=3, iters=30, n_on=8, precision=mgar.MGAR_FP64, guess="zero")
    acc = [g for k, g, o, *_ in out if g["accepted"]]
    assert len(out) == 30 and len(acc) > 0
    for k, g, o, rg, ro, tg, to, synced in out:
        assert abs(g["compliance"] - o["compliance"]) / o["compliance"] < 1e-9, k
        assert np.max(np.abs(rg - ro)) < 1e-8, k


def test_fp64_loop_3d():
    out = run_stepwise(16, 16, 16, nl=3, iters=8, n_on=4, precision=mgar.MGAR_FP64, volfrac=0.3)
    assert len(out) == 8
    for k, g, o, rg, ro, tg, to, synced in out:
        assert abs(g["compliance"] - o["compliance"]) / o["compliance"] < 1e-9, k
        assert np.max(np.abs(rg - ro)) < 1e-8, k


def check_mixed(out, iters, eps1, tol, min_accepted):
    """Every cycle of the run is recorded; cycles decided differently are only
    allowed where the oracle's Res lies within rounding of eps1; every cycle
    decided alike matches the oracle's compliance within tol, and at least
    min_accepted of them are accepted MGAR cycles."""
    assert len(out) == iters
    for k, g, o, rg, ro, tg, to, synced in out:
        if not synced:
            assert abs(o["res"] - eps1) < 1e-3 * eps1, k
            continue
        assert abs(g["compliance"] - o["compliance"]) / o["compliance"] < tol, k
        if o["res"] == o["res"]:  # an MGAR attempt, accepted or not: its reduced compliance
            assert abs(g["compliance_mgar"] - o["compliance_mgar"]) / o["compliance_mgar"] < tol, k
        else:
            assert g["compliance_mgar"] != g["compliance_mgar"], k  # NaN: no attempt
    n_same, n_acc = counts(out)
    n_near = sum(1 for e in out if abs(e[2]["res"] - eps1) < 1e-3 * eps1)
    assert n_same >= iters - n_near
    assert n_acc >= min_accepted


# eps1 per reading of Eq. 17 so that MGAR is accepted in several cycles of
# the 24 (the oracle accepts 4 with the literal basis at 2.0, 4 with the
# zero-guess basis at 0.8 and 2 at the paper's 0.5, where the literal basis
# is accepted in none)
@pytest.mark.parametrize("guess,eps1,min_acc", [("previous", 2.0, 4), ("zero", 0.8, 4),
                                                 ("zero", 0.5, 2)])
def test_mixed_loop_compliance_within_1e6(guess, eps1, min_acc):
    out = run_stepwise(100, 100, 0, nl=4, iters=24, n_on=13, precision=mgar.MGAR_MIXED,
                       eps1=eps1, eps2=1e-10, guess=guess)
    check_mixed(out, 24, eps1, 1e-6, min_acc)


@pytest.mark.parametrize("dims,nl,precision,tol,eps1,min_acc", [
    ((48, 40, 0), 3, "fp64", 1e-9, 1.5, 1), ((48, 40, 0), 3, "mixed", 1e-6, 1.5, 1),
    ((16, 16, 12), 3, "mixed", 1e-6, 1.5, 3)])
def test_loop_continuous_filter(dims, nl, precision, tol, eps1, min_acc):
    """Continuous filter radius (Eq. 22-23): r^(0) = 0.2 L shrinking to
    r_min = 1.5 over 5 cycles; the GPU rebuilds its filter tables each cycle
    and follows the oracle's loop (MGAR from cycle 4 on)."""
    prec = mgar.MGAR_FP64 if precision == "fp64" else mgar.MGAR_MIXED
    nx, ny, nz = dims
    out = run_stepwise(nx, ny, nz, nl=nl, iters=8, n_on=4, precision=prec, guess="zero",
                       eps1=eps1, eps2=1e-12 if precision == "fp64" else 1e-10, volfrac=0.4,
                       filter_alpha=0.2, filter_lp=5)
    check_mixed(out, 8, eps1, tol, min_acc)
    if precision == "fp64":
        for k, g, o, rg, ro, tg, to, synced in out:
            assert synced and np.max(np.abs(rg - ro)) < 1e-8, k


# A 3D loop of the mixed path (tiled FP32 V-cycle and CG iterations with
# df64 reliable updates, df64 MGAR projection) on 49^3 nodes with accepted
# MGAR cycles under both readings of Eq. 17 (the oracle accepts 3 of the 11
# attempts in each).
@pytest.mark.parametrize("guess,eps1,min_acc", [("zero", 1.0, 3), ("previous", 2.5, 3)])
def test_mixed_loop_3d_accepts_mgar(guess, eps1, min_acc):
    out = run_stepwise(48, 48, 48, nl=4, iters=14, n_on=4, precision=mgar.MGAR_MIXED, eps1=eps1,
                       eps2=1e-10, guess=guess, volfrac=0.3)
    check_mixed(out, 14, eps1, 1e-6, min_acc)
