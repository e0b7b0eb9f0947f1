"""Kernel-class timing (mgar_profile_*): every class that a solve launches
reports launches and a positive time, and timing a solve does not change
its result (a timed solve runs the host-driven loop instead of the
device-side graph, with the same arithmetic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2210_00947_gb300 import mgar, workloads  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _solver(dims, nl):
    nx, ny, nz = dims
    fixed = workloads.heat_sink_mask(nx, ny, nz)
    q = workloads.nodal_load(fixed)
    rho = workloads.random_density(workloads.num_elements(nx, ny, nz), 0.2, 0.9, seed=7)
    p = mgar.default_params(nx=nx, ny=ny, nz=nz, nl=nl, eps2=1e-10, cg_max=300,
                            precision=mgar.MGAR_MIXED)
    s = mgar.Solver(p, fixed, q)
    s.set_density(torch.tensor(rho, device=DEV))
    return s


def _solve(s):
    T = torch.zeros(s.n_nodes, dtype=torch.float64, device=DEV)
    it, rr, ok = s.solve_mgcg(T)
    assert ok
    return T.cpu().numpy(), it


# 2D: the finest smoothing class nests the sweep's own scope inside the
# V-cycle's (one timed interval each); the df64 products are APPLY64.
# 3D: the tiled passes, the FP32 CG product and the df64 residuals.
@pytest.mark.parametrize("dims,nl,classes", [
    ((96, 80, 0), 4, [mgar.KC_SMOOTH0, mgar.KC_RESID0, mgar.KC_APPLY64]),
    ((24, 20, 16), 3, [mgar.KC_SMOOTH0, mgar.KC_APPLY32, mgar.KC_RESID64]),
])
def test_profiled_classes_report_and_leave_results_unchanged(dims, nl, classes):
    with _solver(dims, nl) as s:
        ref, it_ref = _solve(s)
        for kc in classes:
            s.profile_start(kc)
            t, it = _solve(s)
            ms, n = s.profile_stop()
            assert n >= 1 and ms > 0.0, (kc, n, ms)
            assert it == it_ref
            np.testing.assert_array_equal(t, ref)
        s.profile_start(mgar.KC_TIMELINE)
        t, _ = _solve(s)
        ms, n = s.profile_stop()
        assert n >= 10 and ms > 0.0
        assert "ms" in s.profile_report()
        np.testing.assert_array_equal(t, ref)
