"""Independent designs run concurrently (one handle, stream and host thread
each) give exactly the results of running them one after another, and each
follows the oracle's loop."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import loop  # noqa: E402
from paper_2210_00947_gb300 import batch, mgar  # noqa: E402

pytestmark = pytest.mark.gpu


def _designs():
    return [batch.Design(48, 32, 0, 0.5, 0.4), batch.Design(64, 48, 1, 0.2, 0.3),
            batch.Design(32, 64, 2, 0.7, 0.45), batch.Design(80, 80, 3, 0.0, 0.35),
            batch.Design(64, 64, 0, 0.9, 0.5)]


@pytest.mark.parametrize("precision", [mgar.MGAR_FP64, mgar.MGAR_MIXED])
def test_concurrent_designs_equal_sequential(precision):
    ds = _designs()
    seq, _ = batch.run_designs(ds, cycles=8, workers=1, precision=precision)
    par, _ = batch.run_designs(ds, cycles=8, workers=len(ds), precision=precision)
    for (rs, hs), (rp, hp) in zip(seq, par):
        np.testing.assert_array_equal(rs, rp)
        assert [h["compliance"] for h in hs] == [h["compliance"] for h in hp]


def test_batched_design_follows_the_oracle():
    d = _designs()[1]
    cycles = 6
    res, _ = batch.run_designs([d], cycles=cycles, workers=1, precision=mgar.MGAR_FP64,
                               eps2=1e-12)
    rho_g, hist = res[0]
    p = d.params(cycles, mgar.MGAR_FP64)
    s = loop.LoopSettings(nx=d.nx, ny=d.ny, nz=0, volfrac=d.volfrac, iters=cycles, n_on=p.n_on,
                          nl=p.nl, eps2=1e-12, eps1=p.eps1)
    rho_o, _, hist_o = loop.optimise(s, d.fixed(), d.q(), d.density())
    for g, o in zip(hist, hist_o):
        assert g["used_mgcg"] == o["mgcg"]
        assert abs(g["compliance"] - o["compliance"]) / o["compliance"] < 1e-9
    assert np.max(np.abs(rho_g - rho_o)) < 1e-8


# ------------------------------------------- batched MGCG (mgar_batch_*)
from oracle import design as odesign, fem, solvers  # noqa: E402
from paper_2210_00947_gb300 import workloads  # noqa: E402

UNEVEN = [batch.Design(64, 96, 0, 0.3, 0.35), batch.Design(128, 80, 1, 0.6, 0.3),
          batch.Design(96, 160, 2, 0.1, 0.45), batch.Design(160, 144, 3, 0.8, 0.25)]


def _batch_problem(designs, nl, eps2, seed=31):
    """Mixed-precision handles at random densities (different per design)."""
    solvers_, rhos = [], []
    for i, d in enumerate(designs):
        p = d.params(30, mgar.MGAR_MIXED, nl=nl, eps2=eps2, cg_max=300)
        s = mgar.Solver(p, d.fixed(), d.q())
        rho = workloads.random_density(d.nx * d.ny, 0.1, 1.0, seed=seed + i)
        s.set_density(torch.tensor(rho, device="cuda:0"))
        solvers_.append(s)
        rhos.append(rho)
    return solvers_, rhos


@pytest.mark.parametrize("nl", [5, 0])
def test_batched_solve_equals_one_at_a_time(nl):
    """Each design's batched solution and iteration count are bit-identical
    whether it is solved with the others or alone (nl 0: each design's own
    depth from the 300-node coarsest rule, so the depths differ)."""
    levels = [nl or workloads.levels_for_direct_coarsest(d.nx, d.ny, max_nodes=300)
              for d in UNEVEN]
    sv = []
    for d, l in zip(UNEVEN, levels):
        s, _ = _batch_problem([d], l, 1e-10)
        sv.append(s[0])
    rhos = [workloads.random_density(d.nx * d.ny, 0.1, 1.0, seed=31) for d in UNEVEN]
    for s, rho in zip(sv, rhos):
        s.set_density(torch.tensor(rho, device="cuda:0"))
    Ts = [torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda:0") for s in sv]
    with mgar.BatchSolver(sv) as b:
        res_all = b.solve(Ts)
        assert "level 0" in b.report()
    together = [t.cpu().numpy() for t in Ts]
    for i, s in enumerate(sv):
        T1 = torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda:0")
        with mgar.BatchSolver([s]) as b1:
            (it1, rr1, ok1), = b1.solve([T1])
        assert ok1 and res_all[i][2]
        assert it1 == res_all[i][0]
        np.testing.assert_array_equal(T1.cpu().numpy(), together[i])
    for s in sv:
        s.close()


def test_batched_solve_matches_the_oracle():
    """Four uneven designs (64 x 96 .. 160 x 144, nl 5, random densities),
    solved together to eps2 = 1e-11: each against the oracle's exact solve
    of its own system, element by element."""
    sv, rhos = _batch_problem(UNEVEN, 5, 1e-11)
    Ts = [torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda:0") for s in sv]
    with mgar.BatchSolver(sv) as b:
        res = b.solve(Ts)
        # warm start from the solutions: each design starts at the recomputed
        # true residual of its solution (the recursive one stopped the first
        # solve; in double-float arithmetic the two differ by a few units of
        # eps2 here), so it needs at most two more iterations
        res2 = b.solve(Ts)
    for d, s, rho, T, (it, rr, ok), (it2, _, ok2) in zip(UNEVEN, sv, rhos, Ts, res, res2):
        assert ok and rr <= 1e-11 and it > 0
        assert ok2 and it2 <= 2
        g = fem.Grid(d.nx, d.ny, 0)
        H, Hs = odesign.filter_matrix(g, s.params.rmin)
        A = fem.system_matrix(g, odesign.filter_forward(H, Hs, rho), d.fixed())
        q = d.q()
        t_ex = solvers.exact_solve(A, q)
        t = T.cpu().numpy()
        np.testing.assert_allclose(t, t_ex, rtol=0, atol=1e-9 * np.abs(t_ex).max())
        assert abs(q @ t - q @ t_ex) <= 1e-10 * abs(q @ t_ex)
    for s in sv:
        s.close()


def test_batched_solve_iteration_cap_per_design():
    """cg_max is per design: a design capped at 2 iterations stops there
    (status MAXIT) while the others converge."""
    sv, _ = _batch_problem(UNEVEN[:3], 5, 1e-10)
    d = UNEVEN[1]
    capped = mgar.Solver(d.params(30, mgar.MGAR_MIXED, nl=5, eps2=1e-10, cg_max=2), d.fixed(), d.q())
    capped.set_density(torch.tensor(workloads.random_density(d.nx * d.ny, 0.1, 1.0, seed=32),
                                    device="cuda:0"))
    sv[1].close()
    sv[1] = capped
    Ts = [torch.zeros(s.n_nodes, dtype=torch.float64, device="cuda:0") for s in sv]
    with mgar.BatchSolver(sv) as b:
        res = b.solve(Ts)
    assert res[1][0] == 2 and not res[1][2]
    assert res[0][2] and res[2][2] and res[0][0] > 2
    for s in sv:
        s.close()


def test_batched_design_loop_follows_the_per_handle_loop():
    """Design cycles with the batched solve (filter, batched MGCG,
    sensitivities, OC) against the same designs' per-handle loops (MGCG in
    every cycle): compliances within 1e-6 each cycle, densities within 1e-5."""
    ds = UNEVEN[:3]
    cycles = 5
    bat, _, report = batch.run_designs_batched(ds, cycles=cycles, workers=3, nl=5, eps2=1e-10)
    ref, _ = batch.run_designs(ds, cycles=cycles, workers=3, precision=mgar.MGAR_MIXED, nl=5,
                               eps2=1e-10, n_on=cycles + 1)
    assert "coarsest solve" in report
    for (rb, hb), (rr, hr) in zip(bat, ref):
        assert len(hb) == cycles
        for a, b in zip(hb, hr):
            assert a["converged"]
            assert abs(a["compliance"] - b["compliance"]) <= 1e-6 * abs(b["compliance"])
        assert np.max(np.abs(rb - rr)) < 1e-5


def test_batch_cycle_equals_its_steps(monkeypatch):
    """mgar_batch_cycle (filter, batched solve, sensitivities and OC queued for
    every design before any outcome is read) gives bit for bit what the same
    steps give called one by one: as graphs of per-design branches (captured
    again when the solution vectors move), and launched eagerly on the
    handles' streams."""
    ds = UNEVEN[:3]
    cycles = 4
    runs = []
    for mode in ("graphs", "eager", "steps"):
        fused = mode != "steps"
        if mode == "eager":
            monkeypatch.setenv("MGAR_NO_GRAPHS", "1")
        else:
            monkeypatch.delenv("MGAR_NO_GRAPHS", raising=False)
        sv, rh, Ts, vf = [], [], [], []
        for d in ds:
            p = d.params(cycles, mgar.MGAR_MIXED, nl=5, n_on=cycles + 1, eps2=1e-10)
            sv.append(mgar.Solver(p, d.fixed(), d.q(), stream=torch.cuda.Stream()))
            rh.append(torch.tensor(d.density(), device="cuda:0"))
            Ts.append(torch.zeros(sv[-1].n_nodes, dtype=torch.float64, device="cuda:0"))
            vf.append(d.volfrac)
        comps = []
        with mgar.BatchSolver(sv, stream=torch.cuda.Stream()) as b:
            for k in range(cycles):
                if k == 2:
                    Ts = [T.clone() for T in Ts]
                if fused:
                    comps.append([inf["compliance"] for inf in b.cycle(rh, Ts, vf, 0.2)])
                else:
                    for s, r in zip(sv, rh):
                        s.set_density(r)
                    torch.cuda.synchronize()
                    b.solve(Ts)
                    row = []
                    for s, r, T, v in zip(sv, rh, Ts, vf):
                        dc = torch.empty_like(r)
                        row.append(s.sensitivity(T, dc))
                        s.oc_update(r, dc, v, 0.2)
                    comps.append(row)
        torch.cuda.synchronize()
        runs.append(([r.cpu().numpy() for r in rh], comps))
        for s in sv:
            s.close()
    (ra, ca), *others = runs
    for rb, cb in others:
        assert ca == cb
        for a, b_ in zip(ra, rb):
            np.testing.assert_array_equal(a, b_)
