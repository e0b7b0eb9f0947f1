"""Many independent designs on one GPU at once.

Independent topology-optimisation problems (different grids, sinks and
volume fractions) share nothing, so they batch without any exchange: each
design gets its own handle (device buffers, multigrid hierarchy, CUDA graphs)
and its own CUDA stream, and a host thread drives its design cycles through
the C ABI.  ctypes releases the interpreter lock for the duration of each
library call, so the threads' host waits overlap and the GPU interleaves the
designs' kernels; small designs that cannot fill the GPU alone fill it
together.  Results do not depend on the interleaving: every reduction in the
library has a fixed order.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import math
import threading

import numpy as np

from . import mgar, workloads


@dataclasses.dataclass
class Design:
    """One 2D heat-sink design: an nx x ny grid with a sink patch of a tenth
    of one edge (edge 0..3, relative offset in [0, 1)) and a volume fraction."""
    nx: int
    ny: int
    edge: int
    offset: float
    volfrac: float

    def fixed(self) -> np.ndarray:
        return workloads.edge_patch_mask(self.nx, self.ny, self.edge, self.offset)

    def q(self) -> np.ndarray:
        return workloads.nodal_load(self.fixed())

    def density(self) -> np.ndarray:
        return workloads.uniform_density(self.nx * self.ny, self.volfrac)

    def params(self, cycles: int, precision: int = mgar.MGAR_MIXED, **overrides) -> mgar.Params:
        nl = workloads.levels_for_direct_coarsest(self.nx, self.ny, max_nodes=300)
        p = mgar.default_params(nx=self.nx, ny=self.ny, nz=0, nl=nl, volfrac=self.volfrac,
                                move=0.2, precision=precision,
                                n_on=int(math.floor(2.0 * cycles / 15.0 + 0.5)))
        for k, v in overrides.items():
            setattr(p, k, v)
        return p


def designs_from_workload(count: int = 64, seed: int = 2210) -> list[Design]:
    """The seeded set of uneven designs of the workload module."""
    return [Design(**d) for d in workloads.batched_designs(count, seed)]


def run_designs(designs: list[Design], cycles: int, workers: int = 16,
                precision: int = mgar.MGAR_MIXED, device: int = 0, **overrides):
    """Optimise every design for `cycles` design cycles, `workers` at a time
    (workers = 1: one after another) on CUDA device `device`.  Returns, per
    design, the final densities and the per-cycle reports, and the seconds
    the runs took (after every handle has been created, before any is
    destroyed)."""
    import time

    import torch

    n = len(designs)
    workers = max(1, min(workers, n))
    # every worker builds its handles, all start together, and the clock
    # stops when all have finished (before any handle is destroyed); a
    # failing worker breaks the barriers so that nobody waits for it
    ready = threading.Barrier(workers + 1, timeout=600)
    finished = threading.Barrier(workers + 1, timeout=3600)
    out = [None] * n
    per = -(-n // workers)
    chunks = [list(range(w * per, min(n, (w + 1) * per))) for w in range(workers)]

    def worker(jobs):
        built = []
        try:
            torch.cuda.set_device(device)
            stream = torch.cuda.Stream()
            for i in jobs:
                d = designs[i]
                s = mgar.Solver(d.params(cycles, precision, **overrides), d.fixed(), d.q(),
                                stream=stream)
                rho_in = torch.from_numpy(d.density()).pin_memory()
                rho_out = torch.empty_like(rho_in).pin_memory()
                built.append((i, s, rho_in, rho_out))
            ready.wait()
            for i, s, rho_in, rho_out in built:
                infos = s.run(rho_in, cycles, rho_out)
                out[i] = (rho_out.numpy().copy(), infos)
            stream.synchronize()
            finished.wait()
        except BaseException:
            ready.abort()
            finished.abort()
            raise
        finally:
            for _, s, _, _ in built:
                s.close()

    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = [ex.submit(worker, chunks[w]) for w in range(workers)]
        try:
            ready.wait()
            t0 = time.perf_counter()
            finished.wait()
            seconds = time.perf_counter() - t0
        except threading.BrokenBarrierError:
            seconds = float("nan")
        for f in futs:
            f.result()  # re-raises a worker's error
    return out, seconds


def run_designs_batched(designs: list[Design], cycles: int, workers: int = 16, device: int = 0,
                        nl: int = 0, **overrides):
    """Optimise every design for `cycles` design cycles, MGCG in every cycle,
    one mgar_batch_cycle per cycle for the whole set: each design's filter and
    SIMP on its own stream, the batched solve (one launch per V-cycle level
    and operation for all designs), then every design's sensitivities and OC
    update queued on its stream before any outcome is read.  Mixed precision
    (FP32 V-cycle, FP64 CG).  Returns, per design, the final densities and
    compliances, the seconds of the cycles, and the batched solver's
    autotuner report.  nl = 0: each design's own depth (coarsest level of
    at most 300 nodes, as the per-handle runner's).  `workers` is accepted
    for the per-handle runner's signature."""
    import time

    import torch

    del workers
    torch.cuda.set_device(device)
    dev = torch.device("cuda", device)
    solvers, rhos, Ts = [], [], []
    for d in designs:
        depth = {"nl": nl} if nl else {}
        p = d.params(cycles, mgar.MGAR_MIXED, n_on=cycles + 1, **depth, **overrides)
        solvers.append(mgar.Solver(p, d.fixed(), d.q(), stream=torch.cuda.Stream(dev)))
        rhos.append(torch.tensor(d.density(), device=dev))
        Ts.append(torch.zeros(solvers[-1].n_nodes, dtype=torch.float64, device=dev))
    bs = mgar.BatchSolver(solvers, stream=torch.cuda.Stream(dev))
    volfracs = [d.volfrac for d in designs]
    hist = [[] for _ in designs]
    try:
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(cycles):
            for i, inf in enumerate(bs.cycle(rhos, Ts, volfracs, 0.2)):
                hist[i].append(dict(compliance=inf["compliance"], cg_iters=inf["cg_iters"],
                                    converged=inf["status"] == mgar.MGAR_OK))
        torch.cuda.synchronize(dev)
        seconds = time.perf_counter() - t0
        out = [(rhos[i].cpu().numpy(), hist[i]) for i in range(len(designs))]
        report = bs.report()
    finally:
        bs.close()
        for s in solvers:
            s.close()
    return out, seconds, report
