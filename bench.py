"""Benchmark: ms per topology-optimisation iteration on the 3D H8 128^3
heat-sink workload (2,146,689 nodal temperatures), the mixed-precision path
against plain FP64 MGCG on the same GPU at equal compliance (1e-6), with the
dominant kernel's roofline.

One step = one whole optimisation run of the workload (50 design cycles from
rho = 0.3: filter, solve, sensitivities, OC), inputs resident in HBM; value =
mean device time per design cycle.  On this workload no acceptance threshold
of Eq. 28 lets an MGAR reanalysis within 1e-6 of the FP64 MGCG compliance, so
the timed path solves every cycle by MGCG (--mgar zero|previous times the
MGAR loop instead); the MGAR legs report the paper's setting (eps1 = 0.5,
both readings of Eq. 17) with their compliance errors, and the best error an
attempt reaches in any cycle.  The e2e figure runs the timed path through
mgar_run from pinned host memory (design in, design and per-cycle reports
out).  --impl reference times the FP64 CPU oracle on a bounded sample of the
same workload instead.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mgar|reference]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms per TO iteration, 3D H8 128^3, MGAR vs FP64 MGCG @1e-6 rel err; HBM %"
UNIT = "ms/iteration"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mgar", choices=["mgar", "reference"])
    ap.add_argument("--workload", default="heat3d_128")
    ap.add_argument("--cycles", type=int, default=0, help="design cycles per step (0 = workload's)")
    ap.add_argument("--mgar", default="off", choices=["off", "zero", "previous"],
                    help="timed path: MGCG every cycle (off), or the MGAR loop with this "
                         "reading of Eq. 17 (zero-guess or literal basis)")
    ap.add_argument("--eps1", type=float, default=None, help="Eq. 28 threshold with --mgar")
    ap.add_argument("--no-mgar-legs", action="store_true",
                    help="skip the paper-setting MGAR legs (eps1 = 0.5, both readings)")
    ap.add_argument("--cpu-all-cores", action="store_true",
                    help="also time the oracle with BLAS/OpenMP on every host core")
    ap.add_argument("--cpu-cycles", type=int, default=1,
                    help="design cycles of the oracle's loop in the CPU baseline")
    ap.add_argument("--kernel", default=None,
                    choices=["df3d", "apply64", "apply32", "resid64", "smooth0", "galerkin0"],
                    help="kernel class of the roofline (default: the dominant one of the path)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 MGCG comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-check", action="store_true", help="skip the equal-compliance check")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--timeline", action="store_true",
                    help="after timing, print a per-launch-site device-time table to stderr")
    ap.add_argument("--replay", default=None,
                    help="comma-separated paper-setting workloads (e.g. paper2d_m1,paper2d_m2): "
                         "MGAR against pure MGCG as in Table 2, one JSON line each")
    ap.add_argument("--nl", type=int, default=0, help="replay: number of levels (0 = workload's)")
    ap.add_argument("--batch", type=int, default=0,
                    help="run this many seeded independent 2D designs concurrently and one after "
                         "another (--cycles each, default 30); one JSON line")
    ap.add_argument("--batch-workers", type=int, default=16)
    ap.add_argument("--postprocess", default=None,
                    help="time the boundary post-processing (Eq. 24-27) after --cycles design "
                         "cycles of this workload; one JSON line")
    ap.add_argument("--autograd", default=None,
                    help="time the differentiable compliance (forward solve + adjoint gradient) "
                         "on this workload; one JSON line")
    ap.add_argument("--random-density", action="store_true",
                    help="autograd: start from i.i.d. U[0.05, 1] densities (the differentiation "
                         "workload) instead of the workload's uniform field")
    ap.add_argument("--replay-precisions", default="mixed,fp64")
    ap.add_argument("--replay-guesses", default="previous,zero")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------ distributed
def dist_setup(args=None, backend=None):
    """Ranks of a torchrun launch (one process per GPU; replicas, no
    collective on the data path): NCCL between GPUs, gloo without CUDA."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend is None:
            backend = "nccl" if torch.cuda.is_available() else "gloo"
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(items, rank, world):
    """Independent problems over ranks: item i goes to rank i mod world."""
    return list(items)[rank::world]


# ------------------------------------------------------------- roofline
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu capture of the kernel as it stands; a kernel changed since its
# capture has no entry (traffic null).
TRAFFIC = {
    # cold-cache ncu capture (43 x 5 tiles, layer-split stencil) of one
    # pre-smoothing (27.73 MB) and one post-smoothing pass (36.34 MB) of the
    # 128^3 workload: their mean
    "smooth0": 32.03e6,
    # the same capture, FP32 CG product
    "apply32": 27.74e6,
}

def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def fp64_peak_tflops(sm_mhz):
    """FP64 peak of GB300 from its unit count and clock: the nominal
    1.25 TFLOP/s at the 2070 MHz maximum SM clock is 604 FLOP per clock for
    the chip (152 SMs x 2 FP64 FMA per clock x 2 FLOP); scaled to the clock
    seen under load."""
    mhz = sm_mhz or 2070.0
    return 152 * 2 * 2 * mhz * 1e6 / 1e12


def fp32_peak_tops(sm_mhz):
    """FP32-pipe peak of GB300 from its unit count and clock: 152 SMs x 128
    FP32 lanes, one add, multiply or fused multiply-add each per clock
    (counted as one operation, as the df64 operation counts are)."""
    mhz = sm_mhz or 2070.0
    return 152 * 128 * mhz * 1e6 / 1e12


def kernel_model(kernel, w):
    """Algorithmic work per launch of a kernel class on workload w:
    (bytes, operations, bound, pipe), from the per-unit figures derived
    below."""
    n = w.n_nodes
    e = w.n_elems
    if kernel == "df3d":
        # mixed path, tiled df64 H8 product with the fused CG direction update
        # (p = z + beta p_old, y = A p, p.y), element form, per node in
        # FP32-pipe operations: direction update 18 (df mul 7 + df add 11),
        # 8 element sums f_e 192 (TwoSum chain of four pairs, 24 each), 8
        # products k_e f_e in two accumulators 80 (first term TwoProd with
        # cross terms 4, the others 4 + TwoSum accumulation 8), joining the
        # accumulators 11, diagonal product with the per-node 4 sum k_e 7,
        # subtraction 11, 1/12 scale 7, p.y 18: 344.  Bytes: p_old and y and
        # p (8 B each), z (4 B), one k_e (8 B), 4 sum k_e (8 B), mask (1 B):
        # 45.
        return 45 * n, 344 * n, "alu", "fp32"
    if kernel == "apply32":
        # mixed path, 3D: FP32 product of a CG iteration with the fused
        # direction update and p.Ap (tiled, 21-point H8 stencil): read z,
        # p_old, k_e (4 B each) and the mask (1 B), write p and A p (4 B
        # each): 21 B per node
        return 21 * n, 0, "hbm", None
    if kernel == "resid64":
        # mixed path, 3D: df64 residual r = q - A x in the difference form,
        # per node in FP32-pipe operations: 12 face-diagonal weight sums 96
        # (TwoSum pair 8), 20 terms 380 (exact difference 8, TwoProd with
        # cross terms 4, TwoSum accumulation 8 minus the shared 1), 1/12
        # scale 7, q - A x 11, r.r 18, FP32 copy 1: 513.  Bytes: x, q, one
        # k_e (8 B each), mask (1 B), FP32 r (4 B): 29.
        return 29 * n, 513 * n, "alu", "fp32"
    if kernel == "apply64":
        # 3D H8 y = A x in FP64, node-centred: read x (8 B) and one k_e per
        # node (8 B, each element read once) and the fixed-node mask (1 B),
        # write y (8 B); 62 FP64 FLOP per node (7 adds for sum k, 12 pair
        # sums, 20 FMA, 3 multiplies), + 2 for the fused p.Ap dot.
        return 25 * n, 64 * n, "alu", "fp64"
    if kernel == "smooth0":
        # FP32 level-0 passes of the V-cycle, per node 21 B for either: the
        # pre-smoothing pass reads b, D^-1, one k_e (4 B each) and the mask
        # (1 B) and writes x and r (4 B each); the post-smoothing sweep reads
        # x, b, D^-1, one k_e and the mask and writes x'
        return 21 * n, 0, "hbm", None
    if kernel == "galerkin0":
        return 8 * e + 64 * 4 * e // 8, 0, "hbm", None
    raise ValueError(kernel)


KC = {"df3d": 1, "apply64": 1, "smooth0": 2, "galerkin0": 5, "apply32": 8, "resid64": 9}


# ------------------------------------------------------------- GPU arm
def _timed(stream, fn, flush=None):
    """Device time (ms) of fn() with CUDA events on the stream, L2 flushed
    before the first event."""
    import torch
    if flush is not None:
        flush.zero_()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    out = fn()
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b), out


def run_gpu(args):
    import numpy as np
    import torch

    from paper_2210_00947_gb300 import mgar, workloads

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workloads.WORKLOADS[args.workload]
    cycles = args.cycles or w.iters
    fixed = w.fixed()
    q = w.q()
    rho0 = w.density()
    stream = torch.cuda.current_stream(dev)
    prec = mgar.MGAR_MIXED if args.precision == "mixed" else mgar.MGAR_FP64
    GUESS = {"zero": mgar.MGAR_GUESS_ZERO, "previous": mgar.MGAR_GUESS_PREVIOUS}

    def params(mode, eps1=None, precision=prec, **kw):
        """mode "off": MGCG every cycle (no MGAR attempt); "zero" / "previous":
        the MGAR loop of Figure 5 from N_on with that reading of Eq. 17."""
        if mode == "off":
            return mgar.params_for(w, precision=precision, n_on=cycles + 1, **kw)
        extra = {} if eps1 is None else {"eps1": eps1}
        return mgar.params_for(w, precision=precision, basis_guess=GUESS[mode], **extra, **kw)

    p_head = params(args.mgar, args.eps1)
    solver = mgar.Solver(p_head, fixed, q, stream=stream)
    rho0_d = torch.tensor(rho0, device=dev)
    rho = torch.empty_like(rho0_d)
    T = torch.zeros(solver.n_nodes, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_run(s, rho_t, T_t):
        rho_t.copy_(rho0_d)
        T_t.zero_()
        return [s.step(rho_t, T_t, k) for k in range(1, cycles + 1)]

    for _ in range(args.warmup):
        one_run(solver, rho, T)
    torch.cuda.synchronize()

    # timed region: K whole runs, L2 flushed between them (outside the events)
    sampler = ClockSampler(local)
    if args.kernel:
        kernels = [args.kernel]
    elif prec == mgar.MGAR_MIXED and w.nz:
        kernels = ["apply32", "smooth0", "resid64"]
    else:
        kernels = ["apply64"]
    times = []
    infos = []
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    launches0 = mgar.kernel_launches()
    for _ in range(args.steps):
        ms, infos = _timed(stream, lambda: one_run(solver, rho, T), flush)
        times.append(ms)
    launches = mgar.kernel_launches() - launches0
    torch.cuda.synchronize()
    barrier(world)
    # The launches of each candidate kernel class are timed with CUDA events
    # on the handle's stream, each class over one more timed region of the
    # same K runs: events between launches keep the CG on its host-driven
    # loop, so they stay out of the region that gives `value`.  The class
    # with the largest share of its region is the dominant kernel.
    prof = {}
    for kname in kernels:
        solver.profile_start(KC[kname])
        prof_times = [_timed(stream, lambda: one_run(solver, rho, T), flush)[0]
                      for _ in range(args.steps)]
        k_ms, k_n = solver.profile_stop()
        prof[kname] = (k_ms, k_n, sum(prof_times))
    torch.cuda.synchronize()
    kernel = max(prof, key=lambda k: prof[k][0] / prof[k][2])
    kern_ms, kern_launches, prof_total = prof[kernel]
    clocks = sampler.stop()
    step_ms = max_over_ranks(statistics.mean(times), world)
    value = step_ms / (cycles * world)

    if args.timeline:
        solver.profile_start(mgar.KC_TIMELINE)
        one_run(solver, rho, T)
        tl_ms, tl_n = solver.profile_stop()
        print(f"[timeline] one run: {tl_ms:.2f} ms over {tl_n} marks\n" + solver.profile_report(),
              file=sys.stderr, flush=True)

    # e2e: mgar_run from pinned host memory, copies inside the timed region
    e2e_ms = float("nan")
    if not args.no_e2e:
        rho_h = torch.from_numpy(rho0.copy()).pin_memory()
        rho_out = torch.empty_like(rho_h).pin_memory()
        solver.run(rho_h, cycles, rho_out)
        e2e_times = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            solver.run(rho_h, cycles, rho_out)
            e2e_times.append((time.perf_counter() - t0) * 1e3)
        e2e_ms = max_over_ranks(statistics.mean(e2e_times), world)

    # plain FP64 MGCG on the same workload (MGCG every cycle)
    fp64 = None
    if not args.no_fp64:
        s64 = mgar.Solver(params("off", precision=mgar.MGAR_FP64), fixed, q, stream=stream)
        rho64 = torch.empty_like(rho0_d)
        T64 = torch.zeros_like(T)
        one_run(s64, rho64, T64)
        t64 = []
        for _ in range(max(1, min(args.steps, 2))):
            ms, inf64 = _timed(stream, lambda: one_run(s64, rho64, T64), flush)
            t64.append(ms)
        fp64 = {"ms_per_iteration": statistics.mean(t64) / cycles,
                "cg_iters_mean": statistics.mean(i["cg_iters"] for i in inf64),
                "final_compliance": inf64[-1]["compliance"]}
        s64.close()

    # Equal compliance: replay a run's trajectory; at every cycle solve the same
    # design with FP64 MGCG to eps2 = 1e-10 and compare compliances.
    pc = params("off", precision=mgar.MGAR_FP64, eps2=1e-10)
    sc = mgar.Solver(pc, fixed, q, stream=stream) if not args.no_check else None

    def compliance_trace(s):
        rho.copy_(rho0_d)
        T.zero_()
        Tc = torch.zeros_like(T)
        rows = []
        for k in range(1, cycles + 1):
            sc.set_density(rho)
            Tc.zero_()
            sc.solve_mgcg(Tc)
            c_ref = sc.sensitivity(Tc)
            inf = s.step(rho, T, k)
            rows.append((k, inf, c_ref))
        return rows

    check = None
    if sc is not None:
        rows = compliance_trace(solver)
        errs = [abs(i["compliance"] - c) / abs(c) for k, i, c in rows]
        acc = [e for e, (k, i, c) in zip(errs, rows) if i["accepted"]]
        check = {"max_rel_err_all_cycles": max(errs),
                 "max_rel_err_accepted_mgar": max(acc) if acc else None,
                 "accepted_mgar_cycles": len(acc),
                 "reference": "FP64 MGCG (eps2 1e-10) on the same design each cycle"}
        print("[check] cycle, solve (mgcg / mgar accepted), CG iterations, Res, compliance, "
              "FP64 MGCG compliance, relative error:\n" +
              "\n".join(f"  {k:3d} {'mgar' if i['accepted'] else 'mgcg'} {i['cg_iters']:3d} "
                        f"{i['res']:9.3e} {i['compliance']:.12e} {c:.12e} {e:.3e}"
                        for e, (k, i, c) in zip(errs, rows)),
              file=sys.stderr, flush=True)

    # MGAR at the paper's acceptance threshold (Eq. 28, eps1 = 0.5) under both
    # readings of Eq. 17 (timed, with the compliance error of every accepted
    # cycle), and the best compliance error any threshold could reach: every
    # cycle from N_on attempts MGAR and rejects it (eps1 = 0, so K0 is always
    # the previous cycle's matrix, the freshest MGAR ever sees), the attempt's
    # reduced compliance q^T t~ against this cycle's MGCG solution.
    mgar_legs = None
    if not args.no_mgar_legs and sc is not None and prec == mgar.MGAR_MIXED:
        mgar_legs = []
        for reading in ("zero", "previous"):
            sp = mgar.Solver(params(reading, 0.5), fixed, q, stream=stream)
            rp = torch.empty_like(rho0_d)
            Tp = torch.zeros_like(T)
            one_run(sp, rp, Tp)
            tp = [_timed(stream, lambda: one_run(sp, rp, Tp), flush)[0] for _ in range(2)]
            rows = compliance_trace(sp)
            errs = [abs(i["compliance"] - c) / abs(c) for k, i, c in rows if i["accepted"]]
            sp.close()
            sa = mgar.Solver(params(reading, 0.0), fixed, q, stream=stream)
            att = [(k, i["res"], (i["compliance"] - i["compliance_mgar"]) / i["compliance"])
                   for k, i in enumerate(one_run(sa, rp, Tp), start=1)
                   if i["compliance_mgar"] == i["compliance_mgar"]]
            sa.close()
            best = min(att, key=lambda a: a[2])
            mgar_legs.append({
                "basis_guess": reading, "eps1": 0.5,
                "ms_per_iteration": statistics.mean(tp) / cycles,
                "mgar_accepted": len(errs),
                "max_rel_err_accepted": max(errs) if errs else None,
                "attempts_every_cycle": {"attempts": len(att),
                                         "best_rel_err": best[2], "best_cycle": best[0],
                                         "res_at_best": best[1],
                                         "within_1e-6": sum(1 for a in att if a[2] <= 1e-6)}})
            print(f"[mgar {reading}] cycle, Res, relative compliance error of the attempt:\n" +
                  "\n".join(f"  {k:3d} {r:8.4f} {e:.3e}" for k, r, e in att),
                  file=sys.stderr, flush=True)
    if sc is not None:
        sc.close()

    peaks = load_peaks()
    bytes_, flops, bound, pipe = kernel_model(kernel, w)
    avg_ms = kern_ms / max(kern_launches, 1)
    if bound == "alu" and pipe == "fp32":
        achieved = flops / (avg_ms * 1e-3) / 1e12
        peak = fp32_peak_tops(clocks.get("sm_mhz"))
        roof = {"bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "Top/s (FP32-pipe operations of the df64 arithmetic)",
                "frac": achieved / peak, "traffic": TRAFFIC.get(kernel),
                "peak_source": "152 SMs x 128 FP32 lanes x SM clock under load (derived)",
                "hbm_gbs": bytes_ / (avg_ms * 1e-3) / 1e9}
    elif bound == "alu":
        achieved = flops / (avg_ms * 1e-3) / 1e12
        peak = fp64_peak_tflops(clocks.get("sm_mhz"))
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s (fp64)",
                "frac": achieved / peak, "traffic": TRAFFIC.get(kernel),
                "peak_source": "FP64 unit count x SM clock under load (derived)",
                "hbm_gbs": bytes_ / (avg_ms * 1e-3) / 1e9}
    else:
        achieved = bytes_ / (avg_ms * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": TRAFFIC.get(kernel),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy)" if "hbm_gbs" in peaks
                else "fallback"}
    roof.update({"kernel": kernel, "launches": kern_launches, "avg_launch_us": avg_ms * 1e3,
                 "share_of_step": kern_ms / prof_total,
                 "timed_region": "one more timed region of the same runs per kernel class, "
                                 "events around each launch",
                 "classes": [{"kernel": k, "launches": v[1],
                              "avg_launch_us": v[0] / max(v[1], 1) * 1e3,
                              "share_of_step": v[0] / v[2]} for k, v in prof.items()]})

    n_mgcg = sum(1 for i in infos if i["used_mgcg"])
    n_acc = sum(1 for i in infos if i["accepted"])
    if args.mgar == "off":
        mgar_cfg = ("off in the timed path: no acceptance threshold of Eq. 28 gives a "
                    "reanalysis within 1e-6 of FP64 MGCG on this workload (see mgar_legs)")
    else:
        mgar_cfg = {"basis_guess": args.mgar, "eps1": p_head.eps1, "m": w.m, "n_on": w.n_on}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": args.workload, "grid": f"{w.nx}x{w.ny}x{w.nz} H8" if w.nz else
                   f"{w.nx}x{w.ny} Q4", "dofs": w.n_nodes, "cycles_per_step": cycles,
                   "nl": w.nl, "eps2": w.eps2, "omega": p_head.omega, "mgar": mgar_cfg,
                   "precision": "mixed (FP32 V-cycle and CG with df64 reliable updates; FP64 scalars, "
                                "Gram-Schmidt and reduced system)" if prec == mgar.MGAR_MIXED
                   else "fp64",
                   "parallelism": f"replicas x{world}", "l2": "flushed (256 MB write) between steps"},
        "cycles": {"mgcg": n_mgcg, "mgar_accepted": n_acc,
                   "cg_iters_mean": statistics.mean([i["cg_iters"] for i in infos if i["used_mgcg"]] or [0]),
                   "final_compliance": infos[-1]["compliance"]},
        "fp64_mgcg": fp64, "compliance_check": check, "mgar_legs": mgar_legs,
        "e2e": {"value": e2e_ms / (cycles * world), "unit": UNIT,
                "h2d_bytes_per_step": 8 * w.n_elems,
                "d2h_bytes_per_step": 8 * w.n_elems + ctypes.sizeof(mgar.StepInfo) * cycles},
        "gpu_launches": launches, "roofline": roof, "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu:
        cb = cpu_baseline(args.workload, cycles=args.cpu_cycles)
        # the oracle's own loop from the same rho0: its compliances beside the
        # timed path's for the cycles it ran (free-running, each side its own
        # trajectory)
        oc = cb.pop("compliance", None)
        line["cpu_baseline"] = cb
        if oc:
            errs = [abs(i["compliance"] - c) / abs(c) for i, c in zip(infos, oc)]
            line["oracle_compliance"] = {"cycles": len(errs), "max_rel_err": max(errs),
                                         "rel_err": errs,
                                         "note": "oracle loop and timed path, each from rho0"}
        if args.cpu_all_cores:
            cba = cpu_baseline(args.workload, cycles=args.cpu_cycles, threads=os.cpu_count() or 1)
            cba.pop("compliance", None)
            line["cpu_baseline_all_cores"] = cba
    if rank == 0:
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------ CPU oracle
ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
from oracle import loop
from paper_2210_00947_gb300 import workloads
w = workloads.WORKLOADS[{name!r}]
s = loop.LoopSettings(nx=w.nx, ny=w.ny, nz=w.nz, volfrac=w.volfrac, iters=w.iters, n_on=w.n_on,
                      nl=w.nl, eps2=w.eps2, cg_max=w.cg_max, eps1=w.eps1, m=w.m)
an = loop.Analysis(s, w.fixed(), w.q())
rho = w.density(); t = np.zeros(an.grid.n_nodes)
out = []
for k in range(1, {cycles} + 1):
    t0 = time.perf_counter()
    rho, t, info = an.cycle(k, rho, t)
    out.append(dict(seconds=time.perf_counter() - t0, mgcg=bool(info["mgcg"]),
                    compliance=float(info["compliance"])))
print(json.dumps(out))
"""


def cpu_baseline(name, cycles=1, threads=1):
    """The FP64 oracle as it stands, on the host cores, one process with BLAS
    and OpenMP limited to `threads` threads: design cycles 1..cycles of the
    workload."""
    th = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=th, OPENBLAS_NUM_THREADS=th, MKL_NUM_THREADS=th)
    code = ORACLE_SNIPPET.format(root=ROOT, name=name, cycles=cycles)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if res.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": threads, "kind": "oracle",
                "sample": "failed: " + res.stderr.strip().splitlines()[-1][:200]}
    cyc = json.loads(res.stdout.strip().splitlines()[-1])
    ms = 1e3 * statistics.mean(c["seconds"] for c in cyc)
    return {"value": ms, "unit": UNIT, "cores": threads, "kind": "oracle",
            "compliance": [c["compliance"] for c in cyc],
            "sample": f"design cycles 1..{cycles} of {name} (MGCG cycles incl. assembly and "
                      f"hierarchy), mean per cycle, numpy/scipy FP64, BLAS/OpenMP threads "
                      f"{threads} (scipy.sparse kernels run on one thread regardless)"}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    times = []
    for i in range(args.warmup + args.steps):
        b = cpu_baseline(args.workload, cycles=1)
        b.pop("compliance", None)
        if b["value"] is None:
            print(json.dumps({"impl": "reference", "unavailable": b["sample"]}))
            return
        if i >= args.warmup:
            times.append(b["value"])
    value = statistics.mean(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "sample": "design cycle 1 per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": "design cycle 1 (MGCG) of the workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------ paper-setting replay
# Tables 2 and 3 of the paper (2D heat sink, nl 3, eps1 0.5, eps2 1e-6, 300 cycles):
# costs normalised to Model 1's MGAR run, MGCG evaluations inside MGAR,
# efficiency improvement and relative objective difference of MGAR against
# pure MGCG.  Context only: another machine, FP64 Matlab.
PAPER_TABLE2 = {
    "paper2d_m1": dict(cost_mgar=1.0, cost_mgcg=1.71, mgcg_evaluations=107,
                       efficiency_improvement=0.4165, relative_difference=0.0015),
    "paper2d_m2": dict(cost_mgar=5.58, cost_mgcg=9.16, mgcg_evaluations=115,
                       efficiency_improvement=0.3911, relative_difference=0.00037),
    "paper2d_m3": dict(cost_mgar=42.25, cost_mgcg=65.17, mgcg_evaluations=125,
                       efficiency_improvement=0.3518, relative_difference=0.000040),
    "paper2d_m4": dict(cost_mgar=102.81, cost_mgcg=156.01, mgcg_evaluations=127,
                       efficiency_improvement=0.3410, relative_difference=0.000033),
    # Table 3 (Section 4.2, four sub-domain sources)
    "paper2d_q480_v04": dict(mgcg_evaluations=112, efficiency_improvement=0.4050,
                             relative_difference=0.0013, cg_iters=7.71, cg_iters_mgcg=7.38),
    "paper2d_q480_v06": dict(mgcg_evaluations=102, efficiency_improvement=0.4546,
                             relative_difference=0.000050, cg_iters=7.69, cg_iters_mgcg=7.32),
    "paper2d_q960_v04": dict(mgcg_evaluations=124, efficiency_improvement=0.3593,
                             relative_difference=0.00028, cg_iters=7.81, cg_iters_mgcg=7.51),
    "paper2d_q960_v06": dict(mgcg_evaluations=109, efficiency_improvement=0.4368,
                             relative_difference=0.000015, cg_iters=7.47, cg_iters_mgcg=7.24),
}
# Section 4.3 (3D quarter model): efficiency improvement and MGAR objective
PAPER_TABLE2["paper3d_quarter"] = dict(efficiency_improvement=0.5125, objective_mgar=5792.03)
PAPER_TABLE2["paper2d_m1c"] = PAPER_TABLE2["paper2d_m1"]
PAPER_TABLE2["paper2d_m2c"] = PAPER_TABLE2["paper2d_m2"]


def run_replay(args):
    """MGAR against pure MGCG on the paper's 2D models: one whole run of
    each (after a short warm-up run), device time with CUDA events, for both
    precisions and both readings of Eq. 17's initial guess."""
    import torch

    from paper_2210_00947_gb300 import mgar, workloads

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    base_ms = {}
    for name in args.replay.split(","):
        w = workloads.WORKLOADS[name]
        cycles = args.cycles or w.iters
        fixed, q, rho0 = w.fixed(), w.q(), w.density()
        rho0_d = torch.tensor(rho0, device=dev)
        nl = args.nl or w.nl
        for prec_name in args.replay_precisions.split(","):
            prec = mgar.MGAR_MIXED if prec_name == "mixed" else mgar.MGAR_FP64
            for guess_name in args.replay_guesses.split(","):
                guess = (mgar.MGAR_GUESS_PREVIOUS if guess_name == "previous"
                         else mgar.MGAR_GUESS_ZERO)
                runs = {}
                for mode, n_on in (("mgar", w.n_on), ("mgcg", cycles + 1)):
                    p = mgar.params_for(w, precision=prec, basis_guess=guess, n_on=n_on, nl=nl)
                    solver = mgar.Solver(p, fixed, q, stream=stream)
                    rho = torch.empty_like(rho0_d)
                    T = torch.zeros(solver.n_nodes, dtype=torch.float64, device=dev)

                    def one_run(nc):
                        rho.copy_(rho0_d)
                        T.zero_()
                        return [solver.step(rho, T, k) for k in range(1, nc + 1)]

                    one_run(min(cycles, 3))  # graphs and buffers
                    torch.cuda.synchronize()
                    start = torch.cuda.Event(enable_timing=True)
                    end = torch.cuda.Event(enable_timing=True)
                    start.record(stream)
                    infos = one_run(cycles)
                    end.record(stream)
                    end.synchronize()
                    runs[mode] = (start.elapsed_time(end), infos)
                    solver.close()
                t_mgar, inf_a = runs["mgar"]
                t_mgcg, inf_c = runs["mgcg"]
                key = (prec_name, guess_name)
                base_ms.setdefault(key, t_mgar)
                fa, fc = inf_a[-1]["compliance"], inf_c[-1]["compliance"]
                line = {
                    "replay": name, "dofs": w.n_nodes, "cycles": cycles, "nl": nl,
                    "precision": prec_name,
                    "basis_guess": guess_name, "mgar_ms": t_mgar, "mgcg_ms": t_mgcg,
                    "savings_ms": t_mgcg - t_mgar,
                    "cost_mgar": t_mgar / base_ms[key], "cost_mgcg": t_mgcg / base_ms[key],
                    "mgcg_evaluations": sum(1 for i in inf_a if i["used_mgcg"]),
                    "mgar_accepted": sum(1 for i in inf_a if i["accepted"]),
                    "efficiency_improvement": 1.0 - t_mgar / t_mgcg,
                    "relative_difference": abs(fa - fc) / abs(fc),
                    "objective_mgar": fa, "objective_mgcg": fc,
                    "cg_iters_mean_mgcg": statistics.mean(i["cg_iters"] for i in inf_c),
                    "cg_iters_mean_in_mgar": statistics.mean(
                        [i["cg_iters"] for i in inf_a if i["used_mgcg"]] or [0]),
                    "filter": ("continuous, alpha %.4g, lp %d" % (w.filter_alpha, w.filter_lp)
                               if w.filter_alpha > 0 else "plain, r_min %.3g" % w.rmin),
                    "paper": PAPER_TABLE2.get(name),
                    "data": "synthetic (the paper's geometry, source and settings)",
                }
                print(json.dumps(line), flush=True)


def run_batch(args):
    """Independent designs (the workload module's seeded uneven 2D set): the
    batched solve (one launch per V-cycle level and operation over all
    designs, one CUDA graph per solve, autotuned V-cycle block sizes), against
    the same designs run concurrently with one handle, stream and host thread
    each, and one after another."""
    from paper_2210_00947_gb300 import batch, mgar

    world, rank, local = dist_setup(args)
    designs = shard(batch.designs_from_workload(args.batch), rank, world)
    cycles = args.cycles or 30
    prec = mgar.MGAR_MIXED if args.precision == "mixed" else mgar.MGAR_FP64
    # warm-up: library load, graphs of a small set
    batch.run_designs_batched(designs[:2], cycles=2, workers=2, device=local)
    batch.run_designs(designs[:2], cycles=2, workers=2, precision=prec, device=local)
    bat, t_bat, report = batch.run_designs_batched(designs, cycles=cycles,
                                                   workers=args.batch_workers, device=local)
    n_on = {"n_on": cycles + 1}  # MGCG in every cycle, as the batched run
    par, t_par = batch.run_designs(designs, cycles=cycles, workers=args.batch_workers,
                                   precision=prec, device=local, **n_on)
    seq, t_seq = batch.run_designs(designs, cycles=cycles, workers=1, precision=prec,
                                   device=local, **n_on)
    same = all(np.array_equal(a[0], b[0]) for a, b in zip(seq, par))
    diff = max(abs(hb["compliance"] - hp["compliance"]) / abs(hp["compliance"])
               for (_, hsb), (_, hsp) in zip(bat, par) for hb, hp in zip(hsb, hsp))
    t_bat = max_over_ranks(t_bat, world)
    t_seq = max_over_ranks(t_seq, world)
    t_par = max_over_ranks(t_par, world)
    total = args.batch * cycles
    if rank != 0:
        return
    line = {"batch": args.batch, "n_gpus": world, "cycles": cycles, "precision": args.precision,
            "dofs_total": sum((d.nx + 1) * (d.ny + 1)
                              for d in batch.designs_from_workload(args.batch)),
            "batched": {"seconds": t_bat, "design_cycles_per_s": total / t_bat,
                        "nl": "each design's own depth (coarsest level of at most 300 nodes)",
                        "solve": "one mgar_batch_cycle per cycle: every design's filter, SIMP and "
                                 "hierarchy as one graph of per-design branches; the solve graph, one "
                                 "launch per V-cycle level and operation over all designs, FP32 "
                                 "V-cycle and double-float CG; every design's sensitivities and OC "
                                 "update as one graph; one read of all outcomes",
                        "cg_iters_mean": statistics.mean(h["cg_iters"] for _, hs in bat
                                                         for h in hs),
                        "autotuner": [l for l in report.splitlines() if not l.startswith("  ")]},
            "per_handle_concurrent": {"seconds": t_par, "design_cycles_per_s": total / t_par,
                                      "workers": args.batch_workers},
            "one_after_another": {"seconds": t_seq, "design_cycles_per_s": total / t_seq},
            "speedup_batched_vs_one_after_another": t_seq / t_bat,
            "identical_results_concurrent_vs_sequential": same,
            "max_rel_compliance_diff_batched_vs_per_handle": diff,
            "timing": "host wall clock from the start of the first cycle to the end of the last",
            "data": "synthetic (seeded uneven 2D designs, sides 64-512)"}
    print(json.dumps(line), flush=True)


def run_autograd(args):
    """Forward (filter, SIMP, MGCG from the previous temperatures) and backward
    (adjoint sensitivity) of the compliance of a design, as a PyTorch user
    calls it; device time with CUDA events."""
    import torch

    from paper_2210_00947_gb300 import autograd, mgar, workloads

    w = workloads.WORKLOADS[args.autograd]
    dev = torch.device("cuda", 0)
    prec = mgar.MGAR_MIXED if args.precision == "mixed" else mgar.MGAR_FP64
    comp = autograd.Compliance(mgar.params_for(w, precision=prec), w.fixed(), w.q())
    # the differentiation workload starts from i.i.d. U[0.05, 1] densities
    rho0 = (workloads.random_density(w.n_elems, 0.05, 1.0, seed=2210) if args.random_density
            else w.density())
    rho = torch.tensor(rho0, device=dev, requires_grad=True)
    stream = torch.cuda.current_stream(dev)
    times = []
    for step in range(args.warmup + args.steps):
        rho.grad = None
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        c = comp(rho)
        c.backward()
        end.record(stream)
        end.synchronize()
        if step >= args.warmup:
            times.append(start.elapsed_time(end))
        with torch.no_grad():  # a small descent step, so each solve starts warm but not converged
            rho -= 1e-3 * rho.grad / rho.grad.abs().max()
            rho.clamp_(1e-3, 1.0)
    comp.close()
    # then the workload's design cycles of the MGAR loop (Figure 5) from the same
    # starting field, mixed precision, zero-guess basis of Eq. 17, eps1 0.5
    cycles = args.cycles or w.iters
    sp = mgar.Solver(mgar.params_for(w, precision=prec, basis_guess=mgar.MGAR_GUESS_ZERO),
                     w.fixed(), w.q(), stream=stream)
    r = torch.tensor(rho0, device=dev)
    T = torch.zeros(sp.n_nodes, dtype=torch.float64, device=dev)
    sp.step(r, T, 1)  # graphs and buffers
    r.copy_(torch.tensor(rho0, device=dev))
    T.zero_()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    infos = [sp.step(r, T, k) for k in range(1, cycles + 1)]
    b.record(stream)
    b.synchronize()
    sp.close()
    line = {"autograd": args.autograd, "dofs": w.n_nodes, "precision": args.precision,
            "density": "iid U[0.05, 1], SplitMix64(2210)" if args.random_density else "uniform",
            "ms_forward_backward": statistics.mean(times), "steps": args.steps,
            "compliance": c.item(),
            "mgar_loop": {"cycles": cycles, "ms_per_iteration": a.elapsed_time(b) / cycles,
                          "n_on": w.n_on, "basis_guess": "zero", "eps1": w.eps1,
                          "mgar_accepted": sum(1 for i in infos if i["accepted"]),
                          "cg_iters_mean": statistics.mean(
                              [i["cg_iters"] for i in infos if i["used_mgcg"]] or [0]),
                          "final_compliance": infos[-1]["compliance"]},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)


def run_postprocess(args):
    """A short optimisation (--cycles, default 10), then the post-processing
    of its design, timed with CUDA events (it runs once per optimisation)."""
    import torch

    from paper_2210_00947_gb300 import mgar, workloads

    w = workloads.WORKLOADS[args.postprocess]
    dev = torch.device("cuda", 0)
    prec = mgar.MGAR_MIXED if args.precision == "mixed" else mgar.MGAR_FP64
    cycles = args.cycles or 10
    solver = mgar.Solver(mgar.params_for(w, precision=prec), w.fixed(), w.q())
    rho = torch.tensor(w.density(), device=dev)
    T = torch.zeros(solver.n_nodes, dtype=torch.float64, device=dev)
    for k in range(1, cycles + 1):
        solver.step(rho, T, k)
    solver.set_density(rho)
    solver.solve_mgcg(T)
    out = torch.empty_like(rho)
    stream = torch.cuda.current_stream(dev)
    times = []
    for _ in range(max(args.steps, 1) + 1):
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        level, vol = solver.postprocess(rho, T, w.volfrac, out)
        end.record(stream)
        end.synchronize()
        times.append(start.elapsed_time(end))
    crisp = float(((out == 0) | (out == 1)).double().mean().item())
    line = {"postprocess": args.postprocess, "elements": w.n_elems, "cycles_before": cycles,
            "ms": statistics.mean(times[1:]), "level": level, "volume": vol,
            "volfrac": w.volfrac, "crisp_share": crisp, "data": "synthetic"}
    print(json.dumps(line), flush=True)
    solver.close()


if __name__ == "__main__":
    a = parse()
    if a.postprocess:
        run_postprocess(a)
    elif a.autograd:
        run_autograd(a)
    elif a.batch:
        run_batch(a)
    elif a.replay:
        run_replay(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)
