"""Python binding of libmgar (include/mgar.h): argument marshalling only.

Device arrays are torch CUDA tensors (float64, contiguous); their data
pointers are passed straight to the C ABI, and every call is ordered on the
stream the solver was created with (default: torch's current stream).  There
is no CPU fallback: if the CUDA library cannot be loaded, every entry point
raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np

from . import build as _build

MGAR_OK = 0
MGAR_ERR_ARG = -1
MGAR_ERR_CUDA = -2
MGAR_ERR_NOT_SPD = -3
MGAR_ERR_MAXIT = -4
MGAR_ERR_NONFINITE = -5
MGAR_ERR_STATE = -6
MGAR_ERR_TOO_LARGE = -7
MGAR_FP64 = 0
MGAR_MIXED = 1
MGAR_GUESS_PREVIOUS = 0
MGAR_GUESS_ZERO = 1

ERROR_NAMES = {MGAR_ERR_ARG: "MGAR_ERR_ARG", MGAR_ERR_CUDA: "MGAR_ERR_CUDA",
               MGAR_ERR_NOT_SPD: "MGAR_ERR_NOT_SPD", MGAR_ERR_MAXIT: "MGAR_ERR_MAXIT",
               MGAR_ERR_NONFINITE: "MGAR_ERR_NONFINITE", MGAR_ERR_STATE: "MGAR_ERR_STATE",
               MGAR_ERR_TOO_LARGE: "MGAR_ERR_TOO_LARGE"}

# every entry point of include/mgar.h, in declaration order
EXPORTS = ("mgar_default_params", "mgar_create", "mgar_destroy", "mgar_set_stream",
           "mgar_last_error", "mgar_filter", "mgar_set_density", "mgar_set_load", "mgar_apply_K",
           "mgar_build_hierarchy", "mgar_vcycle", "mgar_solve_mgcg", "mgar_solve_mgar",
           "mgar_sensitivity", "mgar_postprocess", "mgar_oc_update", "mgar_step", "mgar_sizes", "mgar_run",
           "mgar_profile_start", "mgar_profile_stop", "mgar_profile_report",
           "mgar_kernel_launches", "mgar_batch_create", "mgar_batch_destroy",
           "mgar_batch_last_error", "mgar_batch_solve_mgcg", "mgar_batch_cycle", "mgar_batch_report",
           "mgar_sensitivity_noalloc")

# kernel classes of mgar_profile_start
KC_APPLY64, KC_SMOOTH0, KC_RESID0, KC_OC, KC_GALERKIN0, KC_FILTER, KC_SENS = range(1, 8)
KC_APPLY32, KC_RESID64 = 8, 9
KC_TIMELINE = 100


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("k0", ctypes.c_double), ("kmin", ctypes.c_double), ("penal", ctypes.c_double),
                ("rmin", ctypes.c_double), ("nl", ctypes.c_int32), ("m", ctypes.c_int32),
                ("eps1", ctypes.c_double), ("eps2", ctypes.c_double), ("cg_max", ctypes.c_int32),
                ("omega", ctypes.c_double), ("nu_pre", ctypes.c_int32), ("nu_post", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("basis_guess", ctypes.c_int32),
                ("n_on", ctypes.c_int32), ("volfrac", ctypes.c_double), ("move", ctypes.c_double),
                ("filter_alpha", ctypes.c_double), ("filter_lp", ctypes.c_int32),
                ("filter_L", ctypes.c_double)]


class StepInfo(ctypes.Structure):
    _fields_ = [("compliance", ctypes.c_double), ("res", ctypes.c_double),
                ("relres", ctypes.c_double), ("lambda_", ctypes.c_double),
                ("used_mgcg", ctypes.c_int32), ("accepted", ctypes.c_int32),
                ("cg_iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("compliance_mgar", ctypes.c_double)]

    def as_dict(self):
        return dict(compliance=self.compliance, res=self.res, relres=self.relres,
                    lam=self.lambda_, used_mgcg=bool(self.used_mgcg),
                    accepted=bool(self.accepted), cg_iters=self.cg_iters, status=self.status,
                    compliance_mgar=self.compliance_mgar)


_LIB = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libmgar.so (building it first if it is missing or stale)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if os.environ.get("MGAR_CHECKED") == "1":
        path = _build.LIB_CHECKED  # bounds-checked debug build
        if not os.path.exists(path):
            _build.build_checked()
    else:
        if build_if_missing and not _build.up_to_date():
            _build.build()
        path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libmgar.so not found at {path}; run paper_2210_00947_gb300/build.py")
    lib = ctypes.CDLL(path)
    P, vp, i32, dp = ctypes.POINTER, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
    sig = {
        "mgar_default_params": (None, [P(Params)]),
        "mgar_create": (i32, [P(vp), P(Params), vp, vp, vp]),
        "mgar_destroy": (i32, [vp]),
        "mgar_set_stream": (i32, [vp, vp]),
        "mgar_last_error": (ctypes.c_char_p, [vp]),
        "mgar_filter": (i32, [vp, vp, vp, i32]),
        "mgar_set_density": (i32, [vp, vp, i32]),
        "mgar_set_load": (i32, [vp, vp]),
        "mgar_apply_K": (i32, [vp, vp, vp]),
        "mgar_build_hierarchy": (i32, [vp]),
        "mgar_vcycle": (i32, [vp, vp, vp]),
        "mgar_solve_mgcg": (i32, [vp, vp, P(i32), dp]),
        "mgar_solve_mgar": (i32, [vp, vp, vp, dp, P(i32)]),
        "mgar_sensitivity": (i32, [vp, vp, vp, vp, dp]),
        "mgar_oc_update": (i32, [vp, vp, vp, ctypes.c_double, ctypes.c_double, dp, dp]),
        "mgar_postprocess": (i32, [vp, vp, vp, ctypes.c_double, vp, dp, dp]),
        "mgar_step": (i32, [vp, vp, vp, i32, P(StepInfo)]),
        "mgar_sizes": (i32, [vp, P(ctypes.c_int64), P(ctypes.c_int64)]),
        "mgar_run": (i32, [vp, vp, i32, vp, P(StepInfo)]),
        "mgar_profile_start": (i32, [vp, i32]),
        "mgar_profile_stop": (i32, [vp, dp, P(ctypes.c_int64)]),
        "mgar_profile_report": (i32, [vp, ctypes.c_char_p, ctypes.c_int64]),
        "mgar_kernel_launches": (ctypes.c_int64, []),
        "mgar_batch_create": (i32, [P(vp), P(vp), i32, vp]),
        "mgar_batch_destroy": (i32, [vp]),
        "mgar_batch_last_error": (ctypes.c_char_p, [vp]),
        "mgar_batch_solve_mgcg": (i32, [vp, P(vp), P(i32), dp, P(i32)]),
        "mgar_batch_cycle": (i32, [vp, P(vp), P(vp), dp, ctypes.c_double, P(StepInfo)]),
        "mgar_batch_report": (i32, [vp, ctypes.c_char_p, ctypes.c_int64]),
        "mgar_sensitivity_noalloc": (i32, [P(Params), vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class MgarError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def default_params(**overrides) -> Params:
    p = Params()
    load().mgar_default_params(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def _ptr(t):
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a):
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("expected a contiguous float64 array")
        return a.ctypes.data_as(ctypes.c_void_p)
    import torch
    if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous():
        raise ValueError("expected a contiguous float64 host tensor")
    return ctypes.c_void_p(a.data_ptr())


class Solver:
    """One design domain on the GPU (a mgar_t handle)."""

    def __init__(self, params: Params, fixed: np.ndarray, q: np.ndarray, stream=None):
        import torch
        self._lib = load()
        self.params = params
        fixed = np.ascontiguousarray(fixed, dtype=np.uint8)
        q = np.ascontiguousarray(q, dtype=np.float64)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        rc = self._lib.mgar_create(ctypes.byref(h), ctypes.byref(params),
                                   fixed.ctypes.data_as(ctypes.c_void_p),
                                   q.ctypes.data_as(ctypes.c_void_p),
                                   ctypes.c_void_p(stream.cuda_stream))
        if rc != MGAR_OK:
            raise MgarError(rc, self._lib.mgar_last_error(None).decode())
        self._h = h
        n = ctypes.c_int64()
        e = ctypes.c_int64()
        self._check(self._lib.mgar_sizes(h, ctypes.byref(n), ctypes.byref(e)))
        self.n_nodes, self.n_elems = n.value, e.value

    def _check(self, rc, ok=(MGAR_OK,)):
        if rc not in ok:
            raise MgarError(rc, self._lib.mgar_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mgar_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ------------------------------------------------------------ entry points
    def filter(self, x, out, transpose=False):
        self._check(self._lib.mgar_filter(self._h, _ptr(x), _ptr(out), int(transpose)))
        return out

    def set_density(self, rho, physical=False):
        self._check(self._lib.mgar_set_density(self._h, _ptr(rho), int(physical)))

    def set_load(self, q):
        """mgar_set_load: q is a float64 CUDA tensor of n entries."""
        self._check(self._lib.mgar_set_load(self._h, _ptr(q)))

    def apply_K(self, x, y):
        self._check(self._lib.mgar_apply_K(self._h, _ptr(x), _ptr(y)))
        return y

    def build_hierarchy(self):
        self._check(self._lib.mgar_build_hierarchy(self._h))

    def vcycle(self, b, x):
        self._check(self._lib.mgar_vcycle(self._h, _ptr(b), _ptr(x)))
        return x

    def solve_mgcg(self, T):
        it = ctypes.c_int32()
        rr = ctypes.c_double()
        rc = self._check(self._lib.mgar_solve_mgcg(self._h, _ptr(T), ctypes.byref(it),
                                                   ctypes.byref(rr)),
                         ok=(MGAR_OK, MGAR_ERR_MAXIT))
        return it.value, rr.value, rc == MGAR_OK

    def solve_mgar(self, T_prev, T):
        res = ctypes.c_double()
        acc = ctypes.c_int32()
        self._check(self._lib.mgar_solve_mgar(self._h, _ptr(T_prev), _ptr(T), ctypes.byref(res),
                                              ctypes.byref(acc)))
        return res.value, bool(acc.value)

    def sensitivity(self, T, dc=None, dv=None):
        c = ctypes.c_double()
        self._check(self._lib.mgar_sensitivity(self._h, _ptr(T), _ptr(dc), _ptr(dv),
                                               ctypes.byref(c)))
        return c.value

    def oc_update(self, rho, dc, volfrac, move):
        lam = ctypes.c_double()
        ch = ctypes.c_double()
        self._check(self._lib.mgar_oc_update(self._h, _ptr(rho), _ptr(dc), float(volfrac),
                                             float(move), ctypes.byref(lam), ctypes.byref(ch)))
        return lam.value, ch.value

    def postprocess(self, rho, T, volfrac, rho_out):
        """mgar_postprocess (Eq. 24-27); returns (level, volume)."""
        lev = ctypes.c_double()
        vol = ctypes.c_double()
        self._check(self._lib.mgar_postprocess(self._h, _ptr(rho), _ptr(T), float(volfrac),
                                               _ptr(rho_out), ctypes.byref(lev),
                                               ctypes.byref(vol)))
        return lev.value, vol.value

    def run(self, rho_host, cycles, rho_out_host):
        """mgar_run: host arrays in and out (numpy arrays or pinned CPU
        tensors, float64, contiguous); returns the per-cycle reports."""
        infos = (StepInfo * max(cycles, 1))()
        self._check(self._lib.mgar_run(self._h, _host_ptr(rho_host), int(cycles),
                                       _host_ptr(rho_out_host), infos))
        return [infos[i].as_dict() for i in range(cycles)]

    def profile_start(self, kernel_class):
        self._check(self._lib.mgar_profile_start(self._h, int(kernel_class)))

    def profile_stop(self):
        ms = ctypes.c_double()
        n = ctypes.c_int64()
        self._check(self._lib.mgar_profile_stop(self._h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def profile_report(self) -> str:
        buf = ctypes.create_string_buffer(1 << 16)
        self._check(self._lib.mgar_profile_report(self._h, buf, len(buf)))
        return buf.value.decode()

    def step(self, rho, T, cycle):
        info = StepInfo()
        self._check(self._lib.mgar_step(self._h, _ptr(rho), _ptr(T), int(cycle),
                                        ctypes.byref(info)))
        return info.as_dict()


class BatchSolver:
    """Batched MGCG over several 2D mixed-precision Solvers (mgar_batch_*):
    one launch per V-cycle level and operation over all designs."""

    def __init__(self, solvers, stream=None):
        import torch
        self._lib = load()
        self.solvers = list(solvers)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        hs = (ctypes.c_void_p * len(self.solvers))(*[s._h.value for s in self.solvers])
        b = ctypes.c_void_p()
        rc = self._lib.mgar_batch_create(ctypes.byref(b), hs, len(self.solvers),
                                         ctypes.c_void_p(stream.cuda_stream))
        if rc != MGAR_OK:
            raise MgarError(rc, self._lib.mgar_batch_last_error(None).decode())
        self._b = b

    def solve(self, Ts):
        """mgar_batch_solve_mgcg: Ts are the designs' temperature tensors (warm
        start in, solution out); returns per design (iters, relres, ok)."""
        n = len(self.solvers)
        if len(Ts) != n:
            raise ValueError("one temperature tensor per design")
        ptrs = (ctypes.c_void_p * n)(*[_ptr(t).value for t in Ts])
        it = (ctypes.c_int32 * n)()
        rr = (ctypes.c_double * n)()
        st = (ctypes.c_int32 * n)()
        rc = self._lib.mgar_batch_solve_mgcg(self._b, ptrs, it, rr, st)
        if rc not in (MGAR_OK, MGAR_ERR_MAXIT):
            raise MgarError(rc, self._lib.mgar_batch_last_error(self._b).decode())
        return [(it[d], rr[d], st[d] == MGAR_OK) for d in range(n)]

    def cycle(self, rhos, Ts, volfracs, move=0.2):
        """mgar_batch_cycle: one MGCG design cycle of every design (filter,
        batched solve, sensitivities, OC); rhos and Ts are updated in place;
        returns the per-design reports."""
        n = len(self.solvers)
        if len(rhos) != n or len(Ts) != n or len(volfracs) != n:
            raise ValueError("one density, temperature tensor and volume fraction per design")
        rp = (ctypes.c_void_p * n)(*[_ptr(r).value for r in rhos])
        tp = (ctypes.c_void_p * n)(*[_ptr(t).value for t in Ts])
        vf = (ctypes.c_double * n)(*[float(v) for v in volfracs])
        infos = (StepInfo * n)()
        rc = self._lib.mgar_batch_cycle(self._b, rp, tp, vf, float(move), infos)
        if rc not in (MGAR_OK, MGAR_ERR_MAXIT):
            raise MgarError(rc, self._lib.mgar_batch_last_error(self._b).decode())
        return [infos[d].as_dict() for d in range(n)]

    def report(self) -> str:
        buf = ctypes.create_string_buffer(1 << 14)
        rc = self._lib.mgar_batch_report(self._b, buf, len(buf))
        if rc != MGAR_OK:
            raise MgarError(rc, self._lib.mgar_batch_last_error(self._b).decode())
        return buf.value.decode()

    def close(self):
        if getattr(self, "_b", None):
            self._lib.mgar_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def kernel_launches() -> int:
    """Kernels libmgar has launched in this process so far."""
    return int(load().mgar_kernel_launches())


def params_for(workload, precision=MGAR_FP64, basis_guess=MGAR_GUESS_PREVIOUS, **overrides) -> Params:
    """Solver parameters of a named workload (paper_2210_00947_gb300.workloads)."""
    w = workload
    p = default_params(nx=w.nx, ny=w.ny, nz=w.nz, k0=w.k0, kmin=w.kmin, penal=w.penal,
                       rmin=w.rmin, nl=w.nl, m=w.m, eps1=w.eps1, eps2=w.eps2, cg_max=w.cg_max,
                       precision=precision, basis_guess=basis_guess, n_on=w.n_on,
                       volfrac=w.volfrac, move=w.move,
                       filter_alpha=getattr(w, "filter_alpha", 0.0),
                       filter_lp=getattr(w, "filter_lp", 0))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p
