"""mgar_sensitivity_noalloc, the entry point for callers that cannot
allocate device memory (its intermediate lives in a static device array),
called through the C ABI and checked against mgar_sensitivity of a handle on
the same inputs, twice in a row (the static array keeps the previous call's
contents), and against the oracle's sensitivities (Eq. 9-11).  Kept in its
own file, collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import design, fem  # noqa: E402
from paper_2210_00947_gb300 import mgar, workloads  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("dims,rmin", [((37, 23, 0), 1.5), ((13, 11, 9), 1.5), ((40, 30, 0), 2.5)])
def test_noalloc_matches_handle_sensitivity(dims, rmin):
    nx, ny, nz = dims
    fixed = workloads.heat_sink_mask(nx, ny, nz)
    q = workloads.nodal_load(fixed)
    ne = workloads.num_elements(nx, ny, nz)
    nn = workloads.num_nodes(nx, ny, nz)
    rng = np.random.default_rng(21)
    p = mgar.default_params(nx=nx, ny=ny, nz=nz, nl=2, rmin=rmin)
    lib = mgar.load()
    with mgar.Solver(p, fixed, q) as s:
        rho = torch.tensor(rng.uniform(0.05, 1.0, ne), device=DEV)
        T = torch.tensor(rng.uniform(0.0, 300.0, nn), device=DEV)
        rho_phys = torch.empty(ne, dtype=torch.float64, device=DEV)
        s.filter(rho, rho_phys)
        s.set_density(rho)
        dc_ref = torch.empty(ne, dtype=torch.float64, device=DEV)
        s.sensitivity(T, dc_ref)
        ref = dc_ref.cpu().numpy()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for _ in range(2):
            dc = torch.full((ne,), float("nan"), dtype=torch.float64, device=DEV)
            rc = lib.mgar_sensitivity_noalloc(ctypes.byref(p), _ptr(rho_phys), _ptr(T), _ptr(dc),
                                              stream)
            assert rc == mgar.MGAR_OK
            torch.cuda.synchronize()
            got = dc.cpu().numpy()
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())


def test_noalloc_rejects_grids_beyond_its_scratch():
    lib = mgar.load()
    p = mgar.default_params(nx=1024, ny=1025, nz=0)  # 1,049,600 elements > 2^20
    small = torch.zeros(4, dtype=torch.float64, device=DEV)
    rc = lib.mgar_sensitivity_noalloc(ctypes.byref(p), _ptr(small), _ptr(small), _ptr(small),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == mgar.MGAR_ERR_TOO_LARGE


@pytest.mark.parametrize("dims,rmin", [((37, 23, 0), 1.5), ((13, 11, 9), 2.2)])
def test_noalloc_matches_oracle(dims, rmin):
    """The same call against the oracle's filtered sensitivities, on the
    oracle's physical density, twice in a row."""
    nx, ny, nz = dims
    g = fem.Grid(nx, ny, nz)
    rng = np.random.default_rng(22)
    H, Hs = design.filter_matrix(g, rmin)
    rho_phys = design.filter_forward(H, Hs, rng.uniform(0.05, 1.0, g.n_elems))
    t = rng.uniform(0.0, 300.0, g.n_nodes)
    dc_ref, _ = design.sensitivities(g, H, Hs, rho_phys, t)
    p = mgar.default_params(nx=nx, ny=ny, nz=nz, rmin=rmin)
    lib = mgar.load()
    rho_d = torch.tensor(rho_phys, device=DEV)
    T_d = torch.tensor(t, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        dc = torch.full((g.n_elems,), float("nan"), dtype=torch.float64, device=DEV)
        rc = lib.mgar_sensitivity_noalloc(ctypes.byref(p), _ptr(rho_d), _ptr(T_d), _ptr(dc), stream)
        assert rc == mgar.MGAR_OK
        torch.cuda.synchronize()
        np.testing.assert_allclose(dc.cpu().numpy(), dc_ref, rtol=1e-11,
                                   atol=1e-13 * np.abs(dc_ref).max())


def test_noalloc_refuses_a_filter_schedule():
    """The entry point filters with the fixed radius rmin; parameters that ask
    for the continuation schedule of Eq. 22-23 are refused, not ignored."""
    lib = mgar.load()
    p = mgar.default_params(nx=8, ny=8, nz=0, filter_alpha=0.2, filter_lp=5)
    small = torch.zeros(81, dtype=torch.float64, device=DEV)
    rc = lib.mgar_sensitivity_noalloc(ctypes.byref(p), _ptr(small), _ptr(small), _ptr(small),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == mgar.MGAR_ERR_ARG
