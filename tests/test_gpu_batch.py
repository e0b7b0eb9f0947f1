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
