"""The paper-setting workloads against the figures the paper prints for
them (Table 2: DOF counts of Models 1-4; Section 4.3: the 3D model's DOF
count; Section 3.2: source, sink patch, N_on).  The printed counts are the
fixture tests/golden/paper_dof_counts.txt, one cited record per model."""
import os

import numpy as np
import pytest

from paper_2210_00947_gb300 import workloads


def _golden_dofs():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_dof_counts.txt")
    dofs = {}
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, count = line.split()[:2]
                dofs[name] = int(count)
    return dofs


GOLDEN_DOFS = _golden_dofs()


@pytest.mark.parametrize("name", ["paper2d_m1", "paper2d_m2", "paper2d_m3", "paper2d_m4"])
def test_paper_models_match_table2_dofs(name):
    dofs = GOLDEN_DOFS[name]
    w = workloads.WORKLOADS[name]
    assert w.n_nodes == dofs
    # the axial element count is a multiple of 2^(3-1) for the paper's nl = 3
    # (Section 3.2); the level count used here keeps the coarsest grid small
    # enough for the explicit coarse inverse
    assert w.nx % 4 == 0 and w.ny % 4 == 0
    assert w.nl >= 3
    ex = w.nx
    for _ in range(w.nl - 1):
        ex = (ex + 1) // 2
    assert (ex + 1) ** 2 <= workloads.COARSEST_TARGET_NODES
    # and one level fewer would not be
    ex2 = w.nx
    for _ in range(w.nl - 2):
        ex2 = (ex2 + 1) // 2
    assert w.nl == 3 or (ex2 + 1) ** 2 > workloads.COARSEST_TARGET_NODES
    # N_on is 2/15 of the 300 design cycles
    assert w.iters == 300 and w.n_on == 40


def test_paper_model_load_and_sink():
    w = workloads.WORKLOADS["paper2d_m1"]
    fixed = w.fixed()
    q = w.q()
    # sink: the middle tenth of the left edge (j in [162, 198] of 0..360)
    sink = np.flatnonzero(fixed)
    NX = w.nx + 1
    assert np.all(sink % NX == 0)
    rows = sink // NX
    assert rows.min() == 162 and rows.max() == 198 and len(rows) == 37
    # 1e-4 per unit volume over 360^2 unit elements, each node receiving a
    # quarter of each adjacent element's share; sink nodes receive nothing
    # the 37 sink nodes lie on the left edge, each touching two elements (the
    # end nodes of the edge would touch one; the patch is in the middle)
    assert abs(q.sum() - (1e-4 * 360 * 360 - 37 * 2 * 1e-4 / 4)) < 1e-12
    full = workloads.volumetric_load(w.nx, w.ny, 0, 1e-4, np.zeros_like(fixed))
    assert abs(full.sum() - 1e-4 * 360 * 360) < 1e-12
    assert np.all(q[fixed != 0] == 0.0)
    np.testing.assert_allclose(q[fixed == 0], full[fixed == 0])
    # interior node: four elements x 1e-4 / 4
    assert abs(full[NX * 100 + 100] - 1e-4) < 1e-18


def test_quarter_model_matches_section_4_3():
    w = workloads.WORKLOADS["paper3d_quarter"]
    assert w.n_nodes == GOLDEN_DOFS["paper3d_quarter"]  # the DOF count the paper prints
    fixed = w.fixed()
    NX, NY, NZ = w.nx + 1, w.ny + 1, w.nz + 1
    f = fixed.reshape(NZ, NY, NX)
    # a 14 x 14-element square (15 x 15 nodes) in the corner of the x = 0 face
    # at the symmetry planes: a quarter of the L/8 = 28-element sink
    assert f[:, :, 1:].sum() == 0
    assert f[98:, 98:, 0].all() and f[:, :, 0].sum() == 15 * 15
    # source 1e-4 per unit volume: the whole load less the sink nodes' shares
    q = w.q()
    full = workloads.volumetric_load(w.nx, w.ny, w.nz, 1e-4, np.zeros_like(fixed))
    assert abs(full.sum() - 1e-4 * 224 * 112 * 112) < 1e-9
    assert abs(q.sum() - (full.sum() - full[fixed != 0].sum())) < 1e-9
