"""Seeded synthetic inputs for the heat-sink topology-optimisation workloads.

This module holds inputs only: grid sizes, the Dirichlet (heat-sink) node
mask, nodal heat loads, initial and random density fields, and the solver
settings of each named workload.  It contains none of the method's
arithmetic (no conductivity, no operator, no solver), so both the CUDA path
and the CPU oracle may draw their inputs from it.

Numbering conventions shared by every consumer:
  * nodes are numbered x-fastest: node(i, j, k) = i + (nx+1)*(j + (ny+1)*k)
  * elements likewise: elem(i, j, k) = i + nx*(j + ny*k)
  * a 2D grid has nz = 0 (one layer of nodes, no z index)

The boundary conditions follow the paper's heat-sink problem (Section 3.2,
Figure 6: T = 0 on the middle tenth of the left edge, adiabatic elsewhere,
uniform internal heat source; Section 4.3 for the 3D cube with a centred
square sink on one face).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), written from its
    published definition: add the golden-ratio increment, then two
    xor-shift-multiply rounds and a final xor-shift."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniform_array(self, count: int) -> np.ndarray:
        """`count` consecutive draws, vectorised (same stream as uniform())."""
        idx = np.arange(1, count + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + idx * np.uint64(0x9E3779B97F4A7C15)
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + count * 0x9E3779B97F4A7C15) & _MASK64
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def node_dims(nx: int, ny: int, nz: int = 0) -> tuple[int, int, int]:
    return nx + 1, ny + 1, (nz + 1) if nz > 0 else 1


def num_nodes(nx: int, ny: int, nz: int = 0) -> int:
    a, b, c = node_dims(nx, ny, nz)
    return a * b * c


def num_elements(nx: int, ny: int, nz: int = 0) -> int:
    return nx * ny * (nz if nz > 0 else 1)


def heat_sink_mask(nx: int, ny: int, nz: int = 0, *, lo: float | None = None,
                   hi: float | None = None) -> np.ndarray:
    """uint8 per node, 1 where T = 0 is imposed.

    2D: nodes on x = 0 with lo*ny <= j <= hi*ny (default 0.45..0.55, the
    middle tenth of the left edge).  3D: nodes on x = 0 with lo*n <= j, k <=
    hi*n (default 0.4..0.6, a centred square of side 0.2)."""
    NX, NY, NZ = node_dims(nx, ny, nz)
    mask = np.zeros((NZ, NY, NX), dtype=np.uint8)
    if nz == 0:
        lo = 0.45 if lo is None else lo
        hi = 0.55 if hi is None else hi
        j = np.arange(NY)
        sel = (j >= lo * ny - 1e-9) & (j <= hi * ny + 1e-9)
        mask[0, sel, 0] = 1
    else:
        lo = 0.4 if lo is None else lo
        hi = 0.6 if hi is None else hi
        j = np.arange(NY)
        k = np.arange(NZ)
        sj = (j >= lo * ny - 1e-9) & (j <= hi * ny + 1e-9)
        sk = (k >= lo * nz - 1e-9) & (k <= hi * nz + 1e-9)
        mask[np.ix_(sk, sj, np.array([0]))] = 1
    return mask.reshape(-1)


def edge_patch_mask(nx: int, ny: int, edge: int, offset: float, frac: float = 0.1) -> np.ndarray:
    """2D sink patch of length frac*side on one edge (0 = x=0, 1 = x=nx,
    2 = y=0, 3 = y=ny) starting at relative position `offset`."""
    NX, NY = nx + 1, ny + 1
    mask = np.zeros((NY, NX), dtype=np.uint8)
    side = ny if edge in (0, 1) else nx
    start = offset * (1.0 - frac) * side
    idx = np.arange(side + 1)
    sel = (idx >= start - 1e-9) & (idx <= start + frac * side + 1e-9)
    if edge == 0:
        mask[sel, 0] = 1
    elif edge == 1:
        mask[sel, NX - 1] = 1
    elif edge == 2:
        mask[0, sel] = 1
    else:
        mask[NY - 1, sel] = 1
    return mask.reshape(-1)


def quarter_sink_mask(nx: int, ny: int, nz: int, half_side: int) -> np.ndarray:
    """3D quarter model of a cube with a centred square sink on its x = 0
    face (Section 4.3): the quarter keeps y, z in [0, L/2] with the symmetry
    planes y = ny, z = nz (adiabatic), so the sink is the corner square
    ny - half_side <= j <= ny, nz - half_side <= k <= nz of the x = 0 face."""
    NX, NY, NZ = node_dims(nx, ny, nz)
    mask = np.zeros((NZ, NY, NX), dtype=np.uint8)
    mask[nz - half_side:, ny - half_side:, 0] = 1
    return mask.reshape(-1)


def nodal_load(fixed: np.ndarray, value: float = 0.01) -> np.ndarray:
    """Uniform nodal heat load `value` on every free node, 0 on sink nodes."""
    q = np.full(fixed.shape[0], value, dtype=np.float64)
    q[fixed != 0] = 0.0
    return q


def volumetric_load(nx: int, ny: int, nz: int, source, fixed: np.ndarray) -> np.ndarray:
    """Nodal loads of a heat source given per unit volume on unit elements
    (source: scalar, or per-element array): each element hands source/2^d
    to each of its nodes (the integral of a bilinear/trilinear hat function
    over one unit element is 1/2^d).  Sink nodes get 0."""
    NX, NY, NZ = node_dims(nx, ny, nz)
    d = 2 if nz == 0 else 3
    nz_e = max(nz, 1)
    src = np.broadcast_to(np.asarray(source, dtype=np.float64), (nz_e * ny * nx,))
    src = src.reshape(nz_e, ny, nx) / (2 ** d)
    q = np.zeros((NZ, NY, NX))
    if d == 2:
        for dj in (0, 1):
            for di in (0, 1):
                q[0, dj:dj + ny, di:di + nx] += src[0]
    else:
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    q[dk:dk + nz, dj:dj + ny, di:di + nx] += src
    q = q.reshape(-1)
    q[fixed != 0] = 0.0
    return q


def quadrant_source(nx: int, ny: int, values=(5e-5, 1e-4, 1.5e-4, 3e-4)) -> np.ndarray:
    """Per-element source of the four-subdomain problem (Section 4.2):
    quadrants (x<1/2,y<1/2), (x>=1/2,y<1/2), (x<1/2,y>=1/2), (x>=1/2,y>=1/2)."""
    ex = (np.arange(nx) + 0.5) / nx
    ey = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(ex, ey)
    quad = (X >= 0.5).astype(int) + 2 * (Y >= 0.5).astype(int)
    return np.asarray(values, dtype=np.float64)[quad].reshape(-1)


def uniform_density(nel: int, value: float) -> np.ndarray:
    return np.full(nel, value, dtype=np.float64)


def random_density(nel: int, lo: float = 0.05, hi: float = 1.0, seed: int = 2210) -> np.ndarray:
    """i.i.d. uniform densities in [lo, hi) drawn element by element (element
    order) from SplitMix64(seed)."""
    return lo + (hi - lo) * SplitMix64(seed).uniform_array(nel)


def batched_designs(count: int = 64, seed: int = 2210):
    """Uneven 2D designs: per design draw nx, ny (multiples of 16 in
    64..512), sink edge (0..3), patch offset in [0,1), volume fraction in
    [0.2, 0.5), in that order, from one SplitMix64(seed) stream."""
    g = SplitMix64(seed)
    sides = list(range(64, 513, 16))
    out = []
    for _ in range(count):
        nx = sides[min(int(g.uniform() * len(sides)), len(sides) - 1)]
        ny = sides[min(int(g.uniform() * len(sides)), len(sides) - 1)]
        edge = min(int(g.uniform() * 4), 3)
        offset = g.uniform()
        vol = 0.2 + 0.3 * g.uniform()
        out.append(dict(nx=nx, ny=ny, edge=edge, offset=offset, volfrac=vol))
    return out


@dataclasses.dataclass
class Workload:
    """One named synthetic workload: grid, boundary conditions, loads and
    the solver settings it is run with."""
    name: str
    nx: int
    ny: int
    nz: int
    volfrac: float
    rho0: float
    nl: int
    iters: int
    eps2: float = 1e-8
    cg_max: int = 200
    k0: float = 1.0
    kmin: float = 1e-3
    penal: float = 3.0
    rmin: float = 1.5
    move: float = 0.2
    m: int = 2
    eps1: float = 0.5
    load: float = 0.01
    # heat source per unit volume (Section 3.2), or "quadrants" for the four
    # sub-domain sources of Section 4.2; None: the uniform nodal load
    source: float | str | None = None
    # continuous filter radius (Eq. 22-23): alpha (0 = off) and lp cycles
    filter_alpha: float = 0.0
    filter_lp: int = 0
    # sink: "centre" (heat_sink_mask) or "quarter" (quarter_sink_mask with
    # half side sink_half)
    sink: str = "centre"
    sink_half: int = 0

    @property
    def dim(self) -> int:
        return 2 if self.nz == 0 else 3

    @property
    def n_nodes(self) -> int:
        return num_nodes(self.nx, self.ny, self.nz)

    @property
    def n_elems(self) -> int:
        return num_elements(self.nx, self.ny, self.nz)

    @property
    def n_on(self) -> int:
        # MGCG is used for design cycles below N_on = 2/15 of the maximum
        # number of cycles (Section 3.2).
        return int(math.floor(2.0 * self.iters / 15.0 + 0.5))

    def fixed(self) -> np.ndarray:
        if self.sink == "quarter":
            return quarter_sink_mask(self.nx, self.ny, self.nz, self.sink_half)
        return heat_sink_mask(self.nx, self.ny, self.nz)

    def q(self) -> np.ndarray:
        if isinstance(self.source, str):
            return volumetric_load(self.nx, self.ny, self.nz, quadrant_source(self.nx, self.ny),
                                   self.fixed())
        if self.source is not None:
            return volumetric_load(self.nx, self.ny, self.nz, self.source, self.fixed())
        return nodal_load(self.fixed(), self.load)

    def density(self) -> np.ndarray:
        return uniform_density(self.n_elems, self.rho0)


# largest coarsest grid (nodes) the explicit coarse inverse is built for
COARSEST_MAX_NODES = 8192


# coarsest grid size (nodes) the paper-setting workloads aim for
COARSEST_TARGET_NODES = 300


def levels_for_direct_coarsest(nx: int, ny: int, nz: int = 0, nl_min: int = 3,
                               max_nodes: int = COARSEST_MAX_NODES) -> int:
    """Fewest levels >= nl_min whose coarsest grid (ceil coarsening) has at
    most max_nodes nodes."""
    nl = nl_min
    while True:
        ex, ey, ez = nx, ny, nz
        for _ in range(nl - 1):
            ex, ey, ez = (ex + 1) // 2, (ey + 1) // 2, (ez + 1) // 2 if nz else 0
        if num_nodes(ex, ey, ez) <= max_nodes:
            return nl
        nl += 1


def _paper2d(name: str, n: int, volfrac: float = 0.5, source=1e-4,
             continuous: bool = False) -> Workload:
    # The 2D heat-sink models of Table 2 (Sections 3.2 and 4.1): n x n
    # elements, volume fraction 0.5, r_min 3, two basis vectors, eps1 0.5,
    # eps2 1e-6, cg_max 200, source 1e-4 per unit volume, 300 design cycles
    # (the figures' run length), N_on = 2/15 of them.  The paper uses nl = 3
    # (coarsest 91^2 .. 511^2 nodes, a sparse direct solve).  Here the
    # coarsest level is factorised (a chain of sequential pivots on one SM)
    # at every MGCG call, so nl is the fewest levels >= 3 whose coarsest grid
    # holds at most 300 nodes (on Model 1, nl 4 with a 2116-node coarsest
    # grid costs 14.5 ms per MGCG design cycle, nl 6 with 169 nodes 1.8 ms).
    # With continuous=True the filter radius follows Eq. 22-23 with the
    # paper's defaults alpha = 1.4/50 and lp = 5/6 of the cycles.
    return Workload(name, n, n, 0, volfrac=volfrac, rho0=volfrac,
                    nl=levels_for_direct_coarsest(n, n, max_nodes=COARSEST_TARGET_NODES),
                    iters=300, eps2=1e-6, cg_max=200, rmin=3.0, source=source,
                    filter_alpha=1.4 / 50 if continuous else 0.0, filter_lp=250 if continuous else 0)


WORKLOADS = {
    "paper2d_m1": _paper2d("paper2d_m1", 360),
    "paper2d_m2": _paper2d("paper2d_m2", 720),
    "paper2d_m3": _paper2d("paper2d_m3", 1560),
    "paper2d_m4": _paper2d("paper2d_m4", 2040),
    # the same with the continuous filter (Section 2.3 defaults)
    "paper2d_m1c": _paper2d("paper2d_m1c", 360, continuous=True),
    "paper2d_m2c": _paper2d("paper2d_m2c", 720, continuous=True),
    # Section 4.2: four sub-domain sources, 480^2 and 960^2, volume 0.4 / 0.6
    "paper2d_q480_v04": _paper2d("paper2d_q480_v04", 480, 0.4, "quadrants", True),
    "paper2d_q480_v06": _paper2d("paper2d_q480_v06", 480, 0.6, "quadrants", True),
    "paper2d_q960_v04": _paper2d("paper2d_q960_v04", 960, 0.4, "quadrants", True),
    "paper2d_q960_v06": _paper2d("paper2d_q960_v06", 960, 0.6, "quadrants", True),
    # Section 4.3: the 224^3 cube as its quarter 224 x 112 x 112 (2,873,025
    # nodes), sink of side L/8 centred on the x = 0 face, volume 0.3, r_min 3
    # with the continuous filter (L = 224), cg_max 50, source 1e-4
    "paper3d_quarter": Workload("paper3d_quarter", 224, 112, 112, volfrac=0.3, rho0=0.3,
                                nl=levels_for_direct_coarsest(224, 112, 112, max_nodes=300),
                                iters=300, eps2=1e-6, cg_max=50, rmin=3.0, source=1e-4,
                                filter_alpha=1.4 / 50, filter_lp=250, sink="quarter",
                                sink_half=14),
    "heat2d_100": Workload("heat2d_100", 100, 100, 0, volfrac=0.4, rho0=0.4, nl=4, iters=100),
    "heat2d_1024": Workload("heat2d_1024", 1024, 1024, 0, volfrac=0.4, rho0=0.4, nl=7, iters=50),
    "heat3d_128": Workload("heat3d_128", 128, 128, 128, volfrac=0.3, rho0=0.3, nl=6, iters=50),
    "heat3d_256": Workload("heat3d_256", 256, 256, 256, volfrac=0.3, rho0=0.3, nl=7, iters=20),
}
