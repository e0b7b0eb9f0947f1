// Tiled kernels for the finest 3D (H8) level of the V-cycle.
//
// A block of TX x TY threads owns a TX x TY column of nodes and walks along z
// through a run of node planes.  Rotating planes of the operand
// (x^ = x with fixed nodes zeroed, zero off the grid) and rotating layers of
// element conductivities (zero off the grid) sit in shared memory, so the
// 21-point H8 stencil of each node
//   (A x)_i = (4 sum_e k_e x_i - sum_facediag (k_a + k_b) x^_j - sum_bodydiag k_e x^_j) / 12
// is evaluated without bounds tests; a fixed row is the identity.  Two fused
// forms cover the V-cycle with a zero initial guess (Table 1 with one pre- and
// one post-sweep):
//   pre:  x = w D^-1 b  and  r = b - A x             (jacobi from zero + residual)
//   post: x' = v + w D^-1 (b - A v),  v = x + P x_c   (interpolation + post-smooth)
// and a generic form computes r = b - A x or one damped-Jacobi sweep.  A
// fifth form serves the FP32 conjugate-gradient iteration of the mixed path:
//   dir:  p = z + beta p_old,  y = A p,  p . y       (direction update + product)
//
// Latency: the global loads of plane k+2 (and element layer k+1) are issued
// into registers before the block computes plane k, and are turned into the
// operand and stored to shared memory one step later, so each step overlaps
// its memory round trip with the previous step's arithmetic.  A step reads
// one plane and one layer of the tile (the rows are split by element layer
// and the lower layer's share, with plane k's in-plane neighbours, is carried
// in registers), and four slots of each let one barrier per step suffice.
// Each thread loads its own node; the one-node ring around the tile is
// loaded by a few warps, so no thread divides to find its halo cell.  The z
// extent is split evenly into as many runs as fill the GPU once.
#include "common.cuh"
#include "tile3d.cuh"
#include "df64.cuh"

namespace mgar {
namespace f3d {
using namespace tile;

enum Mode { PRE = 0, POST = 1, RESID = 2, SWEEP = 3, DIR = 4 };

struct FineArgs {
  int ex, ey, ez, NX, NY, NZ;
  int gz;  // z runs
  const uint8_t* fixed;
  const void* ke;
  const void* b;    // DIR: z
  const void* dinv;
  const void* x;    // RESID / SWEEP: iterate; POST: x before interpolation; DIR: p_old
  const void* xc;   // POST: coarse correction
  int cNX, cNY, cNZ;  // POST: coarse node dims
  void* out0;       // PRE: x, RESID: r, SWEEP/POST: x', DIR: p
  void* out1;       // PRE: r, DIR: A p
  double omega;
  // POST / SWEEP, optional (dout given): r . x' with r in double-float
  // pairs (the CG's r . z), or with r = b when rdot is null
  const float2* rdot;
  double* partials;
  unsigned int* counter;
  double* dout;     // POST / SWEEP: r . x'; DIR: p . A p
  // DIR: beta = rz_new / rz_old, or 0 while *first is nonzero; with *parity
  // odd, p_old is x_alt and p goes to out_alt (the two direction buffers swap
  // each iteration); rz_set, when given, receives *rz_new once every block
  // has read it
  const double* rz_new;
  const double* rz_old;
  const double* first;
  const double* parity;
  const void* x_alt;
  void* out_alt;
  double* rz_set;
};

// 1D interpolation taps onto fine node i (nf fine elements): coarse index of
// the first tap and whether the node sits halfway between two coarse nodes.
__device__ __forceinline__ int ptap0(int i, int nf, bool& half) {
  half = (i & 1) && i < nf;
  return (i & 1) ? (half ? (i - 1) >> 1 : (i + 1) >> 1) : i >> 1;
}

// A node column (i, j): everything about its loads that does not depend on
// the plane, computed once per thread.
struct Column {
  int base;      // clamped i + NX * clamped j
  bool on;       // (i, j) inside the grid
  int cxy[4];    // POST: coarse offsets of (x0|x1) + cNX * (y0|y1)
  uint8_t hxy;   // POST: half flags of x (bit 0) and y (bit 1)
};

__device__ __forceinline__ Column make_column(const FineArgs& a, int i, int j, bool post) {
  Column c;
  c.on = i >= 0 && i < a.NX && j >= 0 && j < a.NY;
  const int ic = min(max(i, 0), a.NX - 1), jc = min(max(j, 0), a.NY - 1);
  c.base = ic + a.NX * jc;
  c.hxy = 0;
  c.cxy[0] = c.cxy[1] = c.cxy[2] = c.cxy[3] = 0;
  if (post) {
    bool hx, hy;
    const int x0 = ptap0(ic, a.ex, hx), y0 = ptap0(jc, a.ey, hy);
    c.hxy = (uint8_t)(hx | (hy << 1));
    c.cxy[0] = x0 + a.cNX * y0;
    c.cxy[1] = x0 + hx + a.cNX * y0;
    c.cxy[2] = x0 + a.cNX * (y0 + hy);
    c.cxy[3] = x0 + hx + a.cNX * (y0 + hy);
  }
  return c;
}

// Raw loads of one node of a plane, issued one step before use.
template <typename Real, int MODE>
struct NodeFetch {
  Real v0 = Real(0), v1 = Real(0);  // PRE: b, dinv; DIR: z, p_old; else x (v1 unused)
  Real c[8];                        // POST: coarse values
  uint8_t f = 1;                    // fixed (or off the grid: treated as zero)
  uint8_t hz = 0;                   // POST: half flag of z
  bool on = false;

  // xsrc: DIR's p_old (null on the first iteration)
  __device__ __forceinline__ void issue(const FineArgs& a, const Column& col, int k,
                                        const Real* xsrc = nullptr) {
    on = col.on && k >= 0 && k < a.NZ;
    const int kc = min(max(k, 0), a.NZ - 1);
    const int idx = col.base + a.NX * a.NY * kc;
    if (!CK(idx, (int64_t)a.NX * a.NY * a.NZ)) return;
    f = a.fixed[idx];
    if (MODE == PRE) {
      v0 = ((const Real*)a.b)[idx];
      v1 = ((const Real*)a.dinv)[idx];
    } else if (MODE == DIR) {
      v0 = ((const Real*)a.b)[idx];
      if (xsrc) v1 = xsrc[idx];
    } else {
      v0 = ((const Real*)a.x)[idx];
    }
    if (MODE == POST) {
      bool h;
      const int z0 = ptap0(kc, a.ez, h);
      hz = h;
      const int P = a.cNX * a.cNY;
      const Real* xc = (const Real*)a.xc;
      const int z0o = z0 * P, z1o = (z0 + h) * P;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (CK(col.cxy[q] + z1o, (int64_t)P * a.cNZ)) {
          c[q] = xc[col.cxy[q] + z0o];
          c[4 + q] = xc[col.cxy[q] + z1o];
        }
      }
    }
  }

  // operand value before masking (PRE: w D^-1 b; POST: x + P x_c, fixed
  // nodes keep x; DIR: z + beta p_old, beta passed as omega; else x)
  __device__ __forceinline__ Real value(Real omega, uint8_t hxy) const {
    if (MODE == PRE) return omega * v1 * v0;
    if (MODE == DIR) return v0 + omega * v1;
    if (MODE == POST) {
      if (f) return v0;
      const Real wx = (hxy & 1) ? Real(0.5) : Real(1), ux = (hxy & 1) ? Real(0.5) : Real(0);
      const Real wy = (hxy & 2) ? Real(0.5) : Real(1), uy = (hxy & 2) ? Real(0.5) : Real(0);
      const Real wz = hz ? Real(0.5) : Real(1), uz = hz ? Real(0.5) : Real(0);
      // c[q + 4 cz] with q = x-tap + 2 y-tap
      const Real r00 = wx * c[0] + ux * c[1], r01 = wx * c[2] + ux * c[3];
      const Real r10 = wx * c[4] + ux * c[5], r11 = wx * c[6] + ux * c[7];
      const Real s0 = wy * r00 + uy * r01, s1 = wy * r10 + uy * r11;
      return v0 + (wz * s0 + uz * s1);
    }
    return v0;
  }
  __device__ __forceinline__ Real masked(Real omega, uint8_t hxy) const {
    return (on && !f) ? value(omega, hxy) : Real(0);
  }
};

template <typename Real>
struct ElemFetch {
  Real v = Real(0);
  bool on = false;
  __device__ __forceinline__ void issue(const FineArgs& a, int ebase, bool eon, int l) {
    on = eon && l >= 0 && l < a.ez;
    const int idx = ebase + a.ex * a.ey * min(max(l, 0), a.ez - 1);
    if (CK(idx, (int64_t)a.ex * a.ey * a.ez)) v = ((const Real*)a.ke)[idx];
  }
  __device__ __forceinline__ Real get() const { return on ? v : Real(0); }
};

// The eight in-plane neighbours of node (tx, ty) of a plane tile: the four
// diagonal ones (-x-y, +x-y, -x+y, +x+y), then -x, +x, -y, +y.
template <typename Real, int TX, int TY>
__device__ __forceinline__ void plane_ring8(const Real (&Xp)[TY + 2][TX + 2], int tx, int ty,
                                            Real (&h)[8]) {
  const int cx = tx + 1, cy = ty + 1;
  h[0] = Xp[cy - 1][cx - 1];
  h[1] = Xp[cy - 1][cx + 1];
  h[2] = Xp[cy + 1][cx - 1];
  h[3] = Xp[cy + 1][cx + 1];
  h[4] = Xp[cy][cx - 1];
  h[5] = Xp[cy][cx + 1];
  h[6] = Xp[cy - 1][cx];
  h[7] = Xp[cy + 1][cx];
}

// The four elements e_q of one layer around a node column, q = (qy, qx) for
// the element at (i - 1 + qx, j - 1 + qy), give the H8 rows (times 12) of the
// column's nodes below (plane lo) and above (plane hi) the layer:
//   up   = 4 S x_lo - C - E(hi),   down = 4 S x_hi - C - E(lo),
// with S = sum_q e_q, C = sum_q e_q (x_lo + x_hi at the in-plane diagonal
// neighbour q) and E(p) = sum over the four in-plane edge neighbours of plane
// p of the two elements sharing that edge times its value.  Row (i,j,k) is
// up(layer k) + down(layer k-1).  nb holds plane lo's neighbours on entry
// and plane hi's on return.
template <typename Real, int TX, int TY>
__device__ __forceinline__ void layer_rows(const Real (&Kl)[TY + 1][TX + 1],
                                           const Real (&Xhi)[TY + 2][TX + 2], int tx, int ty,
                                           Real (&nb)[8], Real x_lo, Real x_hi, Real& up,
                                           Real& down) {
  const Real e00 = Kl[ty][tx], e01 = Kl[ty][tx + 1], e10 = Kl[ty + 1][tx], e11 = Kl[ty + 1][tx + 1];
  Real h[8];
  plane_ring8<Real, TX, TY>(Xhi, tx, ty, h);
  const Real ew = e00 + e10, ee = e01 + e11, es = e00 + e01, en = e10 + e11;
  const Real s4 = Real(4) * (es + en);
  const Real cc = e00 * (nb[0] + h[0]) + e01 * (nb[1] + h[1]) + e10 * (nb[2] + h[2]) +
                  e11 * (nb[3] + h[3]);
  const Real elo = ew * nb[4] + ee * nb[5] + es * nb[6] + en * nb[7];
  const Real ehi = ew * h[4] + ee * h[5] + es * h[6] + en * h[7];
  up = s4 * x_lo - cc - ehi;
  down = s4 * x_hi - cc - elo;
#pragma unroll
  for (int q = 0; q < 8; ++q) nb[q] = h[q];
}

// Plane slots are relative to the block's first plane: plane p lives in slot
// (p - kb + 1) & 3, and so does element layer p.  The z loop is unrolled by
// four, so every slot index is a compile-time constant.
// resident blocks per SM the registers are budgeted for (POST holds the
// interpolation's coarse values and needs more)
constexpr int f3d_minb(int mode, int nt) {
  return mode == POST ? (nt <= 256 ? 3 : (nt <= 400 ? 2 : 1)) : (nt <= 256 ? 4 : 2);
}

template <typename Real, int MODE, class T>
__global__ void __launch_bounds__(T::NTB, f3d_minb(MODE, T::NT)) k_fine3d(FineArgs a) {
  constexpr int TX = T::TX, TY = T::TY, NT = T::NT;
  constexpr int XRING = T::XRING, KRING = T::KRING, KRING0 = T::KRING0;
  __shared__ Real X[4][TY + 2][TX + 2];
  __shared__ Real K[4][TY + 1][TX + 1];
  pdl_wait();  // one wave: the successor may be dispatched right away
  pdl_trigger();

  // 1D block of whole warps; threads past TX * TY only help with the ring
  // loads and the reduction
  const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
  const bool real = tid < NT;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int kb = (int)(((int64_t)blockIdx.z * a.NZ) / a.gz);
  const int kend = (int)(((int64_t)(blockIdx.z + 1) * a.NZ) / a.gz);
  const int i = i0 + tx, j = j0 + ty;
  // DIR: beta takes omega's place, and the direction buffers follow the parity
  Real om = (Real)a.omega;
  const Real* dsrc = nullptr;
  Real* pdst = nullptr;
  if (MODE == DIR) {
    const bool first = *a.first != 0.0;
    const bool odd = a.parity && (((int)*a.parity) & 1);
    const float q = block_div_f(a.rz_new, a.rz_old);  // once per block
    om = first ? Real(0) : (Real)q;
    dsrc = first ? nullptr : (const Real*)(odd ? a.x_alt : a.x);
    pdst = (Real*)(odd ? a.out_alt : a.out0);
  }
  const bool xr = tid < XRING, kr = tid >= KRING0 && tid < KRING0 + KRING;
  int rxh = 0, ryh = 0, kxh = 0, kyh = 0;
  if (xr) T::xring(tid, rxh, ryh);
  if (kr) T::kring(tid - KRING0, kxh, kyh);
  const bool mine = real && i < a.NX && j < a.NY;
  const int NXY = a.NX * a.NY;

  const Column ocol = make_column(a, i, j, MODE == POST);
  const Column rcol = make_column(a, i0 - 1 + rxh, j0 - 1 + ryh, MODE == POST);
  const int ke_i = i, ke_j = j, kr_i = i0 - 1 + kxh, kr_j = j0 - 1 + kyh;
  const bool keon = ke_i < a.ex && ke_j < a.ey;
  const bool kron = kr_i >= 0 && kr_i < a.ex && kr_j >= 0 && kr_j < a.ey;
  const int kebase = min(ke_i, a.ex - 1) + a.ex * min(ke_j, a.ey - 1);
  const int krbase = min(max(kr_i, 0), a.ex - 1) + a.ex * min(max(kr_j, 0), a.ey - 1);

  NodeFetch<Real, MODE> own, ring;
  ElemFetch<Real> kown, kring_;
  Real ownb = Real(0), ownd = Real(0);
  // centre values per slot: unmasked operand, b, D^-1, fixed flag (and r
  // for the fused r . x')
  Real cv[4], cb[4], cd[4], mv[4];
  bool cf[4];
  const bool rdot = (MODE == POST || MODE == SWEEP || MODE == DIR) && a.dout != nullptr;
  // the thread's terms of p . Ap, or of r . x' with r in FP32, are few (one z
  // run, about 20): summed in FP32 and combined across threads in df64; r in
  // df64 pairs keeps a df64 sum
  df dacc{0.f, 0.f};
  float facc = 0.f;

  auto issue_plane_to = [&](int p, NodeFetch<Real, MODE>& o, NodeFetch<Real, MODE>& rg, Real& ob,
                            Real& od) {
    o.issue(a, ocol, p, dsrc);
    if (MODE != PRE && MODE != DIR) {
      const int idx = ocol.base + NXY * min(max(p, 0), a.NZ - 1);
      if (CK(idx, (int64_t)NXY * a.NZ)) {
        ob = ((const Real*)a.b)[idx];
        if (MODE == POST || MODE == SWEEP) od = ((const Real*)a.dinv)[idx];
      }
    }
    if (xr) rg.issue(a, rcol, p, dsrc);
  };
  auto issue_plane = [&](int p) { issue_plane_to(p, own, ring, ownb, ownd); };
  auto issue_layer = [&](int l) {
    kown.issue(a, kebase, keon, l);
    if (kr) kring_.issue(a, krbase, kron, l);
  };

#define F3D_FINISH_FROM(S, O, RG, OB, OD)                              \
  {                                                                    \
    mv[S] = O.masked(om, ocol.hxy);                                    \
    if (real) X[S][ty + 1][tx + 1] = mv[S];                            \
    cv[S] = O.value(om, ocol.hxy);                                     \
    cb[S] = MODE == PRE ? O.v0 : OB;                                   \
    cd[S] = OD;                                                        \
    cf[S] = O.f != 0;                                                  \
    if (xr) X[S][ryh][rxh] = RG.masked(om, rcol.hxy);                  \
  }
#define F3D_FINISH(S) F3D_FINISH_FROM(S, own, ring, ownb, ownd)
#define F3D_FINISH_LAYER(S)                                            \
  {                                                                    \
    if (real) K[S][ty + 1][tx + 1] = kown.get();                       \
    if (kr) K[S][kyh][kxh] = kring_.get();                             \
  }

  // prologue: planes kb-1 (slot 0), kb (slot 1) and layer kb-1 (slot 0) in
  // place, their loads in flight together; then plane kb+1 and layer kb in
  // flight
  {
    NodeFetch<Real, MODE> own2, ring2;
    Real ownb2 = Real(0), ownd2 = Real(0);
    issue_plane(kb - 1);
    issue_plane_to(kb, own2, ring2, ownb2, ownd2);
    issue_layer(kb - 1);
    F3D_FINISH(0);
    F3D_FINISH_FROM(1, own2, ring2, ownb2, ownd2);
    F3D_FINISH_LAYER(0);
  }
  issue_plane(kb + 1);
  issue_layer(kb);

  // Row (i,j,k) of the operator is split by element layer: the layer between
  // planes k and k+1 gives its "up" part and the next row's "down" part
  // (layer_rows).  The down part and plane k's in-plane neighbours come from
  // the step before, so a step reads one layer and one plane of the tile.
  // Prologue: planes kb-1 and kb and layer kb-1 are in place.
  __syncthreads();
  Real nb[8], dk = Real(0);
  if (mine) {
    Real up;
    plane_ring8<Real, TX, TY>(X[0], tx, ty, nb);
    layer_rows<Real, TX, TY>(K[0], X[1], tx, ty, nb, mv[0], mv[1], up, dk);
  }

  // one step for plane k in slot S1 = (S + 1) & 3 (plane k+1 in slot S2,
  // layer k in slot S1)
#define F3D_STEP(S)                                                                        \
  {                                                                                        \
    constexpr int S1 = ((S) + 1) & 3, S2 = ((S) + 2) & 3;                                  \
    const int k = kk + (S);                                                                \
    if (k >= kend) break;                                                                  \
    F3D_FINISH(S2);                                                                        \
    F3D_FINISH_LAYER(S1);                                                                  \
    issue_plane(k + 2);                                                                    \
    issue_layer(k + 1);                                                                    \
    __syncthreads();                                                                       \
    if (mine) {                                                                            \
      const int idx = i + a.NX * (j + a.NY * k);                                           \
      /* r for the fused r . x' (its load overlaps the stencil) */                         \
      const float2 rv = (rdot && a.rdot) ? a.rdot[idx] : make_float2(0.f, 0.f);           \
      Real up, down;                                                                       \
      layer_rows<Real, TX, TY>(K[S1], X[S2], tx, ty, nb, mv[S1], mv[S2], up, down);        \
      const Real acc = up + dk;                                                            \
      dk = down;                                                                           \
      const Real xi = cv[S1]; /* a fixed row is the identity */                            \
      const Real ax = cf[S1] ? xi : acc * Real(1.0 / 12.0);                                \
      const Real bi = cb[S1];                                                              \
      /* r = 0 on fixed nodes: the restriction P^T = (Z P)^T does not read them */       \
      if (MODE == PRE) {                                                                   \
        ((Real*)a.out0)[idx] = xi;                                                         \
        ((Real*)a.out1)[idx] = cf[S1] ? Real(0) : bi - ax;                                 \
      } else if (MODE == RESID) {                                                          \
        ((Real*)a.out0)[idx] = cf[S1] ? Real(0) : bi - ax;                                 \
      } else if (MODE == DIR) {                                                            \
        pdst[idx] = xi;                                                                    \
        ((Real*)a.out1)[idx] = ax;                                                         \
        if (rdot) facc = fmaf((float)xi, (float)ax, facc);                                  \
      } else {                                                                             \
        const Real xo = xi + om * cd[S1] * (bi - ax);                                      \
        ((Real*)a.out0)[idx] = xo;                                                         \
        if (rdot) {                                                                        \
          if (a.rdot) dacc = df_add(dacc, df_mulf(df{rv.x, rv.y}, (float)xo));              \
          else facc = fmaf((float)bi, (float)xo, facc);                                    \
        }                                                                                  \
      }                                                                                    \
    }                                                                                      \
  }

  for (int kk = kb; kk < kend; kk += 4) {
    F3D_STEP(0)
    F3D_STEP(1)
    F3D_STEP(2)
    F3D_STEP(3)
  }
#undef F3D_STEP
#undef F3D_FINISH
#undef F3D_FINISH_FROM
#undef F3D_FINISH_LAYER
  if (rdot) {
    double t;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    const df v = df_add(dacc, df{facc, 0.f});
    if (block_sum_last_df(v, a.partials, a.counter, t, tid, T::NTB, bid, nb) && tid == 0) {
      a.dout[0] = t;
      if (MODE == DIR && a.rz_set) *a.rz_set = *a.rz_new;  // every block has read rz_new
    }
  }
}

// z runs so that the grid fills the GPU once: resident blocks per SM x SMs,
// split over the column tiles
template <typename Real, int MODE, class T>
int runs_for(const Dims& d, int sms) {
  int per_sm = 0;
  MGAR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fine3d<Real, MODE, T>, T::NTB, 0));
  per_sm = std::max(per_sm, 1);
  const int64_t cols = (int64_t)((d.NX + T::TX - 1) / T::TX) * ((d.NY + T::TY - 1) / T::TY);
  const int64_t want = (int64_t)per_sm * sms;
  // at most one wave: a few blocks past it would run as a second wave
  const int64_t gz = std::max<int64_t>(1, want / cols);
  return (int)std::min<int64_t>(gz, d.NZ);
}

}  // namespace f3d

// The tile: 32 x 8, or 43 x 5 where that leaves fewer lanes idle (129-node
// planes: 95 % of the lanes busy instead of 76 %).
void fine3d_prepare(Ctx& c) {
  using namespace f3d;
  int dev = 0, sms = 0;
  MGAR_CUDA(cudaGetDevice(&dev));
  MGAR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const Dims& d = c.L[0];
  c.f3d_tile = tile_use(d.NX, d.NY, T43x5::TX, T43x5::TY) > tile_use(d.NX, d.NY, T32x8::TX, T32x8::TY);
  if (c.f3d_tile) {
    c.f3d_gz[PRE] = runs_for<float, PRE, T43x5>(d, sms);
    c.f3d_gz[POST] = runs_for<float, POST, T43x5>(d, sms);
    c.f3d_gz[RESID] = runs_for<float, RESID, T43x5>(d, sms);
    c.f3d_gz[SWEEP] = runs_for<float, SWEEP, T43x5>(d, sms);
    c.f3d_gz[DIR] = runs_for<float, DIR, T43x5>(d, sms);
  } else {
    c.f3d_gz[PRE] = runs_for<float, PRE, T32x8>(d, sms);
    c.f3d_gz[POST] = runs_for<float, POST, T32x8>(d, sms);
    c.f3d_gz[RESID] = runs_for<float, RESID, T32x8>(d, sms);
    c.f3d_gz[SWEEP] = runs_for<float, SWEEP, T32x8>(d, sms);
    c.f3d_gz[DIR] = runs_for<float, DIR, T32x8>(d, sms);
  }
}

namespace f3d {
template <int MODE, class T>
void launch_t(Ctx& c, FineArgs& a) {
  const Dims& d = c.L[0];
  a.gz = std::max(1, std::min(c.f3d_gz[MODE], d.NZ));
  const dim3 grid((d.NX + T::TX - 1) / T::TX, (d.NY + T::TY - 1) / T::TY, a.gz);
  launch_pdl(c.stream, c.use_pdl, k_fine3d<float, MODE, T>, grid, dim3(T::NTB), a);
}
template <int MODE>
void launch(Ctx& c, FineArgs& a) {
  if (c.f3d_tile) launch_t<MODE, T43x5>(c, a);
  else launch_t<MODE, T32x8>(c, a);
}
}  // namespace f3d

// Launch one tiled finest-level pass of the FP32 V-cycle (3D only).
// mode: 0 pre, 1 post, 2 residual, 3 sweep.
void fine3d(Ctx& c, int mode, const float* ke, const float* b, const float* dinv, const float* x,
            const float* xc, float* out0, float* out1, const float2* rdot, double* dout) {
  using namespace f3d;
  const Dims& d = c.L[0];
  FineArgs a{};
  a.ex = d.ex;
  a.ey = d.ey;
  a.ez = d.ez;
  a.NX = d.NX;
  a.NY = d.NY;
  a.NZ = d.NZ;
  a.fixed = c.fixed;
  a.ke = ke;
  a.b = b;
  a.dinv = dinv;
  a.x = x;
  a.xc = xc;
  a.cNX = c.nl > 1 ? c.L[1].NX : 0;
  a.cNY = c.nl > 1 ? c.L[1].NY : 0;
  a.cNZ = c.nl > 1 ? c.L[1].NZ : 0;
  a.out0 = out0;
  a.out1 = out1;
  a.omega = c.p.omega;
  a.rdot = rdot;
  a.dout = dout;
  a.partials = c.partials;
  a.counter = c.counter;
  switch (mode) {
    case PRE: launch<PRE>(c, a); break;
    case POST: launch<POST>(c, a); break;
    case RESID: launch<RESID>(c, a); break;
    default: launch<SWEEP>(c, a); break;
  }
  MGAR_LAUNCH_CHECK_AT(level_site(6 + (mode == PRE ? 0 : mode == POST ? 1 : mode == SWEEP ? 2 : 3), 0));
}

// p = z + (rz_new / rz_old) p_old (p = z while *first is nonzero), y = A p,
// p . y into *dot; FP32 vectors
void fine3d_dir(Ctx& c, const float* z, const float* p_old, float* p, const double* rz_new,
                const double* rz_old, const double* first, const double* parity, float* y,
                double* dot, double* rz_set) {
  using namespace f3d;
  const Dims& d = c.L[0];
  FineArgs a{};
  a.ex = d.ex;
  a.ey = d.ey;
  a.ez = d.ez;
  a.NX = d.NX;
  a.NY = d.NY;
  a.NZ = d.NZ;
  a.fixed = c.fixed;
  a.ke = c.ke_f;
  a.b = z;
  a.x = p_old;
  a.out0 = p;
  a.x_alt = p;  // odd parity: the buffers swap roles
  a.out_alt = const_cast<float*>(p_old);
  a.out1 = y;
  a.rz_new = rz_new;
  a.rz_old = rz_old;
  a.first = first;
  a.parity = parity;
  a.rz_set = rz_set;
  a.dout = dot;
  a.partials = c.partials;
  a.counter = c.counter;
  launch<DIR>(c, a);
  MGAR_LAUNCH_CHECK();
}

}  // namespace mgar
