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
// and a generic form computes r = b - A x or one damped-Jacobi sweep.
//
// Latency: the global loads of plane k+2 (and element layer k+1) are issued
// into registers before the block computes plane k, and are turned into the
// operand and stored to shared memory one step later, so each step overlaps
// its memory round trip with the previous step's arithmetic.  Four plane
// slots and three layer slots let one barrier per step suffice.  Each thread
// loads its own node; the one-node ring around the tile is loaded by a few
// warps, so no thread divides to find its halo cell.  The z extent is split
// evenly into as many runs as fill the GPU once.
#include "common.cuh"
#include "tile3d.cuh"

namespace mgar {
namespace f3d {
using namespace tile;

enum Mode { PRE = 0, POST = 1, RESID = 2, SWEEP = 3 };

struct FineArgs {
  int ex, ey, ez, NX, NY, NZ;
  int gz;  // z runs
  const uint8_t* fixed;
  const void* ke;
  const void* b;
  const void* dinv;
  const void* x;    // RESID / SWEEP: iterate; POST: x before interpolation
  const void* xc;   // POST: coarse correction
  int cNX, cNY, cNZ;  // POST: coarse node dims
  void* out0;       // PRE: x, RESID: r, SWEEP/POST: x'
  void* out1;       // PRE: r
  double omega;
};

// 1D interpolation taps onto fine node i (nf fine elements): coarse index of
// the first tap and whether the node sits halfway between two coarse nodes.
__device__ __forceinline__ int ptap0(int i, int nf, bool& half) {
  half = (i & 1) && i < nf;
  return (i & 1) ? (half ? (i - 1) >> 1 : (i + 1) >> 1) : i >> 1;
}

// Raw loads of one node of a plane, issued one step before use.
template <typename Real, int MODE>
struct NodeFetch {
  Real v0 = Real(0), v1 = Real(0);  // PRE: b, dinv; else x (v1 unused)
  Real c[8];                        // POST: coarse values
  uint8_t f = 1;                    // fixed (or off the grid: treated as zero)
  uint8_t hm = 0;                   // POST: half flags (x, y, z)
  bool on = false;

  __device__ __forceinline__ void issue(const FineArgs& a, int i, int j, int k) {
    on = i >= 0 && i < a.NX && j >= 0 && j < a.NY && k >= 0 && k < a.NZ;
    const int ic = min(max(i, 0), a.NX - 1), jc = min(max(j, 0), a.NY - 1),
              kc = min(max(k, 0), a.NZ - 1);
    const int idx = ic + a.NX * (jc + a.NY * kc);
    if (!CK(idx, (int64_t)a.NX * a.NY * a.NZ)) return;
    f = a.fixed[idx];
    if (MODE == PRE) {
      v0 = ((const Real*)a.b)[idx];
      v1 = ((const Real*)a.dinv)[idx];
    } else {
      v0 = ((const Real*)a.x)[idx];
    }
    if (MODE == POST) {
      bool hx, hy, hz;
      const int x0 = ptap0(ic, a.ex, hx), y0 = ptap0(jc, a.ey, hy), z0 = ptap0(kc, a.ez, hz);
      hm = (uint8_t)(hx | (hy << 1) | (hz << 2));
      const int x1 = x0 + hx, y1 = y0 + hy, z1 = z0 + hz;
      const int P = a.cNX * a.cNY;
      const Real* xc = (const Real*)a.xc;
      const int zz[2] = {z0 * P, z1 * P}, yy[2] = {y0 * a.cNX, y1 * a.cNX};
#pragma unroll
      for (int cz = 0; cz < 2; ++cz)
#pragma unroll
        for (int cy = 0; cy < 2; ++cy) {
          const int base = zz[cz] + yy[cy];
          if (CK(base + x1, (int64_t)P * a.cNZ)) {
            c[4 * cz + 2 * cy] = xc[base + x0];
            c[4 * cz + 2 * cy + 1] = xc[base + x1];
          }
        }
    }
  }

  // operand value before masking (PRE: w D^-1 b; POST: x + P x_c, fixed
  // nodes keep x; else x)
  __device__ __forceinline__ Real value(Real omega) const {
    if (MODE == PRE) return omega * v1 * v0;
    if (MODE == POST) {
      if (f) return v0;
      const Real wx = (hm & 1) ? Real(0.5) : Real(1), wy = (hm & 2) ? Real(0.5) : Real(1),
                 wz = (hm & 4) ? Real(0.5) : Real(1);
      const Real ux = (hm & 1) ? Real(0.5) : Real(0), uy = (hm & 2) ? Real(0.5) : Real(0),
                 uz = (hm & 4) ? Real(0.5) : Real(0);
      const Real r00 = wx * c[0] + ux * c[1], r01 = wx * c[2] + ux * c[3];
      const Real r10 = wx * c[4] + ux * c[5], r11 = wx * c[6] + ux * c[7];
      const Real s0 = wy * r00 + uy * r01, s1 = wy * r10 + uy * r11;
      return v0 + (wz * s0 + uz * s1);
    }
    return v0;
  }
  __device__ __forceinline__ Real masked(Real omega) const {
    return (on && !f) ? value(omega) : Real(0);
  }
};

template <typename Real>
struct ElemFetch {
  Real v = Real(0);
  bool on = false;
  __device__ __forceinline__ void issue(const FineArgs& a, int e, int f, int l) {
    on = e >= 0 && e < a.ex && f >= 0 && f < a.ey && l >= 0 && l < a.ez;
    const int idx = min(max(e, 0), a.ex - 1) + a.ex * (min(max(f, 0), a.ey - 1) + a.ey * min(max(l, 0), a.ez - 1));
    if (CK(idx, (int64_t)a.ex * a.ey * a.ez)) v = ((const Real*)a.ke)[idx];
  }
  __device__ __forceinline__ Real get() const { return on ? v : Real(0); }
};

template <typename Real, int MODE>
__global__ void __launch_bounds__(NT, sizeof(Real) == 4 ? 4 : 2) k_fine3d(FineArgs a) {
  __shared__ Real X[XS][TY + 2][TX + 2];
  __shared__ Real K[KS][TY + 1][TX + 1];
  __shared__ Real Cx[XS][TY][TX];  // centre operand value, unmasked
  __shared__ Real Cb[XS][TY][TX];  // centre right-hand side
  __shared__ Real Cd[(MODE == POST || MODE == SWEEP) ? XS : 1][TY][TX];  // centre D^-1
  __shared__ uint8_t Cf[XS][TY][TX];                                       // centre fixed flag

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int kb = (int)(((int64_t)blockIdx.z * a.NZ) / a.gz);
  const int kend = (int)(((int64_t)(blockIdx.z + 1) * a.NZ) / a.gz);
  const int i = i0 + tx, j = j0 + ty;
  const Real om = (Real)a.omega;
  const bool xr = tid < XRING, kr = tid >= KRING0 && tid < KRING0 + KRING;
  int rxh = 0, ryh = 0, kxh = 0, kyh = 0;
  if (xr) xring(tid, rxh, ryh);
  if (kr) kring(tid - KRING0, kxh, kyh);

  NodeFetch<Real, MODE> own, ring;
  ElemFetch<Real> kown, kring_;
  Real ownb = Real(0), ownd = Real(0);

  auto issue_plane = [&](int p) {
    own.issue(a, i, j, p);
    if (MODE != PRE) {
      // centre data beyond the operand
      const int idx = min(i, a.NX - 1) + a.NX * (min(j, a.NY - 1) + a.NY * min(max(p, 0), a.NZ - 1));
      if (CK(idx, (int64_t)a.NX * a.NY * a.NZ)) {
        ownb = ((const Real*)a.b)[idx];
        if (MODE == POST || MODE == SWEEP) ownd = ((const Real*)a.dinv)[idx];
      }
    }
    if (xr) ring.issue(a, i0 - 1 + rxh, j0 - 1 + ryh, p);
  };
  auto finish_plane = [&](int p) {
    const int s = (p + XS) % XS;
    X[s][ty + 1][tx + 1] = own.masked(om);
    const Real v = own.value(om);
    Cx[s][ty][tx] = v;
    Cb[s][ty][tx] = MODE == PRE ? own.v0 : ownb;
    if (MODE == POST || MODE == SWEEP) Cd[s][ty][tx] = ownd;
    Cf[s][ty][tx] = own.f;
    if (xr) X[s][ryh][rxh] = ring.masked(om);
  };
  auto issue_layer = [&](int l) {
    kown.issue(a, i, j, l);
    if (kr) kring_.issue(a, i0 - 1 + kxh, j0 - 1 + kyh, l);
  };
  auto finish_layer = [&](int l) {
    const int s = (l + KS) % KS;
    K[s][ty + 1][tx + 1] = kown.get();
    if (kr) K[s][kyh][kxh] = kring_.get();
  };

  // prologue: planes kb-1, kb and layer kb-1 in place; plane kb+1 and layer
  // kb in flight
  issue_plane(kb - 1);
  finish_plane(kb - 1);
  issue_plane(kb);
  issue_layer(kb - 1);
  finish_plane(kb);
  finish_layer(kb - 1);
  issue_plane(kb + 1);
  issue_layer(kb);

  const bool mine = i < a.NX && j < a.NY;
  for (int k = kb; k < kend; ++k) {
    finish_plane(k + 1);
    finish_layer(k);
    issue_plane(k + 2);
    issue_layer(k + 1);
    __syncthreads();
    if (mine) {
      const int idx = i + a.NX * (j + a.NY * k);
      const auto& Xm = X[(k + XS - 1) % XS];
      const auto& X0 = X[k % XS];
      const auto& Xp = X[(k + 1) % XS];
      const auto& Km = K[(k + KS - 1) % KS];
      const auto& Kp = K[k % KS];
      const Real k000 = Km[ty][tx], k001 = Km[ty][tx + 1], k010 = Km[ty + 1][tx],
                 k011 = Km[ty + 1][tx + 1];
      const Real k100 = Kp[ty][tx], k101 = Kp[ty][tx + 1], k110 = Kp[ty + 1][tx],
                 k111 = Kp[ty + 1][tx + 1];
      const int cx = tx + 1, cy = ty + 1;
      const Real ksum = ((k000 + k001) + (k010 + k011)) + ((k100 + k101) + (k110 + k111));
      const Real xc = X0[cy][cx];
      Real acc = Real(4) * ksum * xc;
      acc -= (k000 + k100) * X0[cy - 1][cx - 1];
      acc -= (k001 + k101) * X0[cy - 1][cx + 1];
      acc -= (k010 + k110) * X0[cy + 1][cx - 1];
      acc -= (k011 + k111) * X0[cy + 1][cx + 1];
      acc -= (k000 + k010) * Xm[cy][cx - 1];
      acc -= (k001 + k011) * Xm[cy][cx + 1];
      acc -= (k100 + k110) * Xp[cy][cx - 1];
      acc -= (k101 + k111) * Xp[cy][cx + 1];
      acc -= (k000 + k001) * Xm[cy - 1][cx];
      acc -= (k010 + k011) * Xm[cy + 1][cx];
      acc -= (k100 + k101) * Xp[cy - 1][cx];
      acc -= (k110 + k111) * Xp[cy + 1][cx];
      acc -= k000 * Xm[cy - 1][cx - 1];
      acc -= k001 * Xm[cy - 1][cx + 1];
      acc -= k010 * Xm[cy + 1][cx - 1];
      acc -= k011 * Xm[cy + 1][cx + 1];
      acc -= k100 * Xp[cy - 1][cx - 1];
      acc -= k101 * Xp[cy - 1][cx + 1];
      acc -= k110 * Xp[cy + 1][cx - 1];
      acc -= k111 * Xp[cy + 1][cx + 1];
      const int s = k % XS;
      const bool fx = Cf[s][ty][tx];
      const Real xi = Cx[s][ty][tx];  // a fixed row is the identity
      const Real ax = fx ? xi : acc * Real(1.0 / 12.0);
      const Real bi = Cb[s][ty][tx];
      if (MODE == PRE) {
        ((Real*)a.out0)[idx] = xi;
        ((Real*)a.out1)[idx] = bi - ax;
      } else if (MODE == RESID) {
        ((Real*)a.out0)[idx] = bi - ax;
      } else {  // POST, SWEEP
        ((Real*)a.out0)[idx] = xi + om * Cd[s][ty][tx] * (bi - ax);
      }
    }
  }
}

// z runs so that the grid fills the GPU once: resident blocks per SM x SMs,
// split over the column tiles
template <typename Real, int MODE>
int runs_for(const Dims& d, int sms) {
  int per_sm = 0;
  MGAR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fine3d<Real, MODE>, NT, 0));
  per_sm = std::max(per_sm, 1);
  const int64_t cols = (int64_t)((d.NX + TX - 1) / TX) * ((d.NY + TY - 1) / TY);
  const int64_t want = (int64_t)per_sm * sms;
  const int64_t gz = std::max<int64_t>(1, (want + cols / 2) / cols);
  return (int)std::min<int64_t>(gz, d.NZ);
}

}  // namespace f3d

void fine3d_prepare(Ctx& c) {
  using namespace f3d;
  int dev = 0, sms = 0;
  MGAR_CUDA(cudaGetDevice(&dev));
  MGAR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const Dims& d = c.L[0];
  c.f3d_gz[0][PRE] = runs_for<float, PRE>(d, sms);
  c.f3d_gz[0][POST] = runs_for<float, POST>(d, sms);
  c.f3d_gz[0][RESID] = runs_for<float, RESID>(d, sms);
  c.f3d_gz[0][SWEEP] = runs_for<float, SWEEP>(d, sms);
  c.f3d_gz[1][PRE] = runs_for<double, PRE>(d, sms);
  c.f3d_gz[1][POST] = runs_for<double, POST>(d, sms);
  c.f3d_gz[1][RESID] = runs_for<double, RESID>(d, sms);
  c.f3d_gz[1][SWEEP] = runs_for<double, SWEEP>(d, sms);
}

// Launch one tiled finest-level pass (3D only).  mode: 0 pre, 1 post,
// 2 residual, 3 sweep.
template <typename Real>
void fine3d(Ctx& c, int mode, const Real* ke, const Real* b, const Real* dinv, const Real* x,
            const Real* xc, Real* out0, Real* out1) {
  using namespace f3d;
  const Dims& d = c.L[0];
  FineArgs a;
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
  const dim3 block(TX, TY);
  const int gx = (d.NX + TX - 1) / TX, gy = (d.NY + TY - 1) / TY;
  a.gz = std::max(1, std::min(c.f3d_gz[sizeof(Real) == 8][mode & 3], d.NZ));
  const dim3 grid(gx, gy, a.gz);
  switch (mode) {
    case PRE: k_fine3d<Real, PRE><<<grid, block, 0, c.stream>>>(a); break;
    case POST: k_fine3d<Real, POST><<<grid, block, 0, c.stream>>>(a); break;
    case RESID: k_fine3d<Real, RESID><<<grid, block, 0, c.stream>>>(a); break;
    default: k_fine3d<Real, SWEEP><<<grid, block, 0, c.stream>>>(a); break;
  }
  MGAR_LAUNCH_CHECK_AT(level_site(6 + (mode == PRE ? 0 : mode == POST ? 1 : mode == SWEEP ? 2 : 3), 0));
}
template void fine3d<float>(Ctx&, int, const float*, const float*, const float*, const float*,
                            const float*, float*, float*);
template void fine3d<double>(Ctx&, int, const double*, const double*, const double*, const double*,
                             const double*, double*, double*);

}  // namespace mgar
