// Tiled kernels for the finest 3D (H8) level of the V-cycle.
//
// A block of TX x TY threads owns a TX x TY column of nodes and walks along z
// through a chunk of ZCH node planes.  Three rotating planes of the operand
// (x^ = x with fixed nodes zeroed, zero off the grid) and two rotating layers
// of element conductivities (zero off the grid) sit in shared memory, so the
// 21-point H8 stencil of each node
//   (A x)_i = (4 sum_e k_e x_i - sum_facediag (k_a + k_b) x^_j - sum_bodydiag k_e x^_j) / 12
// is evaluated without bounds tests or per-neighbour mask loads; a fixed row
// is the identity.  Two fused forms cover the V-cycle with a zero initial
// guess (Table 1 with one pre- and one post-sweep):
//   pre:  x = w D^-1 b  and  r = b - A x             (jacobi from zero + residual)
//   post: x' = v + w D^-1 (b - A v),  v = x + P x_c   (interpolation + post-smooth)
// and a generic form computes r = b - A x or one damped-Jacobi sweep.
#include "common.cuh"

namespace mgar {
namespace {

constexpr int TX = 32, TY = 8, ZCH = 16;

// 1D interpolation taps onto fine node i from coarse nodes (unused slot has
// weight 0 and a valid index).
__device__ __forceinline__ void ptaps(int i, int nf, int& i0, int& i1, float& w0, float& w1) {
  if ((i & 1) == 0) {
    i0 = i1 = i >> 1;
    w0 = 1.f;
    w1 = 0.f;
  } else if (i < nf) {
    i0 = (i - 1) >> 1;
    i1 = (i + 1) >> 1;
    w0 = w1 = 0.5f;
  } else {
    i0 = i1 = (i + 1) >> 1;
    w0 = 1.f;
    w1 = 0.f;
  }
}

enum Mode { PRE = 0, POST = 1, RESID = 2, SWEEP = 3 };

struct FineArgs {
  int ex, ey, ez, NX, NY, NZ;
  const uint8_t* fixed;
  const void* ke;
  const void* b;
  const void* dinv;
  const void* x;    // RESID / SWEEP: iterate; POST: x before interpolation
  const void* xc;   // POST: coarse correction
  int cNX, cNY;     // POST: coarse node dims
  void* out0;       // PRE: x, RESID: r, SWEEP/POST: x'
  void* out1;       // PRE: r
  double omega;
};

// operand value at node (i, j, k) before masking
template <typename Real, int MODE>
__device__ __forceinline__ Real operand(const FineArgs& a, int i, int j, int k, int idx) {
  if (MODE == PRE) {
    return (Real)a.omega * ((const Real*)a.dinv)[idx] * ((const Real*)a.b)[idx];
  } else if (MODE == POST) {
    Real v = ((const Real*)a.x)[idx];
    if (!a.fixed[idx]) {
      int x0, x1, y0, y1, z0, z1;
      float wx0, wx1, wy0, wy1, wz0, wz1;
      ptaps(i, a.ex, x0, x1, wx0, wx1);
      ptaps(j, a.ey, y0, y1, wy0, wy1);
      ptaps(k, a.ez, z0, z1, wz0, wz1);
      const Real* xc = (const Real*)a.xc;
      const int P = a.cNX * a.cNY;
      const int zz[2] = {z0 * P, z1 * P};
      const int yy[2] = {y0 * a.cNX, y1 * a.cNX};
      const float wz[2] = {wz0, wz1}, wy[2] = {wy0, wy1};
      Real acc = Real(0);
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const Real wyz = (Real)(wz[c] * wy[b]);
          acc += wyz * ((Real)wx0 * xc[zz[c] + yy[b] + x0] + (Real)wx1 * xc[zz[c] + yy[b] + x1]);
        }
      v += acc;
    }
    return v;
  } else {
    return ((const Real*)a.x)[idx];
  }
}

template <typename Real, int MODE>
__global__ void __launch_bounds__(TX * TY) k_fine3d(FineArgs a) {
  __shared__ Real X[3][TY + 2][TX + 2];
  __shared__ Real K[2][TY + 1][TX + 1];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, kb = blockIdx.z * ZCH;
  const int ke_ = min(kb + ZCH, a.NZ);
  const int i = i0 + tx, j = j0 + ty;
  const bool mine = i < a.NX && j < a.NY;
  const int NXY = a.NX * a.NY;
  const Real* kev = (const Real*)a.ke;

  auto load_plane = [&](int p) {
    const int slot = (p + 3) % 3;
    for (int t = tid; t < (TX + 2) * (TY + 2); t += TX * TY) {
      const int hy = t / (TX + 2), hx = t - hy * (TX + 2);
      const int ii = i0 - 1 + hx, jj = j0 - 1 + hy;
      Real v = Real(0);
      if (ii >= 0 && ii < a.NX && jj >= 0 && jj < a.NY && p >= 0 && p < a.NZ) {
        const int idx = ii + a.NX * jj + NXY * p;
        if (CK(idx, (int64_t)NXY * a.NZ) && !a.fixed[idx]) v = operand<Real, MODE>(a, ii, jj, p, idx);
      }
      X[slot][hy][hx] = v;
    }
  };
  auto load_layer = [&](int l) {
    const int slot = (l + 2) % 2;
    for (int t = tid; t < (TX + 1) * (TY + 1); t += TX * TY) {
      const int hy = t / (TX + 1), hx = t - hy * (TX + 1);
      const int ei = i0 - 1 + hx, ej = j0 - 1 + hy;
      Real v = Real(0);
      if (ei >= 0 && ei < a.ex && ej >= 0 && ej < a.ey && l >= 0 && l < a.ez) {
        const int e = ei + a.ex * (ej + a.ey * l);
        if (CK(e, (int64_t)a.ex * a.ey * a.ez)) v = kev[e];
      }
      K[slot][hy][hx] = v;
    }
  };

  load_plane(kb - 1);
  load_plane(kb);
  load_layer(kb - 1);
  for (int k = kb; k < ke_; ++k) {
    load_plane(k + 1);
    load_layer(k);
    __syncthreads();
    if (mine) {
      const int idx = i + a.NX * j + NXY * k;
      const auto& Xm = X[(k + 2) % 3];
      const auto& X0 = X[k % 3];
      const auto& Xp = X[(k + 1) % 3];
      const auto& Km = K[(k + 1) % 2];
      const auto& Kp = K[k % 2];
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
      Real ax = acc * Real(1.0 / 12.0);
      const bool fx = a.fixed[idx];
      // the centre value unmasked (a fixed row is the identity)
      const Real xi = fx ? operand<Real, MODE>(a, i, j, k, idx) : xc;
      if (fx) ax = xi;
      const Real bi = ((const Real*)a.b)[idx];
      if (MODE == PRE) {
        ((Real*)a.out0)[idx] = xi;
        ((Real*)a.out1)[idx] = bi - ax;
      } else if (MODE == RESID) {
        ((Real*)a.out0)[idx] = bi - ax;
      } else {  // POST, SWEEP
        ((Real*)a.out0)[idx] = xi + (Real)a.omega * ((const Real*)a.dinv)[idx] * (bi - ax);
      }
    }
    __syncthreads();
  }
}

}  // namespace

// Launch one tiled finest-level pass (3D only).  mode: 0 pre, 1 post,
// 2 residual, 3 sweep.
template <typename Real>
void fine3d(Ctx& c, int mode, const Real* ke, const Real* b, const Real* dinv, const Real* x,
            const Real* xc, Real* out0, Real* out1) {
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
  a.out0 = out0;
  a.out1 = out1;
  a.omega = c.p.omega;
  const dim3 block(TX, TY);
  const dim3 grid((d.NX + TX - 1) / TX, (d.NY + TY - 1) / TY, (d.NZ + ZCH - 1) / ZCH);
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
