// Per-node operations of the multigrid levels (Table 1), shared by the
// single-design V-cycle and the batched one: restriction P^T, interpolation
// P, the residual and the fused interpolation + post-smoothing on assembled
// levels, and the coarsest solve by the explicit inverse.
#pragma once
#include "common.cuh"

namespace mgar {

// Loads of data written earlier in the same launch by other thread blocks
// of a cluster go through L2 (CG = true); everything else may use L1.
template <bool CG, typename Real>
__device__ __forceinline__ Real ldv(const Real* p) {
  if (CG) return __ldcg(p);
  return *p;
}

// 1D interpolation taps.  Coarse node I sits at fine node min(2I, nf).
// Restriction (P^T) gathers from fine nodes 2I - 1, 2I, 2I + 1 (weights 1/2,
// 1, 1/2); the last fine node nf of an odd axis is injected (weight 1) into
// the last coarse node.  All three slots are always read: an unused slot
// points at a valid node with weight 0, so the loads need no branches.
__device__ __forceinline__ void restrict_taps(int I, int nf, int* idx, float* w) {
  const int f = 2 * I;
  idx[0] = min(max(f - 1, 0), nf);
  w[0] = (f - 1 >= 1 && f - 1 <= nf) ? ((f - 1 < nf) ? 0.5f : 1.f) : 0.f;
  idx[1] = min(f, nf);
  w[1] = (f <= nf) ? 1.f : 0.f;
  idx[2] = min(f + 1, nf);
  w[2] = (f + 1 < nf) ? 0.5f : 0.f;
}

// Interpolation (P) onto fine node i from coarse nodes.
__device__ __forceinline__ int prolong_taps(int i, int nf, int* idx, float* w) {
  if ((i & 1) == 0) { idx[0] = idx[1] = i >> 1; w[0] = 1.f; w[1] = 0.f; return 1; }
  if (i < nf) { idx[0] = (i - 1) >> 1; w[0] = 0.5f; idx[1] = (i + 1) >> 1; w[1] = 0.5f; return 2; }
  idx[0] = idx[1] = (i + 1) >> 1; w[0] = 1.f; w[1] = 0.f; return 1;
}

// dst = cur + P xc at fine node idx (a fixed fine node keeps cur).
template <typename Real, int DIM>
__device__ __forceinline__ void prolong_node(const Real* __restrict__ xc, const Real* cur, Real* dst,
                                             const Dims& f, const Dims& cd,
                                             const uint8_t* __restrict__ fixed, int idx) {
  if (fixed && fixed[idx]) {
    dst[idx] = cur[idx];
    return;
  }
  int i, j, k;
  coords(idx, f.fNX, f.fNXY, i, j, k);
  int ix[2], iy[2], iz[2] = {0, 0};
  float wx[2], wy[2], wz[2] = {1.f, 0.f};
  prolong_taps(i, f.ex, ix, wx);
  prolong_taps(j, f.ey, iy, wy);
  if (DIM == 3) prolong_taps(k, f.ez, iz, wz);
  Real acc = Real(0);
#pragma unroll
  for (int c = 0; c < (DIM == 3 ? 2 : 1); ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int base = cd.NX * (iy[b] + cd.NY * iz[c]);
      const Real wyz = (Real)(wy[b] * wz[c]);
#pragma unroll
      for (int a = 0; a < 2; ++a)
        if (CK(base + ix[a], cd.n)) acc += (wyz * (Real)wx[a]) * xc[base + ix[a]];
    }
  dst[idx] = cur[idx] + acc;
}

// b_c = P^T r at coarse node idx (fixed fine nodes excluded when given);
// with xc, also the zero-guess smoothing x_c = w D_c^-1 b_c of the coarse
// level, so its first sweep reduces to a residual.  The 3^d fine values are
// loaded before the first product.
template <typename Real, int DIM, bool CG>
__device__ __forceinline__ void restrict_node(const Real* __restrict__ r, Real* __restrict__ bc,
                                              const Dims& f, const Dims& cd,
                                              const uint8_t* __restrict__ fixed, int idx,
                                              const Real* __restrict__ dinvc = nullptr,
                                              Real omega = Real(0), Real* __restrict__ xc = nullptr) {
  constexpr int NZ3 = DIM == 3 ? 3 : 1, NV = 9 * NZ3;
  int I, J, K;
  coords(idx, cd.fNX, cd.fNXY, I, J, K);
  int ix[3], iy[3], iz[3] = {0, 0, 0};
  float wx[3], wy[3], wz[3] = {1.f, 0.f, 0.f};
  restrict_taps(I, f.ex, ix, wx);
  restrict_taps(J, f.ey, iy, wy);
  if (DIM == 3) restrict_taps(K, f.ez, iz, wz);
  Real rv[NV];
  bool fx[NV];
#pragma unroll
  for (int c = 0; c < NZ3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int base = f.NX * (iy[b] + f.NY * iz[c]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int q = a + 3 * b + 9 * c, fi = base + ix[a];
        const bool ok = CK(fi, f.n);
        rv[q] = ok ? ldv<CG>(r + fi) : Real(0);
        fx[q] = ok && fixed ? fixed[fi] != 0 : false;
      }
    }
  Real acc = Real(0);
#pragma unroll
  for (int c = 0; c < NZ3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const Real wyz = (Real)(wy[b] * wz[c]);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int q = a + 3 * b + 9 * c;
        acc += fx[q] ? Real(0) : (wyz * (Real)wx[a]) * rv[q];
      }
    }
  bc[idx] = acc;
  if (xc) xc[idx] = omega * dinvc[idx] * acc;
}

// Residual r = b - A x on an assembled level.  Below the finest level the
// V-cycle's first sweep starts from zero, x = w D^-1 b, and the restriction
// that made b has already written that x, so the sweep and its residual
// reduce to this.
template <typename Real, int DIM, bool CG>
__device__ __forceinline__ void resid_node(const StencilOp<Real>& op, const Real* __restrict__ b,
                                           const Real* __restrict__ x, Real* __restrict__ r, int idx) {
  int i, j, k;
  coords(idx, op.fNX, op.fNXY, i, j, k);
  const Real ax = DIM == 3 ? stencil_row3<Real, CG>(op, x, i, j, k) : stencil_row2<Real, CG>(op, x, i, j);
  r[idx] = ldv<CG>(b + idx) - ax;
}

// Per axis: the coarse nodes c0, c0+1, c0+2 that interpolate onto the fine
// positions f-1, f, f+1 (clamped to 0..nf), and the 3x3 weights w[t][u] of
// coarse node c0+u at fine position f-1+t.
__device__ __forceinline__ void interp_axis(int f, int nf, int& c0, float (&w)[3][3]) {
  int t0[3];
  bool hf[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const int p = min(max(f - 1 + t, 0), nf);
    hf[t] = (p & 1) && p < nf;
    t0[t] = (p & 1) ? (hf[t] ? (p - 1) >> 1 : (p + 1) >> 1) : p >> 1;
  }
  c0 = t0[0];
#pragma unroll
  for (int t = 0; t < 3; ++t)
#pragma unroll
    for (int u = 0; u < 3; ++u)
      w[t][u] = (t0[t] == c0 + u ? (hf[t] ? 0.5f : 1.f) : 0.f) + (hf[t] && t0[t] + 1 == c0 + u ? 0.5f : 0.f);
}

// Fused interpolation and post-smooth on an assembled level:
// v = x + P x_c at the node and its neighbours, x' = v + w D^-1 (b - A v).
// The 3^d coarse values around the node are read once and interpolated
// separably onto the 3^d fine positions.
// PRE: the row's coefficients were gathered already (sv, slot order).
template <typename Real, int DIM, bool CG, bool PRE = false>
__device__ __forceinline__ void post_node(const StencilOp<Real>& op, const Real* __restrict__ xc,
                                          const Real* __restrict__ cur, const Real* __restrict__ b,
                                          const Real* __restrict__ dinv, Real omega,
                                          Real* __restrict__ dst, const Dims& f, const Dims& cd,
                                          int idx, const Real* sv = nullptr) {
  int i, j, k;
  coords(idx, op.fNX, op.fNXY, i, j, k);
  constexpr int NZ3 = DIM == 3 ? 3 : 1;
  int cx0, cy0, cz0 = 0;
  float wx[3][3], wy[3][3], wz[3][3] = {{1.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
  interp_axis(i, f.ex, cx0, wx);
  interp_axis(j, f.ey, cy0, wy);
  if (DIM == 3) interp_axis(k, f.ez, cz0, wz);
  // coarse values C[u][v][w] (z, y, x), clamped: weights of clamped slots are 0
  Real C[NZ3][3][3];
#pragma unroll
  for (int uz = 0; uz < NZ3; ++uz)
#pragma unroll
    for (int uy = 0; uy < 3; ++uy)
#pragma unroll
      for (int ux = 0; ux < 3; ++ux) {
        const int ci = min(cx0 + ux, cd.NX - 1) + cd.NX * (min(cy0 + uy, cd.NY - 1) +
                                                           cd.NY * min(cz0 + uz, cd.NZ - 1));
        C[uz][uy][ux] = CK(ci, cd.n) ? ldv<CG>(xc + ci) : Real(0);
      }
  // along x, then y, then z
  Real T1[NZ3][3][3];
#pragma unroll
  for (int uz = 0; uz < NZ3; ++uz)
#pragma unroll
    for (int uy = 0; uy < 3; ++uy)
#pragma unroll
      for (int tx = 0; tx < 3; ++tx)
        T1[uz][uy][tx] = (Real)wx[tx][0] * C[uz][uy][0] + (Real)wx[tx][1] * C[uz][uy][1] +
                         (Real)wx[tx][2] * C[uz][uy][2];
  Real T2[NZ3][3][3];
#pragma unroll
  for (int uz = 0; uz < NZ3; ++uz)
#pragma unroll
    for (int ty = 0; ty < 3; ++ty)
#pragma unroll
      for (int tx = 0; tx < 3; ++tx)
        T2[uz][ty][tx] = (Real)wy[ty][0] * T1[uz][0][tx] + (Real)wy[ty][1] * T1[uz][1][tx] +
                         (Real)wy[ty][2] * T1[uz][2][tx];
  const int NX = op.NX, NXY = op.NX * op.NY;
  Real acc = Real(0), vc = Real(0);
#pragma unroll
  for (int tz = 0; tz < NZ3; ++tz) {
    const int kk = DIM == 3 ? min(max(k - 1 + tz, 0), op.NZ - 1) : 0;
#pragma unroll
    for (int ty = 0; ty < 3; ++ty) {
      const int jj = min(max(j - 1 + ty, 0), op.NY - 1);
#pragma unroll
      for (int tx = 0; tx < 3; ++tx) {
        const int ii = min(max(i - 1 + tx, 0), op.NX - 1);
        Real pv;
        if (DIM == 3)
          pv = (Real)wz[tz][0] * T2[0][ty][tx] + (Real)wz[tz][1] * T2[NZ3 > 1 ? 1 : 0][ty][tx] +
               (Real)wz[tz][2] * T2[NZ3 > 2 ? 2 : 0][ty][tx];
        else
          pv = T2[0][ty][tx];
        const int nb = ii + NX * jj + NXY * kk;
        if (!CK(nb, op.n)) continue;
        const Real v = ldv<CG>(cur + nb) + pv;
        const int s = tx + 3 * ty + 9 * tz;
        const bool in = ii == i - 1 + tx && jj == j - 1 + ty && (DIM == 2 || kk == k - 1 + tz);
        acc += (PRE ? sv[s] : st_coef<DIM>(op, s, idx, nb, in)) * v;
        if (tx == 1 && ty == 1 && tz == (DIM == 3 ? 1 : 0)) vc = v;
      }
    }
  }
  dst[idx] = vc + omega * dinv[idx] * (ldv<CG>(b + idx) - acc);
}

// x = C b with the explicit inverse of the coarsest operator (FP64 sums).
template <typename Real, bool CG, typename M>
__device__ __forceinline__ void coarse_row(const M* __restrict__ cinv, const Real* __restrict__ b,
                                           Real* __restrict__ x, int n, int row, int lane) {
  M s = M(0);
  for (int j = lane; j < n; j += 32)
    if (CK((int64_t)row * n + j, (int64_t)n * n)) s += cinv[(int64_t)row * n + j] * (M)ldv<CG>(b + j);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = (Real)s;
}

}  // namespace mgar
