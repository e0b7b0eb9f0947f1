// Multigrid hierarchy of the reference matrix K0 (Section 2.2, Table 1).
//
// Coarse operators are Galerkin products A_{l+1} = P_l^T A_l P_l with
// P_0 = Z P (no coarse correction reaches a fixed fine node).  They are
// built element by element: every fine element lies inside exactly one
// coarse element, and the interpolation onto its nodes uses only that coarse
// element's nodes, so each coarse element matrix is
//   sum over its sub-elements s of  P_s^T M_s P_s,
// with M_s = k_s Z k0 Z on the finest level and the stored element matrix
// below it.  P_s is the tensor product of 1D 2x2 weights chosen by the
// position of s inside the coarse element (first half, second half, or the
// single fine element of a truncated coarse element on an odd axis).
// Node stencils are then assembled from the element matrices.  The coarsest
// operator is factorised by a banded Cholesky and inverted explicitly, so the
// coarse solve of every V-cycle is one small dense product.
#include "common.cuh"

#include <vector>

namespace mgar {

// 1D interpolation weight of coarse local node c onto fine local node f of a
// sub-element of position type t (0: first half, 1: second half, 2: the
// single fine element of a truncated coarse element).  Values are exact in
// any precision.
__host__ __device__ __forceinline__ float w1(int t, int f, int c) {
  if (t == 0) return f == 0 ? (c == 0 ? 1.f : 0.f) : 0.5f;
  if (t == 1) return f == 1 ? (c == 1 ? 1.f : 0.f) : 0.5f;
  return f == c ? 1.f : 0.f;
}

template <int DIM>
__device__ __forceinline__ float pw(const int (&t)[3], int a, int I) {
  float w = w1(t[0], a & 1, I & 1) * w1(t[1], (a >> 1) & 1, (I >> 1) & 1);
  if (DIM == 3) w *= w1(t[2], (a >> 2) & 1, (I >> 2) & 1);
  return w;
}

// Unit element matrix k0 (Galerkin integral of grad N_a . grad N_b).
static void unit_element(int dim, double* k) {
  const int nen = 1 << dim;
  for (int a = 0; a < nen; ++a)
    for (int b = 0; b < nen; ++b) {
      const int d = __builtin_popcount(a ^ b);
      if (dim == 2) k[a * nen + b] = (d == 0 ? 4.0 : d == 1 ? -1.0 : -2.0) / 6.0;
      else k[a * nen + b] = (d == 0 ? 4.0 : d == 1 ? 0.0 : -1.0) / 12.0;
    }
}

// Sub-element s of coarse element (cx, cy, cz): fine element index, validity
// and 1D position types.
template <int DIM>
__device__ __forceinline__ bool sub_element(const Dims& f, int cx, int cy, int cz, int s, int& e,
                                            int (&t)[3]) {
  const int sx = s & 1, sy = (s >> 1) & 1, sz = (s >> 2) & 1;
  const int fx = 2 * cx + sx, fy = 2 * cy + sy, fz = 2 * cz + sz;
  const bool ok = !(fx >= f.ex || fy >= f.ey || (DIM == 3 && fz >= f.ez));
  e = ok ? fx + f.ex * (fy + f.ey * fz) : 0;  // a valid address either way
  t[0] = (2 * cx + 1 < f.ex) ? sx : 2;
  t[1] = (2 * cy + 1 < f.ey) ? sy : 2;
  t[2] = DIM == 3 ? ((2 * cz + 1 < f.ez) ? sz : 2) : 0;
  return ok;
}

// ------------------------------------------------------------------ kernels
// Level 0 -> 1: element matrices of A_1 from k_e, kGalerkinTPE threads per
// coarse element, each forming every kGalerkinTPE-th group of four entries,
// so the threads of an element store 64 contiguous bytes at a time.
// Sub-elements without fixed nodes use the tables G_type = P_type^T k0 P_type
// (staged in shared memory); a coarse element with any fixed fine node takes
// (Z P)^T k0 (Z P) entry by entry.
constexpr int kGalerkinTPE = 4;

template <typename Real, int DIM>
__global__ void __launch_bounds__(kThreads) k_galerkin_fine(const Real* __restrict__ ke,
                                                             const uint8_t* __restrict__ fixed,
                                                             const uint8_t* __restrict__ efix, Dims f,
                                                             Dims cd, const Real* __restrict__ G,
                                                             const double* __restrict__ k0,
                                                             Real* __restrict__ elem) {
  constexpr int nen = 1 << DIM;
  constexpr int NN = nen * nen;
  constexpr int NT = DIM == 2 ? 9 : 27;
  constexpr int GS = NN + 1;  // padded row: the types of a warp fall in distinct banks
  __shared__ Real Gs[NT * GS];
  for (int u = threadIdx.x; u < NT * NN; u += blockDim.x) Gs[(u / NN) * GS + (u % NN)] = G[u];
  __syncthreads();
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t E = gt / kGalerkinTPE;
  const int part = (int)(gt - E * kGalerkinTPE);
  if (E >= cd.ne) return;
  int cx, cy, cz;
  coords((int)E, cd.fEX, cd.fEXY, cx, cy, cz);
  Real kv[nen];
  int ty[nen];
  int any_fixed = 0;
#pragma unroll
  for (int s = 0; s < nen; ++s) {
    int e = 0, t[3] = {0, 0, 0};
    const bool ok = sub_element<DIM>(f, cx, cy, cz, s, e, t) && CK(e, f.ne);
    kv[s] = ok ? ke[e] : Real(0);
    ty[s] = (t[0] + 3 * t[1] + 9 * t[2]) * GS;
    any_fixed |= ok ? efix[e] : 0;
  }
  Real* dst = elem + E * NN;
  if (!any_fixed) {  // (the others are written by k_galerkin_fixed)
    // A_E = sum_s k_s G_type(s), four entries per store
#pragma unroll
    for (int q = 4 * part; q < NN; q += 4 * kGalerkinTPE) {
      Real a0 = Real(0), a1 = Real(0), a2 = Real(0), a3 = Real(0);
#pragma unroll
      for (int s = 0; s < nen; ++s) {
        const Real* g = Gs + ty[s] + q;
        a0 += kv[s] * g[0];
        a1 += kv[s] * g[1];
        a2 += kv[s] * g[2];
        a3 += kv[s] * g[3];
      }
      if (sizeof(Real) == 4) {
        *reinterpret_cast<float4*>(dst + q) = make_float4((float)a0, (float)a1, (float)a2, (float)a3);
      } else {
        dst[q] = a0;
        dst[q + 1] = a1;
        dst[q + 2] = a2;
        dst[q + 3] = a3;
      }
    }
  }
}

// Level 0 -> 1 for the coarse elements with a fixed fine node (a short list
// fixed at creation), one thread per entry: (Z P)^T k0 (Z P) with the rows
// and columns of fixed fine nodes removed.  k0 sits in shared memory in the
// working precision, and each sub-element's double sum is factored as
// sum_b P_bJ (sum_a P_aI k0_ab) over the free fine nodes a, b.
template <typename Real, int DIM>
__global__ void k_galerkin_fixed(const Real* __restrict__ ke, const uint8_t* __restrict__ fixed,
                                 const int* __restrict__ list, int nlist, Dims f, Dims cd,
                                 const double* __restrict__ k0, Real* __restrict__ elem) {
  constexpr int nen = 1 << DIM;
  constexpr int NN = nen * nen;
  __shared__ Real k0s[NN];
  for (int u = threadIdx.x; u < NN; u += blockDim.x) k0s[u] = (Real)k0[u];
  __syncthreads();
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= (int64_t)nlist * NN) return;
  const int li = (int)(tid / NN);
  const int IJ = (int)(tid - (int64_t)li * NN);
  const int E = list[li];
  if (!CK(E, cd.ne)) return;
  const int I = IJ / nen, J = IJ - (IJ / nen) * nen;
  int cx, cy, cz;
  coords(E, cd.fEX, cd.fEXY, cx, cy, cz);
  Real acc = Real(0);
  for (int s = 0; s < nen; ++s) {
    int e, t[3];
    if (!sub_element<DIM>(f, cx, cy, cz, s, e, t) || !CK(e, f.ne)) continue;
    const int fx = 2 * cx + (s & 1), fy = 2 * cy + ((s >> 1) & 1), fz = 2 * cz + ((s >> 2) & 1);
    unsigned fm = 0;
#pragma unroll
    for (int a = 0; a < nen; ++a) {
      const int nd = (fx + (a & 1)) + f.NX * ((fy + ((a >> 1) & 1)) + f.NY * (fz + ((a >> 2) & 1)));
      if (CK(nd, f.n) && fixed[nd]) fm |= 1u << a;
    }
    Real u[nen];
#pragma unroll
    for (int b = 0; b < nen; ++b) u[b] = Real(0);
#pragma unroll
    for (int a = 0; a < nen; ++a) {
      const Real pa = (fm & (1u << a)) ? Real(0) : (Real)pw<DIM>(t, a, I);
#pragma unroll
      for (int b = 0; b < nen; ++b) u[b] += pa * k0s[a * nen + b];
    }
    Real part = Real(0);
#pragma unroll
    for (int b = 0; b < nen; ++b)
      if (!(fm & (1u << b))) part += (Real)pw<DIM>(t, b, J) * u[b];
    acc += ke[e] * part;
  }
  elem[(int64_t)E * NN + IJ] = acc;
}

// Level l -> l+1 (l >= 1) from stored element matrices:
//   A_E = sum_s P_s^T M_s P_s
// over the sub-elements s of coarse element E.  A block takes 256 / 2^(2d) coarse
// elements, stages their sub-element matrices in shared memory, forms
// T_s = M_s P_s (each thread one entry of every T_s) and then
// A_E[I, J] = sum_s sum_a P_s[a, I] T_s[a, J], with P_s read from the
// per-type interpolation tables.

template <typename Real, int DIM>
__global__ void __launch_bounds__(kThreads) k_galerkin_coarse(const Real* __restrict__ elem_f, Dims f,
                                                               Dims cd, const Real* __restrict__ Ptab,
                                                               Real* __restrict__ elem_c) {
  constexpr int nen = 1 << DIM;
  constexpr int NN = nen * nen;
  constexpr int EPB = kThreads / NN;
  constexpr int NT = DIM == 2 ? 9 : 27;
  __shared__ Real M[EPB][nen][NN];
  __shared__ Real T[EPB][nen][NN];
  __shared__ Real Ps[NT * NN];
  for (int u = threadIdx.x; u < NT * NN; u += blockDim.x) Ps[u] = Ptab[u];
  const int le = threadIdx.x / NN;
  const int IJ = threadIdx.x - le * NN;
  const int I = IJ / nen, J = IJ - (IJ / nen) * nen;
  const int64_t E = (int64_t)blockIdx.x * EPB + le;
  const bool valid = E < cd.ne;
  int cx = 0, cy = 0, cz = 0;
  if (valid) coords((int)E, cd.fEX, cd.fEXY, cx, cy, cz);
  int ty[nen];
#pragma unroll
  for (int s = 0; s < nen; ++s) {
    // sub_element sets e and t on every call, also for the padding threads
    // past the last coarse element (cx = cy = cz = 0 there)
    int e = 0, t[3] = {0, 0, 0};
    const bool in = sub_element<DIM>(f, cx, cy, cz, s, e, t);
    const bool ok = valid && in && CK((int64_t)e * NN + IJ, f.ne * NN);
    ty[s] = t[0] + 3 * t[1] + 9 * t[2];
    M[le][s][IJ] = ok ? elem_f[(int64_t)e * NN + IJ] : Real(0);
  }
  __syncthreads();
  // T_s[I][J] = sum_b M_s[I][b] P_s[b][J]
#pragma unroll
  for (int s = 0; s < nen; ++s) {
    const Real* P = Ps + ty[s] * NN;
    Real acc = Real(0);
#pragma unroll
    for (int b = 0; b < nen; ++b) acc += M[le][s][I * nen + b] * P[b * nen + J];
    T[le][s][IJ] = acc;
  }
  __syncthreads();
  // A[I][J] = sum_s sum_a P_s[a][I] T_s[a][J]
  Real acc = Real(0);
#pragma unroll
  for (int s = 0; s < nen; ++s) {
    const Real* P = Ps + ty[s] * NN;
#pragma unroll
    for (int a = 0; a < nen; ++a) acc += P[a * nen + I] * T[le][s][a * nen + J];
  }
  if (valid) elem_c[E * NN + IJ] = acc;
}

// Node stencils and inverse diagonal of a level from its element matrices.
template <typename Real, int DIM>
__global__ void k_assemble(const Real* __restrict__ elem, Dims d, Real* __restrict__ st,
                           Real* __restrict__ dinv) {
  constexpr int nen = 1 << DIM;
  constexpr int S = DIM == 2 ? 9 : 27;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int)d.n) return;
  int i, j, k;
  coords(idx, d.fNX, d.fNXY, i, j, k);
  Real acc[S];
#pragma unroll
  for (int s = 0; s < S; ++s) acc[s] = Real(0);
#pragma unroll
  for (int o = 0; o < nen; ++o) {
    const int ox = -(o & 1), oy = -((o >> 1) & 1), oz = DIM == 3 ? -((o >> 2) & 1) : 0;
    const int exi = i + ox, eyi = j + oy, ezi = k + oz;
    const bool ok = !(exi < 0 || exi >= d.ex || eyi < 0 || eyi >= d.ey) &&
                    !(DIM == 3 && (ezi < 0 || ezi >= d.ez));
    const int e = ok ? exi + d.ex * (eyi + d.ey * ezi) : 0;  // valid address either way
    if (!ok || !CK(e, d.ne)) continue;
    const int Iloc = o;  // node position inside the element equals -offset
    // the row: nen consecutive entries at a multiple of nen (16-byte loads
    // for FP32; the element matrices are 256-byte aligned allocations)
    Real row[nen];
    const Real* src = elem + (size_t)e * nen * nen + Iloc * nen;
    if (sizeof(Real) == 4) {
#pragma unroll
      for (int J = 0; J < nen; J += 4) {
        const float4 v = *reinterpret_cast<const float4*>(src + J);
        row[J] = (Real)v.x;
        row[J + 1] = (Real)v.y;
        row[J + 2] = (Real)v.z;
        row[J + 3] = (Real)v.w;
      }
    } else {
#pragma unroll
      for (int J = 0; J < nen; ++J) row[J] = src[J];
    }
#pragma unroll
    for (int J = 0; J < nen; ++J) {
      const int dx = (J & 1) + ox, dy = ((J >> 1) & 1) + oy;
      const int dz = DIM == 3 ? ((J >> 2) & 1) + oz : 0;
      const int s = (dx + 1) + 3 * (dy + 1) + (DIM == 3 ? 9 * (dz + 1) : 0);
      acc[s] += row[J];
    }
  }
  // the upper half with the centre (the operator is symmetric)
#pragma unroll
  for (int s = S / 2; s < S; ++s) st[(s - S / 2) * (int)d.n + idx] = acc[s];
  dinv[idx] = Real(1) / acc[S / 2];
}

// Inverse diagonal of the matrix-free finest operator (1 on fixed nodes).
template <typename Real, int DIM>
__global__ void k_fine_dinv(const Real* __restrict__ ke, const uint8_t* __restrict__ fixed, Dims d,
                            Real* __restrict__ dinv) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int)d.n) return;
  if (fixed[idx]) {
    dinv[idx] = Real(1);
    return;
  }
  int i, j, k;
  coords(idx, d.fNX, d.fNXY, i, j, k);
  Real ks = Real(0);
  constexpr int nen = 1 << DIM;
#pragma unroll
  for (int o = 0; o < nen; ++o) {
    const int exi = i - (o & 1), eyi = j - ((o >> 1) & 1), ezi = DIM == 3 ? k - ((o >> 2) & 1) : 0;
    const bool ok = !(exi < 0 || exi >= d.ex || eyi < 0 || eyi >= d.ey) &&
                    !(DIM == 3 && (ezi < 0 || ezi >= d.ez));
    const int e = ok ? exi + d.ex * (eyi + d.ey * ezi) : 0;  // valid address either way
    const Real kv = CK(e, d.ne) ? ke[e] : Real(0);
    if (ok) ks += kv;
  }
  dinv[idx] = Real(1) / (ks * Real(DIM == 2 ? 4.0 / 6.0 : 4.0 / 12.0));
}

// Lower band of the coarsest operator: band[i*(bw+1) + (j - i + bw)].
template <typename Real, int DIM, typename B>
__global__ void k_band_fill(const Real* __restrict__ st, Dims d, int bw, B* __restrict__ band) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int)d.n) return;
  int i, j, k;
  coords(idx, d.fNX, d.fNXY, i, j, k);
  const int S = DIM == 2 ? 9 : 27;
  for (int s = 0; s < S; ++s) {
    const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = DIM == 3 ? s / 9 - 1 : 0;
    const int ii = i + dx, jj = j + dy, kk = k + dz;
    if (ii < 0 || ii >= d.NX || jj < 0 || jj >= d.NY || kk < 0 || kk >= d.NZ) continue;
    const int col = ii + d.NX * (jj + d.NY * kk);  // no load depends on it before the check
    if (col > idx) continue;
    // col <= idx: the centre, or a lower slot held by the neighbour col as
    // its mirror (upper) slot S - 1 - s
    const int64_t at = s == S / 2 ? (int64_t)idx : (int64_t)(S / 2 - s) * d.n + col;
    if (CK((int64_t)idx * (bw + 1) + (col - idx + bw), d.n * (bw + 1)) && CK(col - idx + bw, bw + 1))
      band[(int64_t)idx * (bw + 1) + (col - idx + bw)] = (B)st[at];
  }
}

// Right-looking banded Cholesky in one block of kCholThreads threads, on a
// shared-memory copy of the band when it fits (SMEM) or in place in global
// memory.  Step k: the pivot (reciprocal square root), the scaled column k
// below it, then the rank-1 update of the trailing band triangle, one row
// per warp and one column per lane.  Stores the factor and the reciprocals
// of its diagonal (rdiag).
constexpr int kCholThreads = 1024;  // FP64 latency needs many warps in flight

template <typename B, bool SMEM>
__global__ void __launch_bounds__(kCholThreads) k_band_cholesky(B* __restrict__ gband,
                                                                B* __restrict__ rdiag, int n, int bw,
                                                                int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  B* sband = reinterpret_cast<B*>(smraw);
  __shared__ B rpiv;
  __shared__ int bad;
  const int ld = bw + 1;
  const int64_t size = (int64_t)n * ld;
  B* band = SMEM ? sband : gband;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  if (SMEM)
    for (int64_t t = tid; t < size; t += blockDim.x) band[t] = gband[t];
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const B a = band[(int64_t)k * ld + bw];
      if (!(a > B(0)) || !isfinite(a)) bad = 1;
      const B r = rsqrt_nr(a);
      rpiv = r;
      band[(int64_t)k * ld + bw] = a * r;  // sqrt(a)
      rdiag[k] = r;
    }
    __syncthreads();
    if (bad) break;
    const int last = min(k + bw, n - 1);
    const int m = last - k;
    const B rp = rpiv;
    for (int t = tid; t < m; t += blockDim.x) {
      const int64_t at = (int64_t)(k + 1 + t) * ld + (bw - 1 - t);  // L(k+1+t, k)
      if (CK(at, size)) band[at] *= rp;
    }
    __syncthreads();
    // A(i, j) -= L(i, k) L(j, k) for k < j <= i <= last
    for (int ii = warp; ii < m; ii += nw) {
      const int i = k + 1 + ii;
      const B lik = band[(int64_t)i * ld + (k - i + bw)];
      for (int jj = lane; jj <= ii; jj += 32) {
        const int j = k + 1 + jj;
        const int64_t at = (int64_t)i * ld + (j - i + bw);
        const int64_t bt = (int64_t)j * ld + (k - j + bw);
        if (CK(at, size) && CK(bt, size)) band[at] -= lik * band[bt];
      }
    }
    __syncthreads();
  }
  if (SMEM)
    for (int64_t t = tid; t < size; t += blockDim.x) gband[t] = band[t];
  if (tid == 0 && bad) *err = MGAR_ERR_NOT_SPD;
}

// Columns of the inverse, one warp per column, by forward then backward
// substitution with the band factor in column-oriented form: once x_p is
// known, each lane removes its term from one of the next bw right-hand
// sides (no reductions on the critical path).  With SMEM the band is staged
// in shared memory once per block and each warp keeps its column there.
template <typename B, bool SMEM>
__global__ void k_band_inverse(const B* __restrict__ gband, const B* __restrict__ rdiag, int n, int bw,
                               B* inv) {
  extern __shared__ __align__(16) unsigned char smraw[];
  B* sband = reinterpret_cast<B*>(smraw);
  const int ld = bw + 1;
  const int64_t size = (int64_t)n * ld;
  const int warps = blockDim.x >> 5;
  const int wid = threadIdx.x >> 5;
  const B* band = gband;
  B* colbuf = nullptr;
  if (SMEM) {
    for (int64_t t = threadIdx.x; t < size; t += blockDim.x) sband[t] = gband[t];
    __syncthreads();
    band = sband;
    colbuf = sband + size + (int64_t)wid * n;
  }
  const int col = blockIdx.x * warps + wid;
  const int lane = threadIdx.x & 31;
  if (col >= n) return;
  // column values live in colbuf (shared) or in inv itself (global)
  auto cv = [&](int i) -> B& { return SMEM ? colbuf[i] : inv[(int64_t)i * n + col]; };
  for (int i = lane; i < n; i += 32) cv(i) = (i == col) ? B(1) : B(0);
  __syncwarp();
  // forward: L y = e_col (y_p = 0 for p < col)
  for (int p = col; p < n; ++p) {
    const B yp = cv(p) * rdiag[p];
    __syncwarp();
    if (lane == 0) cv(p) = yp;
    const int last = min(n - 1, p + bw);
    for (int i = p + 1 + lane; i <= last; i += 32) {
      const int64_t at = (int64_t)i * ld + (p - i + bw);  // L(i, p)
      if (CK(at, size)) cv(i) -= band[at] * yp;
    }
    __syncwarp();
  }
  // backward: L^T x = y
  for (int i = n - 1; i >= 0; --i) {
    const B xi = cv(i) * rdiag[i];
    __syncwarp();
    if (lane == 0) cv(i) = xi;
    const int first = max(0, i - bw);
    for (int p = first + lane; p < i; p += 32) {
      const int64_t at = (int64_t)i * ld + (p - i + bw);  // L(i, p)
      if (CK(at, size)) cv(p) -= band[at] * xi;
    }
    __syncwarp();
  }
  if (SMEM)
    for (int i = lane; i < n; i += 32) inv[(int64_t)i * n + col] = colbuf[i];
}

// The same factorisation and inverse in double-float arithmetic (df64: two
// FP32 words, ~48 bits) on the FP32 pipe, for the FP32 V-cycle.  GB300 runs
// FP64 at 1/58 of the FP32 rate, and the chain of 125 dependent pivots is
// bound by that rate; a df64 operation costs a handful of FP32 operations.
// The band arrives in FP64 (gband), is factorised in shared memory, and the
// factor (band, rdiag) is stored as df64 pairs in the same buffers; the
// inverse is written in FP64.
__device__ __forceinline__ df df_ld(const float2* p) {
  const float2 v = *p;
  return df{v.x, v.y};
}
__device__ __forceinline__ void df_st(float2* p, df v) { *p = make_float2(v.hi, v.lo); }

__global__ void __launch_bounds__(kCholThreads) k_band_cholesky_df(double* __restrict__ gband,
                                                                   double* __restrict__ grdiag,
                                                                   int n, int bw,
                                                                   int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* band = reinterpret_cast<float2*>(smraw);
  float2* out = reinterpret_cast<float2*>(gband);  // same bytes, df64 pairs
  float2* rdiag = reinterpret_cast<float2*>(grdiag);
  __shared__ float2 rpiv;
  __shared__ int bad;
  const int ld = bw + 1;
  const int64_t size = (int64_t)n * ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int64_t t = tid; t < size; t += blockDim.x) {
    const df v = df_from_double(gband[t]);
    band[t] = make_float2(v.hi, v.lo);
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      const df a = df_ld(band + (int64_t)k * ld + bw);
      if (!(a.hi > 0.f) || !isfinite(a.hi)) bad = 1;
      const df r = df_rsqrt(a);
      rpiv = make_float2(r.hi, r.lo);
      df_st(band + (int64_t)k * ld + bw, df_mul(a, r));  // sqrt(a)
      df_st(rdiag + k, r);
    }
    __syncthreads();
    if (bad) break;
    const int last = min(k + bw, n - 1);
    const int m = last - k;
    const df rp{rpiv.x, rpiv.y};
    for (int t = tid; t < m; t += blockDim.x) {
      const int64_t at = (int64_t)(k + 1 + t) * ld + (bw - 1 - t);  // L(k+1+t, k)
      if (CK(at, size)) df_st(band + at, df_mul(df_ld(band + at), rp));
    }
    __syncthreads();
    // A(i, j) -= L(i, k) L(j, k) for k < j <= i <= last
    for (int ii = warp; ii < m; ii += nw) {
      const int i = k + 1 + ii;
      const df lik = df_ld(band + (int64_t)i * ld + (k - i + bw));
      for (int jj = lane; jj <= ii; jj += 32) {
        const int j = k + 1 + jj;
        const int64_t at = (int64_t)i * ld + (j - i + bw);
        const int64_t bt = (int64_t)j * ld + (k - j + bw);
        if (CK(at, size) && CK(bt, size))
          df_st(band + at, df_sub(df_ld(band + at), df_mul(lik, df_ld(band + bt))));
      }
    }
    __syncthreads();
  }
  for (int64_t t = tid; t < size; t += blockDim.x) out[t] = band[t];
  if (tid == 0 && bad) *err = MGAR_ERR_NOT_SPD;
}

// Columns of the inverse from the df64 factor, one warp per column, as
// k_band_inverse does in FP64; the result is written in FP64.
__global__ void k_band_inverse_df(const double* __restrict__ gband_d,
                                  const double* __restrict__ grdiag_d, int n, int bw,
                                  double* __restrict__ inv) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const float2* gband = reinterpret_cast<const float2*>(gband_d);
  const float2* rdiag = reinterpret_cast<const float2*>(grdiag_d);
  float2* sband = reinterpret_cast<float2*>(smraw);
  const int ld = bw + 1;
  const int64_t size = (int64_t)n * ld;
  const int warps = blockDim.x >> 5;
  const int wid = threadIdx.x >> 5;
  for (int64_t t = threadIdx.x; t < size; t += blockDim.x) sband[t] = gband[t];
  __syncthreads();
  float2* colbuf = sband + size + (int64_t)wid * n;
  const int col = blockIdx.x * warps + wid;
  const int lane = threadIdx.x & 31;
  if (col >= n) return;
  for (int i = lane; i < n; i += 32) colbuf[i] = make_float2(i == col ? 1.f : 0.f, 0.f);
  __syncwarp();
  // forward: L y = e_col (y_p = 0 for p < col)
  for (int p = col; p < n; ++p) {
    const df yp = df_mul(df_ld(colbuf + p), df_ld(rdiag + p));
    __syncwarp();
    if (lane == 0) df_st(colbuf + p, yp);
    const int last = min(n - 1, p + bw);
    for (int i = p + 1 + lane; i <= last; i += 32) {
      const int64_t at = (int64_t)i * ld + (p - i + bw);  // L(i, p)
      if (CK(at, size)) df_st(colbuf + i, df_sub(df_ld(colbuf + i), df_mul(df_ld(sband + at), yp)));
    }
    __syncwarp();
  }
  // backward: L^T x = y
  for (int i = n - 1; i >= 0; --i) {
    const df xi = df_mul(df_ld(colbuf + i), df_ld(rdiag + i));
    __syncwarp();
    if (lane == 0) df_st(colbuf + i, xi);
    const int first = max(0, i - bw);
    for (int p = first + lane; p < i; p += 32) {
      const int64_t at = (int64_t)i * ld + (p - i + bw);  // L(i, p)
      if (CK(at, size)) df_st(colbuf + p, df_sub(df_ld(colbuf + p), df_mul(df_ld(sband + at), xi)));
    }
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) inv[(int64_t)i * n + col] = df_to_double(df_ld(colbuf + i));
}

// Band widths below one warp (every coarsest level the V-cycles build here:
// 5^3 nodes in 3D, up to 17^2 in 2D): the same factorisation and inverse,
// the same df64 operations on every entry in the same order (bit-identical
// results), with shorter dependency chains.
constexpr int kWinBw = 32;

// The pivot of column k: sqrt(A(k,k)) into the band, 1/sqrt into rdiag and
// *rp; *bad set when A(k,k) is not positive.
__device__ __forceinline__ void chol_pivot_df(float2* band, float2* rdiag, int k, int ld, int bw,
                                              float2* rp, int* bad) {
  const df a = df_ld(band + (int64_t)k * ld + bw);
  if (!(a.hi > 0.f) || !isfinite(a.hi)) *bad = 1;
  const df r = df_rsqrt(a);
  *rp = make_float2(r.hi, r.lo);
  df_st(band + (int64_t)k * ld + bw, df_mul(a, r));
  df_st(rdiag + k, r);
}

// Right-looking band Cholesky for bw < 32, one barrier per column: warp w
// takes row i = k+1+w of column k's rank-1 update (lane l the entry j =
// k+1+l <= i), scaling A(i,k) and A(j,k) by the pivot as it reads them; the
// scaled column is stored after the barrier, when no thread reads the
// unscaled one any more.  The first lane of warp 0, which updates A(k+1,k+1),
// computes the next pivot at once (double-buffered pivot and flag), so the
// pivot's rsqrt chain overlaps the other rows' updates.
__global__ void __launch_bounds__(kCholThreads) k_band_cholesky_df_win(double* __restrict__ gband,
                                                                       double* __restrict__ grdiag,
                                                                       int n, int bw,
                                                                       int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* band = reinterpret_cast<float2*>(smraw);
  float2* out = reinterpret_cast<float2*>(gband);  // same bytes, df64 pairs
  float2* rdiag = reinterpret_cast<float2*>(grdiag);
  __shared__ float2 rpiv[2];
  __shared__ int bad[2];
  const int ld = bw + 1;
  const int64_t size = (int64_t)n * ld;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int64_t t = tid; t < size; t += blockDim.x) {
    const df v = df_from_double(gband[t]);
    band[t] = make_float2(v.hi, v.lo);
  }
  if (tid == 0) bad[0] = bad[1] = 0;
  __syncthreads();
  if (tid == 0) chol_pivot_df(band, rdiag, 0, ld, bw, &rpiv[0], &bad[0]);
  __syncthreads();
  df lprev{0.f, 0.f};  // lane 0 of warp w: L(i, k-1) of its row in the last column
  int64_t aprev = -1;
  for (int k = 0; k < n; ++k) {
    if (bad[k & 1]) break;
    const df rp{rpiv[k & 1].x, rpiv[k & 1].y};
    if (aprev >= 0) {
      df_st(band + aprev, lprev);
      aprev = -1;
    }
    const int m = min(k + bw, n - 1) - k;
    if (warp < m) {
      const int i = k + 1 + warp;
      const int64_t ai = (int64_t)i * ld + (k - i + bw);  // A(i, k)
      const df lik = df_mul(df_ld(band + ai), rp);
      if (lane <= warp) {
        const int j = k + 1 + lane;
        const int64_t at = (int64_t)i * ld + (j - i + bw);
        const df ljk = df_mul(df_ld(band + (int64_t)j * ld + (k - j + bw)), rp);
        df_st(band + at, df_sub(df_ld(band + at), df_mul(lik, ljk)));
      }
      if (lane == 0) {
        lprev = lik;
        aprev = ai;
        if (warp == 0)
          chol_pivot_df(band, rdiag, k + 1, ld, bw, &rpiv[(k + 1) & 1], &bad[(k + 1) & 1]);
      }
    }
    __syncthreads();
  }
  if (aprev >= 0) df_st(band + aprev, lprev);
  __syncthreads();
  for (int64_t t = tid; t < size; t += blockDim.x) out[t] = band[t];
  if (tid == 0 && (bad[0] || bad[1])) *err = MGAR_ERR_NOT_SPD;
}

// Columns of the inverse for bw < 32, one warp per column, the unknowns of
// the substitutions in registers: lane l holds the row r = l (mod 32) of the
// bw + 1 rows the current step touches, receives the step's solved value by
// shuffle and takes row r + 32 (forward) or r - 32 (backward) once its own
// row is solved, so no step waits on shared memory.  The band and the
// reciprocal pivots are staged in shared memory; a step's coefficient and
// pivot loads do not depend on the chain, and the solved value is stored
// after it has been passed on.
__global__ void k_band_inverse_df_win(const double* __restrict__ gband_d,
                                      const double* __restrict__ grdiag_d, int n, int bw,
                                      double* __restrict__ inv) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const float2* gband = reinterpret_cast<const float2*>(gband_d);
  const float2* grdiag = reinterpret_cast<const float2*>(grdiag_d);
  float2* sband = reinterpret_cast<float2*>(smraw);
  const int ld = bw + 1;
  const int64_t size = (int64_t)n * ld;
  float2* srdiag = sband + size;
  const int warps = blockDim.x >> 5;
  const int wid = threadIdx.x >> 5;
  for (int64_t t = threadIdx.x; t < size; t += blockDim.x) sband[t] = gband[t];
  for (int t = threadIdx.x; t < n; t += blockDim.x) srdiag[t] = grdiag[t];
  __syncthreads();
  float2* colbuf = srdiag + n + (int64_t)wid * n;  // the forward solution y
  const int col = blockIdx.x * warps + wid;
  const int lane = threadIdx.x & 31;
  if (col >= n) return;
  for (int i = lane; i < col; i += 32) colbuf[i] = make_float2(0.f, 0.f);
  // forward: L y = e_col (y_p = 0 for p < col)
  int r = col + ((lane - col) & 31);
  df y = r == col ? df{1.f, 0.f} : df{0.f, 0.f};
  for (int p = col; p < n; ++p) {
    const int owner = p & 31;
    const bool upd = r > p && r <= p + bw && r < n;
    const df lrp = upd ? df_ld(sband + (int64_t)r * ld + (p - r + bw)) : df{0.f, 0.f};  // L(r, p)
    const df rd = df_ld(srdiag + p);
    df yp = df_mul(y, rd);  // the owner's solved value (others discard theirs)
    yp.hi = __shfl_sync(0xffffffffu, yp.hi, owner);
    yp.lo = __shfl_sync(0xffffffffu, yp.lo, owner);
    if (upd) y = df_sub(y, df_mul(lrp, yp));
    if (lane == owner) {
      df_st(colbuf + p, yp);
      r = p + 32;
      y = df{0.f, 0.f};
    }
  }
  __syncwarp();
  // backward: L^T x = y
  r = (n - 1) - ((n - 1 - lane) & 31);
  y = r >= 0 ? df_ld(colbuf + r) : df{0.f, 0.f};
  for (int i = n - 1; i >= 0; --i) {
    const int owner = i & 31;
    const bool upd = r >= 0 && r < i && r >= i - bw;
    const df lir = upd ? df_ld(sband + (int64_t)i * ld + (r - i + bw)) : df{0.f, 0.f};  // L(i, r)
    const df rd = df_ld(srdiag + i);
    df xi = df_mul(y, rd);
    xi.hi = __shfl_sync(0xffffffffu, xi.hi, owner);
    xi.lo = __shfl_sync(0xffffffffu, xi.lo, owner);
    if (upd) y = df_sub(y, df_mul(lir, xi));
    if (lane == owner) {
      inv[(int64_t)i * n + col] = df_to_double(xi);
      r = i - 32;
      y = r >= 0 ? df_ld(colbuf + r) : df{0.f, 0.f};
    }
  }
}

__global__ void k_d2f(const double* a, float* b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// ------------------------------------------------------------------- host
template <typename Real>
static void alloc_levels(Ctx& c, LevelBuf<Real>* h) {
  const int nen = c.nen;
  for (int l = 0; l < c.nl; ++l) {
    const Dims& d = c.L[l];
    MGAR_CUDA(cudaMalloc(&h[l].dinv, d.n * sizeof(Real)));
    MGAR_CUDA(cudaMalloc(&h[l].t, d.n * sizeof(Real)));
    MGAR_CUDA(cudaMalloc(&h[l].r, d.n * sizeof(Real)));
    if (l >= 1) {
      MGAR_CUDA(cudaMalloc(&h[l].st, (size_t)stencil_slots(c.dim) * d.n * sizeof(Real)));
      MGAR_CUDA(cudaMalloc(&h[l].elem, (size_t)d.ne * nen * nen * sizeof(Real)));
      MGAR_CUDA(cudaMalloc(&h[l].x, d.n * sizeof(Real)));
      MGAR_CUDA(cudaMalloc(&h[l].b, d.n * sizeof(Real)));
    }
  }
}

template <typename Real>
static void free_levels(LevelBuf<Real>* h) {
  for (int l = 0; l < kMaxLevels; ++l) {
    cudaFree(h[l].dinv);
    cudaFree(h[l].t);
    cudaFree(h[l].r);
    cudaFree(h[l].st);
    cudaFree(h[l].elem);
    cudaFree(h[l].x);
    cudaFree(h[l].b);
    h[l] = LevelBuf<Real>{};
  }
}

void alloc_hierarchy(Ctx& c) {
  if (c.p.precision == MGAR_FP64) alloc_levels(c, c.h64);
  else alloc_levels(c, c.h32);
  const Dims& dc = c.L[c.nl - 1];
  c.nc = (int)dc.n;
  c.bw = (c.dim == 2) ? dc.NX + 1 : dc.NX * dc.NY + dc.NX + 1;
  if (c.bw > c.nc - 1) c.bw = c.nc - 1 > 0 ? c.nc - 1 : 0;
  MGAR_CUDA(cudaMalloc(&c.band, (size_t)c.nc * (c.bw + 1) * sizeof(double)));
  MGAR_CUDA(cudaMalloc(&c.rdiag, (size_t)c.nc * sizeof(double)));
  MGAR_CUDA(cudaMalloc(&c.cinv, (size_t)c.nc * c.nc * sizeof(double)));
  MGAR_CUDA(cudaFuncSetAttribute(k_band_cholesky<double, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
  MGAR_CUDA(cudaFuncSetAttribute(k_band_inverse<double, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
  MGAR_CUDA(cudaFuncSetAttribute(k_band_cholesky<float, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
  MGAR_CUDA(cudaFuncSetAttribute(k_band_inverse<float, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBandSmemMax));
  MGAR_CUDA(cudaFuncSetAttribute(k_band_cholesky_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kBandSmemMax));
  MGAR_CUDA(cudaFuncSetAttribute(k_band_inverse_df, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kBandSmemMax));
  MGAR_CUDA(cudaFuncSetAttribute(k_band_cholesky_df_win, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kBandSmemMax));
  MGAR_CUDA(cudaFuncSetAttribute(k_band_inverse_df_win, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kBandSmemMax));
  // constant tables: k0 (nen^2) then G (3^dim * nen^2)
  const int nen = c.nen, ntypes = c.dim == 2 ? 9 : 27;
  std::vector<double> k0(nen * nen), G((size_t)ntypes * nen * nen, 0.0),
      Pt((size_t)ntypes * nen * nen, 0.0);
  unit_element(c.dim, k0.data());
  for (int type = 0; type < ntypes; ++type) {
    const int t[3] = {type % 3, (type / 3) % 3, type / 9};
    std::vector<double> P(nen * nen);
    for (int a = 0; a < nen; ++a)
      for (int I = 0; I < nen; ++I) {
        double w = w1(t[0], a & 1, I & 1) * w1(t[1], (a >> 1) & 1, (I >> 1) & 1);
        if (c.dim == 3) w *= w1(t[2], (a >> 2) & 1, (I >> 2) & 1);
        P[a * nen + I] = w;
        Pt[(size_t)type * nen * nen + a * nen + I] = w;
      }
    for (int I = 0; I < nen; ++I)
      for (int J = 0; J < nen; ++J) {
        double s = 0.0;
        for (int a = 0; a < nen; ++a)
          for (int b = 0; b < nen; ++b) s += P[a * nen + I] * k0[a * nen + b] * P[b * nen + J];
        G[(size_t)type * nen * nen + I * nen + J] = s;
      }
  }
  // device layout: k0 | G | P (FP64), G | P (FP32)
  std::vector<double> all(k0);
  all.insert(all.end(), G.begin(), G.end());
  all.insert(all.end(), Pt.begin(), Pt.end());
  MGAR_CUDA(cudaMalloc(&c.tables, all.size() * sizeof(double)));
  MGAR_CUDA(cudaMemcpy(c.tables, all.data(), all.size() * sizeof(double), cudaMemcpyHostToDevice));
  std::vector<float> allf(all.begin() + k0.size(), all.end());
  MGAR_CUDA(cudaMalloc(&c.tables_f, allf.size() * sizeof(float)));
  MGAR_CUDA(cudaMemcpy(c.tables_f, allf.data(), allf.size() * sizeof(float), cudaMemcpyHostToDevice));
}

void free_hierarchy(Ctx& c) {
  free_levels(c.h64);
  free_levels(c.h32);
  cudaFree(c.band);
  cudaFree(c.rdiag);
  cudaFree(c.cinv);
  cudaFree(c.tables);
  cudaFree(c.tables_f);
  c.tables_f = nullptr;
  c.band = nullptr;
  c.rdiag = nullptr;
  c.cinv = nullptr;
  c.tables = nullptr;
}

template <typename Real>
static const Real* g_tables(Ctx& c);
template <>
const double* g_tables<double>(Ctx& c) { return c.tables + c.nen * c.nen; }
template <>
const float* g_tables<float>(Ctx& c) { return c.tables_f; }
// interpolation tables P_type[a * nen + I], after the G tables
template <typename Real>
static const Real* p_tables(Ctx& c) {
  return g_tables<Real>(c) + (size_t)(c.dim == 2 ? 9 : 27) * c.nen * c.nen;
}

// Band Cholesky of the coarsest operator and its explicit inverse, in B
// (the V-cycle's working precision).  On the side stream when there is one:
// the factorisation is a chain of 125 dependent pivots on one SM, and the
// solve's first kernels (the df64 residual) do not need it; join_coarse
// orders the main stream after it.
template <typename Real, int DIM, typename B>
static void coarse_factor(Ctx& c, const Real* st, const Dims& dcst) {
  cudaStream_t s = c.stream;
  if (c.side_stream) {
    MGAR_CUDA(cudaEventRecord(c.ev_fork, c.stream));
    MGAR_CUDA(cudaStreamWaitEvent(c.side_stream, c.ev_fork, 0));
    s = c.side_stream;
  }
  B* band = CoarseT<Real>::band(c);
  B* rdiag = CoarseT<Real>::rdiag(c);
  B* inv = CoarseT<Real>::inv(c);
  zero_async(band, (int64_t)c.nc * (c.bw + 1), s);
  MGAR_LAUNCH_CHECK();
  k_band_fill<Real, DIM, B><<<blocks_for(dcst.n), kThreads, 0, s>>>(st, dcst, c.bw, band);
  MGAR_LAUNCH_CHECK();
  const size_t band_bytes = (size_t)c.nc * (c.bw + 1) * sizeof(B);
  const bool smem = band_bytes <= kBandSmemMax;
  const size_t inv_smem = band_bytes + (size_t)8 * c.nc * sizeof(B);
  // the FP32 V-cycle's coarsest factor and inverse in df64 on the FP32 pipe
  // (same band bytes: a df64 pair is the size of a double)
  if (sizeof(Real) == 4 && sizeof(B) == 8 && smem && inv_smem <= kBandSmemMax && c.df_coarse) {
    // the windowed inverse also stages the n reciprocal pivots
    const size_t win_smem = inv_smem + (size_t)c.nc * sizeof(B);
    if (c.bw < kWinBw)
      k_band_cholesky_df_win<<<1, 32 * std::max(c.bw, 1), band_bytes, s>>>(
          (double*)band, (double*)rdiag, c.nc, c.bw, c.derr);
    else
      k_band_cholesky_df<<<1, kCholThreads, band_bytes, s>>>((double*)band, (double*)rdiag, c.nc,
                                                             c.bw, c.derr);
    MGAR_LAUNCH_CHECK();
    if (c.bw < kWinBw && win_smem <= kBandSmemMax)
      k_band_inverse_df_win<<<(c.nc + 7) / 8, 256, win_smem, s>>>(
          (const double*)band, (const double*)rdiag, c.nc, c.bw, (double*)inv);
    else
      k_band_inverse_df<<<(c.nc + 7) / 8, 256, inv_smem, s>>>((const double*)band,
                                                             (const double*)rdiag, c.nc, c.bw,
                                                             (double*)inv);
    MGAR_LAUNCH_CHECK();
    if (c.side_stream) {
      MGAR_CUDA(cudaEventRecord(c.ev_join, s));
      c.coarse_pending = true;
      c.derr_fresh = false;
    }
    return;
  }
  if (smem) {
    k_band_cholesky<B, true><<<1, kCholThreads, band_bytes, s>>>(band, rdiag, c.nc, c.bw, c.derr);
  } else {
    k_band_cholesky<B, false><<<1, kCholThreads, 0, s>>>(band, rdiag, c.nc, c.bw, c.derr);
  }
  MGAR_LAUNCH_CHECK();
  MGAR_CUDA(cudaMemsetAsync(inv, 0, (size_t)c.nc * c.nc * sizeof(B), s));
  if (smem && inv_smem <= kBandSmemMax)
    k_band_inverse<B, true><<<(c.nc + 7) / 8, 256, inv_smem, s>>>(band, rdiag, c.nc, c.bw, inv);
  else
    k_band_inverse<B, false><<<(c.nc + 7) / 8, 256, 0, s>>>(band, rdiag, c.nc, c.bw, inv);
  MGAR_LAUNCH_CHECK();
  if (c.side_stream) {
    MGAR_CUDA(cudaEventRecord(c.ev_join, s));
    c.coarse_pending = true;
    c.derr_fresh = false;
  }
}

template <typename Real, int DIM>
static void build_levels(Ctx& c, const Real* ke0, LevelBuf<Real>* h) {
  cudaStream_t s = c.stream;
  const int nen = 1 << DIM;
  const double* k0 = c.tables;
  const Real* G = g_tables<Real>(c);
  k_fine_dinv<Real, DIM><<<blocks_for(c.L[0].n), kThreads, 0, s>>>(ke0, c.fixed, c.L[0], h[0].dinv);
  MGAR_LAUNCH_CHECK();
  for (int l = 0; l + 1 < c.nl; ++l) {
    const Dims& f = c.L[l];
    const Dims& cd = c.L[l + 1];
    ProfScope ps(c, l == 0 ? MGAR_KC_GALERKIN0 : -1);
    const int64_t entries = cd.ne * nen * nen;  // coarse levels: one thread per entry
    if (l == 0) {
      k_galerkin_fine<Real, DIM><<<blocks_for(cd.ne * kGalerkinTPE), kThreads, 0, s>>>(
          ke0, c.fixed, c.efix, f, cd, G, k0, h[1].elem);
      MGAR_LAUNCH_CHECK();
      if (c.n_gfix > 0)
        k_galerkin_fixed<Real, DIM><<<blocks_for((int64_t)c.n_gfix * nen * nen), kThreads, 0, s>>>(
            ke0, c.fixed, c.gfix, c.n_gfix, f, cd, k0, h[1].elem);
    }
    else
      k_galerkin_coarse<Real, DIM><<<blocks_for(entries), kThreads, 0, s>>>(
          h[l].elem, f, cd, p_tables<Real>(c), h[l + 1].elem);
    MGAR_LAUNCH_CHECK();
    k_assemble<Real, DIM><<<blocks_for(cd.n), kThreads, 0, s>>>(h[l + 1].elem, cd, h[l + 1].st,
                                                                 h[l + 1].dinv);
    MGAR_LAUNCH_CHECK();
  }
  const Dims& dcst = c.L[c.nl - 1];
  coarse_factor<Real, DIM, typename CoarseT<Real>::T>(c, h[c.nl - 1].st, dcst);
}

void build_hierarchy(Ctx& c) {
  cudaStream_t s = c.stream;
  if (c.p.precision == MGAR_FP64) {
    // the reference k_e of MGAR's K - K0 (the mixed path keeps only its FP32 copy)
    copy_async((const double*)c.ke, c.ke0, c.ne, s);
    MGAR_LAUNCH_CHECK();
    if (c.dim == 2) build_levels<double, 2>(c, c.ke0, c.h64);
    else build_levels<double, 3>(c, c.ke0, c.h64);
  } else {
    // the FP32 copy of k_e is already fl32(k_e) (set_density writes both)
    copy_async((const float*)c.ke_f, c.ke0_f, c.ne, s);
    MGAR_LAUNCH_CHECK();
    if (c.dim == 2) build_levels<float, 2>(c, c.ke0_f, c.h32);
    else build_levels<float, 3>(c, c.ke0_f, c.h32);
  }
  c.have_ref = true;
}

}  // namespace mgar
