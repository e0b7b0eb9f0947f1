// Density filter (Eq. 6-8), SIMP conductivities (Eq. 4), compliance and
// sensitivities (Eq. 5, 9-11), and the optimality-criteria update.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "df64.cuh"

#include <vector>

namespace mgar {

// ----------------------------------------------------------------- kernels
// out_e = inv_hs_e * sum_o w_o in_{e+o}            (forward, Eq. 6)
// out_j = sum_o w_o in_{j+o} inv_hs_{j+o}           (transpose, Eq. 9/11)
// over in-domain neighbours; the offset set is symmetric.
template <bool TRANSPOSE>
__global__ void k_filter(const double* __restrict__ in, double* __restrict__ out,
                         const double* __restrict__ inv_hs, const int4* __restrict__ offs,
                         const double* __restrict__ w, int noff, Dims d) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int)d.ne) return;
  const int ex = d.ex, ey = d.ey, ez = d.ez;
  int i, j, k;
  coords(e, d.fEX, d.fEXY, i, j, k);
  double acc = 0.0;
  for (int o = 0; o < noff; ++o) {
    const int4 d = offs[o];
    const int ii = i + d.x, jj = j + d.y, kk = k + d.z;
    const bool ok = !(ii < 0 || ii >= ex || jj < 0 || jj >= ey || kk < 0 || kk >= ez);
    const int nb = ok ? ii + ex * (jj + ey * kk) : e;  // valid address either way
    if (!CK(nb, ex * ey * ez)) continue;
    const double wo = ok ? w[o] : 0.0;
    if (TRANSPOSE) acc += wo * (in[nb] * inv_hs[nb]);
    else acc += wo * in[nb];
  }
  out[e] = TRANSPOSE ? acc : acc * inv_hs[e];
}

// ---- mixed path: filter and sensitivities in double-float on the FP32 pipe
// (FP64 runs at 1/58 of the FP32 rate here).  Weights and inputs are
// non-negative (densities) or non-positive (sensitivities), so the sums have
// no cancellation and the pairs' 2^-46 relative precision carries through.

__device__ __forceinline__ df dfk2(float2 v) { return df{v.x, v.y}; }

// (ah, al) += w * x, unnormalised
__device__ __forceinline__ void acc_prod(float& ah, float& al, df w, df x) {
  float p, pe;
  two_prod(w.hi, x.hi, p, pe);
  pe = __fmaf_rn(w.hi, x.lo, pe);
  pe = __fmaf_rn(w.lo, x.hi, pe);
  float t, te;
  two_sum(ah, p, t, te);
  ah = t;
  al = __fadd_rn(al, __fadd_rn(te, pe));
}

// sum over in-domain offsets o of w_o in_{e+o}.  Every lane of the warp
// must call it (a warp vote): a warp whose elements all lie at least reach
// (reach_z along z) from the boundary takes every offset without bounds
// tests; the sum is taken in the same order either way.
__device__ __forceinline__ df filter_sum_df(const float2* __restrict__ in, const df* w, const char4* offs,
                                            int noff, int e, int i, int j, int k, const Dims& d,
                                            int reach, int reach_z) {
  float ah = 0.f, al = 0.f;
  const bool inner = i >= reach && i < d.ex - reach && j >= reach && j < d.ey - reach &&
                     k >= reach_z && k < d.ez - reach_z;
  if (__all_sync(0xffffffffu, inner)) {
#pragma unroll 4
    for (int o = 0; o < noff; ++o) {
      const char4 dd = offs[o];
      const int nb = e + dd.x + d.ex * (dd.y + d.ey * dd.z);
      if (!CK(nb, d.ne)) continue;
      acc_prod(ah, al, w[o], dfk2(in[nb]));
    }
    return df_make(ah, al);
  }
  // unrolled: the neighbours' loads of several offsets in flight together
#pragma unroll 4
  for (int o = 0; o < noff; ++o) {
    const char4 dd = offs[o];
    const int ii = i + dd.x, jj = j + dd.y, kk = k + dd.z;
    const bool ok = !(ii < 0 || ii >= d.ex || jj < 0 || jj >= d.ey || kk < 0 || kk >= d.ez);
    const int nb = ok ? ii + d.ex * (jj + d.ey * kk) : e;  // valid address either way
    if (!CK(nb, d.ne)) continue;
    const df x = dfk2(in[nb]);
    if (ok) acc_prod(ah, al, w[o], x);
  }
  return df_make(ah, al);
}

// Forward filter (Eq. 6) fused with the SIMP conductivities (Eq. 4):
// rho~_e = inv_hs_e sum_o w_o rho_{e+o}, k_e = kmin + (k0 - kmin) rho~^3,
// written as FP64 (rho~, k_e), FP32 and df64 copies of k_e.
// The constants come as double-float pairs (kmin_df, dk_df = k0 - kmin) and
// 1/Hs as pairs, so no thread converts from FP64 (1/58 of the FP32 rate).
__global__ void k_filter_simp_df(const float2* __restrict__ rho, const float2* __restrict__ inv_hs,
                                 const int4* __restrict__ offs, const double* __restrict__ w, int noff,
                                 Dims d, int reach, int reach_z, double k0, double kmin, double penal,
                                 float2 kmin_df, float2 dk_df, double* __restrict__ rho_phys,
                                 float2* __restrict__ rho_df, double* __restrict__ ke,
                                 float* __restrict__ kf, float2* __restrict__ kdf) {
  // offsets staged as bytes: |d| <= 127 for any radius the tables allow
  __shared__ df ws[kMaxFilterOffsets];
  __shared__ char4 os[kMaxFilterOffsets];
  for (int o = threadIdx.x; o < noff; o += blockDim.x) {
    ws[o] = df_from_double(w[o]);
    const int4 v = offs[o];
    os[o] = make_char4((signed char)v.x, (signed char)v.y, (signed char)v.z, 0);
  }
  __syncthreads();
  // lanes past the last element work on the last one (the warp vote in
  // filter_sum_df needs every lane) and store nothing
  const int e0 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = e0 < (int)d.ne;
  const int e = valid ? e0 : (int)d.ne - 1;
  int i, j, k;
  coords(e, d.fEX, d.fEXY, i, j, k);
  const df r = df_mul(filter_sum_df(rho, ws, os, noff, e, i, j, k, d, reach, reach_z),
                      dfk2(inv_hs[e]));
  if (!valid) return;
  rho_phys[e] = df_to_double(r);
  rho_df[e] = make_float2(r.hi, r.lo);  // the pair k_e comes from (rho_phys: its FP64 rounding)
  df kv;
  if (penal == 3.0) {
    kv = df_add(dfk2(kmin_df), df_mul(dfk2(dk_df), df_mul(df_mul(r, r), r)));
  } else {
    kv = df_from_double(kmin + (k0 - kmin) * pow(df_to_double(r), penal));
  }
  ke[e] = df_to_double(kv);
  kf[e] = __fadd_rn(kv.hi, kv.lo);
  kdf[e] = make_float2(kv.hi, kv.lo);
}

// Element sensitivity (Eq. 10) times inv_hs, as the transpose filter's input:
// out_e = -p (k0 - kmin) rho~_e^(p-1) t_e^T k0 t_e / sum_e', with the energy
// from exact pair differences (k0 has zero row sums).
template <int DIM>
__global__ void k_sens_df(const float2* __restrict__ T, const double* __restrict__ rho,
                          const float2* __restrict__ rho_df, const float2* __restrict__ inv_hs,
                          float2* __restrict__ out, Dims d, float2 mcoef_df, double penal) {
  constexpr int nen = 1 << DIM;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int)d.ne) return;
  int i, j, k;
  coords(e, d.fEX, d.fEXY, i, j, k);
  float2 t[nen];
#pragma unroll
  for (int a = 0; a < nen; ++a) {
    const int nd = (i + (a & 1)) + d.NX * ((j + ((a >> 1) & 1)) + d.NY * (k + ((a >> 2) & 1)));
    t[a] = CK(nd, d.n) ? T[nd] : make_float2(0.f, 0.f);
  }
  // sum over pairs of c_ab (t_a - t_b)^2 with c = 1 (Q4 edges), 2 (Q4
  // diagonals), 1 (H8 face and body diagonals); scale 1/6 (Q4) or 1/12 (H8)
  float ah = 0.f, al = 0.f;
#pragma unroll
  for (int a = 0; a < nen; ++a)
#pragma unroll
    for (int b = a + 1; b < nen; ++b) {
      const int pc = __popc(a ^ b);
      const float cab = DIM == 2 ? (pc == 1 ? 1.f : 2.f) : (pc >= 2 ? 1.f : 0.f);
      if (cab == 0.f) continue;
      float s, er;
      two_sum(t[a].x, -t[b].x, s, er);
      er = __fadd_rn(er, __fsub_rn(t[a].y, t[b].y));
      // (s + er)^2 ~ s^2 + 2 s er
      float p, pe;
      two_prod(s, s, p, pe);
      pe = __fmaf_rn(2.f * s, er, pe);
      p *= cab;
      pe *= cab;
      float u, ue;
      two_sum(ah, p, u, ue);
      ah = u;
      al = __fadd_rn(al, __fadd_rn(ue, pe));
    }
  const df energy = df_mul(df_make(ah, al), df_from_double(DIM == 2 ? 1.0 / 6.0 : 1.0 / 12.0));
  const df r = dfk2(rho_df[e]);
  const df rp = penal == 3.0 ? df_mul(r, r) : df_from_double(pow(rho[e], penal - 1.0));
  const df v = df_mul(df_mul(dfk2(mcoef_df), rp), df_mul(energy, dfk2(inv_hs[e])));
  out[e] = make_float2(v.hi, v.lo);
}

// Transpose filter (Eq. 9/11) of a df64 input already scaled by inv_hs.
__global__ void k_filter_t_df(const float2* __restrict__ in, const int4* __restrict__ offs,
                              const double* __restrict__ w, int noff, Dims d, int reach, int reach_z,
                              double* __restrict__ out, float2* __restrict__ out_df) {
  // offsets staged as bytes: |d| <= 127 for any radius the tables allow
  __shared__ df ws[kMaxFilterOffsets];
  __shared__ char4 os[kMaxFilterOffsets];
  for (int o = threadIdx.x; o < noff; o += blockDim.x) {
    ws[o] = df_from_double(w[o]);
    const int4 v = offs[o];
    os[o] = make_char4((signed char)v.x, (signed char)v.y, (signed char)v.z, 0);
  }
  __syncthreads();
  // lanes past the last element work on the last one (warp vote) and store nothing
  const int e0 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = e0 < (int)d.ne;
  const int e = valid ? e0 : (int)d.ne - 1;
  int i, j, k;
  coords(e, d.fEX, d.fEXY, i, j, k);
  const df v = filter_sum_df(in, ws, os, noff, e, i, j, k, d, reach, reach_z);
  if (!valid) return;
  if (out_df) {
    // renormalised by TwoSum: the pair an FP64 round trip of hi + lo gives
    float sh, se;
    two_sum(v.hi, v.lo, sh, se);
    out_df[e] = make_float2(sh, se);
  } else {
    out[e] = df_to_double(v);
  }
}

__global__ void k_to_df(const double* __restrict__ a, float2* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const df v = df_from_double(a[i]);
    b[i] = make_float2(v.hi, v.lo);
  }
}

__global__ void k_filter_norm(double* __restrict__ inv_hs, const int4* __restrict__ offs,
                              const double* __restrict__ w, int noff, Dims d) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int)d.ne) return;
  const int ex = d.ex, ey = d.ey, ez = d.ez;
  int i, j, k;
  coords(e, d.fEX, d.fEXY, i, j, k);
  double hs = 0.0;
  for (int o = 0; o < noff; ++o) {
    const int4 d = offs[o];
    const int ii = i + d.x, jj = j + d.y, kk = k + d.z;
    if (ii < 0 || ii >= ex || jj < 0 || jj >= ey || kk < 0 || kk >= ez) continue;
    hs += w[o];
  }
  inv_hs[e] = 1.0 / hs;
}

// Eq. 4: k_e = kmin + (k0 - kmin) rho~^p (FP32 copy in mixed mode)
__global__ void k_simp(const double* __restrict__ rho, double* __restrict__ ke, float* __restrict__ kf,
                       int64_t ne, double k0, double kmin, double p) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const double r = rho[e];
  const double rp = (p == 3.0) ? r * r * r : pow(r, p);
  const double k = kmin + (k0 - kmin) * rp;
  ke[e] = k;
  if (kf) kf[e] = (float)k;
}

// Eq. 10: df/drho~_e = -p (k0 - kmin) rho~_e^(p-1) t_e^T k0 t_e
template <int DIM>
__global__ void k_elem_sens(const double* __restrict__ T, const double* __restrict__ rho,
                            double* __restrict__ out, Dims d, double coef, double p) {
  constexpr int nen = 1 << DIM;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int)d.ne) return;
  int i, j, k;
  coords(e, d.fEX, d.fEXY, i, j, k);
  double t[nen];
#pragma unroll
  for (int a = 0; a < nen; ++a) {
    const int nd = (i + (a & 1)) + d.NX * ((j + ((a >> 1) & 1)) + d.NY * (k + ((a >> 2) & 1)));
    t[a] = CK(nd, d.n) ? T[nd] : 0.0;
  }
  // k0 has zero row sums, so t^T k0 t = -sum_{a<b} k0_ab (t_a - t_b)^2:
  // differences first, no cancellation between large temperatures.
  double energy = 0.0;
  if (DIM == 2) {
    // -k0_ab = 1/6 between edge neighbours, 2/6 between opposite corners
    const double d01 = t[0] - t[1], d02 = t[0] - t[2], d13 = t[1] - t[3], d23 = t[2] - t[3];
    const double d03 = t[0] - t[3], d12 = t[1] - t[2];
    energy = ((d01 * d01 + d02 * d02) + (d13 * d13 + d23 * d23) + 2.0 * (d03 * d03 + d12 * d12)) *
             (1.0 / 6.0);
  } else {
    // -k0_ab = 1/12 between face- and body-diagonal corners, 0 along edges
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = a + 1; b < 8; ++b)
        if (__popc(a ^ b) >= 2) {
          const double dd = t[a] - t[b];
          energy += dd * dd;
        }
    energy *= 1.0 / 12.0;
  }
  const double r = rho[e];
  const double rp = (p == 3.0) ? r * r : pow(r, p - 1.0);
  out[e] = -coef * rp * energy;
}

// The OC update's per-element values are kept as double-float pairs (df64,
// about 48 bits) and its per-element arithmetic runs on the FP32 pipe: GB300
// runs FP64 arithmetic and FP32<->FP64 conversions at about 1.6 per SM and
// clock against 110 FP32 operations, and each FP64 operation per element
// costs about 4 us on 2.1 M elements.  The design's rho and dc arrive in
// FP64 and the new rho leaves in FP64 (one conversion each); the scalars
// (lambda, the bracket, the volume sums across blocks) stay FP64.
__device__ __forceinline__ df ld2(const float2* p, int64_t i) {
  const float2 v = p[i];
  return df{v.x, v.y};
}
__device__ __forceinline__ void st2(float2* p, int64_t i, df v) { p[i] = make_float2(v.hi, v.lo); }

// OC preparation: s_e = rho_e sqrt(max(-dc_e, 0) / dv_e) and the move box
// [max(0, rho - move), min(1, rho + move)], with their FP32 copies for the
// multisection and rho itself for the apply; rsdv = 1 / sqrt(dv) is fixed by
// the filter and computed once.
__global__ void k_oc_prep(const double* __restrict__ rho, const double* __restrict__ dc,
                          const float2* __restrict__ dc_df, const float2* __restrict__ rsdv, float2* __restrict__ s,
                          float2* __restrict__ lo, float2* __restrict__ hi,
                          float2* __restrict__ rdf, float* __restrict__ s32,
                          float* __restrict__ lo32, float* __restrict__ hi32, int64_t ne,
                          df move) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const df r = df_from_double(rho[e]);
  const df x = dc_df ? df_neg(ld2(dc_df, e)) : df_from_double(-dc[e]);
  // sqrt(x) = x / sqrt(x); x <= 0 (or NaN) gives 0
  const df sq = x.hi > 0.f ? df_mul(x, df_rsqrt(x)) : df{0.f, 0.f};
  const df sv = df_mul(df_mul(r, sq), ld2(rsdv, e));
  df l = df_sub(r, move);
  if (l.hi < 0.f) l = df{0.f, 0.f};
  df h = df_add(r, move);
  if (df_le(df{1.f, 0.f}, h)) h = df{1.f, 0.f};
  st2(s, e, sv);
  st2(lo, e, l);
  st2(hi, e, h);
  st2(rdf, e, r);
  s32[e] = sv.hi;
  lo32[e] = l.hi;
  hi32[e] = h.hi;
}

// One bisection step on lambda: volume sum_e dv_e clamp(s_e / sqrt(lambda))
// at the geometric midpoint of the bracket; the last block moves the
// bracket and raises the done flag once (hi - lo) / (hi + lo) <= tol.  The
// fallback of the fast solve: FP64 arithmetic on the pairs' values.
__global__ void k_oc_pass(const float2* __restrict__ s, const float2* __restrict__ lo,
                          const float2* __restrict__ hi, const float2* __restrict__ dv, int64_t ne,
                          double volfrac, double tol, double* dsc, double* partials,
                          unsigned int* counter) {
  if (dsc[S_OC_DONE] != 0.0) return;
  const double blo = dsc[S_OC_LO], bhi = dsc[S_OC_HI];
  const double lam = sqrt(blo * bhi);
  const double mu = 1.0 / sqrt(lam);
  double v[1] = {0.0};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x)
    v[0] += df_to_double(ld2(dv, e)) *
            fmin(fmax(df_to_double(ld2(s, e)) * mu, df_to_double(ld2(lo, e))),
                 df_to_double(ld2(hi, e)));
  double vol[1];
  if (block_sum_last<1>(v, partials, counter, vol) && threadIdx.x == 0) {
    double nlo = blo, nhi = bhi;
    if (vol[0] > volfrac) nlo = lam;
    else nhi = lam;
    dsc[S_OC_LO] = nlo;
    dsc[S_OC_HI] = nhi;
    dsc[S_OC_VOL] = vol[0];
    dsc[S_OC_STEPS] += 1.0;
    if ((nhi - nlo) / (nhi + nlo) <= tol) dsc[S_OC_DONE] = 1.0;
  }
}

__global__ void k_oc_mu_from_bracket(double* dsc) {
  const double lam = sqrt(dsc[S_OC_LO] * dsc[S_OC_HI]);
  dsc[S_OC_MU] = 1.0 / sqrt(lam);
}

__global__ void k_oc_init(double* dsc, double lo, double hi) {
  dsc[S_OC_LO] = lo;
  dsc[S_OC_HI] = hi;
  dsc[S_OC_DONE] = 0.0;
  dsc[S_OC_STEPS] = 0.0;
  dsc[S_OC_FAIL] = 0.0;  // the update by the plain bisection is applied
}

// ---- OC solve for mu = 1/sqrt(lambda) without 50 FP64 passes ----------
// g(mu) = sum_e dv_e clamp(s_e mu, lo_e, hi_e) is continuous, monotone and
// piecewise linear.  (1) FP32 multisection on ln(mu) narrows the bracket by
// 32x per pass; (2) one FP64 pass splits the elements into constant
// (clamped over the whole bracket), linear, and ambiguous (a breakpoint
// inside the bracket) and sums the first two; (3) one warp bisects in FP64
// over the few ambiguous elements.  Any failed check falls back to the plain
// bisection of k_oc_pass.

// candidates mu_k, k = 0..kOcCand-1, at fractions (k+1)/(kOcCand+1) of [La, Lb]
// evenly spaced candidates strictly inside the ln-bracket [La, Lb]
__device__ __forceinline__ void oc_candidates(double* dsc) {
  const double La = dsc[S_OC_LA], Lb = dsc[S_OC_LB];
  for (int k = threadIdx.x; k < kOcCand; k += blockDim.x) {
    const double L = La + (Lb - La) * (double)(k + 1) / (double)(kOcCand + 1);
    dsc[S_OC_CANDL + k] = L;
    dsc[S_OC_CAND + k] = exp(L);
  }
}

// First pass.  Cold: evenly spaced over [La, Lb].  Warm (ln mu of the
// previous update known): a two-sided geometric ladder L0 +- 1e-3 * 2^(j-1),
// j = 1..14, around it, with the range ends as outermost candidates, so the
// first pass brackets the root anywhere in the range and finely near L0.
__global__ void k_oc_start(double* dsc, double La, double Lb, int warm, int* namb) {
  const bool w = warm && dsc[S_OC_HAVEPREV] != 0.0;
  const double L0 = fmin(fmax(dsc[S_OC_LPREV], La), Lb);
  if (threadIdx.x == 0) {
    *namb = 0;  // the classification's ambiguous count
    dsc[S_OC_LA] = La;
    dsc[S_OC_LB] = Lb;
    dsc[S_OC_FAIL] = 0.0;
  }
  if (!w) {
    __syncthreads();
    oc_candidates(dsc);
    return;
  }
  for (int k = threadIdx.x; k < kOcCand; k += blockDim.x) {
    const int j = k - kOcCand / 2;
    double L;
    if (k == 0) L = La;
    else if (k == kOcCand - 1) L = Lb;
    else if (j == 0) L = L0;
    else L = L0 + (j > 0 ? 1.0 : -1.0) * 1e-3 * exp2((double)(abs(j) - 1));
    L = fmin(fmax(L, La), Lb);
    dsc[S_OC_CANDL + k] = L;
    dsc[S_OC_CAND + k] = exp(L);
  }
}

__global__ void k_oc_multisect(const float* __restrict__ s, const float* __restrict__ lo,
                               const float* __restrict__ hi, const float* __restrict__ dv, int ne,
                               double volfrac, double* dsc, double* partials,
                               unsigned int* counter) {
  // the bracket is read by every block before the last one moves it
  if (dsc[S_OC_LB] - dsc[S_OC_LA] <= kOcTarget) return;  // narrow enough: pass skipped
  __shared__ float mu[kOcCand];
  if (threadIdx.x < kOcCand) mu[threadIdx.x] = (float)dsc[S_OC_CAND + threadIdx.x];
  __syncthreads();
  float acc[kOcCand];
#pragma unroll
  for (int k = 0; k < kOcCand; ++k) acc[k] = 0.f;
  const int stride = gridDim.x * blockDim.x;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  // four elements per iteration: their loads are in flight together
  for (; e + 3 * stride < ne; e += 4 * stride) {
    float sv[4], lv[4], hv[4], dd[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      sv[u] = s[e + u * stride];
      lv[u] = lo[e + u * stride];
      hv[u] = hi[e + u * stride];
      dd[u] = dv[e + u * stride];
    }
#pragma unroll
    for (int k = 0; k < kOcCand; ++k)
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[k] += dd[u] * fminf(fmaxf(sv[u] * mu[k], lv[u]), hv[u]);
  }
  for (; e < ne; e += stride) {
    const float se = s[e], l = lo[e], h = hi[e], d = dv[e];
#pragma unroll
    for (int k = 0; k < kOcCand; ++k) acc[k] += d * fminf(fmaxf(se * mu[k], l), h);
  }
  double tot[kOcCand];
  const bool last = block_sum_last_f32<kOcCand>(acc, partials, counter, tot);
  if (!last) return;
  if (threadIdx.x == 0) {
    int ks = kOcCand;
    for (int k = 0; k < kOcCand; ++k)
      if (tot[k] >= volfrac) {
        ks = k;
        break;
      }
    const double La = dsc[S_OC_LA], Lb = dsc[S_OC_LB];
    dsc[S_OC_LA] = ks == 0 ? La : dsc[S_OC_CANDL + ks - 1];
    dsc[S_OC_LB] = ks == kOcCand ? Lb : dsc[S_OC_CANDL + ks];
  }
  __syncthreads();
  oc_candidates(dsc);
}

// Split elements for the bracket [mu_a, mu_b] (ln bracket widened by
// margin): constant part C, slope B, and the ambiguous list.  The tests and
// sums run in df64; an element whose breakpoint lies within rounding of a
// bracket end is either listed as ambiguous or contributes an error of that
// rounding's size (the root lies well inside the bracket).
__global__ void k_oc_classify(const float2* __restrict__ s, const float2* __restrict__ lo,
                              const float2* __restrict__ hi, const float2* __restrict__ dv, int ne,
                              double margin, double Lmin, double Lmax, double* dsc, int* amb,
                              int* namb, double* partials, unsigned int* counter) {
  __shared__ float2 mua, mub;
  if (threadIdx.x == 0) {
    const double La = fmax(dsc[S_OC_LA] - margin, Lmin), Lb = fmin(dsc[S_OC_LB] + margin, Lmax);
    const double ea = exp(La), eb = exp(Lb);
    if (blockIdx.x == 0) {
      dsc[S_OC_MUA] = ea;
      dsc[S_OC_MUB] = eb;
    }
    const df da = df_from_double(ea), db = df_from_double(eb);
    mua = make_float2(da.hi, da.lo);
    mub = make_float2(db.hi, db.lo);
  }
  __syncthreads();
  const df A{mua.x, mua.y}, Bv{mub.x, mub.y};
  df v0{0.f, 0.f}, v1{0.f, 0.f};
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
    const df se = ld2(s, e), l = ld2(lo, e), h = ld2(hi, e);
    const df ta = df_mul(se, A), tb = df_mul(se, Bv);
    if (df_le(tb, l)) v0 = df_add(v0, df_mul(ld2(dv, e), l));
    else if (df_le(h, ta)) v0 = df_add(v0, df_mul(ld2(dv, e), h));
    else if (df_le(l, ta) && df_le(tb, h)) v1 = df_add(v1, df_mul(ld2(dv, e), se));
    else {
      const int slot = atomicAdd(namb, 1);
      if (slot < kOcAmbMax && CK(slot, kOcAmbMax)) amb[slot] = e;
    }
  }
  // warp sums in df64, FP64 across warps and blocks
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 = df_add(v0, df{__shfl_down_sync(0xffffffffu, v0.hi, o), __shfl_down_sync(0xffffffffu, v0.lo, o)});
    v1 = df_add(v1, df{__shfl_down_sync(0xffffffffu, v1.hi, o), __shfl_down_sync(0xffffffffu, v1.lo, o)});
  }
  double w[2] = {0.0, 0.0};
  if ((threadIdx.x & 31) == 0) {
    w[0] = df_to_double(v0);
    w[1] = df_to_double(v1);
  }
  double tot[2];
  if (block_sum_last_core<2>(w, partials, counter, tot, threadIdx.x, blockDim.x, blockIdx.x,
                             gridDim.x) &&
      threadIdx.x == 0) {
    dsc[S_OC_C] = tot[0];
    dsc[S_OC_B] = tot[1];
  }
}

// Sort the ambiguous list (bitonic, shared memory), then one warp bisects
// g(mu) = C + B mu + sum_amb dv clamp(s mu, lo, hi) = volfrac on [mu_a, mu_b].
__global__ void k_oc_finish(const float2* __restrict__ s, const float2* __restrict__ lo,
                            const float2* __restrict__ hi, const float2* __restrict__ dv, int ne,
                            double volfrac, double* dsc, int* amb, int* namb_p) {
  __shared__ int key[kOcAmbMax];
  const int namb = *namb_p;
  if (namb > kOcAmbMax) {
    if (threadIdx.x == 0) dsc[S_OC_FAIL] = 1.0;
    return;
  }
  int size = 1;
  while (size < namb) size <<= 1;
  for (int i = threadIdx.x; i < size; i += blockDim.x)
    if (CK(i, kOcAmbMax)) key[i] = i < namb ? amb[i] : 0x7fffffff;
  __syncthreads();
  for (int k = 2; k <= size; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < size; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i && CK(ixj, kOcAmbMax) && CK(i, kOcAmbMax)) {
          const bool up = (i & k) == 0;
          const int a = key[i], b = key[ixj];
          if ((a > b) == up) {
            key[i] = b;
            key[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const double C = dsc[S_OC_C], B = dsc[S_OC_B];
  double a = dsc[S_OC_MUA], b = dsc[S_OC_MUB];
  // up to kCache ambiguous elements are staged in shared memory, so the
  // bisection steps do not wait on global loads; the same elements in the
  // same order as the loads below otherwise
  constexpr int kCache = 256;
  __shared__ double cs[kCache], cl[kCache], ch[kCache], cd[kCache];
  const bool cached = namb <= kCache;
  if (cached) {
    for (int i = lane; i < namb; i += 32) {
      const int e = CK(i, kOcAmbMax) ? key[i] : 0;
      const bool ok = CK(e, ne);
      cs[i] = ok ? df_to_double(ld2(s, e)) : 0.0;
      cl[i] = ok ? df_to_double(ld2(lo, e)) : 0.0;
      ch[i] = ok ? df_to_double(ld2(hi, e)) : 0.0;
      cd[i] = ok ? df_to_double(ld2(dv, e)) : 0.0;
    }
    __syncwarp();
  }
  auto g = [&](double mu) {
    double acc = 0.0;
    if (cached) {
      for (int i = lane; i < namb; i += 32) acc += cd[i] * fmin(fmax(cs[i] * mu, cl[i]), ch[i]);
    } else {
      for (int i = lane; i < namb; i += 32) {
        if (!CK(i, kOcAmbMax)) continue;
        const int e = key[i];
        if (!CK(e, ne)) continue;
        acc += df_to_double(ld2(dv, e)) *
               fmin(fmax(df_to_double(ld2(s, e)) * mu, df_to_double(ld2(lo, e))),
                    df_to_double(ld2(hi, e)));
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return C + B * mu + acc;
  };
  const double ga = g(a), gb = g(b);
  if (!(ga <= volfrac && volfrac <= gb)) {
    if (lane == 0) dsc[S_OC_FAIL] = 1.0;
    return;
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (a + b);
    if (!(mid > a && mid < b)) break;
    if ((b - a) <= 1e-15 * b) break;
    if (g(mid) >= volfrac) b = mid;
    else a = mid;
  }
  if (lane == 0) dsc[S_OC_MU] = 0.5 * (a + b);
}

// rho <- clamp(s mu) for mu = dsc[S_OC_MU]; max |change| into dsc.  Skipped
// (every block) while the fast solve's failure flag is up: the host then
// runs the plain bisection and this kernel again.  rho_old is the pair the
// preparation kept; the clamp and the change are formed in df64.
__global__ void k_oc_apply(double* __restrict__ rho, const float2* __restrict__ s,
                           const float2* __restrict__ lo, const float2* __restrict__ hi,
                           const float2* __restrict__ rdf, int ne, double* dsc, double* partials,
                           unsigned int* counter) {
  if (dsc[S_OC_FAIL] != 0.0) return;
  const double mu = dsc[S_OC_MU];
  const df M = df_from_double(mu);
  df chd{0.f, 0.f};
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
    const df rn = df_min(df_max(df_mul(ld2(s, e), M), ld2(lo, e)), ld2(hi, e));
    chd = df_max(chd, df_abs(df_sub(rn, ld2(rdf, e))));
    rho[e] = df_to_double(rn);
  }
  block_max_finish(df_to_double(chd), partials, counter, dsc + S_OC_CHANGE);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    dsc[S_OC_LAM] = 1.0 / (mu * mu);
    // ln mu for the next update's warm start
    const double L = log(mu);
    const bool ok = isfinite(L) && fabs(L) < 20.0 * 2.302585092994046;
    dsc[S_OC_LPREV] = ok ? L : 0.0;
    dsc[S_OC_HAVEPREV] = ok ? 1.0 : 0.0;
  }
}

// dv and 1 / sqrt(dv) as double-float pairs for the OC update
__global__ void k_dv_df(const double* __restrict__ dv, float2* __restrict__ dvdf,
                        float2* __restrict__ rsdv, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  st2(dvdf, i, df_from_double(dv[i]));
  st2(rsdv, i, df_from_double(1.0 / sqrt(dv[i])));
}

__global__ void k_d2f_e(const double* __restrict__ a, float* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// ------------------------------------------------------------------- host
// Offsets and weights max(0, r - |d|) of a radius-r filter (Eq. 7), in the
// order dz, dy, dx.
// The largest |offset| component of the current tables (filter_tables
// reaches ceil(r) along each axis).
static int filter_reach(const Ctx& c) { return (int)std::ceil(c.filter_r); }

static void filter_tables(double r, int dim, std::vector<int4>& offs, std::vector<double>& w) {
  const int reach = (int)std::ceil(r);
  offs.clear();
  w.clear();
  const int zr = dim == 3 ? reach : 0;
  for (int dz = -zr; dz <= zr; ++dz)
    for (int dy = -reach; dy <= reach; ++dy)
      for (int dx = -reach; dx <= reach; ++dx) {
        const double wt = r - std::sqrt((double)(dx * dx + dy * dy + dz * dz));
        if (wt > 0.0) {
          offs.push_back(make_int4(dx, dy, dz, 0));
          w.push_back(wt);
        }
      }
}

// Eq. 22-23, applied as a recursion from r^(0) = alpha L exactly as written
// (the same sequence of multiplications as the oracle); r_min throughout
// when alpha L <= r_min.
double filter_radius(const Ctx& c, int k) {
  const double L = c.p.filter_L > 0.0 ? c.p.filter_L : (double)std::max(std::max(c.p.nx, c.p.ny), c.p.nz);
  const double r0 = c.p.filter_alpha * L, rmin = c.p.rmin;
  if (!(r0 > rmin) || c.p.filter_lp <= 0) return rmin;
  const double eta = std::exp((std::log(rmin) - std::log(r0)) / c.p.filter_lp);
  double r = r0;
  for (int i = 0; i < k; ++i) r = std::max(rmin, eta * r);
  return r;
}

__global__ void k_fill(double* __restrict__ a, double v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

// 1/Hs and dv = F^T (1/E) (with its FP32 copy and 1/sqrt) for the current tables
static void filter_derived(Ctx& c) {
  const Dims& d = c.L[0];
  k_filter_norm<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(c.inv_hs, c.f_offs, c.f_w, c.n_filter,
                                                             d);
  MGAR_LAUNCH_CHECK();
  k_to_df<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(c.inv_hs, c.inv_hs_df, (int)c.ne);
  MGAR_LAUNCH_CHECK();
  k_fill<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(c.tmp_e, 1.0 / (double)c.ne, (int)c.ne);
  MGAR_LAUNCH_CHECK();
  filter(c, c.tmp_e, c.dv, true);
  k_d2f_e<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(c.dv, c.dv32, (int)c.ne);
  MGAR_LAUNCH_CHECK();
  k_dv_df<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(c.dv, c.dv_df, c.rsdv, (int)c.ne);
  MGAR_LAUNCH_CHECK();
}

void setup_filter(Ctx& c) {
  // room for the largest radius the run will use
  double rcap = c.p.rmin;
  if (c.p.filter_alpha > 0.0) rcap = std::max(rcap, filter_radius(c, 0));
  std::vector<int4> offs;
  std::vector<double> w;
  filter_tables(rcap, c.dim, offs, w);
  require((int)offs.size() <= kMaxFilterOffsets, MGAR_ERR_ARG, "filter radius too large");
  c.filter_cap = (int)offs.size();
  MGAR_CUDA(cudaMalloc(&c.f_offs, offs.size() * sizeof(int4)));
  MGAR_CUDA(cudaMalloc(&c.f_w, w.size() * sizeof(double)));
  if (c.p.filter_alpha > 0.0) {
    MGAR_CUDA(cudaHostAlloc(&c.f_offs_h, offs.size() * sizeof(int4), cudaHostAllocDefault));
    MGAR_CUDA(cudaHostAlloc(&c.f_w_h, w.size() * sizeof(double), cudaHostAllocDefault));
  }
  filter_tables(c.p.rmin, c.dim, offs, w);
  c.n_filter = (int)offs.size();
  c.filter_r = c.p.rmin;
  MGAR_CUDA(cudaMemcpy(c.f_offs, offs.data(), offs.size() * sizeof(int4), cudaMemcpyHostToDevice));
  MGAR_CUDA(cudaMemcpy(c.f_w, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
  filter_derived(c);
  MGAR_CUDA(cudaStreamSynchronize(c.stream));
}

// New tables through the pinned staging buffers.  The previous copy out of
// them has completed: every design cycle waits on the stream (scalar
// fetches) after its filter work.
void set_filter_radius(Ctx& c, double r) {
  std::vector<int4> offs;
  std::vector<double> w;
  filter_tables(r, c.dim, offs, w);
  require((int)offs.size() <= c.filter_cap && c.f_offs_h, MGAR_ERR_ARG,
          "filter radius beyond the tables' capacity");
  std::copy(offs.begin(), offs.end(), c.f_offs_h);
  std::copy(w.begin(), w.end(), c.f_w_h);
  MGAR_CUDA(cudaMemcpyAsync(c.f_offs, c.f_offs_h, offs.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, c.stream));
  MGAR_CUDA(cudaMemcpyAsync(c.f_w, c.f_w_h, w.size() * sizeof(double), cudaMemcpyHostToDevice,
                            c.stream));
  c.n_filter = (int)offs.size();
  c.filter_r = r;
  filter_derived(c);
}

void filter(Ctx& c, const double* in, double* out, bool transpose) {
  const Dims& d = c.L[0];
  ProfScope ps(c, MGAR_KC_FILTER);
  if (transpose)
    k_filter<true><<<blocks_for(c.ne), kThreads, 0, c.stream>>>(in, out, c.inv_hs, c.f_offs, c.f_w,
                                                                c.n_filter, d);
  else
    k_filter<false><<<blocks_for(c.ne), kThreads, 0, c.stream>>>(in, out, c.inv_hs, c.f_offs, c.f_w,
                                                                 c.n_filter, d);
  MGAR_LAUNCH_CHECK();
}

void set_density(Ctx& c, const double* rho, bool physical) {
  if (c.p.precision == MGAR_MIXED && !physical) {
    // filter + SIMP in one df64 pass
    ProfScope ps(c, MGAR_KC_FILTER);
    k_to_df<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(rho, c.df_e, (int)c.ne);
    MGAR_LAUNCH_CHECK();
    const df kmin_df = df_from_double(c.p.kmin), dk_df = df_from_double(c.p.k0 - c.p.kmin);
    k_filter_simp_df<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(
        c.df_e, c.inv_hs_df, c.f_offs, c.f_w, c.n_filter, c.L[0], filter_reach(c),
        c.dim == 3 ? filter_reach(c) : 0, c.p.k0, c.p.kmin, c.p.penal,
        make_float2(kmin_df.hi, kmin_df.lo), make_float2(dk_df.hi, dk_df.lo), c.rho_phys,
        c.rho_phys_df, c.ke, c.ke_f, c.ke_df);
    MGAR_LAUNCH_CHECK();
    if (c.dim == 3) df3d_node_diag(c);
    return;
  }
  if (physical)
    MGAR_CUDA(cudaMemcpyAsync(c.rho_phys, rho, c.ne * sizeof(double), cudaMemcpyDeviceToDevice,
                              c.stream));
  else
    filter(c, rho, c.rho_phys, false);
  k_simp<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(c.rho_phys, c.ke,
                                                      c.p.precision == MGAR_FP64 ? nullptr : c.ke_f,
                                                      c.ne, c.p.k0, c.p.kmin, c.p.penal);
  MGAR_LAUNCH_CHECK();
  if (c.p.precision == MGAR_MIXED) {
    ke_to_df(c);
    k_to_df<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(c.rho_phys, c.rho_phys_df, (int)c.ne);
    MGAR_LAUNCH_CHECK();
    if (c.dim == 3) df3d_node_diag(c);
  }
}

void sensitivity(Ctx& c, const double* T, double* dc, double* dv, double* compliance,
                 const float2* T_df, float2* dc_df) {
  const Dims& d = c.L[0];
  const double coef = c.p.penal * (c.p.k0 - c.p.kmin);
  require(!dc_df || c.p.precision == MGAR_MIXED, MGAR_ERR_ARG, "dc pairs need the mixed path");
  if ((dc || dc_df) && c.p.precision == MGAR_MIXED) {
    ProfScope ps(c, MGAR_KC_SENS);
    if (!T_df) {
      k_to_df<<<blocks_for(c.n), kThreads, 0, c.stream>>>(T, c.df_p2, (int)c.n);
      MGAR_LAUNCH_CHECK();
      T_df = c.df_p2;
    }
    const df mc = df_from_double(-coef);
    const float2 mcoef_df = make_float2(mc.hi, mc.lo);
    if (c.dim == 2)
      k_sens_df<2><<<blocks_for(c.ne), kThreads, 0, c.stream>>>(T_df, c.rho_phys, c.rho_phys_df,
                                                                c.inv_hs_df, c.df_e, d, mcoef_df,
                                                                c.p.penal);
    else
      k_sens_df<3><<<blocks_for(c.ne), kThreads, 0, c.stream>>>(T_df, c.rho_phys, c.rho_phys_df,
                                                                c.inv_hs_df, c.df_e, d, mcoef_df,
                                                                c.p.penal);
    MGAR_LAUNCH_CHECK();
    k_filter_t_df<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(
        c.df_e, c.f_offs, c.f_w, c.n_filter, d, filter_reach(c), c.dim == 3 ? filter_reach(c) : 0,
        dc_df ? nullptr : dc, dc_df);
    MGAR_LAUNCH_CHECK();
  } else if (dc) {
    ProfScope ps(c, MGAR_KC_SENS);
    if (c.dim == 2)
      k_elem_sens<2><<<blocks_for(c.ne), kThreads, 0, c.stream>>>(T, c.rho_phys, c.tmp_e, d, coef,
                                                                  c.p.penal);
    else
      k_elem_sens<3><<<blocks_for(c.ne), kThreads, 0, c.stream>>>(T, c.rho_phys, c.tmp_e, d, coef,
                                                                  c.p.penal);
    MGAR_LAUNCH_CHECK();
    filter(c, c.tmp_e, dc, true);
  }
  if (dv)
    MGAR_CUDA(cudaMemcpyAsync(dv, c.dv, c.ne * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  if (compliance) {
    dot(c, c.q, T, c.n, c.dsc + S_COMPL);
    fetch_scalars(c, S_COMPL, 1);
    *compliance = c.hsc[S_COMPL];
  }
}

}  // namespace mgar

namespace mgar {

// The fast solve for lambda and its application to rho, queued on the
// handle's stream without a host read (the apply does nothing if the solve
// failed; oc_complete reads the outcome).
void oc_issue(Ctx& c, double* rho, const double* dc, double volfrac, double move,
              const float2* dc_df) {
  const int ne = (int)c.ne;
  const int rb = c.grid_blocks_e;
  k_oc_prep<<<blocks_for(ne), kThreads, 0, c.stream>>>(rho, dc, dc_df, c.rsdv, c.oc_s, c.oc_lo, c.oc_hi,
                                                       c.oc_rho, c.oc_s32, c.oc_lo32, c.oc_hi32,
                                                       ne, df_from_double(move));
  MGAR_LAUNCH_CHECK();
  // lambda in [1e-40, 1e40]  <=>  ln(mu) in [-20 ln 10, 20 ln 10]
  const double Lmax = 20.0 * std::log(10.0), Lmin = -Lmax;
  ProfScope ps(c, MGAR_KC_OC);
  k_oc_start<<<1, 32, 0, c.stream>>>(c.dsc, Lmin, Lmax, 1, c.oc_namb);
  MGAR_LAUNCH_CHECK();
  // three blocks per SM (the 80 registers of the 31 accumulators allow
  // three): more loads in flight; the last block's sum over the partials
  // stays short
  const int msb = std::min(blocks_for(ne), c.sms * 3);
  for (int pass = 0; pass < kOcPasses; ++pass) {
    k_oc_multisect<<<msb, kThreads, 0, c.stream>>>(c.oc_s32, c.oc_lo32, c.oc_hi32, c.dv32, ne,
                                                  volfrac, c.dsc, c.partials, c.counter);
    MGAR_LAUNCH_CHECK();
  }
  k_oc_classify<<<rb, kThreads, 0, c.stream>>>(c.oc_s, c.oc_lo, c.oc_hi, c.dv_df, ne, kOcMargin, Lmin,
                                               Lmax, c.dsc, c.oc_amb, c.oc_namb, c.partials,
                                               c.counter);
  MGAR_LAUNCH_CHECK();
  k_oc_finish<<<1, 1024, 0, c.stream>>>(c.oc_s, c.oc_lo, c.oc_hi, c.dv_df, ne, volfrac, c.dsc,
                                        c.oc_amb, c.oc_namb);
  MGAR_LAUNCH_CHECK();
  k_oc_apply<<<rb, kThreads, 0, c.stream>>>(rho, c.oc_s, c.oc_lo, c.oc_hi, c.oc_rho, ne, c.dsc,
                                            c.partials, c.counter);
  MGAR_LAUNCH_CHECK();
}

// One host read from S_OC_LAM on brings the check, lambda, the change and a
// compliance dot launched before the update; if the fast solve failed, the
// plain bisection on lambda over the whole range and the apply again.
void oc_complete(Ctx& c, double* rho, double volfrac, double* lambda, double* change) {
  fetch_scalars(c, S_OC_LAM, S_OC_FAIL - S_OC_LAM + 1);
  oc_finish(c, rho, volfrac, lambda, change);
}

// The rest of oc_complete once the host mirror holds S_OC_LAM, S_OC_CHANGE
// and S_OC_FAIL of this update (read by oc_complete, or gathered for many
// designs at once by the batched design cycle).
void oc_finish(Ctx& c, double* rho, double volfrac, double* lambda, double* change) {
  const int ne = (int)c.ne;
  const int rb = c.grid_blocks_e;
  const bool fast_ok = c.hsc[S_OC_FAIL] == 0.0;
  if (!fast_ok) {
    k_oc_init<<<1, 1, 0, c.stream>>>(c.dsc, 1e-40, 1e40);
    MGAR_LAUNCH_CHECK();
    const int max_steps = 200, batch = 16;
    for (int done = 0; done < max_steps; done += batch) {
      for (int b = 0; b < batch; ++b) {
        k_oc_pass<<<rb, kThreads, 0, c.stream>>>(c.oc_s, c.oc_lo, c.oc_hi, c.dv_df, ne, volfrac, 1e-13,
                                                 c.dsc, c.partials, c.counter);
        MGAR_LAUNCH_CHECK();
      }
      fetch_scalars(c, S_OC_DONE, 1);
      if (c.hsc[S_OC_DONE] != 0.0) break;
    }
    k_oc_mu_from_bracket<<<1, 1, 0, c.stream>>>(c.dsc);
    MGAR_LAUNCH_CHECK();
    k_oc_apply<<<rb, kThreads, 0, c.stream>>>(rho, c.oc_s, c.oc_lo, c.oc_hi, c.oc_rho, ne, c.dsc,
                                              c.partials, c.counter);
    MGAR_LAUNCH_CHECK();
    fetch_scalars(c, S_OC_LAM, 3);
  }
  if (lambda) *lambda = c.hsc[S_OC_LAM];
  if (change) *change = c.hsc[S_OC_CHANGE];
  c.oc_fallbacks += fast_ok ? 0 : 1;
}

void oc_update(Ctx& c, double* rho, const double* dc, double volfrac, double move, double* lambda,
               double* change, const float2* dc_df) {
  oc_issue(c, rho, dc, volfrac, move, dc_df);
  oc_complete(c, rho, volfrac, lambda, change);
}


// ---------------------------------------------------------------------------
// Projection-based boundary post-processing, Section 2.3, Eq. 24-27 (run once
// after the loop).  s_e = -df/drho~_e of the final design (Eq. 10) is
// projected onto the nodes with the filter's weights, ns_i = sum_e w_ie s_e /
// sum_e w_ie, w_ie = max(0, r - |x_i - c_e|); an element is solid when all
// its nodes have ns > level, void when all have ns < level, and otherwise
// gets the share of the (S+1)^d points of a lattice over the element (the
// original nodes included) at which the bilinear / trilinear interpolation
// of ns exceeds the level (Eq. 25-27); the level is bisected so that the
// mean density stays at or below the volume fraction.

constexpr int kPpLattice = 4;  // S: lattice intervals per axis

template <int DIM>
__global__ void k_pp_nodal(const double* __restrict__ dcp, double* __restrict__ ns, Dims d,
                           double r, int reach) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int)d.n) return;
  int i, j, k;
  coords(idx, d.fNX, d.fNXY, i, j, k);
  double num = 0.0, den = 0.0;
  // element (i + ox, j + oy, k + oz) has its centroid at offset o + 1/2
  for (int ox = -reach; ox < reach; ++ox)
    for (int oy = -reach; oy < reach; ++oy)
      for (int oz = (DIM == 3 ? -reach : 0); oz < (DIM == 3 ? reach : 1); ++oz) {
        const double dz = DIM == 3 ? oz + 0.5 : 0.0;
        const double w = r - sqrt((ox + 0.5) * (ox + 0.5) + (oy + 0.5) * (oy + 0.5) + dz * dz);
        const int ei = i + ox, ej = j + oy, ek = k + oz;
        if (w <= 0.0 || ei < 0 || ei >= d.ex || ej < 0 || ej >= d.ey || ek < 0 || ek >= d.ez)
          continue;
        const int e = ei + d.ex * (ej + d.ey * ek);
        if (!CK(e, d.ne)) continue;
        num += w * -dcp[e];
        den += w;
      }
  ns[idx] = num / den;
}

// Eq. 24 with ev of Eq. 25-27; the densities into rho (may be null) and their
// sum into *sum
template <int DIM>
__global__ void k_pp_density(const double* __restrict__ ns, Dims d, double level,
                             double* __restrict__ rho, double* partials, unsigned int* counter,
                             double* sum) {
  constexpr int nen = 1 << DIM, P = kPpLattice + 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (e < (int)d.ne) {
    int i, j, k;
    coords(e, d.fEX, d.fEXY, i, j, k);
    double t[nen];
    bool all_above = true, all_below = true;
#pragma unroll
    for (int a = 0; a < nen; ++a) {
      const int nd = (i + (a & 1)) + d.NX * ((j + ((a >> 1) & 1)) + d.NY * (k + ((a >> 2) & 1)));
      t[a] = CK(nd, d.n) ? ns[nd] : 0.0;
      all_above = all_above && t[a] > level;
      all_below = all_below && t[a] < level;
    }
    double val;
    if (all_above) {
      val = 1.0;
    } else if (all_below) {
      val = 0.0;
    } else {
      int count = 0, total = 0;
      for (int pz = 0; pz < (DIM == 3 ? P : 1); ++pz)
        for (int px = 0; px < P; ++px)
          for (int py = 0; py < P; ++py) {
            // local coordinates of the lattice point
            const double xi = -1.0 + 2.0 * px / kPpLattice;
            const double eta = -1.0 + 2.0 * py / kPpLattice;
            const double zeta = DIM == 3 ? -1.0 + 2.0 * pz / kPpLattice : 0.0;
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < nen; ++a) {
              const double lx = 2 * (a & 1) - 1, ly = 2 * ((a >> 1) & 1) - 1,
                           lz = 2 * ((a >> 2) & 1) - 1;
              double nval = (1.0 + xi * lx) * (1.0 + eta * ly);
              if (DIM == 3) nval *= (1.0 + zeta * lz);
              s += nval / nen * t[a];
            }
            count += s > level ? 1 : 0;
            ++total;
          }
      val = (double)count / (double)total;
    }
    if (rho) rho[e] = val;
    v[0] = val;
  }
  block_sum_finish<1>(v, partials, counter, sum);
}

__global__ void k_pp_max(const double* __restrict__ ns, int n, double* partials,
                         unsigned int* counter, double* out) {
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = fmax(m, ns[i]);
  block_max_finish(m, partials, counter, out);
}

void postprocess(Ctx& c, const double* rho, const double* T, double volfrac, double* rho_out,
                 double* level_out, double* volume_out) {
  const Dims& d = c.L[0];
  const int ne = (int)c.ne;
  set_density(c, rho, false);
  const double coef = c.p.penal * (c.p.k0 - c.p.kmin);
  if (c.dim == 2)
    k_elem_sens<2><<<blocks_for(ne), kThreads, 0, c.stream>>>(T, c.rho_phys, c.tmp_e, d, coef,
                                                              c.p.penal);
  else
    k_elem_sens<3><<<blocks_for(ne), kThreads, 0, c.stream>>>(T, c.rho_phys, c.tmp_e, d, coef,
                                                              c.p.penal);
  MGAR_LAUNCH_CHECK();
  const double r = c.p.rmin;
  const int reach = (int)std::ceil(r + 0.5);
  double* ns = c.tm;
  if (c.dim == 2)
    k_pp_nodal<2><<<blocks_for(c.n), kThreads, 0, c.stream>>>(c.tmp_e, ns, d, r, reach);
  else
    k_pp_nodal<3><<<blocks_for(c.n), kThreads, 0, c.stream>>>(c.tmp_e, ns, d, r, reach);
  MGAR_LAUNCH_CHECK();
  k_pp_max<<<c.grid_blocks, kThreads, 0, c.stream>>>(ns, (int)c.n, c.partials, c.counter,
                                                      c.dsc + S_TMP);
  MGAR_LAUNCH_CHECK();
  fetch_scalars(c, S_TMP, 1);
  auto volume = [&](double level, double* out) {
    if (c.dim == 2)
      k_pp_density<2><<<blocks_for(ne), kThreads, 0, c.stream>>>(ns, d, level, out, c.partials,
                                                                 c.counter, c.dsc + S_TMP);
    else
      k_pp_density<3><<<blocks_for(ne), kThreads, 0, c.stream>>>(ns, d, level, out, c.partials,
                                                                 c.counter, c.dsc + S_TMP);
    MGAR_LAUNCH_CHECK();
    fetch_scalars(c, S_TMP, 1);
    return c.hsc[S_TMP] / (double)ne;
  };
  // ns >= 0: below -1 every node is above the level (volume 1), at max(ns)
  // none is (volume 0)
  double lo = -1.0, hi = c.hsc[S_TMP];
  for (int step = 0; step < 200; ++step) {
    const double mid = 0.5 * (lo + hi);
    if (!(lo < mid && mid < hi)) break;
    if (volume(mid, nullptr) > volfrac) lo = mid;
    else hi = mid;
  }
  const double v = volume(hi, rho_out);
  if (level_out) *level_out = hi;
  if (volume_out) *volume_out = v;
}
}  // namespace mgar
