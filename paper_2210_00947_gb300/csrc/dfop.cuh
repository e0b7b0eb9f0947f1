// The df64 (double-float) matrix-free operator of the finest level in the
// difference form: K has zero row sums, so
//   (A x)_i = c * sum_j w_ij (x_i - x^_j),   x^_j = 0 on a fixed node,
// with w_ij = k_a + k_b for the face diagonals and k_e for the body diagonals
// of an H8 node (c = 1/12), w_ij = k_a + k_b along the edges and 2 k_e across
// the diagonals of a Q4 node (c = 1/6); a fixed row is the identity.  Each
// term's difference is exact (TwoSum) and each product exact (TwoProd), so a
// term is rounded relative to its own size, not relative to |x|; the terms
// are summed with their rounding errors gathered apart and one
// renormalisation at the end.  Shared by the single-design CG and the
// batched CG.
#pragma once

#include "common.cuh"
#include "df64.cuh"

namespace mgar {

struct DfOp {
  const float2* ke;
  const uint8_t* fixed;
  int ex, ey, ez, NX, NY, NZ, n;
  FastDiv fNX, fNXY;
  df scale;  // 1/6 (2D) or 1/12 (3D)
};

__device__ __forceinline__ df ld_kdf(const DfOp& op, int e, bool ok) {
  const int ee = (ok && CK(e, op.ex * op.ey * op.ez)) ? e : 0;
  const float2 v = op.ke[ee];
  return ok ? df{v.x, v.y} : df{0.f, 0.f};
}

// neighbour value x^_j (0 when fixed or off the grid; off-grid terms also
// have zero weight)
__device__ __forceinline__ df ld_xdf(const DfOp& op, const float2* __restrict__ x, int idx, bool ok) {
  const int j = (ok && CK(idx, op.n)) ? idx : 0;
  const float2 v = x[j];
  return (ok && !op.fixed[j]) ? df{v.x, v.y} : df{0.f, 0.f};
}

// (ah, al) += w * (xi - xj) with the pair left unnormalised: the difference
// formed exactly (TwoSum), the product's high part added by TwoSum and every
// rounding error gathered in al (the compensated dot product of Ogita, Rump
// and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005:
// as accurate as twice the working precision, with one renormalisation at
// the end instead of one per term).
__device__ __forceinline__ void df_acc_term(float& ah, float& al, df w, df xi, df xj) {
  float s, e;
  two_sum(xi.hi, -xj.hi, s, e);
  e = __fadd_rn(e, __fsub_rn(xi.lo, xj.lo));
  float p, pe;
  two_prod(w.hi, s, p, pe);
  pe = __fmaf_rn(w.hi, e, pe);
  pe = __fmaf_rn(w.lo, s, pe);
  float t, te;
  two_sum(ah, p, t, te);
  ah = t;
  al = __fadd_rn(al, __fadd_rn(te, pe));
}

// k_a + k_b as an unnormalised pair (df_acc_term multiplies both halves)
__device__ __forceinline__ df df_wsum(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return df{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}

// 2 k, exactly
__device__ __forceinline__ df df_twice(df a) { return df{2.f * a.hi, 2.f * a.lo}; }

__device__ __forceinline__ df df_row2(const DfOp& op, const float2* __restrict__ x, int i, int j) {
  const int idx = i + op.NX * j;
  const float2 xv = x[idx];
  const df xi{xv.x, xv.y};
  if (op.fixed[idx]) return xi;
  const bool xm = i > 0, xp = i < op.ex, ym = j > 0, yp = j < op.ey;
  const int e00 = (i - 1) + op.ex * (j - 1);
  const df k00 = ld_kdf(op, e00, xm && ym), k01 = ld_kdf(op, e00 + 1, xp && ym);
  const df k10 = ld_kdf(op, e00 + op.ex, xm && yp), k11 = ld_kdf(op, e00 + op.ex + 1, xp && yp);
  const int NX = op.NX;
  float ah = 0.f, al = 0.f;
  df_acc_term(ah, al, df_wsum(k00, k10), xi, ld_xdf(op, x, idx - 1, xm));
  df_acc_term(ah, al, df_wsum(k01, k11), xi, ld_xdf(op, x, idx + 1, xp));
  df_acc_term(ah, al, df_wsum(k00, k01), xi, ld_xdf(op, x, idx - NX, ym));
  df_acc_term(ah, al, df_wsum(k10, k11), xi, ld_xdf(op, x, idx + NX, yp));
  df_acc_term(ah, al, df_twice(k00), xi, ld_xdf(op, x, idx - NX - 1, xm && ym));
  df_acc_term(ah, al, df_twice(k01), xi, ld_xdf(op, x, idx - NX + 1, xp && ym));
  df_acc_term(ah, al, df_twice(k10), xi, ld_xdf(op, x, idx + NX - 1, xm && yp));
  df_acc_term(ah, al, df_twice(k11), xi, ld_xdf(op, x, idx + NX + 1, xp && yp));
  return df_mul(df_make(ah, al), op.scale);
}

__device__ __forceinline__ df df_row3(const DfOp& op, const float2* __restrict__ x, int i, int j, int k) {
  const int NX = op.NX, NXY = op.NX * op.NY;
  const int idx = i + NX * j + NXY * k;
  const float2 xv = x[idx];
  const df xi{xv.x, xv.y};
  if (op.fixed[idx]) return xi;
  const bool xm = i > 0, xp = i < op.ex, ym = j > 0, yp = j < op.ey, zm = k > 0, zp = k < op.ez;
  const int EX = op.ex, EXY = op.ex * op.ey;
  const int e000 = (i - 1) + EX * (j - 1) + EXY * (k - 1);
  const df k000 = ld_kdf(op, e000, xm && ym && zm);
  const df k001 = ld_kdf(op, e000 + 1, xp && ym && zm);
  const df k010 = ld_kdf(op, e000 + EX, xm && yp && zm);
  const df k011 = ld_kdf(op, e000 + EX + 1, xp && yp && zm);
  const df k100 = ld_kdf(op, e000 + EXY, xm && ym && zp);
  const df k101 = ld_kdf(op, e000 + EXY + 1, xp && ym && zp);
  const df k110 = ld_kdf(op, e000 + EXY + EX, xm && yp && zp);
  const df k111 = ld_kdf(op, e000 + EXY + EX + 1, xp && yp && zp);
  float ah = 0.f, al = 0.f;
  // face diagonals in the xy, xz and yz planes (two elements each)
  df_acc_term(ah, al, df_wsum(k000, k100), xi, ld_xdf(op, x, idx - 1 - NX, xm && ym));
  df_acc_term(ah, al, df_wsum(k001, k101), xi, ld_xdf(op, x, idx + 1 - NX, xp && ym));
  df_acc_term(ah, al, df_wsum(k010, k110), xi, ld_xdf(op, x, idx - 1 + NX, xm && yp));
  df_acc_term(ah, al, df_wsum(k011, k111), xi, ld_xdf(op, x, idx + 1 + NX, xp && yp));
  df_acc_term(ah, al, df_wsum(k000, k010), xi, ld_xdf(op, x, idx - 1 - NXY, xm && zm));
  df_acc_term(ah, al, df_wsum(k001, k011), xi, ld_xdf(op, x, idx + 1 - NXY, xp && zm));
  df_acc_term(ah, al, df_wsum(k100, k110), xi, ld_xdf(op, x, idx - 1 + NXY, xm && zp));
  df_acc_term(ah, al, df_wsum(k101, k111), xi, ld_xdf(op, x, idx + 1 + NXY, xp && zp));
  df_acc_term(ah, al, df_wsum(k000, k001), xi, ld_xdf(op, x, idx - NX - NXY, ym && zm));
  df_acc_term(ah, al, df_wsum(k010, k011), xi, ld_xdf(op, x, idx + NX - NXY, yp && zm));
  df_acc_term(ah, al, df_wsum(k100, k101), xi, ld_xdf(op, x, idx - NX + NXY, ym && zp));
  df_acc_term(ah, al, df_wsum(k110, k111), xi, ld_xdf(op, x, idx + NX + NXY, yp && zp));
  // body diagonals (one element each)
  df_acc_term(ah, al, k000, xi, ld_xdf(op, x, idx - 1 - NX - NXY, xm && ym && zm));
  df_acc_term(ah, al, k001, xi, ld_xdf(op, x, idx + 1 - NX - NXY, xp && ym && zm));
  df_acc_term(ah, al, k010, xi, ld_xdf(op, x, idx - 1 + NX - NXY, xm && yp && zm));
  df_acc_term(ah, al, k011, xi, ld_xdf(op, x, idx + 1 + NX - NXY, xp && yp && zm));
  df_acc_term(ah, al, k100, xi, ld_xdf(op, x, idx - 1 - NX + NXY, xm && ym && zp));
  df_acc_term(ah, al, k101, xi, ld_xdf(op, x, idx + 1 - NX + NXY, xp && ym && zp));
  df_acc_term(ah, al, k110, xi, ld_xdf(op, x, idx - 1 + NX + NXY, xm && yp && zp));
  df_acc_term(ah, al, k111, xi, ld_xdf(op, x, idx + 1 + NX + NXY, xp && yp && zp));
  return df_mul(df_make(ah, al), op.scale);
}

template <int DIM>
__device__ __forceinline__ df df_row(const DfOp& op, const float2* __restrict__ x, int idx) {
  int i, j, k;
  coords(idx, op.fNX, op.fNXY, i, j, k);
  return DIM == 2 ? df_row2(op, x, i, j) : df_row3(op, x, i, j, k);
}

__device__ __forceinline__ float2 pack(df a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ df unpack(float2 v) { return df{v.x, v.y}; }

// The operator of a handle's finest level at its current design.
inline DfOp make_op(Ctx& c) {
  const Dims& d = c.L[0];
  DfOp op;
  op.ke = c.ke_df;
  op.fixed = c.fixed;
  op.ex = d.ex;
  op.ey = d.ey;
  op.ez = d.ez;
  op.NX = d.NX;
  op.NY = d.NY;
  op.NZ = d.NZ;
  op.n = (int)d.n;
  op.fNX = d.fNX;
  op.fNXY = d.fNXY;
  op.scale = df_from_double(c.dim == 2 ? 1.0 / 6.0 : 1.0 / 12.0);
  return op;
}

}  // namespace mgar
