// Tiled double-float (df64) finest-level operator for 3D (H8) grids, used
// by the outer CG of the mixed path (Sections 1 and 3.2).
//
// Same z-marching tile as the V-cycle's finest-level kernels: a TX x TY
// block (43 x 11 on 129-node planes, else 32 x 8) walks a run of node
// planes, the operand planes (float2 hi/lo pairs, zero on fixed nodes and
// off the grid) and element-conductivity layers rotate in shared memory,
// and the loads of plane k+2 are in flight while plane k is computed.  The
// product and direction forms use the element form of the conductivity
// stencil:
//   (A x)_i = (1/12) (4 x_i sum_e k_e - sum_e k_e f_e),
// summed over the 8 elements e around node i, where f_e is the sum of the
// operand x^ over the four nodes of e that are not edge neighbours of i
// (three face diagonals and the body diagonal); a fixed row is the
// identity.  4 sum_e k_e is a per-node input computed once per design
// (k_node_kdiag).  Each f_e is a TwoSum chain of the (hi, lo) pairs, each
// k_e f_e is a TwoProd with its cross terms, and the products are summed
// with TwoSum into two unnormalised (hi, lo) accumulators (elements below
// and above the node's plane, for instruction-level parallelism).  Rounding
// errors are of order 2^-47 |x| sum_e k_e (those of the FP64 operator, which
// sums the same terms, are of order 2^-53 |x| sum_e k_e); the form needs
// about a third fewer FP32 operations than the difference form below.
//
// The residual form keeps the difference form of the stencil,
//   (A x)_i = (1/12) sum_j w_ij (x_i - x^_j)
// (w_ij = k_a + k_b over the 12 face diagonals, k_e over the 8 body
// diagonals), each difference formed exactly, so its rounding is relative to
// the differences and not to |x|: a residual recomputed from x keeps its
// accuracy far below 2^-47 ||A|| ||x||, which the reliable updates of the CG
// need when they drive ||r|| / ||q|| to 1e-11.
//
// Three fused forms:
//   APPLY : y = A x with FP64 x and y (the MGAR projection; converted on
//           load and store)                       [x . y]
//   DIR   : p = z + beta p_old, y = A p           [p . y]   (CG direction update + product)
//   RESID : r = q - A x, r32 = fl32(r)            [r . r]   (r optional)
// p is written to a buffer other than p_old, because neighbouring blocks
// still read p_old.
#include "common.cuh"
#include "tile3d.cuh"
#include "df64.cuh"

namespace mgar {
namespace d3d {
using namespace tile;

enum Mode { APPLY = 0, DIR = 1, RESID = 2 };

struct DfArgs {
  int ex, ey, ez, NX, NY, NZ, gz;
  const uint8_t* fixed;
  const float2* ke;
  const float2* kd;     // per node: 4 sum_e k_e (df64)
  const float2* x;      // RESID: operand; DIR: p_old (unused when first)
  const double* x64;    // APPLY: operand
  double* y64;          // APPLY: A x
  const float* z;       // DIR
  const float2* q;      // RESID
  const double* rz_new; // DIR: beta = rz_new / rz_old
  const double* rz_old;
  int first;            // DIR: p = z
  float2* y;            // APPLY/DIR: A x; RESID: r
  float2* p;            // DIR: new direction
  float* r32;           // RESID
  double* partials;
  unsigned int* counter;
  double* out;          // dot product (may be null for APPLY)
  // DIR inside the device-side CG loop: with parity odd, p_old is x_alt and
  // the new p goes to p_alt (the two direction buffers swap each iteration);
  // rz_set, when given, receives rz_new once every block has read it
  const float2* x_alt;
  float2* p_alt;
  const double* parity;
  double* rz_set;
};

template <int MODE>
struct NodeFetch {
  float2 v = make_float2(0.f, 0.f);  // x, or p_old
  float zf = 0.f;                    // DIR: z
  double xd = 0.0;                   // APPLY: x
  uint8_t f = 1;
  bool on = false;
  // col: clamped i + NX * clamped j; con: (i, j) inside the grid
  // xsrc: the operand (RESID) or p_old (DIR)
  __device__ __forceinline__ void issue(const DfArgs& a, const float2* xsrc, int col, bool con, int k) {
    on = con && k >= 0 && k < a.NZ;
    const int idx = col + a.NX * a.NY * min(max(k, 0), a.NZ - 1);
    if (!CK(idx, (int64_t)a.NX * a.NY * a.NZ)) return;
    f = a.fixed[idx];
    if (MODE == DIR) {
      zf = a.z[idx];
      if (!a.first) v = xsrc[idx];
    } else if (MODE == APPLY) {
      xd = a.x64[idx];
    } else {
      v = xsrc[idx];
    }
  }
  __device__ __forceinline__ df value(df beta) const {
    if (MODE == DIR) return df_add(df{zf, 0.f}, df_mul(beta, df{v.x, v.y}));
    if (MODE == APPLY) return df_from_double(xd);
    return df{v.x, v.y};
  }
};

__device__ __forceinline__ df dfk(float2 v) { return df{v.x, v.y}; }

// acc (unnormalised hi, lo) += w * (xi - xj), the difference formed exactly
__device__ __forceinline__ void acc_term(float& ah, float& al, df w, float2 xi, float2 xj) {
  float s, e;
  two_sum(xi.x, -xj.x, s, e);
  e = __fadd_rn(e, __fsub_rn(xi.y, xj.y));
  float p, pe;
  two_prod(w.hi, s, p, pe);
  pe = __fmaf_rn(w.hi, e, pe);
  pe = __fmaf_rn(w.lo, s, pe);
  float t, te;
  two_sum(ah, p, t, te);
  ah = t;
  al = __fadd_rn(al, __fadd_rn(te, pe));
}

// k_a + k_b as an unnormalised pair (acc_term multiplies both halves)
__device__ __forceinline__ df wsum(df a, df b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return df{s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}

// a + b + c + d as an unnormalised (hi, lo) pair: TwoSum chain of the high
// words, low words and rounding errors added in FP32
__device__ __forceinline__ df far4(float2 a, float2 b, float2 c, float2 d) {
  float s, e, t;
  two_sum(a.x, b.x, s, e);
  t = __fadd_rn(e, __fadd_rn(a.y, b.y));
  two_sum(s, c.x, s, e);
  t = __fadd_rn(t, __fadd_rn(e, c.y));
  two_sum(s, d.x, s, e);
  t = __fadd_rn(t, __fadd_rn(e, d.y));
  return df{s, t};
}

// acc (unnormalised hi, lo) = k * f
__device__ __forceinline__ void acc_kf_first(float& ah, float& al, df k, df f) {
  two_prod(k.hi, f.hi, ah, al);
  al = __fmaf_rn(k.hi, f.lo, al);
  al = __fmaf_rn(k.lo, f.hi, al);
}

// acc (unnormalised hi, lo) += k * f
__device__ __forceinline__ void acc_kf(float& ah, float& al, df k, df f) {
  float p, pe;
  two_prod(k.hi, f.hi, p, pe);
  pe = __fmaf_rn(k.hi, f.lo, pe);
  pe = __fmaf_rn(k.lo, f.hi, pe);
  float t, te;
  two_sum(ah, p, t, te);
  ah = t;
  al = __fadd_rn(al, __fadd_rn(te, pe));
}

// Plane p and element layer p live in slot (p - kb + 1) & 3; the z loop is
// unrolled by four, so every slot index is a compile-time constant and the
// centre values of the planes in flight stay in registers.
template <int MODE, class T>
__global__ void __launch_bounds__(T::NTB, T::NT <= 256 ? 4 : 2) k_df3d(DfArgs a) {
  constexpr int TX = T::TX, TY = T::TY, NT = T::NT;
  constexpr int XRING = T::XRING, KRING = T::KRING, KRING0 = T::KRING0;
  __shared__ float2 X[4][TY + 2][TX + 2];
  __shared__ float2 K[4][TY + 1][TX + 1];
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
  const bool mine = real && i < a.NX && j < a.NY;
  const bool xr = tid < XRING, kr = tid >= KRING0 && tid < KRING0 + KRING;
  int rxh = 0, ryh = 0, kxh = 0, kyh = 0;
  if (xr) T::xring(tid, rxh, ryh);
  if (kr) T::kring(tid - KRING0, kxh, kyh);
  df beta{0.f, 0.f};
  if (MODE == DIR) {
    const df q = block_div_df(a.rz_new, a.rz_old);  // once per block
    if (!a.first) beta = q;
  }
  const bool odd = MODE == DIR && a.parity && (((int)*a.parity) & 1);
  const float2* const xsrc = odd ? a.x_alt : a.x;
  float2* const pdst = odd ? a.p_alt : a.p;
  const int NXY = a.NX * a.NY;

  // per-thread column offsets (plane-independent)
  const int ocol = min(i, a.NX - 1) + a.NX * min(j, a.NY - 1);
  const int ri = i0 - 1 + rxh, rj = j0 - 1 + ryh;
  const bool ron = ri >= 0 && ri < a.NX && rj >= 0 && rj < a.NY;
  const int rcol = min(max(ri, 0), a.NX - 1) + a.NX * min(max(rj, 0), a.NY - 1);
  const bool keon = i < a.ex && j < a.ey;
  const int kebase = min(i, a.ex - 1) + a.ex * min(j, a.ey - 1);
  const int ki = i0 - 1 + kxh, kj = j0 - 1 + kyh;
  const bool kron = ki >= 0 && ki < a.ex && kj >= 0 && kj < a.ey;
  const int krbase = min(max(ki, 0), a.ex - 1) + a.ex * min(max(kj, 0), a.ey - 1);
  const int EXY = a.ex * a.ey;

  NodeFetch<MODE> own, ring;
  float2 kown = make_float2(0.f, 0.f), kring_v = make_float2(0.f, 0.f);
  bool kown_on = false, kring_on = false;
  float2 ownq = make_float2(0.f, 0.f), ownkd = make_float2(0.f, 0.f);
  float2 cv[4], cq[4], ckd[4];
  bool cf[4];
  df dot{0.f, 0.f};

  auto issue_plane_to = [&](int p, NodeFetch<MODE>& o, NodeFetch<MODE>& rg, float2& oq, float2& okd) {
    o.issue(a, xsrc, ocol, mine, p);
    {
      const int idx = ocol + NXY * min(max(p, 0), a.NZ - 1);
      if (CK(idx, (int64_t)NXY * a.NZ)) {
        if (MODE != RESID) okd = a.kd[idx];
        if (MODE == RESID) oq = a.q[idx];
      }
    }
    if (xr) rg.issue(a, xsrc, rcol, ron, p);
  };
  auto issue_plane = [&](int p) { issue_plane_to(p, own, ring, ownq, ownkd); };
  auto issue_layer = [&](int l) {
    const int lc = EXY * min(max(l, 0), a.ez - 1);
    const bool lon = l >= 0 && l < a.ez;
    kown_on = keon && lon;
    if (CK(kebase + lc, (int64_t)EXY * a.ez)) kown = a.ke[kebase + lc];
    if (kr) {
      kring_on = kron && lon;
      if (CK(krbase + lc, (int64_t)EXY * a.ez)) kring_v = a.ke[krbase + lc];
    }
  };

#define D3D_FINISH_FROM(S, P, O, RG, OQ, OKD)                                              \
  {                                                                                        \
    const df v = O.value(beta);                                                            \
    const float2 v2 = make_float2(v.hi, v.lo);                                             \
    if (real) X[S][ty + 1][tx + 1] = (O.on && !O.f) ? v2 : make_float2(0.f, 0.f);          \
    cv[S] = v2;                                                                            \
    cf[S] = O.f != 0;                                                                      \
    cq[S] = OQ;                                                                            \
    ckd[S] = OKD;                                                                          \
    if (MODE == DIR && mine && (P) >= kb && (P) < kend) pdst[ocol + NXY * (P)] = v2;       \
    if (xr) {                                                                              \
      const df w = RG.value(beta);                                                         \
      X[S][ryh][rxh] = (RG.on && !RG.f) ? make_float2(w.hi, w.lo) : make_float2(0.f, 0.f); \
    }                                                                                      \
  }
#define D3D_FINISH(S, P) D3D_FINISH_FROM(S, P, own, ring, ownq, ownkd)
#define D3D_FINISH_LAYER(S)                                                                \
  {                                                                                        \
    if (real) K[S][ty + 1][tx + 1] = kown_on ? kown : make_float2(0.f, 0.f);               \
    if (kr) K[S][kyh][kxh] = kring_on ? kring_v : make_float2(0.f, 0.f);                   \
  }

  // prologue: planes kb-1 and kb and layer kb-1, their loads in flight together
  {
    NodeFetch<MODE> own2, ring2;
    float2 ownq2 = make_float2(0.f, 0.f), ownkd2 = make_float2(0.f, 0.f);
    issue_plane(kb - 1);
    issue_plane_to(kb, own2, ring2, ownq2, ownkd2);
    issue_layer(kb - 1);
    D3D_FINISH(0, kb - 1);
    D3D_FINISH_FROM(1, kb, own2, ring2, ownq2, ownkd2);
    D3D_FINISH_LAYER(0);
  }
  issue_plane(kb + 1);
  issue_layer(kb);

  const df scale = df_from_double(1.0 / 12.0);
#define D3D_STEP(S)                                                                        \
  {                                                                                        \
    constexpr int S0 = (S) & 3, S1 = ((S) + 1) & 3, S2 = ((S) + 2) & 3;                    \
    const int k = kk + (S);                                                                \
    if (k >= kend) break;                                                                  \
    D3D_FINISH(S2, k + 1);                                                                 \
    D3D_FINISH_LAYER(S1);                                                                  \
    issue_plane(k + 2);                                                                    \
    issue_layer(k + 1);                                                                    \
    __syncthreads();                                                                       \
    if (mine) {                                                                            \
      const int idx = ocol + NXY * k;                                                      \
      const float2 xi = cv[S1];                                                            \
      df yv;                                                                               \
      if (cf[S1]) {                                                                        \
        yv = dfk(xi);                                                                      \
      } else {                                                                             \
        const int cx = tx + 1, cy = ty + 1;                                                \
        const df k000 = dfk(K[S0][ty][tx]), k001 = dfk(K[S0][ty][tx + 1]),                 \
                 k010 = dfk(K[S0][ty + 1][tx]), k011 = dfk(K[S0][ty + 1][tx + 1]);         \
        const df k100 = dfk(K[S1][ty][tx]), k101 = dfk(K[S1][ty][tx + 1]),                 \
                 k110 = dfk(K[S1][ty + 1][tx]), k111 = dfk(K[S1][ty + 1][tx + 1]);         \
        if (MODE == RESID) {                                                               \
          /* difference form: each term rounded relative to its own size */               \
          float ah = 0.f, al = 0.f;                                                        \
          acc_term(ah, al, wsum(k000, k100), xi, X[S1][cy - 1][cx - 1]);                 \
          acc_term(ah, al, wsum(k001, k101), xi, X[S1][cy - 1][cx + 1]);                 \
          acc_term(ah, al, wsum(k010, k110), xi, X[S1][cy + 1][cx - 1]);                 \
          acc_term(ah, al, wsum(k011, k111), xi, X[S1][cy + 1][cx + 1]);                 \
          acc_term(ah, al, wsum(k000, k010), xi, X[S0][cy][cx - 1]);                     \
          acc_term(ah, al, wsum(k001, k011), xi, X[S0][cy][cx + 1]);                     \
          acc_term(ah, al, wsum(k100, k110), xi, X[S2][cy][cx - 1]);                     \
          acc_term(ah, al, wsum(k101, k111), xi, X[S2][cy][cx + 1]);                     \
          acc_term(ah, al, wsum(k000, k001), xi, X[S0][cy - 1][cx]);                     \
          acc_term(ah, al, wsum(k010, k011), xi, X[S0][cy + 1][cx]);                     \
          acc_term(ah, al, wsum(k100, k101), xi, X[S2][cy - 1][cx]);                     \
          acc_term(ah, al, wsum(k110, k111), xi, X[S2][cy + 1][cx]);                     \
          acc_term(ah, al, k000, xi, X[S0][cy - 1][cx - 1]);                               \
          acc_term(ah, al, k001, xi, X[S0][cy - 1][cx + 1]);                               \
          acc_term(ah, al, k010, xi, X[S0][cy + 1][cx - 1]);                               \
          acc_term(ah, al, k011, xi, X[S0][cy + 1][cx + 1]);                               \
          acc_term(ah, al, k100, xi, X[S2][cy - 1][cx - 1]);                               \
          acc_term(ah, al, k101, xi, X[S2][cy - 1][cx + 1]);                               \
          acc_term(ah, al, k110, xi, X[S2][cy + 1][cx - 1]);                               \
          acc_term(ah, al, k111, xi, X[S2][cy + 1][cx + 1]);                               \
          yv = df_mul(df_make(ah, al), scale);                                             \
        } else {                                                                           \
          /* f_e: in-plane face diagonal, two out-of-plane face diagonals, body diagonal */\
          const df f000 = far4(X[S1][cy - 1][cx - 1], X[S0][cy][cx - 1], X[S0][cy - 1][cx],\
                               X[S0][cy - 1][cx - 1]);                                     \
          const df f001 = far4(X[S1][cy - 1][cx + 1], X[S0][cy][cx + 1], X[S0][cy - 1][cx],\
                               X[S0][cy - 1][cx + 1]);                                     \
          const df f010 = far4(X[S1][cy + 1][cx - 1], X[S0][cy][cx - 1], X[S0][cy + 1][cx],\
                               X[S0][cy + 1][cx - 1]);                                     \
          const df f011 = far4(X[S1][cy + 1][cx + 1], X[S0][cy][cx + 1], X[S0][cy + 1][cx],\
                               X[S0][cy + 1][cx + 1]);                                     \
          const df f100 = far4(X[S1][cy - 1][cx - 1], X[S2][cy][cx - 1], X[S2][cy - 1][cx],\
                               X[S2][cy - 1][cx - 1]);                                     \
          const df f101 = far4(X[S1][cy - 1][cx + 1], X[S2][cy][cx + 1], X[S2][cy - 1][cx],\
                               X[S2][cy - 1][cx + 1]);                                     \
          const df f110 = far4(X[S1][cy + 1][cx - 1], X[S2][cy][cx - 1], X[S2][cy + 1][cx],\
                               X[S2][cy + 1][cx - 1]);                                     \
          const df f111 = far4(X[S1][cy + 1][cx + 1], X[S2][cy][cx + 1], X[S2][cy + 1][cx],\
                               X[S2][cy + 1][cx + 1]);                                     \
          /* two independent accumulators (elements below and above the plane) */          \
          float ah, al, bh, bl;                                                            \
          acc_kf_first(ah, al, k000, f000);                                                \
          acc_kf_first(bh, bl, k100, f100);                                                \
          acc_kf(ah, al, k001, f001);                                                      \
          acc_kf(bh, bl, k101, f101);                                                      \
          acc_kf(ah, al, k010, f010);                                                      \
          acc_kf(bh, bl, k110, f110);                                                      \
          acc_kf(ah, al, k011, f011);                                                      \
          acc_kf(bh, bl, k111, f111);                                                      \
          float sh, se;                                                                    \
          two_sum(ah, bh, sh, se);                                                         \
          const df acc = df_make(sh, __fadd_rn(se, __fadd_rn(al, bl)));                    \
          const df diag = df_mul(dfk(ckd[S1]), dfk(xi));                                   \
          yv = df_mul(df_sub(diag, acc), scale);                                           \
        }                                                                                  \
      }                                                                                    \
      if (MODE == RESID) {                                                                 \
        const df ri = df_sub(dfk(cq[S1]), yv);                                             \
        if (a.y) a.y[idx] = make_float2(ri.hi, ri.lo);                                     \
        a.r32[idx] = __fadd_rn(ri.hi, ri.lo);                                              \
        dot = df_add(dot, df_mul(ri, ri));                                                 \
      } else if (MODE == APPLY) {                                                          \
        a.y64[idx] = df_to_double(yv);                                                     \
        if (a.out) dot = df_add(dot, df_mul(dfk(xi), yv));                                 \
      } else {                                                                             \
        a.y[idx] = make_float2(yv.hi, yv.lo);                                              \
        dot = df_add(dot, df_mul(dfk(xi), yv));                                            \
      }                                                                                    \
    }                                                                                      \
  }

  for (int kk = kb; kk < kend; kk += 4) {
    D3D_STEP(0)
    D3D_STEP(1)
    D3D_STEP(2)
    D3D_STEP(3)
  }
#undef D3D_STEP
#undef D3D_FINISH
#undef D3D_FINISH_FROM
#undef D3D_FINISH_LAYER
  if (a.out) {
    double t;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    if (block_sum_last_df(dot, a.partials, a.counter, t, tid, T::NTB, bid, nb) && tid == 0) {
      a.out[0] = t;
      if (MODE == DIR && a.rz_set) *a.rz_set = *a.rz_new;  // every block has read rz_new
    }
  }
}

template <int MODE, class T>
int runs_for(const Dims& d, int sms) {
  int per_sm = 0;
  MGAR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_df3d<MODE, T>, T::NTB, 0));
  per_sm = std::max(per_sm, 1);
  const int64_t cols = (int64_t)((d.NX + T::TX - 1) / T::TX) * ((d.NY + T::TY - 1) / T::TY);
  const int64_t want = (int64_t)per_sm * sms;
  int64_t gz = std::max<int64_t>(1, (want + cols / 2) / cols);
  gz = std::min<int64_t>(gz, d.NZ);
  // the reduction keeps one partial per block
  gz = std::min<int64_t>(gz, std::max<int64_t>(1, kMinPartialBlocks / cols));
  return (int)gz;
}

DfArgs base_args(Ctx& c) {
  const Dims& d = c.L[0];
  DfArgs a{};
  a.ex = d.ex;
  a.ey = d.ey;
  a.ez = d.ez;
  a.NX = d.NX;
  a.NY = d.NY;
  a.NZ = d.NZ;
  a.fixed = c.fixed;
  a.ke = c.ke_df;
  a.kd = c.kd_df;
  a.partials = c.partials;
  a.counter = c.counter;
  return a;
}

template <int MODE, class T>
void launch_t(Ctx& c, DfArgs& a) {
  const Dims& d = c.L[0];
  a.gz = std::max(1, std::min(c.df3d_gz[MODE], d.NZ));
  const dim3 grid((d.NX + T::TX - 1) / T::TX, (d.NY + T::TY - 1) / T::TY, a.gz);
  launch_pdl(c.stream, c.use_pdl, k_df3d<MODE, T>, grid, dim3(T::NTB), a);
  MGAR_LAUNCH_CHECK();
}

template <int MODE>
void launch(Ctx& c, DfArgs& a) {
  if (c.df3d_tile) launch_t<MODE, T43x11>(c, a);
  else launch_t<MODE, T32x8>(c, a);
}

template <int MODE>
int runs(const Ctx& c, int sms) {
  return c.df3d_tile ? runs_for<MODE, T43x11>(c.L[0], sms) : runs_for<MODE, T32x8>(c.L[0], sms);
}

// kd_i = 4 sum_e k_e over the (up to 8) elements around node i, df64: a
// TwoSum chain of the high words, low words and errors added, then
// normalised; the factor 4 is exact
__global__ void k_node_kdiag(const float2* __restrict__ ke, float2* __restrict__ kd, int ex, int ey,
                             int ez) {
  const int NX = ex + 1, NY = ey + 1, NZ = ez + 1;
  const int64_t n = (int64_t)NX * NY * NZ;
  const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= n) return;
  const int i = (int)(id % NX), j = (int)((id / NX) % NY), k = (int)(id / ((int64_t)NX * NY));
  float s = 0.f, t = 0.f;
  for (int dz = -1; dz <= 0; ++dz)
    for (int dy = -1; dy <= 0; ++dy)
      for (int dx = -1; dx <= 0; ++dx) {
        const int e0 = i + dx, e1 = j + dy, e2 = k + dz;
        if (e0 < 0 || e0 >= ex || e1 < 0 || e1 >= ey || e2 < 0 || e2 >= ez) continue;
        const float2 v = ke[e0 + (int64_t)ex * (e1 + (int64_t)ey * e2)];
        float r;
        two_sum(s, v.x, s, r);
        t = __fadd_rn(t, __fadd_rn(r, v.y));
      }
  const df d = df_make(s, t);
  kd[id] = make_float2(4.f * d.hi, 4.f * d.lo);
}

}  // namespace d3d

// per-node diagonal factor of the df64 operator for the current k_e
void df3d_node_diag(Ctx& c) {
  const Dims& d = c.L[0];
  d3d::k_node_kdiag<<<blocks_for(d.n), kThreads, 0, c.stream>>>(c.ke_df, c.kd_df, d.ex, d.ey, d.ez);
  MGAR_LAUNCH_CHECK();
}

void df3d_prepare(Ctx& c) {
  using namespace d3d;
  int dev = 0, sms = 0;
  MGAR_CUDA(cudaGetDevice(&dev));
  MGAR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const Dims& d = c.L[0];
  c.df3d_tile = tile_use(d.NX, d.NY, T43x11::TX, T43x11::TY) > tile_use(d.NX, d.NY, T32x8::TX, T32x8::TY);
  c.df3d_gz[APPLY] = runs<APPLY>(c, sms);
  c.df3d_gz[DIR] = runs<DIR>(c, sms);
  c.df3d_gz[RESID] = runs<RESID>(c, sms);
}

// y = A x for FP64 x, y; x . y into *dot when given
void df3d_apply(Ctx& c, const double* x, double* y, double* dot) {
  using namespace d3d;
  DfArgs a = base_args(c);
  a.x64 = x;
  a.y64 = y;
  a.out = dot;
  launch<APPLY>(c, a);
}

// p = z + (rz_new / rz_old) p_old (p = z when first), y = A p, p . y into *dot
void df3d_dir(Ctx& c, const float* z, const float2* p_old, float2* p, const double* rz_new,
              const double* rz_old, bool first, float2* y, double* dot, const double* parity,
              double* rz_set) {
  using namespace d3d;
  DfArgs a = base_args(c);
  a.z = z;
  a.x = p_old;
  a.p = p;
  a.x_alt = p;        // odd parity: the buffers swap roles
  a.p_alt = const_cast<float2*>(p_old);
  a.parity = parity;
  a.rz_set = rz_set;
  a.rz_new = rz_new;
  a.rz_old = rz_old;
  a.first = first ? 1 : 0;
  a.y = y;
  a.out = dot;
  launch<DIR>(c, a);
}

// r = q - A x, r32 = fl32(r), r . r into *rr
void df3d_resid(Ctx& c, const float2* q, const float2* x, float2* r, float* r32, double* rr) {
  using namespace d3d;
  DfArgs a = base_args(c);
  a.q = q;
  a.x = x;
  a.y = r;
  a.r32 = r32;
  a.out = rr;
  launch<RESID>(c, a);
}

}  // namespace mgar
