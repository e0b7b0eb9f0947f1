// Tiled double-float (df64) finest-level operator for 3D (H8) grids, used
// by the outer CG of the mixed path (Sections 1 and 3.2).
//
// Same z-marching tile as the V-cycle's finest-level kernels: a 32 x 8 block
// walks a run of node planes, the operand planes (float2 hi/lo pairs, zero on
// fixed nodes and off the grid) and element-conductivity layers rotate in
// shared memory, and the loads of plane k+2 are in flight while plane k is
// computed.  The product uses the difference form of the conductivity
// stencil (K has zero row sums):
//   (A x)_i = (1/12) sum_j w_ij (x_i - x^_j),
// w_ij = k_a + k_b over the 12 face diagonals and k_e over the 8 body
// diagonals; a fixed row is the identity.  Each difference x_i - x^_j is
// formed exactly (TwoSum of the high parts), multiplied by w_ij with TwoProd
// and summed with TwoSum into an unnormalised (hi, lo) accumulator, so every
// term is rounded relative to its own size.
//
// Three fused forms:
//   APPLY : y = A x                              [x . y]
//   DIR   : p = z + beta p_old, y = A p           [p . y]   (CG direction update + product)
//   RESID : r = q - A x, r32 = fl32(r)            [r . r]
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
  const float2* x;      // APPLY/RESID: operand; DIR: p_old (unused when first)
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
};

__device__ __forceinline__ df ld2(const float2* a, int i) {
  const float2 v = a[i];
  return df{v.x, v.y};
}

template <int MODE>
struct NodeFetch {
  float2 v = make_float2(0.f, 0.f);  // x, or p_old
  float zf = 0.f;                    // DIR: z
  uint8_t f = 1;
  bool on = false;
  __device__ __forceinline__ void issue(const DfArgs& a, int i, int j, int k) {
    on = i >= 0 && i < a.NX && j >= 0 && j < a.NY && k >= 0 && k < a.NZ;
    const int idx = min(max(i, 0), a.NX - 1) + a.NX * (min(max(j, 0), a.NY - 1) + a.NY * min(max(k, 0), a.NZ - 1));
    if (!CK(idx, (int64_t)a.NX * a.NY * a.NZ)) return;
    f = a.fixed[idx];
    if (MODE == DIR) {
      zf = a.z[idx];
      if (!a.first) v = a.x[idx];
    } else {
      v = a.x[idx];
    }
  }
  __device__ __forceinline__ df value(df beta) const {
    if (MODE == DIR) return df_add(df{zf, 0.f}, df_mul(beta, df{v.x, v.y}));
    return df{v.x, v.y};
  }
};

// acc (unnormalised hi, lo) += w * (xi - xj)
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

template <int MODE>
__global__ void __launch_bounds__(NT, 4) k_df3d(DfArgs a) {
  __shared__ float2 X[XS][TY + 2][TX + 2];
  __shared__ float2 K[KS][TY + 1][TX + 1];
  __shared__ float2 Cx[XS][TY][TX];  // centre operand, unmasked
  __shared__ uint8_t Cf[XS][TY][TX];

  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int kb = (int)(((int64_t)blockIdx.z * a.NZ) / a.gz);
  const int kend = (int)(((int64_t)(blockIdx.z + 1) * a.NZ) / a.gz);
  const int i = i0 + tx, j = j0 + ty;
  const bool mine = i < a.NX && j < a.NY;
  const bool xr = tid < XRING, kr = tid >= KRING0 && tid < KRING0 + KRING;
  int rxh = 0, ryh = 0, kxh = 0, kyh = 0;
  if (xr) xring(tid, rxh, ryh);
  if (kr) kring(tid - KRING0, kxh, kyh);
  df beta{0.f, 0.f};
  if (MODE == DIR && !a.first) beta = df_from_double(*a.rz_new / *a.rz_old);

  NodeFetch<MODE> own, ring;
  float2 kown = make_float2(0.f, 0.f), kring_v = make_float2(0.f, 0.f);
  bool kown_on = false, kring_on = false;
  df dot{0.f, 0.f};

  auto issue_plane = [&](int p) {
    own.issue(a, i, j, p);
    if (xr) ring.issue(a, i0 - 1 + rxh, j0 - 1 + ryh, p);
  };
  auto finish_plane = [&](int p) {
    const int s = (p + XS) % XS;
    const df v = own.value(beta);
    const float2 v2 = make_float2(v.hi, v.lo);
    X[s][ty + 1][tx + 1] = (own.on && !own.f) ? v2 : make_float2(0.f, 0.f);
    Cx[s][ty][tx] = v2;
    Cf[s][ty][tx] = own.f;
    if (MODE == DIR && mine && p >= kb && p < kend) {
      const int idx = i + a.NX * (j + a.NY * p);
      a.p[idx] = v2;
    }
    if (xr) {
      const df w = ring.value(beta);
      X[s][ryh][rxh] = (ring.on && !ring.f) ? make_float2(w.hi, w.lo) : make_float2(0.f, 0.f);
    }
  };
  auto issue_elem = [&](int e, int f, int l, float2& v, bool& on) {
    on = e >= 0 && e < a.ex && f >= 0 && f < a.ey && l >= 0 && l < a.ez;
    const int idx = min(max(e, 0), a.ex - 1) + a.ex * (min(max(f, 0), a.ey - 1) + a.ey * min(max(l, 0), a.ez - 1));
    if (CK(idx, (int64_t)a.ex * a.ey * a.ez)) v = a.ke[idx];
  };
  auto issue_layer = [&](int l) {
    issue_elem(i, j, l, kown, kown_on);
    if (kr) issue_elem(i0 - 1 + kxh, j0 - 1 + kyh, l, kring_v, kring_on);
  };
  auto finish_layer = [&](int l) {
    const int s = (l + KS) % KS;
    K[s][ty + 1][tx + 1] = kown_on ? kown : make_float2(0.f, 0.f);
    if (kr) K[s][kyh][kxh] = kring_on ? kring_v : make_float2(0.f, 0.f);
  };

  issue_plane(kb - 1);
  finish_plane(kb - 1);
  issue_plane(kb);
  issue_layer(kb - 1);
  finish_plane(kb);
  finish_layer(kb - 1);
  issue_plane(kb + 1);
  issue_layer(kb);

  const df scale = df_from_double(1.0 / 12.0);
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
      const int s = k % XS;
      const float2 xi = Cx[s][ty][tx];
      df yv;
      if (Cf[s][ty][tx]) {
        yv = df{xi.x, xi.y};
      } else {
        const int cx = tx + 1, cy = ty + 1;
        const df k000 = df{Km[ty][tx].x, Km[ty][tx].y}, k001 = df{Km[ty][tx + 1].x, Km[ty][tx + 1].y},
                 k010 = df{Km[ty + 1][tx].x, Km[ty + 1][tx].y},
                 k011 = df{Km[ty + 1][tx + 1].x, Km[ty + 1][tx + 1].y};
        const df k100 = df{Kp[ty][tx].x, Kp[ty][tx].y}, k101 = df{Kp[ty][tx + 1].x, Kp[ty][tx + 1].y},
                 k110 = df{Kp[ty + 1][tx].x, Kp[ty + 1][tx].y},
                 k111 = df{Kp[ty + 1][tx + 1].x, Kp[ty + 1][tx + 1].y};
        float ah = 0.f, al = 0.f;
        // face diagonals (two elements each)
        acc_term(ah, al, df_add(k000, k100), xi, X0[cy - 1][cx - 1]);
        acc_term(ah, al, df_add(k001, k101), xi, X0[cy - 1][cx + 1]);
        acc_term(ah, al, df_add(k010, k110), xi, X0[cy + 1][cx - 1]);
        acc_term(ah, al, df_add(k011, k111), xi, X0[cy + 1][cx + 1]);
        acc_term(ah, al, df_add(k000, k010), xi, Xm[cy][cx - 1]);
        acc_term(ah, al, df_add(k001, k011), xi, Xm[cy][cx + 1]);
        acc_term(ah, al, df_add(k100, k110), xi, Xp[cy][cx - 1]);
        acc_term(ah, al, df_add(k101, k111), xi, Xp[cy][cx + 1]);
        acc_term(ah, al, df_add(k000, k001), xi, Xm[cy - 1][cx]);
        acc_term(ah, al, df_add(k010, k011), xi, Xm[cy + 1][cx]);
        acc_term(ah, al, df_add(k100, k101), xi, Xp[cy - 1][cx]);
        acc_term(ah, al, df_add(k110, k111), xi, Xp[cy + 1][cx]);
        // body diagonals
        acc_term(ah, al, k000, xi, Xm[cy - 1][cx - 1]);
        acc_term(ah, al, k001, xi, Xm[cy - 1][cx + 1]);
        acc_term(ah, al, k010, xi, Xm[cy + 1][cx - 1]);
        acc_term(ah, al, k011, xi, Xm[cy + 1][cx + 1]);
        acc_term(ah, al, k100, xi, Xp[cy - 1][cx - 1]);
        acc_term(ah, al, k101, xi, Xp[cy - 1][cx + 1]);
        acc_term(ah, al, k110, xi, Xp[cy + 1][cx - 1]);
        acc_term(ah, al, k111, xi, Xp[cy + 1][cx + 1]);
        yv = df_mul(df_make(ah, al), scale);
      }
      if (MODE == RESID) {
        const df ri = df_sub(ld2(a.q, idx), yv);
        a.y[idx] = make_float2(ri.hi, ri.lo);
        a.r32[idx] = __fadd_rn(ri.hi, ri.lo);
        dot = df_add(dot, df_mul(ri, ri));
      } else {
        a.y[idx] = make_float2(yv.hi, yv.lo);
        dot = df_add(dot, df_mul(df{xi.x, xi.y}, yv));
      }
    }
  }
  if (a.out) {
    double v[1] = {df_to_double(dot)};
    double t[1];
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int nb = gridDim.x * gridDim.y * gridDim.z;
    if (block_sum_last_ids<1>(v, a.partials, a.counter, t, tid, NT, bid, nb) && tid == 0) a.out[0] = t[0];
  }
}

template <int MODE>
int runs_for(const Dims& d, int sms) {
  int per_sm = 0;
  MGAR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_df3d<MODE>, NT, 0));
  per_sm = std::max(per_sm, 1);
  const int64_t cols = (int64_t)((d.NX + TX - 1) / TX) * ((d.NY + TY - 1) / TY);
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
  a.partials = c.partials;
  a.counter = c.counter;
  return a;
}

template <int MODE>
void launch(Ctx& c, DfArgs& a) {
  const Dims& d = c.L[0];
  a.gz = std::max(1, std::min(c.df3d_gz[MODE], d.NZ));
  const dim3 grid((d.NX + TX - 1) / TX, (d.NY + TY - 1) / TY, a.gz);
  k_df3d<MODE><<<grid, dim3(TX, TY), 0, c.stream>>>(a);
  MGAR_LAUNCH_CHECK();
}

}  // namespace d3d

void df3d_prepare(Ctx& c) {
  using namespace d3d;
  int dev = 0, sms = 0;
  MGAR_CUDA(cudaGetDevice(&dev));
  MGAR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  c.df3d_gz[APPLY] = runs_for<APPLY>(c.L[0], sms);
  c.df3d_gz[DIR] = runs_for<DIR>(c.L[0], sms);
  c.df3d_gz[RESID] = runs_for<RESID>(c.L[0], sms);
}

// y = A x; x . y into *dot when given
void df3d_apply(Ctx& c, const float2* x, float2* y, double* dot) {
  using namespace d3d;
  DfArgs a = base_args(c);
  a.x = x;
  a.y = y;
  a.out = dot;
  launch<APPLY>(c, a);
}

// p = z + (rz_new / rz_old) p_old (p = z when first), y = A p, p . y into *dot
void df3d_dir(Ctx& c, const float* z, const float2* p_old, float2* p, const double* rz_new,
              const double* rz_old, bool first, float2* y, double* dot) {
  using namespace d3d;
  DfArgs a = base_args(c);
  a.z = z;
  a.x = p_old;
  a.p = p;
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
