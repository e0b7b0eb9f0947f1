// V-cycle x <- MG(A, b, x, P) of Table 1 on the reference hierarchy, plus the
// fine-level operator applications used by the solvers.
//
// Per level (Table 1): pre-smooth with damped Jacobi
// x <- x + omega D^-1 (b - A x), residual restricted by P^T, coarse
// correction (recursively one V-cycle with zero initial guess, the coarsest
// level by its explicit inverse), interpolation x <- x + P x^c, post-smooth.
// The finest operator is matrix-free from the element conductivities; the
// coarse ones are assembled 3^d-point stencils.  Every kernel is templated on
// the working precision (FP64, or FP32 for the mixed preconditioner).
#include "common.cuh"
#include "levelops.cuh"

namespace mgar {

const char* level_site(int kind, int level) {
  static const char* names[10] = {"jacobi0", "sweep", "residual", "restrict", "prolong",
                                  "coarse", "pre3d", "post3d", "sweep3d", "resid3d"};
  static char table[10][kMaxLevels][24];
  static bool init = false;
  if (!init) {
    for (int k = 0; k < 10; ++k)
      for (int l = 0; l < kMaxLevels; ++l) snprintf(table[k][l], 24, "vc %s L%d", names[k], l);
    init = true;
  }
  return table[kind % 10][level % kMaxLevels];
}

// ------------------------------------------------------------ row functors
template <typename Real, int DIM>
struct FineRow {
  FineOp<Real> op;
  __device__ __forceinline__ Real operator()(const Real* __restrict__ x, int idx) const {
    int i, j, k;
    coords(idx, op.fNX, op.fNXY, i, j, k);
    Real d;
    if (DIM == 2) return fine_row2(op, x, i, j, d);
    return fine_row3(op, x, i, j, k, d);
  }
  __device__ __forceinline__ int size() const { return op.n; }
};

template <typename Real, int DIM>
struct StencilRow {
  StencilOp<Real> op;
  __device__ __forceinline__ Real operator()(const Real* __restrict__ x, int idx) const {
    int i, j, k;
    coords(idx, op.fNX, op.fNXY, i, j, k);
    if (DIM == 2) return stencil_row2(op, x, i, j);
    return stencil_row3(op, x, i, j, k);
  }
  __device__ __forceinline__ int size() const { return op.n; }
};

// ----------------------------------------------------------------- kernels
template <class Row, typename Real>
__global__ void k_jacobi(Row row, const Real* __restrict__ b, const Real* __restrict__ xin,
                         Real* __restrict__ xout, const Real* __restrict__ dinv, Real omega) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= row.size()) return;
  const Real ax = row(xin, idx);
  xout[idx] = xin[idx] + omega * dinv[idx] * (b[idx] - ax);
}

template <typename Real>
__global__ void k_jacobi_zero(const Real* __restrict__ b, Real* __restrict__ x,
                              const Real* __restrict__ dinv, Real omega, int n) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n) x[idx] = omega * dinv[idx] * b[idx];
}

template <class Row, typename Real>
__global__ void k_residual(Row row, const Real* __restrict__ b, const Real* __restrict__ x,
                           Real* __restrict__ r) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= row.size()) return;
  r[idx] = b[idx] - row(x, idx);
}

// y = A x, optionally with the deterministic sum of x.y into out[0].
template <class Row, typename Real, bool DOT>
__global__ void k_apply(Row row, const Real* __restrict__ x, Real* __restrict__ y, Real scale,
                        double* partials, unsigned int* counter, double* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (idx < row.size()) {
    const Real ax = scale * row(x, idx);
    y[idx] = ax;
    if (DOT) v[0] = (double)x[idx] * (double)ax;
  }
  if (DOT) block_sum_finish<1>(v, partials, counter, out);
}

// The 2D finest-level passes with kNptFine nodes per thread (nodes base,
// base + blockDim.x, ...): each thread has several nodes' loads in flight and
// the launch a quarter of the blocks; the arithmetic per node is that of the
// one-node kernels above.
constexpr int kNptFine = 4;

inline int blocks_npt(int64_t n) {
  const int64_t per = (int64_t)kThreads * kNptFine;
  return (int)((n + per - 1) / per);
}

template <typename Real>
__global__ void k_jacobi_zero_n(const Real* __restrict__ b, Real* __restrict__ x,
                                const Real* __restrict__ dinv, Real omega, int n) {
  const int base = blockIdx.x * blockDim.x * kNptFine + threadIdx.x;
  Real bv[kNptFine], dv[kNptFine];
#pragma unroll
  for (int u = 0; u < kNptFine; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < n) {
      bv[u] = b[idx];
      dv[u] = dinv[idx];
    }
  }
#pragma unroll
  for (int u = 0; u < kNptFine; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < n) x[idx] = omega * dv[u] * bv[u];
  }
}

template <class Row, typename Real>
__global__ void k_residual_n(Row row, const Real* __restrict__ b, const Real* __restrict__ x,
                             Real* __restrict__ r) {
  const int base = blockIdx.x * blockDim.x * kNptFine + threadIdx.x;
#pragma unroll
  for (int u = 0; u < kNptFine; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < row.size()) r[idx] = b[idx] - row(x, idx);
  }
}

template <typename Real, int DIM>
__global__ void k_prolong_n(const Real* __restrict__ xc, const Real* cur, Real* dst, Dims f, Dims cd,
                            const uint8_t* __restrict__ fixed) {
  pdl_wait();
  pdl_trigger();
  const int base = blockIdx.x * blockDim.x * kNptFine + threadIdx.x;
#pragma unroll
  for (int u = 0; u < kNptFine; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < f.n) prolong_node<Real, DIM>(xc, cur, dst, f, cd, fixed, idx);
  }
}

// One damped-Jacobi sweep; with DOT also r . xout (r as df64 pairs: the CG's
// r . z) into *dout, double-float warp sums, FP64 across warps and blocks.
template <class Row, typename Real, bool DOT>
__global__ void k_jacobi_n(Row row, const Real* __restrict__ b, const Real* __restrict__ xin,
                           Real* __restrict__ xout, const Real* __restrict__ dinv, Real omega,
                           const float2* __restrict__ rdot, double* partials,
                           unsigned int* counter, double* dout) {
  const int base = blockIdx.x * blockDim.x * kNptFine + threadIdx.x;
  df acc{0.f, 0.f};
#pragma unroll
  for (int u = 0; u < kNptFine; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < row.size()) {
      const Real ax = row(xin, idx);
      const Real xo = xin[idx] + omega * dinv[idx] * (b[idx] - ax);
      xout[idx] = xo;
      if (DOT) {
        // r . z, or b . z when no r is given
        const float2 rv = rdot ? rdot[idx] : make_float2((float)b[idx], 0.f);
        acc = df_add(acc, df_mulf(df{rv.x, rv.y}, (float)xo));
      }
    }
  }
  if (DOT) block_sum_finish_df(acc, partials, counter, dout);
}

template <typename Real, int DIM>
__global__ void k_restrict(const Real* __restrict__ r, Real* __restrict__ bc, Dims f, Dims cd,
                           const uint8_t* __restrict__ fixed, const Real* __restrict__ dinvc = nullptr,
                           Real omega = Real(0), Real* __restrict__ xc = nullptr) {
  pdl_wait();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < cd.n) restrict_node<Real, DIM, false>(r, bc, f, cd, fixed, idx, dinvc, omega, xc);
  pdl_trigger();
}

// dst = cur + P xc (fixed fine nodes keep cur); dst may equal cur.
template <typename Real, int DIM>
__global__ void k_prolong(const Real* __restrict__ xc, const Real* cur, Real* dst, Dims f, Dims cd,
                          const uint8_t* __restrict__ fixed) {
  pdl_wait();
  pdl_trigger();
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < f.n) prolong_node<Real, DIM>(xc, cur, dst, f, cd, fixed, idx);
}

// 3D interpolation by z-columns: a thread owns the fine nodes (i, j, k0 ..
// k0 + kProlongChunk - 1), k0 even, and interpolates each of the coarse
// planes k0/2 .. k0/2 + kProlongChunk/2 in x and y once (4 loads), so a
// fine node costs one or two plane values instead of 8 coarse loads.  Every
// load of the chunk is issued before the first use (compile-time slots), so
// the column costs one memory round trip.
constexpr int kProlongChunk = 8;

template <typename Real>
__global__ void k_prolong3(const Real* __restrict__ xc, const Real* cur, Real* dst, Dims f, Dims cd,
                           const uint8_t* __restrict__ fixed) {
  constexpr int KC = kProlongChunk, NP = KC / 2 + 1;
  pdl_wait();
  pdl_trigger();
  const int NXY = f.NX * f.NY;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= NXY) return;
  const int i = col % f.NX, j = col / f.NX;
  int ix[2], iy[2];
  float wx[2], wy[2];
  prolong_taps(i, f.ex, ix, wx);
  prolong_taps(j, f.ey, iy, wy);
  const int cNXY = cd.NX * cd.NY;
  const int k0 = blockIdx.y * KC, Kb = k0 >> 1;
  // coarse planes Kb .. Kb + NP - 1, interpolated in x and y
  Real P[NP];
#pragma unroll
  for (int t = 0; t < NP; ++t) {
    P[t] = Real(0);
    const int K = Kb + t;
    if (K < cd.NZ) {
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const int o = ix[a] + cd.NX * iy[b] + cNXY * K;
          if (CK(o, cd.n)) P[t] += (Real)(wx[a] * wy[b]) * xc[o];
        }
    }
  }
  Real cv[KC];
  uint8_t fx[KC];
#pragma unroll
  for (int u = 0; u < KC; ++u) {
    const int k = k0 + u;
    cv[u] = Real(0);
    fx[u] = 0;
    if (k < f.NZ) {
      const int idx = col + NXY * k;
      cv[u] = cur[idx];
      if (fixed) fx[u] = fixed[idx];
    }
  }
#pragma unroll
  for (int u = 0; u < KC; ++u) {
    const int k = k0 + u;
    if (k >= f.NZ) break;
    // taps along z: even k -> plane k/2; odd k -> halfway, or the top node
    // of an odd element count -> plane (k+1)/2
    Real pz;
    if ((u & 1) == 0) pz = P[u >> 1];
    else if (k < f.ez) pz = Real(0.5) * (P[u >> 1] + P[(u >> 1) + 1]);
    else pz = P[(u >> 1) + 1];
    dst[col + NXY * k] = fx[u] ? cv[u] : cv[u] + pz;
  }
}

// The coarse-level kernels gather what the hierarchy build wrote (stencil
// coefficients, D^-1, the coarsest inverse) before they wait on their
// predecessor: a kernel may start while its predecessor runs, and every
// kernel here waits before it lets its own successor start, so everything
// older than the predecessor is complete and visible by then.  The latency
// of those loads overlaps the predecessor's tail; the arithmetic and its
// order are unchanged.
template <typename Real, int DIM>
__global__ void k_resid_coarse(StencilOp<Real> op, const Real* __restrict__ b,
                               const Real* __restrict__ x, Real* __restrict__ r) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const bool on = idx < op.n;
  int i = 0, j = 0, k = 0;
  Real sv[stencil_size<DIM>()];
  if (on) {
    coords(idx, op.fNX, op.fNXY, i, j, k);
    stencil_coefs<DIM>(op, i, j, k, sv);
  }
  pdl_wait();
  if (on) r[idx] = b[idx] - stencil_apply<DIM, Real, false>(op, x, i, j, k, sv);
  pdl_trigger();
}

template <typename Real, int DIM>
__global__ void k_post_coarse(StencilOp<Real> op, const Real* __restrict__ xc,
                              const Real* __restrict__ cur, const Real* __restrict__ b,
                              const Real* __restrict__ dinv, Real omega, Real* __restrict__ dst,
                              Dims f, Dims cd) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const bool on = idx < op.n;
  Real sv[stencil_size<DIM>()];
  if (on) {
    int i, j, k;
    coords(idx, op.fNX, op.fNXY, i, j, k);
    stencil_coefs<DIM>(op, i, j, k, sv);
  }
  pdl_wait();
  if (on) post_node<Real, DIM, false, true>(op, xc, cur, b, dinv, omega, dst, f, cd, idx, sv);
  pdl_trigger();
}

// One damped-Jacobi sweep on an assembled level, x' = x + w D^-1 (b - A x).
template <typename Real, int DIM>
__global__ void k_jacobi_st(StencilOp<Real> op, const Real* __restrict__ b,
                            const Real* __restrict__ xin, Real* __restrict__ xout,
                            const Real* __restrict__ dinv, Real omega) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const bool on = idx < op.n;
  int i = 0, j = 0, k = 0;
  Real sv[stencil_size<DIM>()];
  Real dv = Real(0);
  if (on) {
    coords(idx, op.fNX, op.fNXY, i, j, k);
    stencil_coefs<DIM>(op, i, j, k, sv);
    dv = dinv[idx];
  }
  pdl_wait();
  if (on) {
    const Real ax = stencil_apply<DIM, Real, false>(op, xin, i, j, k, sv);
    xout[idx] = xin[idx] + omega * dv * (b[idx] - ax);
  }
  pdl_trigger();
}

// x = C b with the explicit inverse of the coarsest operator: a warp per
// row, the row's entries loaded before the wait when it has at most 128
// (four per lane), summed in the same order as coarse_row.
template <typename Real, typename M>
__global__ void k_coarse_solve(const M* __restrict__ cinv, const Real* __restrict__ b,
                               Real* __restrict__ x, int n) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  const bool pre = n <= 128;
  M cv[4] = {M(0), M(0), M(0), M(0)};
  if (pre && row < n) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int jj = lane + 32 * q;
      const int jc = min(jj, n - 1);  // a valid address even where the entry is unused
      if (jj < n && CK((int64_t)row * n + jc, (int64_t)n * n)) cv[q] = cinv[(int64_t)row * n + jc];
    }
  }
  pdl_wait();
  pdl_trigger();
  if (row >= n) return;
  if (!pre) {
    coarse_row<Real, false, M>(cinv, b, x, n, row, lane);
    return;
  }
  M s = M(0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int jj = lane + 32 * q;
    if (jj < n) s += cv[q] * (M)b[jj];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[row] = (Real)s;
}

// ------------------------------------------- bottom of the V-cycle, one cluster
// Levels lb .. nl-1 (each at most kBottomNodes nodes) of the zero-guess
// V-cycle in one launch of a thread-block cluster: the CTAs of the cluster
// stride over each level's nodes, and the hardware cluster barrier (release
// on arrive, acquire on wait) separates the phases, so the small levels cost
// no kernel launches and no waits of this code's own.
constexpr int kBottomThreads = 512;
constexpr int kBottomClusterMax = 16;  // non-portable cluster size, used when it fits

template <typename Real>
struct BottomArgs {
  StencilOp<Real> op[kMaxLevels];
  Dims L[kMaxLevels];
  Real* b[kMaxLevels];
  Real* x[kMaxLevels];
  Real* t[kMaxLevels];
  Real* r[kMaxLevels];
  const typename CoarseT<Real>::T* cinv;
  int nc, lb, nl;
  Real omega;
};

__device__ __forceinline__ void cluster_barrier() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n"
      "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

template <typename Real, int DIM>
__global__ void __launch_bounds__(kBottomThreads) k_bottom(BottomArgs<Real> a) {
  pdl_wait();
  pdl_trigger();
  const int nthr = gridDim.x * blockDim.x;
  const int vt = blockIdx.x * blockDim.x + threadIdx.x;
  // x_l = w D^-1 b_l is already in place (left by the restriction)
  for (int l = a.lb; l + 1 < a.nl; ++l) {
    for (int idx = vt; idx < a.L[l].n; idx += nthr)
      resid_node<Real, DIM, true>(a.op[l], a.b[l], a.x[l], a.r[l], idx);
    cluster_barrier();
    Real* xn = l + 2 < a.nl ? a.x[l + 1] : nullptr;  // the coarsest level is solved
    for (int idx = vt; idx < a.L[l + 1].n; idx += nthr)
      restrict_node<Real, DIM, true>(a.r[l], a.b[l + 1], a.L[l], a.L[l + 1], nullptr, idx,
                                     a.op[l + 1].dinv, a.omega, xn);
    cluster_barrier();
  }
  {
    const int l = a.nl - 1;
    const int warp = vt >> 5, nwarps = nthr >> 5, lane = threadIdx.x & 31;
    for (int row = warp; row < a.nc; row += nwarps)
      coarse_row<Real, true, typename CoarseT<Real>::T>(a.cinv, a.b[l], a.x[l], a.nc, row, lane);
  }
  const Real* res = a.x[a.nl - 1];
  for (int l = a.nl - 2; l >= a.lb; --l) {
    cluster_barrier();
    for (int idx = vt; idx < a.L[l].n; idx += nthr)
      post_node<Real, DIM, true>(a.op[l], res, a.x[l], a.b[l], a.op[l].dinv, a.omega, a.t[l], a.L[l],
                                 a.L[l + 1], idx);
    res = a.t[l];
  }
}

__global__ void k_convert_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_convert_f2d(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

// -------------------------------------------------------------------- host
template <typename Real>
static LevelBuf<Real>* levels(Ctx& c);
template <>
LevelBuf<double>* levels<double>(Ctx& c) { return c.h64; }
template <>
LevelBuf<float>* levels<float>(Ctx& c) { return c.h32; }

template <typename Real>
static const Real* ref_ke(Ctx& c);
template <>
const double* ref_ke<double>(Ctx& c) { return c.ke0; }
template <>
const float* ref_ke<float>(Ctx& c) { return c.ke0_f; }

template <typename Real, int DIM>
static FineRow<Real, DIM> fine_row(Ctx& c, const Real* ke, const Real* ksub) {
  FineRow<Real, DIM> r;
  const Dims& d = c.L[0];
  r.op = FineOp<Real>{ke, ksub, c.fixed, d.ex, d.ey, d.ez, d.NX, d.NY, d.NZ, (int)d.n, d.fNX, d.fNXY};
  return r;
}

template <typename Real, int DIM>
static StencilRow<Real, DIM> stencil_row(Ctx& c, int l) {
  StencilRow<Real, DIM> r;
  const Dims& d = c.L[l];
  r.op = StencilOp<Real>{levels<Real>(c)[l].st, levels<Real>(c)[l].dinv, d.NX, d.NY, d.NZ, (int)d.n,
                         d.fNX, d.fNXY};
  return r;
}

// One damped-Jacobi sweep xout = xin + omega D^-1 (b - A xin) on level l.
template <typename Real, int DIM>
static void sweep(Ctx& c, int l, const Real* b, const Real* xin, Real* xout) {
  const Dims& d = c.L[l];
  LevelBuf<Real>* h = levels<Real>(c);
  const Real om = (Real)c.p.omega;
  ProfScope ps(c, l == 0 ? MGAR_KC_SMOOTH0 : -1);
  if (l == 0)
    k_jacobi<<<blocks_for(d.n), kThreads, 0, c.stream>>>(fine_row<Real, DIM>(c, ref_ke<Real>(c), nullptr),
                                                         b, xin, xout, h[0].dinv, om);
  else
    launch_pdl(c.stream, c.use_pdl, k_jacobi_st<Real, DIM>, dim3(blocks_for(d.n)), dim3(kThreads),
               stencil_row<Real, DIM>(c, l).op, b, xin, xout, (const Real*)h[l].dinv, om);
  MGAR_LAUNCH_CHECK_AT(level_site(1, l));
}

template <typename Real, int DIM>
static void residual(Ctx& c, int l, const Real* b, const Real* x, Real* r) {
  const Dims& d = c.L[l];
  ProfScope ps(c, l == 0 ? MGAR_KC_RESID0 : -1);
  if (l == 0)
    k_residual<<<blocks_for(d.n), kThreads, 0, c.stream>>>(fine_row<Real, DIM>(c, ref_ke<Real>(c), nullptr),
                                                           b, x, r);
  else
    k_residual<<<blocks_for(d.n), kThreads, 0, c.stream>>>(stencil_row<Real, DIM>(c, l), b, x, r);
  MGAR_LAUNCH_CHECK_AT(level_site(2, l));
}

// First level handled by the cluster kernel (nl if none).
static int bottom_level(const Ctx& c) {
  if (!c.bottom_ok) return c.nl;
  int lb = c.nl - 1;
  while (lb - 1 >= 1 && c.L[lb - 1].n <= c.bottom_nodes) --lb;
  return lb;
}

template <typename Real, int DIM>
static void launch_bottom(Ctx& c, int lb) {
  LevelBuf<Real>* h = levels<Real>(c);
  BottomArgs<Real> a{};
  for (int l = lb; l < c.nl; ++l) {
    a.op[l] = stencil_row<Real, DIM>(c, l).op;
    a.L[l] = c.L[l];
    a.b[l] = h[l].b;
    a.x[l] = h[l].x;
    a.t[l] = h[l].t;
    a.r[l] = h[l].r;
  }
  a.cinv = CoarseT<Real>::inv(c);
  a.nc = c.nc;
  a.lb = lb;
  a.nl = c.nl;
  a.omega = (Real)c.p.omega;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(c.bottom_cluster);
  cfg.blockDim = dim3(kBottomThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = c.stream;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = c.bottom_cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = c.use_pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  MGAR_CUDA(cudaLaunchKernelEx(&cfg, k_bottom<Real, DIM>, a));
  MGAR_LAUNCH_CHECK_AT("vc bottom");
}

template <typename Real, int DIM>
static bool bottom_fits(int csize) {
  if (csize > 8 &&
      cudaFuncSetAttribute(k_bottom<Real, DIM>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
          cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(kBottomThreads);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, k_bottom<Real, DIM>, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return clusters >= 1;
}

// Whether the cluster kernel can run here (FP32 V-cycle), and with how many
// CTAs (16 if the device allows the non-portable size, else 8); call outside
// stream capture.
void bottom_prepare(Ctx& c) {
  c.bottom_ok = false;
  for (int csize = kBottomClusterMax; csize >= 8 && !c.bottom_ok; csize /= 2) {
    c.bottom_ok = c.dim == 2 ? bottom_fits<float, 2>(csize) : bottom_fits<float, 3>(csize);
    if (c.bottom_ok) c.bottom_cluster = csize;
  }
}

// dst = cur + P xc on level f (P from level cd; fixed nodes of f keep cur).
template <typename Real, int DIM>
static void launch_prolong(Ctx& c, bool pdl, const Real* xc, const Real* cur, Real* dst,
                           const Dims& f, const Dims& cd, const uint8_t* fixed) {
  if (DIM == 3 && c.prolong_col) {
    const int64_t cols = (int64_t)f.NX * f.NY;
    const int gz = (f.NZ + kProlongChunk - 1) / kProlongChunk;
    launch_pdl(c.stream, pdl && c.use_pdl, k_prolong3<Real>, dim3(blocks_for(cols), gz),
               dim3(kThreads), xc, cur, dst, f, cd, fixed);
  } else {
    launch_pdl(c.stream, pdl && c.use_pdl, k_prolong<Real, DIM>, dim3(blocks_for(f.n)),
               dim3(kThreads), xc, cur, dst, f, cd, fixed);
  }
}

// Table 1 with one pre- and one post-sweep and a zero guess below the finest
// level: per level one fused pre kernel (smooth from zero + residual), the
// restriction, and one fused post kernel (interpolation + smooth); the small
// levels at the bottom run in one cluster launch.
template <int DIM>
static void vcycle_fused(Ctx& c, const float* b0, float* x0, bool zero_guess,
                         const float2* rdot = nullptr, double* dout = nullptr) {
  using Real = float;
  LevelBuf<Real>* h = levels<Real>(c);
  const int nl = c.nl;
  const Real om = (Real)c.p.omega;
  const Real* res[kMaxLevels] = {};  // each coarse level's correction
  const Dims& d0 = c.L[0];
  // finest level, pre
  Real* cur0;
  {
    ProfScope ps(c, MGAR_KC_SMOOTH0);
    if (DIM == 3) {
      if (zero_guess) {
        fine3d(c, 0, ref_ke<Real>(c), b0, h[0].dinv, nullptr, nullptr, h[0].t, h[0].r);
      } else {
        fine3d(c, 3, ref_ke<Real>(c), b0, h[0].dinv, x0, nullptr, h[0].t, nullptr);
        fine3d(c, 2, ref_ke<Real>(c), b0, h[0].dinv, h[0].t, nullptr, h[0].r, nullptr);
      }
      cur0 = h[0].t;
    } else {
      if (zero_guess) {
        k_jacobi_zero_n<<<blocks_npt(d0.n), kThreads, 0, c.stream>>>(b0, h[0].t, h[0].dinv, om,
                                                                     (int)d0.n);
        MGAR_LAUNCH_CHECK_AT(level_site(0, 0));
      } else {
        sweep<Real, DIM>(c, 0, b0, x0, h[0].t);
      }
      cur0 = h[0].t;
      ProfScope pr(c, MGAR_KC_RESID0);
      k_residual_n<<<blocks_npt(d0.n), kThreads, 0, c.stream>>>(
          fine_row<Real, DIM>(c, ref_ke<Real>(c), nullptr), b0, (const Real*)cur0, h[0].r);
      MGAR_LAUNCH_CHECK_AT(level_site(2, 0));
    }
  }
  // the tiled 3D kernels leave r = 0 on fixed nodes, which P^T = (Z P)^T ignores
  // each restriction into a level above the coarsest also leaves that
  // level's zero-guess sweep x = w D^-1 b
  launch_pdl(c.stream, c.use_pdl, k_restrict<Real, DIM>, dim3(blocks_for(c.L[1].n)), dim3(kThreads),
             (const Real*)h[0].r, h[1].b, d0, c.L[1], DIM == 3 ? (const uint8_t*)nullptr : c.fixed,
             (const Real*)h[1].dinv, om, nl > 2 ? h[1].x : (Real*)nullptr);
  MGAR_LAUNCH_CHECK_AT(level_site(3, 0));
  const int lb = bottom_level(c);
  // coarse levels, down
  for (int l = 1; l + 1 < nl && l < lb; ++l) {
    const Dims& d = c.L[l];
    launch_pdl(c.stream, c.use_pdl, k_resid_coarse<Real, DIM>, dim3(blocks_for(d.n)), dim3(kThreads),
               stencil_row<Real, DIM>(c, l).op, (const Real*)h[l].b, (const Real*)h[l].x, h[l].r);
    MGAR_LAUNCH_CHECK_AT(level_site(0, l));
    launch_pdl(c.stream, c.use_pdl, k_restrict<Real, DIM>, dim3(blocks_for(c.L[l + 1].n)),
               dim3(kThreads), (const Real*)h[l].r, h[l + 1].b, d, c.L[l + 1],
               (const uint8_t*)nullptr, (const Real*)h[l + 1].dinv, om,
               l + 2 < nl ? h[l + 1].x : (Real*)nullptr);
    MGAR_LAUNCH_CHECK_AT(level_site(3, l));
  }
  if (lb < nl) {
    // levels lb .. nl-1 in one cluster launch
    launch_bottom<Real, DIM>(c, lb);
    res[nl - 1] = h[nl - 1].x;
    for (int l = lb; l + 1 < nl; ++l) res[l] = h[l].t;
  } else {
    // coarsest level
    const int l = nl - 1;
    const int rows_per_block = kThreads / 32;
    k_coarse_solve<Real, typename CoarseT<Real>::T>
        <<<(c.nc + rows_per_block - 1) / rows_per_block, kThreads, 0, c.stream>>>(
            CoarseT<Real>::inv(c), h[l].b, h[l].x, c.nc);
    MGAR_LAUNCH_CHECK_AT(level_site(5, l));
    res[l] = h[l].x;
  }
  // coarse levels, up
  for (int l = std::min(nl - 2, lb - 1); l >= 1; --l) {
    const Dims& d = c.L[l];
    if (d.n > c.split_coarse_nodes) {
      // large level: thin interpolation in place on x_l, then the sweep into t_l
      launch_prolong<Real, DIM>(c, true, res[l + 1], (const Real*)h[l].x, h[l].x, d, c.L[l + 1],
                                (const uint8_t*)nullptr);
      MGAR_LAUNCH_CHECK_AT(level_site(4, l));
      sweep<Real, DIM>(c, l, h[l].b, h[l].x, h[l].t);
    } else {
      launch_pdl(c.stream, c.use_pdl, k_post_coarse<Real, DIM>, dim3(blocks_for(d.n)),
                 dim3(kThreads), stencil_row<Real, DIM>(c, l).op, res[l + 1], (const Real*)h[l].x,
                 (const Real*)h[l].b, (const Real*)h[l].dinv, om, h[l].t, d, c.L[l + 1]);
      MGAR_LAUNCH_CHECK_AT(level_site(4, l));
    }
    res[l] = h[l].t;
  }
  // finest level, post (the timed class is the tiled pass alone)
  if (DIM == 3 && !c.split_post) {
    ProfScope ps(c, MGAR_KC_SMOOTH0);
    fine3d(c, 1, ref_ke<Real>(c), b0, h[0].dinv, cur0, res[1], x0, nullptr, rdot, dout);
  } else if (DIM == 3) {
    // interpolation in place on the pre-smoothed iterate, then the tiled sweep
    launch_prolong<Real, DIM>(c, true, (const Real*)res[1], (const Real*)cur0, cur0, d0, c.L[1],
                              (const uint8_t*)c.fixed);
    MGAR_LAUNCH_CHECK_AT(level_site(4, 0));
    ProfScope ps(c, MGAR_KC_SMOOTH0);
    fine3d(c, 3, ref_ke<Real>(c), b0, h[0].dinv, cur0, nullptr, x0, nullptr, rdot, dout);
  } else {
    ProfScope ps(c, MGAR_KC_SMOOTH0);
    // interpolation in place on the pre-smoothed iterate, then the sweep into
    // x0 (with r . x0 into *dout when asked)
    k_prolong_n<Real, DIM><<<blocks_npt(d0.n), kThreads, 0, c.stream>>>(res[1], cur0, cur0, d0,
                                                                         c.L[1], c.fixed);
    MGAR_LAUNCH_CHECK_AT(level_site(4, 0));
    const FineRow<Real, DIM> row = fine_row<Real, DIM>(c, ref_ke<Real>(c), nullptr);
    if (dout)
      k_jacobi_n<FineRow<Real, DIM>, Real, true><<<blocks_npt(d0.n), kThreads, 0, c.stream>>>(
          row, b0, (const Real*)cur0, x0, (const Real*)h[0].dinv, om, rdot, c.partials, c.counter,
          dout);
    else
      k_jacobi_n<FineRow<Real, DIM>, Real, false><<<blocks_npt(d0.n), kThreads, 0, c.stream>>>(
          row, b0, (const Real*)cur0, x0, (const Real*)h[0].dinv, om, nullptr, nullptr, nullptr,
          nullptr);
    MGAR_LAUNCH_CHECK_AT(level_site(1, 0));
  }
}

// General Table 1 V-cycle (any numbers of pre- and post-sweeps).  The fused
// form is for the FP32 V-cycle: its kernels trade memory passes and launches
// for recomputed arithmetic (the neighbours' smoothed values and
// interpolations), which pays on the FP32 pipe and not at GB300's 1/58-rate
// FP64, where the separate kernels below are faster.
template <typename Real, int DIM>
static void vcycle_dim(Ctx& c, const Real* b0, Real* x0, bool zero_guess) {
  if constexpr (sizeof(Real) == 4) {
    if (c.p.nu_pre == 1 && c.p.nu_post == 1 && c.nl >= 2 && !c.untiled) {
      vcycle_fused<DIM>(c, b0, x0, zero_guess);
      return;
    }
  }
  LevelBuf<Real>* h = levels<Real>(c);
  const int nl = c.nl;
  const Real om = (Real)c.p.omega;
  Real* cur[kMaxLevels];
  // downward leg
  for (int l = 0; l + 1 < nl; ++l) {
    const Dims& d = c.L[l];
    const Real* b = l == 0 ? b0 : h[l].b;
    Real* x = l == 0 ? x0 : h[l].x;
    Real* other = h[l].t;
    Real* cu = x;
    int sweeps = c.p.nu_pre;
    if (l > 0 || zero_guess) {
      if (sweeps > 0) {
        ProfScope ps(c, l == 0 ? MGAR_KC_SMOOTH0 : -1);
        k_jacobi_zero<<<blocks_for(d.n), kThreads, 0, c.stream>>>(b, x, h[l].dinv, om, (int)d.n);
        MGAR_LAUNCH_CHECK_AT(level_site(0, l));
        --sweeps;
      } else {
        MGAR_CUDA(cudaMemsetAsync(x, 0, d.n * sizeof(Real), c.stream));
      }
    }
    for (; sweeps > 0; --sweeps) {
      Real* dst = (cu == x) ? other : x;
      sweep<Real, DIM>(c, l, b, cu, dst);
      cu = dst;
    }
    cur[l] = cu;
    residual<Real, DIM>(c, l, b, cu, h[l].r);
    k_restrict<Real, DIM><<<blocks_for(c.L[l + 1].n), kThreads, 0, c.stream>>>(
        h[l].r, h[l + 1].b, d, c.L[l + 1], l == 0 ? c.fixed : nullptr);
    MGAR_LAUNCH_CHECK_AT(level_site(3, l));
  }
  // coarsest level
  {
    const int l = nl - 1;
    const int rows_per_block = kThreads / 32;
    k_coarse_solve<Real, typename CoarseT<Real>::T>
        <<<(c.nc + rows_per_block - 1) / rows_per_block, kThreads, 0, c.stream>>>(
            CoarseT<Real>::inv(c), h[l].b, h[l].x, c.nc);
    MGAR_LAUNCH_CHECK_AT(level_site(5, l));
  }
  // upward leg
  for (int l = nl - 2; l >= 0; --l) {
    const Dims& d = c.L[l];
    const Real* b = l == 0 ? b0 : h[l].b;
    Real* x = l == 0 ? x0 : h[l].x;
    Real* other = h[l].t;
    const int post = c.p.nu_post;
    Real* dst = (post % 2 == 0) ? x : other;
    launch_prolong<Real, DIM>(c, false, (const Real*)h[l + 1].x, (const Real*)cur[l], dst, d,
                              c.L[l + 1], l == 0 ? (const uint8_t*)c.fixed : nullptr);
    MGAR_LAUNCH_CHECK_AT(level_site(4, l));
    Real* cu = dst;
    for (int s = 0; s < post; ++s) {
      Real* nxt = (cu == x) ? other : x;
      sweep<Real, DIM>(c, l, b, cu, nxt);
      cu = nxt;
    }
  }
}

template <typename Real>
void vcycle(Ctx& c, const Real* b, Real* x, bool zero_guess) {
  if (c.dim == 2) vcycle_dim<Real, 2>(c, b, x, zero_guess);
  else vcycle_dim<Real, 3>(c, b, x, zero_guess);
}
template void vcycle<double>(Ctx&, const double*, double*, bool);
template void vcycle<float>(Ctx&, const float*, float*, bool);

void vcycle_dot(Ctx& c, const float* b, float* x, const float2* r, double* dout) {
  require(vcycle_dot_ok(c), MGAR_ERR_ARG,
          "fused r.z V-cycle needs one pre- and one post-sweep, two levels and the tiled 3D kernels");
  if (c.dim == 2) vcycle_fused<2>(c, b, x, true, r, dout);
  else vcycle_fused<3>(c, b, x, true, r, dout);
}

template <typename Real, int DIM>
static void apply_dim(Ctx& c, const Real* ke, const Real* ksub, const Real* x, Real* y, Real scale,
                      double* dot_out) {
  const Dims& d = c.L[0];
  auto row = fine_row<Real, DIM>(c, ke, ksub);
  if (dot_out)
    k_apply<FineRow<Real, DIM>, Real, true><<<blocks_for(d.n), kThreads, 0, c.stream>>>(
        row, x, y, scale, c.partials, c.counter, dot_out);
  else
    k_apply<FineRow<Real, DIM>, Real, false><<<blocks_for(d.n), kThreads, 0, c.stream>>>(
        row, x, y, scale, nullptr, nullptr, nullptr);
  MGAR_LAUNCH_CHECK();
}

void apply_fine64(Ctx& c, const double* ke, const double* x, double* y, double* dot_out) {
  ProfScope ps(c, MGAR_KC_APPLY64);
  if (c.dim == 2) apply_dim<double, 2>(c, ke, nullptr, x, y, 1.0, dot_out);
  else apply_dim<double, 3>(c, ke, nullptr, x, y, 1.0, dot_out);
}
void apply_fine32(Ctx& c, const float* ke, const float* x, float* y) {
  if (c.dim == 2) apply_dim<float, 2>(c, ke, nullptr, x, y, 1.f, nullptr);
  else apply_dim<float, 3>(c, ke, nullptr, x, y, 1.f, nullptr);
}
// y = -(A - A0) x
void apply_dK64(Ctx& c, const double* x, double* y) {
  if (c.dim == 2) apply_dim<double, 2>(c, c.ke, c.ke0, x, y, -1.0, nullptr);
  else apply_dim<double, 3>(c, c.ke, c.ke0, x, y, -1.0, nullptr);
}
void apply_dK32(Ctx& c, const float* x, float* y) {
  if (c.dim == 2) apply_dim<float, 2>(c, c.ke_f, c.ke0_f, x, y, -1.f, nullptr);
  else apply_dim<float, 3>(c, c.ke_f, c.ke0_f, x, y, -1.f, nullptr);
}

void convert_d2f(Ctx& c, const double* a, float* b, int64_t n) {
  k_convert_d2f<<<blocks_for(n), kThreads, 0, c.stream>>>(a, b, n);
  MGAR_LAUNCH_CHECK();
}
void convert_f2d(Ctx& c, const float* a, double* b, int64_t n) {
  k_convert_f2d<<<blocks_for(n), kThreads, 0, c.stream>>>(a, b, n);
  MGAR_LAUNCH_CHECK();
}

}  // namespace mgar
