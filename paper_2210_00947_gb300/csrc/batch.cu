// Batched MGCG over many independent 2D designs (Section 3.2's solve with
// Table 1's V-cycle as preconditioner), for the uneven designs of a batch.
//
// Every handle keeps its own data (conductivities, hierarchy, vectors); the
// batch only holds device tables of their pointers and sizes.  Each step of
// the solve is one launch over all designs: block b of a launch belongs to
// design bdes[b], and its nodes are (b - b0[design]) * blockDim + thread of
// that design's level.  So one launch per V-cycle level and operation serves
// every design, and the designs' different depths only decide which of them
// take part in a level (a design's coarsest level is solved by one launch
// over all designs' coarsest levels).  The outer CG runs in double-float
// (df64) arithmetic on the FP32 pipe around the FP32 V-cycle (FP32
// preconditioner, FP64-accurate refinement: GB300 runs FP64 at 1/58 of the
// FP32 rate), with FP64 scalars; its per-design scalars
// stay on the device, a design stops when its own ||r|| / ||q|| <= eps2 or
// at cg_max (its blocks then leave at once), and the whole solve after the
// hierarchy builds is one CUDA graph: a WHILE node repeats the iteration
// while any design is still active.
//
// Reductions are per design in a fixed order (each design's blocks write
// partials, the design's last block adds them in block order), and the
// reduction kernels use a fixed block size, so a design's result does not
// depend on the other designs in the batch.  The node kernels of the
// V-cycle (no reductions) take their block size per level from an
// autotuner run at the first solve, which times the candidates on the
// batch's own levels and keeps the fastest.
#include "common.cuh"
#include "dfop.cuh"
#include "levelops.cuh"

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

namespace mgar {
namespace bat {

constexpr int kRedThreads = 256;  // block size of every reducing kernel
constexpr int kBS = 16;           // device scalars per design
enum : int { BS_RZ = 0, BS_PAP = 2, BS_RR = 3, BS_IT = 4, BS_ACT = 5, BS_QN = 6, BS_EPS = 7,
             BS_CGMAX = 8, BS_BAD = 9,
             // gathered from each handle after the solve / the design cycle
             BS_COMPL = 10, BS_LAM = 11, BS_CHANGE = 12, BS_FAIL = 13, BS_DERR = 14 };

// One design at one level of the V-cycle.
struct Lev {
  FineOp<float> f0;      // level 0: FP32 reference conductivities (matrix-free)
  StencilOp<float> op;   // levels >= 1: assembled stencil and 1/diag
  Dims d, dn;            // this level and the next coarser one
  const float* dinv;     // this level's 1/diag
  const float* dinv_n;   // the next level's 1/diag
  float *x, *b, *t, *r;  // level 0: x = V-cycle result, b = its input
  float *bn, *xn;        // the next level's b, and its x (null when it is the coarsest)
  const float* resn;     // the next level's result (x at the coarsest, t above)
  const uint8_t* fixed;  // level 0: Dirichlet mask
  float omega;
};

struct Coarse {
  const double* cinv;  // explicit inverse of the design's coarsest operator (FP64)
  const float* b;
  float* x;
  int nc;
};

struct Des {
  DfOp f;              // current conductivities (df64 pairs, matrix-free difference form)
  const float2* q;     // the load as df64 pairs
  float2 *x, *r, *p, *Ap;  // CG vectors as df64 pairs (the handle's own buffers)
  double* T;           // the caller's solution (FP64): warm start in, solution out
  float *b32, *x32;    // FP32 input and output of the V-cycle at level 0
  const double* dsc;   // the handle's device scalars (compliance, OC outcome)
  const int* derr;     // the handle's factorisation error flag
};

// Launch shape: which design each block serves.
struct Shape {
  int threads = kRedThreads;
  int nblocks = 0;
  int* bdes = nullptr;  // [nblocks]
  int* b0 = nullptr;    // [designs]: first block of the design, -1 if absent
};

__device__ __forceinline__ bool active(const double* bsc, int d) { return bsc[d * kBS + BS_ACT] != 0.0; }

// Nodes per thread of the level-0 launches: a thread takes nodes base,
// base + blockDim.x, ... of its design, so each block's lookups (its design,
// the design's tables and scalars) serve several nodes and each thread has
// several independent loads in flight.
constexpr int kNpt0 = 4;  // V-cycle node kernels at level 0
constexpr int kNptR = 2;  // CG kernels (double-float vectors, reductions)

// The first node of this thread in its design, for npt nodes per thread.
__device__ __forceinline__ int node_base(const int* b0, int d, int npt) {
  return (blockIdx.x - b0[d]) * blockDim.x * npt + threadIdx.x;
}

// The number of blocks of design d's launch over n nodes.
__device__ __forceinline__ int design_blocks(int n, int npt) {
  const int per = blockDim.x * npt;
  return (n + per - 1) / per;
}

// Deterministic per-design sum of one double-float value per thread: the
// design's blocks write partials, its last block adds them in block order
// into *out.  Warp sums in df64 on the FP32 pipe, FP64 only across warps and
// blocks (GB300 runs FP64 at 1/58
// of the FP32 rate; an FP64 value per thread through a shuffle tree costs
// more than the data pass of these kernels).
__device__ __forceinline__ void seg_finish_df(df v, double* partials, unsigned int* counters, int d,
                                              int b0, int nb, double* out) {
  double t = 0.0;
  if (block_sum_last_df(v, partials + b0, counters + d, t, threadIdx.x, blockDim.x,
                        blockIdx.x - b0, nb) &&
      threadIdx.x == 0)
    *out = t;
}

// ------------------------------------------------------------ df64 CG kernels
// The outer CG runs in double-float arithmetic on the FP32 pipe (GB300 runs
// FP64 at 1/58 of the FP32 rate): vectors as df64 pairs, the product in the
// exact difference form, scalars in FP64.
// Per design: scalars of this solve, iteration 0, active.
__global__ void kb_init(double* bsc, const double* consts, int nd) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= nd) return;
  double* s = bsc + d * kBS;
  s[BS_IT] = 0.0;
  s[BS_ACT] = 1.0;
  s[BS_BAD] = 0.0;
  s[BS_QN] = consts[3 * d];
  s[BS_EPS] = consts[3 * d + 1];
  s[BS_CGMAX] = consts[3 * d + 2];
}

// x = T as df64 pairs (the start of each design's CG)
__global__ void kb_t_to_df(const Des* D, const int* bdes, const int* b0) {
  const int d = bdes[blockIdx.x];
  const Des& g = D[d];
  const int base = node_base(b0, d, kNptR);
#pragma unroll
  for (int u = 0; u < kNptR; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < g.f.n) g.x[idx] = pack(df_from_double(g.T[idx]));
  }
}

// T = x (the end of each design's CG)
__global__ void kb_df_to_t(const Des* D, const int* bdes, const int* b0) {
  const int d = bdes[blockIdx.x];
  const Des& g = D[d];
  const int base = node_base(b0, d, kNptR);
#pragma unroll
  for (int u = 0; u < kNptR; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < g.f.n) g.T[idx] = df_to_double(unpack(g.x[idx]));
  }
}

// Each handle's compliance, OC outcome and factorisation flag into the
// batch scalars, so that one copy brings every design's outcome to the host.
__global__ void kb_gather(const Des* D, int nd, double* bsc) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= nd) return;
  const Des& g = D[d];
  double* s = bsc + (size_t)d * kBS;
  s[BS_COMPL] = g.dsc[S_COMPL];
  s[BS_LAM] = g.dsc[S_OC_LAM];
  s[BS_CHANGE] = g.dsc[S_OC_CHANGE];
  s[BS_FAIL] = g.dsc[S_OC_FAIL];
  s[BS_DERR] = (double)*g.derr;
}

// r = q - A x, its FP32 copy, ||r||^2 (the start of each design's CG).
__global__ void kb_resid64(const Des* D, const int* bdes, const int* b0, double* bsc,
                           double* partials, unsigned int* counters) {
  const int d = bdes[blockIdx.x];
  const Des& g = D[d];
  const int base = node_base(b0, d, kNptR);
  df v{0.f, 0.f};
#pragma unroll
  for (int u = 0; u < kNptR; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < g.f.n) {
      const df ri = df_sub(unpack(g.q[idx]), df_row<2>(g.f, g.x, idx));
      g.r[idx] = pack(ri);
      g.b32[idx] = __fadd_rn(ri.hi, ri.lo);
      v = df_add(v, df_mul(ri, ri));
    }
  }
  seg_finish_df(v, partials, counters, d, b0[d], design_blocks(g.f.n, kNptR),
                bsc + d * kBS + BS_RR);
}

// After the initial residual: a design whose start already meets eps2 (or
// whose cg_max is 0) is done; a non-finite residual stops it and is flagged.
__global__ void kb_start(double* bsc, int nd) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= nd) return;
  double* s = bsc + d * kBS;
  const double rel = sqrt(s[BS_RR]) / s[BS_QN];
  if (!isfinite(rel)) s[BS_BAD] = 1.0;
  s[BS_ACT] = (isfinite(rel) && rel > s[BS_EPS] && s[BS_CGMAX] > 0.0) ? 1.0 : 0.0;
}

// Ap = A p and p . Ap.
__global__ void kb_apply_dot(const Des* D, const int* bdes, const int* b0, double* bsc,
                             double* partials, unsigned int* counters) {
  const int d = bdes[blockIdx.x];
  if (!active(bsc, d)) return;
  const Des& g = D[d];
  const int base = node_base(b0, d, kNptR);
  df v{0.f, 0.f};
#pragma unroll
  for (int u = 0; u < kNptR; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < g.f.n) {
      const df ap = df_row<2>(g.f, g.p, idx);
      g.Ap[idx] = pack(ap);
      v = df_add(v, df_mul(unpack(g.p[idx]), ap));
    }
  }
  seg_finish_df(v, partials, counters, d, b0[d], design_blocks(g.f.n, kNptR),
                bsc + d * kBS + BS_PAP);
}

// alpha = r.z / p.Ap; x += alpha p; r -= alpha Ap; ||r||^2; FP32 copy of r.
__global__ void kb_cg_xr(const Des* D, const int* bdes, const int* b0, double* bsc,
                         double* partials, unsigned int* counters) {
  const int d = bdes[blockIdx.x];
  if (!active(bsc, d)) return;
  const Des& g = D[d];
  const double* s = bsc + d * kBS;
  const int par = ((int)s[BS_IT]) & 1;
  const df alpha = block_div_df(s + BS_RZ + par, s + BS_PAP);
  const int base = node_base(b0, d, kNptR);
  // every node's four loads first, then the updates
  float2 xv[kNptR], pv[kNptR], rv[kNptR], qv[kNptR];
#pragma unroll
  for (int u = 0; u < kNptR; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < g.f.n) {
      xv[u] = g.x[idx];
      pv[u] = g.p[idx];
      rv[u] = g.r[idx];
      qv[u] = g.Ap[idx];
    }
  }
  df v{0.f, 0.f};
#pragma unroll
  for (int u = 0; u < kNptR; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < g.f.n) {
      g.x[idx] = pack(df_add(unpack(xv[u]), df_mul(alpha, unpack(pv[u]))));
      const df ri = df_sub(unpack(rv[u]), df_mul(alpha, unpack(qv[u])));
      g.r[idx] = pack(ri);
      g.b32[idx] = __fadd_rn(ri.hi, ri.lo);
      v = df_add(v, df_mul(ri, ri));
    }
  }
  seg_finish_df(v, partials, counters, d, b0[d], design_blocks(g.f.n, kNptR),
                bsc + d * kBS + BS_RR);
}

// One iteration done: count it and decide, per design, whether to go on;
// the WHILE node repeats while any design is active.
__global__ void kb_check(double* bsc, int nd, cudaGraphConditionalHandle loop, int* any_out) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int d = threadIdx.x; d < nd; d += blockDim.x) {
    double* s = bsc + d * kBS;
    if (s[BS_ACT] == 0.0) continue;
    const double it = s[BS_IT] + 1.0;
    s[BS_IT] = it;
    const double rel = sqrt(s[BS_RR]) / s[BS_QN];
    if (!isfinite(rel)) s[BS_BAD] = 1.0;
    const bool go = isfinite(rel) && rel > s[BS_EPS] && it < s[BS_CGMAX];
    s[BS_ACT] = go ? 1.0 : 0.0;
    if (go) atomicOr(&any, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (any_out) *any_out = any;  // a loop driven from the host
    else cudaGraphSetConditional(loop, any ? 1u : 0u);
  }
}

// p = z + (r.z_new / r.z_old) p (p = z in the first iteration), z the FP32
// V-cycle output.
__global__ void kb_cg_p(const Des* D, const int* bdes, const int* b0, const double* bsc) {
  const int d = bdes[blockIdx.x];
  if (!active(bsc, d)) return;
  const Des& g = D[d];
  const double* s = bsc + d * kBS;
  const int it = (int)s[BS_IT];
  const df beta = it == 0 ? df{0.f, 0.f}
                          : block_div_df(s + BS_RZ + (it & 1), s + BS_RZ + ((it - 1) & 1));
  const int base = node_base(b0, d, kNptR);
  float zv[kNptR];
  float2 pv[kNptR];
#pragma unroll
  for (int u = 0; u < kNptR; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < g.f.n) {
      zv[u] = g.x32[idx];
      pv[u] = g.p[idx];
    }
  }
#pragma unroll
  for (int u = 0; u < kNptR; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < g.f.n) {
      const df z{zv[u], 0.f};
      g.p[idx] = pack(it == 0 ? z : df_add(z, df_mul(beta, unpack(pv[u]))));
    }
  }
}

// --------------------------------------------------------- V-cycle kernels
// The design and node of a thread of a level launch (false: nothing to do).
__device__ __forceinline__ bool lev_node(const int* bdes, const int* b0, const double* bsc, int& d,
                                         int& idx) {
  d = bdes[blockIdx.x];
  if (!active(bsc, d)) return false;
  idx = (blockIdx.x - b0[d]) * blockDim.x + threadIdx.x;
  return true;
}

// level 0, zero initial guess: t = w D^-1 b
__global__ void kb_jz0(const Lev* L, const int* bdes, const int* b0, const double* bsc) {
  const int d = bdes[blockIdx.x];
  if (!active(bsc, d)) return;
  const Lev& v = L[d];
  const int base = node_base(b0, d, kNpt0);
  float dv[kNpt0], bv[kNpt0];
#pragma unroll
  for (int u = 0; u < kNpt0; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < v.d.n) {
      dv[u] = v.dinv[idx];
      bv[u] = v.b[idx];
    }
  }
#pragma unroll
  for (int u = 0; u < kNpt0; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < v.d.n) v.t[idx] = v.omega * dv[u] * bv[u];
  }
}

// level 0: r = b - A t (matrix-free FP32 operator)
__global__ void kb_resid0(const Lev* L, const int* bdes, const int* b0, const double* bsc) {
  const int d = bdes[blockIdx.x];
  if (!active(bsc, d)) return;
  const Lev& v = L[d];
  const int base = node_base(b0, d, kNpt0);
#pragma unroll
  for (int u = 0; u < kNpt0; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < v.d.n) {
      int i, j, k;
      coords(idx, v.f0.fNX, v.f0.fNXY, i, j, k);
      float diag;
      v.r[idx] = v.b[idx] - fine_row2(v.f0, v.t, i, j, diag);
    }
  }
}

// b_next = P^T r (fixed fine nodes excluded at level 0), and the next level's
// zero-guess sweep x_next = w D^-1 b_next unless it is the coarsest
__global__ void kb_restrict(const Lev* L, const int* bdes, const int* b0, const double* bsc) {
  int d, idx;
  if (!lev_node(bdes, b0, bsc, d, idx)) return;
  const Lev& v = L[d];
  if (idx < v.dn.n)
    restrict_node<float, 2, false>(v.r, v.bn, v.d, v.dn, v.fixed, idx, v.dinv_n, v.omega, v.xn);
}

// levels >= 1 above the coarsest: r = b - A x (x left by the restriction)
__global__ void kb_resid(const Lev* L, const int* bdes, const int* b0, const double* bsc) {
  int d, idx;
  if (!lev_node(bdes, b0, bsc, d, idx)) return;
  const Lev& v = L[d];
  if (idx < v.d.n) resid_node<float, 2, false>(v.op, v.b, v.x, v.r, idx);
}

// each design's coarsest level: x = C b, one warp per row
__global__ void kb_coarse(const Coarse* C, const int* bdes, const int* b0, const double* bsc) {
  const int d = bdes[blockIdx.x];
  if (!active(bsc, d)) return;
  const Coarse& c = C[d];
  const int wpb = blockDim.x >> 5;
  const int row = (blockIdx.x - b0[d]) * wpb + (threadIdx.x >> 5);
  if (row < c.nc) coarse_row<float, false, double>(c.cinv, c.b, c.x, c.nc, row, threadIdx.x & 31);
}

// levels >= 1 above the coarsest: t = post-smoothing of x + P res_next
__global__ void kb_post(const Lev* L, const int* bdes, const int* b0, const double* bsc) {
  int d, idx;
  if (!lev_node(bdes, b0, bsc, d, idx)) return;
  const Lev& v = L[d];
  if (idx < v.d.n)
    post_node<float, 2, false>(v.op, v.resn, v.x, v.b, v.dinv, v.omega, v.t, v.d, v.dn, idx);
}

// level 0: t += P res_1 (fixed nodes keep t)
__global__ void kb_prolong0(const Lev* L, const int* bdes, const int* b0, const double* bsc) {
  const int d = bdes[blockIdx.x];
  if (!active(bsc, d)) return;
  const Lev& v = L[d];
  const int base = node_base(b0, d, kNpt0);
#pragma unroll
  for (int u = 0; u < kNpt0; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < v.d.n) prolong_node<float, 2>(v.resn, v.t, v.t, v.d, v.dn, v.fixed, idx);
  }
}

// level 0: x = t + w D^-1 (b - A t), z = x in FP64 and r . z (the CG's new
// r.z, slot by iteration parity)
__global__ void kb_sweep0(const Lev* L, const Des* D, const int* bdes, const int* b0,
                          double* bsc, double* partials, unsigned int* counters) {
  const int d = bdes[blockIdx.x];
  if (!active(bsc, d)) return;
  const Lev& v = L[d];
  const Des& g = D[d];
  const int base = node_base(b0, d, kNptR);
  df s{0.f, 0.f};
#pragma unroll
  for (int u = 0; u < kNptR; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < v.d.n) {
      int i, j, k;
      coords(idx, v.f0.fNX, v.f0.fNXY, i, j, k);
      float diag;
      const float ti = v.t[idx];
      const float xo = ti + v.omega * v.dinv[idx] * (v.b[idx] - fine_row2(v.f0, v.t, i, j, diag));
      v.x[idx] = xo;
      s = df_add(s, df_mulf(unpack(g.r[idx]), xo));
    }
  }
  const int par = ((int)bsc[d * kBS + BS_IT]) & 1;
  seg_finish_df(s, partials, counters, d, b0[d], design_blocks(v.d.n, kNptR),
                bsc + d * kBS + BS_RZ + par);
}

// ------------------------------------------------------------------- host
struct Batch {
  std::vector<Ctx*> h;
  int nd = 0, lmax = 0;
  cudaStream_t stream = nullptr, cap = nullptr;
  std::string err;
  Lev* dlev = nullptr;  // [lmax][nd]
  Coarse* dco = nullptr;
  Des* ddes = nullptr;
  std::vector<Des> hdes;       // host copy of the design table
  double* bsc = nullptr;       // [nd][kBS]
  double* consts = nullptr;    // [nd][3] qnorm, eps2, cg_max (device)
  double* hconsts = nullptr;   // pinned
  double* hbsc = nullptr;      // pinned
  double* partials = nullptr;
  unsigned int* counters = nullptr;
  Shape s_red;                 // level 0, reducing kernels
  std::vector<int> tuned;      // threads per level (node kernels); [lmax] + coarse warps last
  std::vector<Shape> shapes;   // all shapes made (freed at destroy)
  // per level l: nodes of l (designs with a level below l), nodes of l + 1
  std::vector<Shape> s_node, s_next;
  Shape s_coarse;
  cudaGraphExec_t exec = nullptr;
  int64_t prologue = 0, body = 0;
  int* any = nullptr;   // device: any design active after a host-driven iteration
  int* hany = nullptr;  // pinned copy
  bool eager = false;   // the last solve was launched from the host
  std::string report;
  // design cycles: each handle's stream -> the batch stream, and back
  std::vector<cudaEvent_t> ev_des;
  cudaEvent_t ev_solved = nullptr, ev_start = nullptr;
  // per-design work of every handle as one graph (a branch per design), kept
  // while the pointers and values captured in it stay the same
  struct DesignGraph {
    std::vector<uint64_t> key;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
  };
  DesignGraph g_hier, g_pre, g_post;  // hierarchy; filter+SIMP+hierarchy; sens+compliance+OC
  // device time of the last graph-launched design cycle's three parts
  cudaEvent_t ev_ph[4] = {nullptr, nullptr, nullptr, nullptr};
  double phase_ms[3] = {0.0, 0.0, 0.0};
  bool have_phases = false;
};

static void free_shape(Shape& s) {
  cudaFree(s.bdes);
  cudaFree(s.b0);
  s.bdes = s.b0 = nullptr;
}

// A shape over per-design unit counts (0: the design takes no part).
static Shape make_shape(const std::vector<int64_t>& units, int per_block, int threads) {
  Shape s;
  s.threads = threads;
  std::vector<int> bdes, b0(units.size(), -1);
  for (size_t d = 0; d < units.size(); ++d) {
    if (units[d] <= 0) continue;
    b0[d] = (int)bdes.size();
    const int64_t nb = (units[d] + per_block - 1) / per_block;
    for (int64_t k = 0; k < nb; ++k) bdes.push_back((int)d);
  }
  s.nblocks = (int)bdes.size();
  MGAR_CUDA(cudaMalloc(&s.b0, b0.size() * sizeof(int)));
  MGAR_CUDA(cudaMemcpy(s.b0, b0.data(), b0.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (s.nblocks > 0) {
    MGAR_CUDA(cudaMalloc(&s.bdes, bdes.size() * sizeof(int)));
    MGAR_CUDA(cudaMemcpy(s.bdes, bdes.data(), bdes.size() * sizeof(int), cudaMemcpyHostToDevice));
  }
  return s;
}

// Nodes of level l per design for the level's own kernels (designs for
// which l is above the coarsest), or of level l + 1 (its restriction).
static std::vector<int64_t> level_units(const Batch& b, int l, bool next) {
  std::vector<int64_t> u(b.nd, 0);
  for (int d = 0; d < b.nd; ++d) {
    const Ctx& c = *b.h[d];
    if (l + 1 < c.nl) u[d] = next ? c.L[l + 1].n : c.L[l].n;
  }
  return u;
}

static void make_level_shapes(Batch& b, int l, int threads) {
  free_shape(b.s_node[l]);
  free_shape(b.s_next[l]);
  b.s_node[l] = make_shape(level_units(b, l, false), threads * (l == 0 ? kNpt0 : 1), threads);
  b.s_next[l] = make_shape(level_units(b, l, true), threads, threads);
}

static void make_coarse_shape(Batch& b, int warps) {
  free_shape(b.s_coarse);
  std::vector<int64_t> rows(b.nd);
  for (int d = 0; d < b.nd; ++d) rows[d] = b.h[d]->nc;
  b.s_coarse = make_shape(rows, warps, warps * 32);
}

template <typename K, typename... Args>
static void launch_shape(Batch& b, const Shape& s, K kernel, Args... args) {
  if (s.nblocks == 0) return;
  kernel<<<s.nblocks, s.threads, 0, b.stream>>>(args..., s.bdes, s.b0, b.bsc);
  MGAR_LAUNCH_CHECK();
}

// The FP32 V-cycle z = M r of every active design (Table 1, zero guess).
static void vcycle(Batch& b) {
  Lev* L0 = b.dlev;
  // down
  for (int l = 0; l + 1 < b.lmax; ++l) {
    Lev* L = b.dlev + (size_t)l * b.nd;
    if (l == 0) {
      launch_shape(b, b.s_node[0], kb_jz0, (const Lev*)L);
      launch_shape(b, b.s_node[0], kb_resid0, (const Lev*)L);
    } else {
      launch_shape(b, b.s_node[l], kb_resid, (const Lev*)L);
    }
    launch_shape(b, b.s_next[l], kb_restrict, (const Lev*)L);
  }
  launch_shape(b, b.s_coarse, kb_coarse, (const Coarse*)b.dco);
  // up
  for (int l = b.lmax - 2; l >= 1; --l)
    launch_shape(b, b.s_node[l], kb_post, (const Lev*)(b.dlev + (size_t)l * b.nd));
  launch_shape(b, b.s_node[0], kb_prolong0, (const Lev*)L0);
  kb_sweep0<<<b.s_red.nblocks, kRedThreads, 0, b.stream>>>(L0, b.ddes, b.s_red.bdes, b.s_red.b0,
                                                           b.bsc, b.partials, b.counters);
  MGAR_LAUNCH_CHECK();
}

static void red_launch_resid(Batch& b) {
  kb_resid64<<<b.s_red.nblocks, kRedThreads, 0, b.stream>>>(b.ddes, b.s_red.bdes, b.s_red.b0, b.bsc,
                                                            b.partials, b.counters);
  MGAR_LAUNCH_CHECK();
}

static void iteration(Batch& b, cudaGraphConditionalHandle loop, int* any_out = nullptr) {
  kb_apply_dot<<<b.s_red.nblocks, kRedThreads, 0, b.stream>>>(b.ddes, b.s_red.bdes, b.s_red.b0,
                                                              b.bsc, b.partials, b.counters);
  MGAR_LAUNCH_CHECK();
  kb_cg_xr<<<b.s_red.nblocks, kRedThreads, 0, b.stream>>>(b.ddes, b.s_red.bdes, b.s_red.b0, b.bsc,
                                                          b.partials, b.counters);
  MGAR_LAUNCH_CHECK();
  kb_check<<<1, 256, 0, b.stream>>>(b.bsc, b.nd, loop, any_out);
  MGAR_LAUNCH_CHECK();
  vcycle(b);
  kb_cg_p<<<b.s_red.nblocks, kRedThreads, 0, b.stream>>>(b.ddes, b.s_red.bdes, b.s_red.b0, b.bsc);
  MGAR_LAUNCH_CHECK();
}

// Per-design scalars, initial residuals, first V-cycle and direction.
static void prologue(Batch& b) {
  const int th = 128;
  kb_init<<<(b.nd + th - 1) / th, th, 0, b.stream>>>(b.bsc, b.consts, b.nd);
  MGAR_LAUNCH_CHECK();
  kb_t_to_df<<<b.s_red.nblocks, kRedThreads, 0, b.stream>>>(b.ddes, b.s_red.bdes, b.s_red.b0);
  MGAR_LAUNCH_CHECK();
  red_launch_resid(b);
  kb_start<<<(b.nd + th - 1) / th, th, 0, b.stream>>>(b.bsc, b.nd);
  MGAR_LAUNCH_CHECK();
  vcycle(b);
  kb_cg_p<<<b.s_red.nblocks, kRedThreads, 0, b.stream>>>(b.ddes, b.s_red.bdes, b.s_red.b0, b.bsc);
  MGAR_LAUNCH_CHECK();
}

// After the loop: the solutions back to the callers' FP64 vectors.
static void epilogue(Batch& b) {
  kb_df_to_t<<<b.s_red.nblocks, kRedThreads, 0, b.stream>>>(b.ddes, b.s_red.bdes, b.s_red.b0);
  MGAR_LAUNCH_CHECK();
}

// The solve launched from the host (handles that time kernel classes or run
// without graphs): the graph's launches in the graph's order, the loop's
// condition read after each iteration as the WHILE node reads it.
static void solve_eager(Batch& b) {
  prologue(b);
  for (;;) {
    iteration(b, 0, b.any);
    MGAR_CUDA(cudaMemcpyAsync(b.hany, b.any, sizeof(int), cudaMemcpyDeviceToHost, b.stream));
    MGAR_CUDA(cudaStreamSynchronize(b.stream));
    if (!*b.hany) break;
  }
  epilogue(b);
}

// The solve after the hierarchy builds as one graph: scalars, initial
// residuals, first V-cycle and direction, then WHILE(any active) iteration.
static void build_graph(Batch& b) {
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle loop = 0;
  MGAR_CUDA(cudaGraphCreate(&g, 0));
  cudaStream_t saved = b.stream;
  const int64_t before = launches_so_far();
  bool ok = false;
  try {
    MGAR_CUDA(cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault));
    MGAR_CUDA(cudaStreamBeginCaptureToGraph(b.cap, g, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
    b.stream = b.cap;
    prologue(b);
    cudaStreamCaptureStatus st;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t ndeps = 0;
    MGAR_CUDA(cudaStreamGetCaptureInfo(b.stream, &st, nullptr, &cg, &deps, &edges, &ndeps));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode = nullptr;
    MGAR_CUDA(cudaGraphAddNode(&wnode, cg, deps, nullptr, ndeps, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    MGAR_CUDA(cudaStreamUpdateCaptureDependencies(b.stream, &wnode, nullptr, 1,
                                                  cudaStreamSetCaptureDependencies));
    epilogue(b);
    cudaGraph_t out = nullptr;
    MGAR_CUDA(cudaStreamEndCapture(b.cap, &out));
    b.stream = saved;
    b.prologue = launches_so_far() - before;
    MGAR_CUDA(cudaStreamBeginCaptureToGraph(b.cap, body, nullptr, nullptr, 0,
                                            cudaStreamCaptureModeThreadLocal));
    b.stream = b.cap;
    const int64_t b0 = launches_so_far();
    iteration(b, loop);
    b.body = launches_so_far() - b0;
    MGAR_CUDA(cudaStreamEndCapture(b.cap, &out));
    b.stream = saved;
    MGAR_CUDA(cudaGraphInstantiate(&b.exec, g, 0));
    ok = true;
  } catch (...) {
    b.stream = saved;
    cudaStreamCaptureStatus st;
    if (cudaStreamIsCapturing(b.cap, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(b.cap, &junk);
      if (junk) cudaGraphDestroy(junk);
    }
    (void)cudaGetLastError();
    count_launches(-(launches_so_far() - before));
    cudaGraphDestroy(g);
    throw;
  }
  count_launches(-(launches_so_far() - before));  // captured, not executed
  cudaGraphDestroy(g);
  (void)ok;
}

// Device time of fn() on the batch stream, best of reps.
template <class F>
static float time_best(Batch& b, int reps, F&& fn) {
  cudaEvent_t e0, e1;
  MGAR_CUDA(cudaEventCreate(&e0));
  MGAR_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    MGAR_CUDA(cudaEventRecord(e0, b.stream));
    fn();
    MGAR_CUDA(cudaEventRecord(e1, b.stream));
    MGAR_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    MGAR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// Autotuner: per level, the block size of its node kernels from 64 / 128 /
// 256 / 512 threads, and the warps per block of the coarsest solve from
// 2 / 4 / 8, each timed on the batch's own levels (the kernels are
// node-parallel without reductions, so the choice changes no result).  The
// device scalars mark every design active while it runs.
static void autotune(Batch& b) {
  std::vector<double> ones((size_t)b.nd * kBS, 0.0);
  for (int d = 0; d < b.nd; ++d) ones[(size_t)d * kBS + BS_ACT] = 1.0;
  MGAR_CUDA(cudaMemcpy(b.bsc, ones.data(), ones.size() * sizeof(double), cudaMemcpyHostToDevice));
  const int cand[4] = {64, 128, 256, 512};
  char line[160];
  b.report = "batched V-cycle autotuner (best of 5 timed runs per candidate)\n";
  for (int l = 0; l + 1 < b.lmax; ++l) {
    Lev* L = b.dlev + (size_t)l * b.nd;
    float best = 1e30f;
    int pick = 256;
    for (int th : cand) {
      make_level_shapes(b, l, th);
      const float ms = time_best(b, 5, [&] {
        if (l == 0) {
          launch_shape(b, b.s_node[0], kb_jz0, (const Lev*)L);
          launch_shape(b, b.s_node[0], kb_resid0, (const Lev*)L);
          launch_shape(b, b.s_next[0], kb_restrict, (const Lev*)L);
          launch_shape(b, b.s_node[0], kb_prolong0, (const Lev*)L);
        } else {
          launch_shape(b, b.s_node[l], kb_resid, (const Lev*)L);
          launch_shape(b, b.s_next[l], kb_restrict, (const Lev*)L);
          launch_shape(b, b.s_node[l], kb_post, (const Lev*)L);
        }
      });
      snprintf(line, sizeof(line), "  level %d: %3d threads %8.2f us\n", l, th, ms * 1e3f);
      b.report += line;
      if (ms < best) {
        best = ms;
        pick = th;
      }
    }
    make_level_shapes(b, l, pick);
    b.tuned[l] = pick;
    snprintf(line, sizeof(line), "level %d: %d threads per block\n", l, pick);
    b.report += line;
  }
  const int wc[3] = {2, 4, 8};
  float best = 1e30f;
  int pick = 8;
  for (int w : wc) {
    make_coarse_shape(b, w);
    const float ms = time_best(b, 5, [&] { launch_shape(b, b.s_coarse, kb_coarse, (const Coarse*)b.dco); });
    snprintf(line, sizeof(line), "  coarsest: %d warps %8.2f us\n", w, ms * 1e3f);
    b.report += line;
    if (ms < best) {
      best = ms;
      pick = w;
    }
  }
  make_coarse_shape(b, pick);
  b.tuned[b.lmax - 1] = pick;
  snprintf(line, sizeof(line), "coarsest solve: %d warps per block\n", pick);
  b.report += line;
}

}  // namespace bat
}  // namespace mgar

using namespace mgar;
using namespace mgar::bat;

namespace {
thread_local std::string g_batch_create_error = "no error";

// Batch calls run one at a time per process (concurrent batches from
// several host threads are not supported; see the header).
std::mutex g_batch_mutex;

template <class F>
int bguard(mgar_batch_t hb, F&& f) {
  Batch* b = reinterpret_cast<Batch*>(hb);
  if (!b) return MGAR_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_batch_mutex);
  try {
    return f(*b);
  } catch (const Error& e) {
    b->err = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    b->err = e.what();
    return MGAR_ERR_CUDA;
  }
}

void free_batch(Batch& b) {
  if (b.exec) cudaGraphExecDestroy(b.exec);
  for (Batch::DesignGraph* g : {&b.g_hier, &b.g_pre, &b.g_post})
    if (g->exec) cudaGraphExecDestroy(g->exec);
  for (cudaEvent_t e : b.ev_ph)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : b.ev_des) cudaEventDestroy(e);
  if (b.ev_solved) cudaEventDestroy(b.ev_solved);
  if (b.ev_start) cudaEventDestroy(b.ev_start);
  for (auto& s : b.s_node) free_shape(s);
  for (auto& s : b.s_next) free_shape(s);
  free_shape(b.s_coarse);
  free_shape(b.s_red);
  cudaFree(b.dlev);
  cudaFree(b.dco);
  cudaFree(b.ddes);
  cudaFree(b.bsc);
  cudaFree(b.consts);
  cudaFree(b.partials);
  cudaFree(b.counters);
  cudaFree(b.any);
  if (b.hany) cudaFreeHost(b.hany);
  if (b.hconsts) cudaFreeHost(b.hconsts);
  if (b.hbsc) cudaFreeHost(b.hbsc);
  if (b.cap) cudaStreamDestroy(b.cap);
}
// Graphs are taken when every handle allows them and none is timing a
// kernel class (a timed class is measured launch by launch).
bool graphable(const Batch& b) {
  for (const Ctx* c : b.h)
    if (!c->use_graphs || c->prof_class != 0) return false;
  return true;
}

// The batch stream after whatever each handle's stream holds, with each
// handle's pending coarsest factorisation joined first.
void order_after_handles(Batch& b) {
  for (int d = 0; d < b.nd; ++d) {
    Ctx& c = *b.h[d];
    join_coarse(c);
    if (c.stream == b.stream) continue;
    MGAR_CUDA(cudaEventRecord(b.ev_des[d], c.stream));
    MGAR_CUDA(cudaStreamWaitEvent(b.stream, b.ev_des[d], 0));
  }
}

uint64_t key_bits(double v) {
  uint64_t u;
  std::memcpy(&u, &v, sizeof u);
  return u;
}

// What a design's captured work depends on besides the batch's own buffers:
// its filter (radius and table size).
void key_filter(std::vector<uint64_t>& key, const Ctx& c) {
  key.push_back(key_bits(c.filter_r));
  key.push_back((uint64_t)c.n_filter);
}

// Launches g on the batch stream, capturing it first if its key changed:
// each design's work is captured on the batch's capture stream (the handle's
// side stream joins it for the coarsest factorisation and is joined back)
// and added to one graph as a child graph without dependencies, so the
// designs' branches run at once and the host issues one launch for all.
template <class F>
void launch_design_graph(Batch& b, Batch::DesignGraph& g, std::vector<uint64_t>&& key,
                                F&& chain) {
  if (!g.exec || g.key != key) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    cudaGraph_t parent = nullptr;
    MGAR_CUDA(cudaGraphCreate(&parent, 0));
    const int64_t before = launches_so_far();
    try {
      for (int d = 0; d < b.nd; ++d) {
        Ctx& c = *b.h[d];
        cudaStream_t saved = c.stream;
        cudaGraph_t gd = nullptr;
        MGAR_CUDA(cudaStreamBeginCapture(b.cap, cudaStreamCaptureModeThreadLocal));
        c.stream = b.cap;
        try {
          chain(d, c);
          join_coarse(c);
        } catch (...) {
          c.stream = saved;
          cudaStreamEndCapture(b.cap, &gd);
          if (gd) cudaGraphDestroy(gd);
          throw;
        }
        c.stream = saved;
        MGAR_CUDA(cudaStreamEndCapture(b.cap, &gd));
        cudaGraphNode_t node;
        const cudaError_t e = cudaGraphAddChildGraphNode(&node, parent, nullptr, 0, gd);
        cudaGraphDestroy(gd);
        MGAR_CUDA(e);
      }
      cudaGraphExec_t exec = nullptr;
      MGAR_CUDA(cudaGraphInstantiate(&exec, parent, 0));
      g.exec = exec;
    } catch (...) {
      cudaGraphDestroy(parent);
      count_launches(-(launches_so_far() - before));
      throw;
    }
    cudaGraphDestroy(parent);
    g.kernels = launches_so_far() - before;
    count_launches(-g.kernels);  // captured, not executed
    g.key = std::move(key);
  }
  MGAR_CUDA(cudaGraphLaunch(g.exec, b.stream));
  count_launches(g.kernels);
}

// Each design's hierarchy from its current design (K0 <- K), ordered after
// what the batch stream and the handle's stream hold; the batch stream
// waits for all of them.  As one graph of per-design branches, or (timed or
// graph-less handles) on the handles' own streams, so that the designs'
// builds (and their coarsest factorisations on the handles' side streams)
// run at once either way.
void build_hierarchies(Batch& b) {
  if (graphable(b)) {
    order_after_handles(b);
    launch_design_graph(b, b.g_hier, {}, [](int, Ctx& c) { build_hierarchy(c); });
    return;
  }
  MGAR_CUDA(cudaEventRecord(b.ev_start, b.stream));
  for (int d = 0; d < b.nd; ++d) {
    Ctx& c = *b.h[d];
    MGAR_CUDA(cudaStreamWaitEvent(c.stream, b.ev_start, 0));
    build_hierarchy(c);
    join_coarse(c);
    MGAR_CUDA(cudaEventRecord(b.ev_des[d], c.stream));
  }
  for (int d = 0; d < b.nd; ++d) MGAR_CUDA(cudaStreamWaitEvent(b.stream, b.ev_des[d], 0));
}

// The batched solve queued on the batch stream after the hierarchies: the
// callers' solution vectors and the per-design constants, the autotuner and
// the solve graph on the first call, the graph's launch.
void solve_issue(Batch& b, double* const* T) {
  std::vector<Des>& des = b.hdes;
  bool moved = false;
  for (int d = 0; d < b.nd; ++d) {
    moved = moved || des[d].T != T[d];
    des[d].T = T[d];
    b.hconsts[3 * d] = b.h[d]->qnorm;
    b.hconsts[3 * d + 1] = b.h[d]->p.eps2;
    b.hconsts[3 * d + 2] = (double)b.h[d]->p.cg_max;
  }
  if (moved)
    MGAR_CUDA(cudaMemcpyAsync(b.ddes, des.data(), b.nd * sizeof(Des), cudaMemcpyHostToDevice,
                              b.stream));
  MGAR_CUDA(cudaMemcpyAsync(b.consts, b.hconsts, (size_t)b.nd * 3 * sizeof(double),
                            cudaMemcpyHostToDevice, b.stream));
  if (!b.exec) {
    MGAR_CUDA(cudaStreamSynchronize(b.stream));
    autotune(b);
    build_graph(b);
  }
  b.eager = !graphable(b);
  if (b.eager) solve_eager(b);
  else MGAR_CUDA(cudaGraphLaunch(b.exec, b.stream));
}

// Every design's outcome to the host once the batch stream holds all the
// work: one gather kernel, one copy, one wait.
void gather_outcomes(Batch& b) {
  kb_gather<<<(b.nd + 127) / 128, 128, 0, b.stream>>>(b.ddes, b.nd, b.bsc);
  MGAR_LAUNCH_CHECK();
  MGAR_CUDA(cudaMemcpyAsync(b.hbsc, b.bsc, (size_t)b.nd * kBS * sizeof(double),
                            cudaMemcpyDeviceToHost, b.stream));
  MGAR_CUDA(cudaStreamSynchronize(b.stream));
}

// The solve's outcome per design from the gathered scalars; a coarsest
// factorisation that met a non-positive pivot is an error of the call.
int solve_read(Batch& b, int* iters, double* relres, int* status) {
  int maxit = 0;
  int rc = MGAR_OK;
  for (int d = 0; d < b.nd; ++d) {
    const double* s = b.hbsc + (size_t)d * kBS;
    const int it = (int)s[BS_IT];
    const double rel = std::sqrt(s[BS_RR]) / s[BS_QN];
    maxit = std::max(maxit, it);
    int st = MGAR_OK;
    if (s[BS_BAD] != 0.0 || !std::isfinite(rel)) st = MGAR_ERR_NONFINITE;
    else if (!(rel <= b.h[d]->p.eps2)) st = MGAR_ERR_MAXIT;
    if (iters) iters[d] = it;
    if (relres) relres[d] = rel;
    if (status) status[d] = st;
    if (st == MGAR_ERR_NONFINITE) rc = MGAR_ERR_NONFINITE;
    else if (st == MGAR_ERR_MAXIT && rc == MGAR_OK) rc = MGAR_ERR_MAXIT;
    // the solution is the handle's new reference
    b.h[d]->have_ref = true;
  }
  if (!b.eager) count_launches(b.prologue + (int64_t)maxit * b.body);
  for (int d = 0; d < b.nd; ++d) {
    const int e = (int)b.hbsc[(size_t)d * kBS + BS_DERR];
    if (e) {
      MGAR_CUDA(cudaMemset(b.h[d]->derr, 0, sizeof(int)));
      throw Error{e, "a coarsest factorisation met a non-positive pivot"};
    }
  }
  if (rc == MGAR_ERR_MAXIT) b.err = "a design reached cg_max";
  if (rc == MGAR_ERR_NONFINITE) b.err = "a design's CG broke down (non-finite residual)";
  return rc;
}

}  // namespace

extern "C" {

int mgar_batch_create(mgar_batch_t* out, const mgar_t* handles, int count, void* stream) {
  if (!out || !handles || count < 1) {
    g_batch_create_error = "mgar_batch_create: bad arguments";
    return MGAR_ERR_ARG;
  }
  *out = nullptr;
  Batch* b = new Batch();
  try {
    b->nd = count;
    b->stream = reinterpret_cast<cudaStream_t>(stream);
    for (int d = 0; d < count; ++d) {
      Ctx* c = reinterpret_cast<Ctx*>(handles[d]);
      require(c != nullptr, MGAR_ERR_ARG, "null handle");
      require(c->dim == 2 && c->p.precision == MGAR_MIXED, MGAR_ERR_ARG,
              "batched solves take 2D handles of the mixed precision");
      for (Ctx* o : b->h) require(o != c, MGAR_ERR_ARG, "a handle appears twice");
      b->h.push_back(c);
      b->lmax = std::max(b->lmax, c->nl);
    }
    const int nd = b->nd, lmax = b->lmax;
    b->s_node.resize(lmax);
    b->s_next.resize(lmax);
    b->tuned.assign(lmax, 256);
    MGAR_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    // tables
    std::vector<Lev> lev((size_t)lmax * nd);
    std::vector<Coarse> co(nd);
    std::vector<Des> des(nd);
    std::vector<int64_t> n0(nd);
    for (int d = 0; d < nd; ++d) {
      Ctx& c = *b->h[d];
      const Dims& d0 = c.L[0];
      n0[d] = d0.n;
      des[d].f = make_op(c);  // k_e pointers only: set_density keeps them current
      des[d].q = c.df_q;
      des[d].x = c.df_x;
      des[d].r = c.df_r;
      des[d].p = c.df_p;
      des[d].Ap = c.df_Ap;
      des[d].b32 = c.b32;
      des[d].x32 = c.x32;
      des[d].T = nullptr;  // the caller's T, set at each solve
      des[d].dsc = c.dsc;
      des[d].derr = c.derr;
      for (int l = 0; l + 1 < c.nl; ++l) {
        Lev& v = lev[(size_t)l * nd + d];
        const Dims& dl = c.L[l];
        const Dims& dn = c.L[l + 1];
        v.d = dl;
        v.dn = dn;
        v.omega = (float)c.p.omega;
        v.dinv = c.h32[l].dinv;
        v.dinv_n = c.h32[l + 1].dinv;
        v.t = c.h32[l].t;
        v.r = c.h32[l].r;
        if (l == 0) {
          v.f0 = FineOp<float>{c.ke0_f, nullptr, c.fixed, dl.ex, dl.ey, dl.ez, dl.NX, dl.NY, dl.NZ,
                               (int)dl.n, dl.fNX, dl.fNXY};
          v.x = c.x32;
          v.b = c.b32;
          v.fixed = c.fixed;
        } else {
          v.op = StencilOp<float>{c.h32[l].st, c.h32[l].dinv, dl.NX, dl.NY, dl.NZ, (int)dl.n,
                                  dl.fNX, dl.fNXY};
          v.x = c.h32[l].x;
          v.b = c.h32[l].b;
          v.fixed = nullptr;
        }
        const bool next_coarsest = l + 2 == c.nl;
        v.bn = c.h32[l + 1].b;
        v.xn = next_coarsest ? nullptr : c.h32[l + 1].x;
        v.resn = next_coarsest ? c.h32[l + 1].x : c.h32[l + 1].t;
      }
      co[d].cinv = c.cinv;
      co[d].b = c.h32[c.nl - 1].b;
      co[d].x = c.h32[c.nl - 1].x;
      co[d].nc = c.nc;
    }
    MGAR_CUDA(cudaMalloc(&b->dlev, lev.size() * sizeof(Lev)));
    MGAR_CUDA(cudaMemcpy(b->dlev, lev.data(), lev.size() * sizeof(Lev), cudaMemcpyHostToDevice));
    MGAR_CUDA(cudaMalloc(&b->dco, co.size() * sizeof(Coarse)));
    MGAR_CUDA(cudaMemcpy(b->dco, co.data(), co.size() * sizeof(Coarse), cudaMemcpyHostToDevice));
    MGAR_CUDA(cudaMalloc(&b->ddes, des.size() * sizeof(Des)));
    MGAR_CUDA(cudaMemcpy(b->ddes, des.data(), des.size() * sizeof(Des), cudaMemcpyHostToDevice));
    b->hdes = des;
    b->s_red = make_shape(n0, kRedThreads * kNptR, kRedThreads);
    for (int l = 0; l + 1 < lmax; ++l) make_level_shapes(*b, l, 256);
    make_coarse_shape(*b, 8);
    MGAR_CUDA(cudaMalloc(&b->bsc, (size_t)nd * kBS * sizeof(double)));
    MGAR_CUDA(cudaMemset(b->bsc, 0, (size_t)nd * kBS * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&b->consts, (size_t)nd * 3 * sizeof(double)));
    MGAR_CUDA(cudaHostAlloc(&b->hconsts, (size_t)nd * 3 * sizeof(double), cudaHostAllocDefault));
    MGAR_CUDA(cudaHostAlloc(&b->hbsc, (size_t)nd * kBS * sizeof(double), cudaHostAllocDefault));
    MGAR_CUDA(cudaMalloc(&b->partials, (size_t)std::max(b->s_red.nblocks, 1) * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&b->counters, (size_t)nd * sizeof(unsigned int)));
    MGAR_CUDA(cudaMemset(b->counters, 0, (size_t)nd * sizeof(unsigned int)));
    MGAR_CUDA(cudaMalloc(&b->any, sizeof(int)));
    MGAR_CUDA(cudaHostAlloc(&b->hany, sizeof(int), cudaHostAllocDefault));
    b->ev_des.assign(nd, nullptr);
    for (int d = 0; d < nd; ++d)
      MGAR_CUDA(cudaEventCreateWithFlags(&b->ev_des[d], cudaEventDisableTiming));
    MGAR_CUDA(cudaEventCreateWithFlags(&b->ev_solved, cudaEventDisableTiming));
    MGAR_CUDA(cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming));
    for (cudaEvent_t& e : b->ev_ph) MGAR_CUDA(cudaEventCreate(&e));
  } catch (const Error& e) {
    g_batch_create_error = e.msg;
    free_batch(*b);
    delete b;
    return e.code;
  }
  *out = reinterpret_cast<mgar_batch_t>(b);
  return MGAR_OK;
}

int mgar_batch_destroy(mgar_batch_t hb) {
  if (!hb) return MGAR_OK;
  Batch* b = reinterpret_cast<Batch*>(hb);
  free_batch(*b);
  delete b;
  return MGAR_OK;
}

const char* mgar_batch_last_error(mgar_batch_t hb) {
  if (!hb) return g_batch_create_error.c_str();
  return reinterpret_cast<Batch*>(hb)->err.c_str();
}

// The batched solve for the designs' current densities.
static int batch_solve(Batch& b, double* const* T, int* iters, double* relres, int* status) {
  require(T != nullptr, MGAR_ERR_ARG, "batch_solve_mgcg: null T");
  for (int d = 0; d < b.nd; ++d) require(T[d] != nullptr, MGAR_ERR_ARG, "batch_solve_mgcg: null T[d]");
  build_hierarchies(b);
  solve_issue(b, T);
  gather_outcomes(b);
  return solve_read(b, iters, relres, status);
}

int mgar_batch_solve_mgcg(mgar_batch_t hb, double* const* T, int* iters, double* relres,
                          int* status) {
  return bguard(hb, [&](Batch& b) { return batch_solve(b, T, iters, relres, status); });
}

int mgar_batch_cycle(mgar_batch_t hb, double* const* rho, double* const* T, const double* volfrac,
                     double move, mgar_step_info* info) {
  return bguard(hb, [&](Batch& b) {
    require(rho && T && volfrac, MGAR_ERR_ARG, "batch_cycle: null argument");
    require(move > 0.0, MGAR_ERR_ARG, "batch_cycle: move must be positive");
    const int nd = b.nd;
    for (int d = 0; d < nd; ++d) {
      require(rho[d] && T[d], MGAR_ERR_ARG, "batch_cycle: null rho[d] or T[d]");
      require(volfrac[d] > 0.0 && volfrac[d] < 1.0, MGAR_ERR_ARG, "batch_cycle: volfrac outside (0, 1)");
      require(!(b.h[d]->p.filter_alpha > 0.0), MGAR_ERR_ARG,
              "batch_cycle: the continuation filter schedule is per cycle of mgar_step");
    }
    // each design's sensitivities (Eq. 10 through the filter), compliance
    // and OC update after the solve
    auto post = [&](int d, Ctx& c) {
      sensitivity(c, T[d], nullptr, nullptr, nullptr, nullptr, dc_pairs(c));
      dot(c, c.q, T[d], c.n, c.dsc + S_COMPL);
      oc_issue(c, rho[d], nullptr, volfrac[d], move, dc_pairs(c));
    };
    if (graphable(b)) {
      // three launches from the host: every design's filter, SIMP and
      // hierarchy as one graph, the solve graph, every design's update as
      // one graph
      std::vector<uint64_t> kpre, kpost;
      for (int d = 0; d < nd; ++d) {
        kpre.push_back((uint64_t)(uintptr_t)rho[d]);
        key_filter(kpre, *b.h[d]);
      }
      kpost = kpre;
      for (int d = 0; d < nd; ++d) {
        kpost.push_back((uint64_t)(uintptr_t)T[d]);
        kpost.push_back(key_bits(volfrac[d]));
      }
      kpost.push_back(key_bits(move));
      order_after_handles(b);
      MGAR_CUDA(cudaEventRecord(b.ev_ph[0], b.stream));
      launch_design_graph(b, b.g_pre, std::move(kpre), [&](int d, Ctx& c) {
        set_density(c, rho[d], false);
        build_hierarchy(c);
      });
      MGAR_CUDA(cudaEventRecord(b.ev_ph[1], b.stream));
      const bool tuning = !b.exec;
      solve_issue(b, T);
      MGAR_CUDA(cudaEventRecord(b.ev_ph[2], b.stream));
      launch_design_graph(b, b.g_post, std::move(kpost), post);
      MGAR_CUDA(cudaEventRecord(b.ev_ph[3], b.stream));
      b.have_phases = !tuning;
    } else {
      // each design's filter and SIMP on its own stream, the hierarchies,
      // the solve, then the updates on the handles' streams again
      for (int d = 0; d < nd; ++d) {
        Ctx& c = *b.h[d];
        set_density(c, rho[d], false);
        MGAR_CUDA(cudaEventRecord(b.ev_des[d], c.stream));
        MGAR_CUDA(cudaStreamWaitEvent(b.stream, b.ev_des[d], 0));
      }
      build_hierarchies(b);
      solve_issue(b, T);
      MGAR_CUDA(cudaEventRecord(b.ev_solved, b.stream));
      for (int d = 0; d < nd; ++d) {
        Ctx& c = *b.h[d];
        MGAR_CUDA(cudaStreamWaitEvent(c.stream, b.ev_solved, 0));
        post(d, c);
        MGAR_CUDA(cudaEventRecord(b.ev_des[d], c.stream));
        MGAR_CUDA(cudaStreamWaitEvent(b.stream, b.ev_des[d], 0));
      }
    }
    gather_outcomes(b);
    if (b.have_phases)
      for (int k = 0; k < 3; ++k) {
        float ms = 0.f;
        MGAR_CUDA(cudaEventElapsedTime(&ms, b.ev_ph[k], b.ev_ph[k + 1]));
        b.phase_ms[k] = ms;
      }
    std::vector<int> it(nd), st(nd);
    std::vector<double> rr(nd);
    const int rc = solve_read(b, it.data(), rr.data(), st.data());
    for (int d = 0; d < nd; ++d) {
      Ctx& c = *b.h[d];
      const double* s = b.hbsc + (size_t)d * kBS;
      c.hsc[S_COMPL] = s[BS_COMPL];
      c.hsc[S_OC_LAM] = s[BS_LAM];
      c.hsc[S_OC_CHANGE] = s[BS_CHANGE];
      c.hsc[S_OC_FAIL] = s[BS_FAIL];
      double lam = 0.0, change = 0.0;
      oc_finish(c, rho[d], volfrac[d], &lam, &change);
      if (info) {
        mgar_step_info& inf = info[d];
        inf = mgar_step_info{};
        inf.compliance = c.hsc[S_COMPL];
        inf.res = NAN;
        inf.relres = rr[d];
        inf.lambda = lam;
        inf.used_mgcg = 1;
        inf.accepted = 0;
        inf.cg_iters = it[d];
        inf.status = st[d];
        inf.compliance_mgar = NAN;
      }
    }
    return rc;
  });
}

int mgar_batch_report(mgar_batch_t hb, char* buf, int64_t len) {
  return bguard(hb, [&](Batch& b) {
    require(buf && len > 0, MGAR_ERR_ARG, "batch_report: bad buffer");
    std::string r = b.report;
    if (b.have_phases) {
      char line[256];
      std::snprintf(line, sizeof line,
                    "last design cycle, device ms: filter+SIMP+hierarchy %.3f, solve %.3f, "
                    "sensitivities+OC %.3f\n",
                    b.phase_ms[0], b.phase_ms[1], b.phase_ms[2]);
      r += line;
    }
    const size_t n = std::min<size_t>((size_t)len - 1, r.size());
    std::memcpy(buf, r.data(), n);
    buf[n] = 0;
    return MGAR_OK;
  });
}

}  // extern "C"
