// MGCG of the mixed-precision path.  3D grids by default run FP32 CG
// iterations with reliable df64 updates (solve_mgcg_ru3, below); the rest of
// this file is the CG in double-float arithmetic (2D grids, and 3D on
// request).
//
// The outer conjugate-gradient iteration (Sections 1 and 3.2) keeps its
// vectors as df64 pairs (about 48 bits) and runs every operation on the FP32
// pipe; only the CG scalars are FP64.  The preconditioner is the FP32
// V-cycle.  The finest-level product uses the difference form of the
// conductivity stencil: K has zero row sums, so
//   (A x)_i = c * sum_j w_ij (x_i - x^_j),   x^_j = 0 on a fixed node,
// with w_ij = k_a + k_b for the face diagonals and k_e for the body diagonals
// of an H8 node (c = 1/12), w_ij = k_a + k_b along the edges and 2 k_e across
// the diagonals of a Q4 node (c = 1/6); a fixed row is the identity.  Each
// term is then rounded relative to its own size, not relative to |x|.
#include "common.cuh"
#include "df64.cuh"
#include "dfop.cuh"

namespace mgar {

namespace {

// y = A x; with DOT, x.y into out (warp sums in df64, FP64 across warps and
// blocks).  NPT nodes per thread: base, base + blockDim.x, ...
template <int DIM, bool DOT, int NPT = 1>
__global__ void k_df_apply(DfOp op, const float2* __restrict__ x, float2* __restrict__ y,
                           double* partials, unsigned int* counter, double* out) {
  const int base = blockIdx.x * blockDim.x * NPT + threadIdx.x;
  df v{0.f, 0.f};
#pragma unroll
  for (int u = 0; u < NPT; ++u) {
    const int idx = base + u * blockDim.x;
    if (idx < op.n) {
      const df yv = df_row<DIM>(op, x, idx);
      y[idx] = pack(yv);
      if (DOT) v = df_add(v, df_mul(unpack(x[idx]), yv));
    }
  }
  if (DOT) block_sum_finish_df(v, partials, counter, out);
}

// The 2D product with p . Ap, two nodes per thread.
constexpr int kNptApply2 = 2;

void df_apply2_dot(const DfOp& op, const float2* x, float2* y, double* partials,
                   unsigned int* counter, double* out, cudaStream_t s) {
  const int per = kThreads * kNptApply2;
  k_df_apply<2, true, kNptApply2><<<(op.n + per - 1) / per, kThreads, 0, s>>>(op, x, y, partials,
                                                                             counter, out);
}

// r = q - A x and ||r||^2
template <int DIM>
__global__ void k_df_residual(DfOp op, const float2* __restrict__ q, const float2* __restrict__ x,
                              float2* __restrict__ r, double* partials, unsigned int* counter,
                              double* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  df v{0.f, 0.f};
  if (idx < op.n) {
    const df ri = df_sub(unpack(q[idx]), df_row<DIM>(op, x, idx));
    r[idx] = pack(ri);
    v = df_mul(ri, ri);
  }
  block_sum_finish_df(v, partials, counter, out);
}

// alpha = rz / pAp; x += alpha p; r -= alpha Ap; ||r||^2; optionally the
// FP32 copy of r for the preconditioner
__global__ void k_df_cg_xr(float2* __restrict__ x, float2* __restrict__ r, const float2* __restrict__ p,
                           const float2* __restrict__ Ap, int n, const double* __restrict__ rz,
                           const double* __restrict__ pap, double* partials, unsigned int* counter,
                           double* out, float* __restrict__ r32,
                           const float2* __restrict__ p_alt = nullptr,
                           const double* parity = nullptr) {
  pdl_wait();
  // device-side CG loop: the two direction buffers swap with the parity
  if (parity && (((int)*parity) & 1)) p = p_alt;
  const df alpha = block_div_df(rz, pap);
  df acc{0.f, 0.f};
  const int stride = gridDim.x * blockDim.x;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  // two nodes per iteration: their eight loads are in flight together
  for (; i + stride < n; i += 2 * stride) {
    const int j = i + stride;
    const float2 xa = x[i], xb = x[j], pa = p[i], pb = p[j];
    const float2 ra = r[i], rb = r[j], qa = Ap[i], qb = Ap[j];
    x[i] = pack(df_add(unpack(xa), df_mul(alpha, unpack(pa))));
    x[j] = pack(df_add(unpack(xb), df_mul(alpha, unpack(pb))));
    const df ria = df_sub(unpack(ra), df_mul(alpha, unpack(qa)));
    const df rib = df_sub(unpack(rb), df_mul(alpha, unpack(qb)));
    r[i] = pack(ria);
    r[j] = pack(rib);
    if (r32) {
      r32[i] = __fadd_rn(ria.hi, ria.lo);
      r32[j] = __fadd_rn(rib.hi, rib.lo);
    }
    acc = df_add(acc, df_mul(ria, ria));
    acc = df_add(acc, df_mul(rib, rib));
  }
  for (; i < n; i += stride) {
    x[i] = pack(df_add(unpack(x[i]), df_mul(alpha, unpack(p[i]))));
    const df ri = df_sub(unpack(r[i]), df_mul(alpha, unpack(Ap[i])));
    r[i] = pack(ri);
    if (r32) r32[i] = __fadd_rn(ri.hi, ri.lo);
    acc = df_add(acc, df_mul(ri, ri));
  }
  block_sum_finish_df(acc, partials, counter, out);
}

// p = z + (rz_new / rz_old) p, z in FP32
__global__ void k_df_cg_p(float2* __restrict__ p, const float* __restrict__ z, int n,
                          const double* __restrict__ rz_new, const double* __restrict__ rz_old) {
  const df beta = block_div_df(rz_new, rz_old);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = pack(df_add(df{z[i], 0.f}, df_mul(beta, unpack(p[i]))));
}

// r . z with z in FP32
__global__ void k_df_dot_f(const float2* __restrict__ r, const float* __restrict__ z, int n,
                           double* partials, unsigned int* counter, double* out) {
  df acc{0.f, 0.f};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    acc = df_add(acc, df_mulf(unpack(r[i]), z[i]));
  block_sum_finish_df(acc, partials, counter, out);
}

__global__ void k_df_to_f32(const float2* __restrict__ a, float* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __fadd_rn(a[i].x, a[i].y);
}

__global__ void k_f32_to_df(const float* __restrict__ a, float2* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2(a[i], 0.f);
}

__global__ void k_d_to_df(const double* __restrict__ a, float2* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = pack(df_from_double(a[i]));
}

__global__ void k_df_to_d(const float2* __restrict__ a, double* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = df_to_double(unpack(a[i]));
}

}  // namespace

// y = A x for FP64 vectors through df64 arithmetic (x converted on the way in,
// y on the way out); the MGAR projection of the mixed path uses it.
void apply_df64(Ctx& c, const double* x, double* y) {
  const int n = (int)c.n;
  ProfScope ps(c, MGAR_KC_APPLY64);
  if (c.dim == 3 && !c.untiled) {
    df3d_apply(c, x, y, nullptr);  // FP64 in and out, converted in the kernel
    return;
  }
  k_d_to_df<<<blocks_for(n), kThreads, 0, c.stream>>>(x, c.df_p, n);
  MGAR_LAUNCH_CHECK();
  const DfOp op = make_op(c);
  {
    if (c.dim == 2)
      k_df_apply<2, false><<<blocks_for(n), kThreads, 0, c.stream>>>(op, c.df_p, c.df_Ap, nullptr,
                                                                     nullptr, nullptr);
    else
      k_df_apply<3, false><<<blocks_for(n), kThreads, 0, c.stream>>>(op, c.df_p, c.df_Ap, nullptr,
                                                                     nullptr, nullptr);
    MGAR_LAUNCH_CHECK();
  }
  k_df_to_d<<<blocks_for(n), kThreads, 0, c.stream>>>(c.df_Ap, y, n);
  MGAR_LAUNCH_CHECK();
}

// k_e of the current design in df64 form
void ke_to_df(Ctx& c) {
  k_d_to_df<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(c.ke, c.ke_df, (int)c.ne);
  MGAR_LAUNCH_CHECK();
}

void q_to_df(Ctx& c) {
  k_d_to_df<<<blocks_for(c.n), kThreads, 0, c.stream>>>(c.q, c.df_q, (int)c.n);
  MGAR_LAUNCH_CHECK();
}

// z32 = M r with r in df64: FP32 copy of r, then the FP32 V-cycle
static void precondition_df(Ctx& c) {
  const int n = (int)c.n;
  const bool prof_inside = c.prof_class == MGAR_KC_SMOOTH0 || c.prof_class == MGAR_KC_RESID0;
  run_graph(c, 6, c.df_r, c.x32, prof_inside, [&] {
    k_df_to_f32<<<blocks_for(n), kThreads, 0, c.stream>>>(c.df_r, c.b32, n);
    MGAR_LAUNCH_CHECK();
    vcycle<float>(c, c.b32, c.x32, true);
  });
}

// Device-side CG loop (one graph per handle): iteration count and buffer
// parity start at zero ...
__global__ void k_cg_reset(double* dsc) {
  dsc[S_CGIT] = 0.0;
  dsc[S_CGPAR] = 0.0;
}

// ... and after each update of x and r: count the iteration, flip the
// parity, and continue while ||r|| / ||q|| > eps2 (the host loop's test,
// same arithmetic) and fewer than cg_max iterations ran; a non-finite
// residual stops the loop and the host reports it.  shift: the iteration's
// r . z (RZ1) becomes the next one's old value (RZ0).
__global__ void k_cg_check(double* dsc, double qnorm, double eps2, int cg_max,
                           cudaGraphConditionalHandle loop, int shift) {
  const double rel = sqrt(dsc[S_RR]) / qnorm;
  const int it = (int)dsc[S_CGIT] + 1;
  dsc[S_CGIT] = (double)it;
  dsc[S_CGPAR] = (double)(((int)dsc[S_CGPAR]) ^ 1);
  if (shift) dsc[S_RZ0] = dsc[S_RZ1];
  const bool go = isfinite(rel) && rel > eps2 && it < cg_max;
  cudaGraphSetConditional(loop, go ? 1u : 0u);
}

// z32 = M r32 (the FP32 copy of r is written by the residual and update
// kernels) and r . z into dsc[slot], fused into the V-cycle's last kernel
static void precondition_f32(Ctx& c, int slot) {
  const bool prof_inside = c.prof_class == MGAR_KC_SMOOTH0 || c.prof_class == MGAR_KC_RESID0;
  double* out = c.dsc + slot;
  run_graph(c, slot == S_RZ0 ? 8 : 9, c.b32, c.x32, prof_inside,
            [&] { vcycle_dot(c, c.b32, c.x32, c.df_r, out); });
}

// 3D: the tiled kernels fuse the direction update into the product
// (p = z + beta p_old, A p, p.Ap in one pass) and write the FP32 copy of r
// beside r, so an iteration is: product, update of x and r, V-cycle, r.z.
// One CG iteration of the device-side loop: V-cycle (r . z into RZ1), the
// direction update and product (beta = RZ1 / RZ0, then RZ0 <- RZ1), the
// update of x and r, the convergence check.
static void cg_iteration(Ctx& c, bool first, cudaGraphConditionalHandle loop) {
  const int n = (int)c.n;
  vcycle_dot(c, c.b32, c.x32, c.df_r, c.dsc + S_RZ1);
  df3d_dir(c, c.x32, c.df_p, c.df_p2, c.dsc + S_RZ1, c.dsc + S_RZ0, first, c.df_Ap, c.dsc + S_PAP,
           c.dsc + S_CGPAR, c.dsc + S_RZ0);
  // parity 0: the new p is in df_p2
  launch_pdl(c.stream, c.use_pdl, k_df_cg_xr, dim3(c.grid_blocks), dim3(kThreads), c.df_x, c.df_r,
             (const float2*)c.df_p2, (const float2*)c.df_Ap, n, (const double*)(c.dsc + S_RZ0),
             (const double*)(c.dsc + S_PAP), c.partials, c.counter, c.dsc + S_RR, c.b32,
             (const float2*)c.df_p, (const double*)(c.dsc + S_CGPAR));
  MGAR_LAUNCH_CHECK();
  k_cg_check<<<1, 1, 0, c.stream>>>(c.dsc, c.qnorm, c.p.eps2, c.p.cg_max, loop, 0);
  MGAR_LAUNCH_CHECK();
}

// 2D: one CG iteration of the device-side loop with the generic kernels,
// the host loop's steps and arithmetic: V-cycle z = M r (r's FP32 copy is
// written by the update of x and r), r . z into RZ1, p = z (first) or
// p = z + (RZ1 / RZ0) p, A p with p . A p, the update of x and r with
// alpha = RZ1 / pAp, the check (which moves RZ1 to RZ0).
static void cg_iteration_2d(Ctx& c, bool first, cudaGraphConditionalHandle loop) {
  const int n = (int)c.n;
  const int rb = c.grid_blocks;
  const DfOp op = make_op(c);
  if (first) {
    k_df_to_f32<<<blocks_for(n), kThreads, 0, c.stream>>>(c.df_r, c.b32, n);
    MGAR_LAUNCH_CHECK();
  }
  if (vcycle_dot_ok(c)) {
    // r . z fused into the V-cycle's last sweep
    vcycle_dot(c, c.b32, c.x32, c.df_r, c.dsc + S_RZ1);
  } else {
    vcycle<float>(c, c.b32, c.x32, true);
    k_df_dot_f<<<rb, kThreads, 0, c.stream>>>(c.df_r, c.x32, n, c.partials, c.counter,
                                              c.dsc + S_RZ1);
    MGAR_LAUNCH_CHECK();
  }
  if (first)
    k_f32_to_df<<<blocks_for(n), kThreads, 0, c.stream>>>(c.x32, c.df_p, n);
  else
    k_df_cg_p<<<rb, kThreads, 0, c.stream>>>(c.df_p, c.x32, n, c.dsc + S_RZ1, c.dsc + S_RZ0);
  MGAR_LAUNCH_CHECK();
  df_apply2_dot(op, c.df_p, c.df_Ap, c.partials, c.counter, c.dsc + S_PAP, c.stream);
  MGAR_LAUNCH_CHECK();
  k_df_cg_xr<<<rb, kThreads, 0, c.stream>>>(c.df_x, c.df_r, c.df_p, c.df_Ap, n, c.dsc + S_RZ1,
                                            c.dsc + S_PAP, c.partials, c.counter, c.dsc + S_RR,
                                            c.b32);
  MGAR_LAUNCH_CHECK();
  k_cg_check<<<1, 1, 0, c.stream>>>(c.dsc, c.qnorm, c.p.eps2, c.p.cg_max, loop, 1);
  MGAR_LAUNCH_CHECK();
}

// Builds the graph of the whole preconditioned CG after the initial
// residual: reset, one peeled iteration, then a WHILE node whose body is one
// iteration and whose condition the check kernel sets.  The host waits once
// per solve instead of once per iteration.  False if the device or driver
// refuses any part (the host loop is used then).
static bool build_cg_graph(Ctx& c) {
  auto iteration = c.dim == 2 ? cg_iteration_2d : cg_iteration;
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle loop = 0;
  cudaStream_t saved = c.stream;
  bool ok = false;
  const int64_t before = launches_so_far();
  auto fail = [&](cudaError_t e) {
    (void)e;
    (void)cudaGetLastError();
    return false;
  };
  do {
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) { fail(e); break; }
    e = cudaGraphConditionalHandleCreate(&loop, g, 0, 0);
    if (e != cudaSuccess) { fail(e); break; }
    e = cudaStreamBeginCaptureToGraph(c.cap_stream, g, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { fail(e); break; }
    c.stream = c.cap_stream;
    bool issued = true;
    cudaGraph_t body = nullptr;
    try {
      k_cg_reset<<<1, 1, 0, c.stream>>>(c.dsc);
      MGAR_LAUNCH_CHECK();
      iteration(c, true, loop);
      // the WHILE node after everything captured so far
      cudaStreamCaptureStatus st;
      cudaGraph_t cg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      const cudaGraphEdgeData* edges = nullptr;
      size_t ndeps = 0;
      MGAR_CUDA(cudaStreamGetCaptureInfo(c.stream, &st, nullptr, &cg, &deps, &edges, &ndeps));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = loop;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      cudaGraphNode_t wnode = nullptr;
      MGAR_CUDA(cudaGraphAddNode(&wnode, cg, deps, nullptr, ndeps, &cp));
      body = cp.conditional.phGraph_out[0];
      MGAR_CUDA(cudaStreamUpdateCaptureDependencies(c.stream, &wnode, nullptr, 1,
                                                    cudaStreamSetCaptureDependencies));
    } catch (...) {
      issued = false;
    }
    cudaGraph_t gout = nullptr;
    e = cudaStreamEndCapture(c.cap_stream, &gout);
    c.stream = saved;
    if (!issued || e != cudaSuccess || !body) { fail(e); break; }
    // the body: one more iteration per pass
    e = cudaStreamBeginCaptureToGraph(c.cap_stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { fail(e); break; }
    c.stream = c.cap_stream;
    const int64_t body_before = launches_so_far();
    try {
      iteration(c, false, loop);
    } catch (...) {
      issued = false;
    }
    c.body_kernels = launches_so_far() - body_before;
    cudaGraph_t bout = nullptr;
    e = cudaStreamEndCapture(c.cap_stream, &bout);
    c.stream = saved;
    if (!issued || e != cudaSuccess) { fail(e); break; }
    e = cudaGraphInstantiate(&c.cg_exec, g, 0);
    if (e != cudaSuccess) { c.cg_exec = nullptr; fail(e); break; }
    c.cg_exec_cgmax = c.p.cg_max;
    ok = true;
  } while (false);
  c.stream = saved;
  const int64_t captured = launches_so_far() - before;
  count_launches(-captured);  // captured, not executed
  c.prologue_kernels = captured - c.body_kernels;
  if (g) cudaGraphDestroy(g);
  return ok;
}

// The graph holds the iteration cap by value: one built for another cap
// (the df64 CG finishing a reliable-update solve gets the iterations left)
// is rebuilt.
static void drop_stale_cg_graph(Ctx& c) {
  if (c.cg_exec && c.cg_exec_cgmax != c.p.cg_max) {
    MGAR_CUDA(cudaGraphExecDestroy(c.cg_exec));
    c.cg_exec = nullptr;
  }
}

static int solve_mgcg_df3(Ctx& c, double* T, int* iters, double* relres) {
  const int n = (int)c.n;
  const int rb = c.grid_blocks;
  k_d_to_df<<<blocks_for(n), kThreads, 0, c.stream>>>(T, c.df_x, n);
  MGAR_LAUNCH_CHECK();
  {
    ProfScope ps(c, MGAR_KC_APPLY64);
    df3d_resid(c, c.df_q, c.df_x, c.df_r, c.b32, c.dsc + S_RR);
  }
  fetch_scalars(c, S_RR, 1);
  double rel = std::sqrt(c.hsc[S_RR]) / c.qnorm;
  int it = 0;
  // the device-side loop while no kernel class is being timed with events
  // (event records cannot sit inside a conditional body)
  if (!(rel <= c.p.eps2) && c.cg_graph && c.prof_class == 0 && c.use_graphs) {
    require(std::isfinite(rel), MGAR_ERR_NONFINITE, "non-finite initial residual");
    drop_stale_cg_graph(c);
    if (!c.cg_exec && !build_cg_graph(c)) c.cg_graph = false;
  }
  if (!(rel <= c.p.eps2) && c.cg_exec && c.prof_class == 0 && c.use_graphs) {
    join_coarse(c);
    MGAR_CUDA(cudaGraphLaunch(c.cg_exec, c.stream));
    fetch_scalars(c, S_RR, S_CGIT - S_RR + 1);
    it = (int)c.hsc[S_CGIT];
    count_launches(c.prologue_kernels + (int64_t)std::max(it - 1, 0) * c.body_kernels);
    rel = std::sqrt(c.hsc[S_RR]) / c.qnorm;
    require(std::isfinite(rel), MGAR_ERR_NONFINITE, "CG breakdown (non-finite residual)");
  } else if (!(rel <= c.p.eps2)) {
    require(std::isfinite(rel), MGAR_ERR_NONFINITE, "non-finite initial residual");
    int a = S_RZ0, b = S_RZ1;
    precondition_f32(c, a);
    float2* pcur = c.df_p;
    float2* pnext = c.df_p2;
    bool first = true;
    while (it < c.p.cg_max) {
      {
        ProfScope ps(c, MGAR_KC_APPLY64);
        df3d_dir(c, c.x32, pcur, pnext, c.dsc + a, c.dsc + b, first, c.df_Ap, c.dsc + S_PAP);
      }
      first = false;
      std::swap(pcur, pnext);
      launch_pdl(c.stream, c.use_pdl, k_df_cg_xr, dim3(rb), dim3(kThreads), c.df_x, c.df_r,
                 (const float2*)pcur, (const float2*)c.df_Ap, n, (const double*)(c.dsc + a),
                 (const double*)(c.dsc + S_PAP), c.partials, c.counter, c.dsc + S_RR, c.b32,
                 (const float2*)nullptr, (const double*)nullptr);
      MGAR_LAUNCH_CHECK();
      ++it;
      fetch_scalars(c, S_RR, 1);
      rel = std::sqrt(c.hsc[S_RR]) / c.qnorm;
      require(std::isfinite(rel), MGAR_ERR_NONFINITE, "CG breakdown (non-finite residual)");
      if (rel <= c.p.eps2) break;
      std::swap(a, b);
      precondition_f32(c, a);
    }
  }
  k_df_to_d<<<blocks_for(n), kThreads, 0, c.stream>>>(c.df_x, T, n);
  MGAR_LAUNCH_CHECK();
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return rel <= c.p.eps2 ? MGAR_OK : MGAR_ERR_MAXIT;
}

// ---------------------------------------------------------------------------
// 3D: FP32 conjugate-gradient iterations with reliable updates.
//
// The Krylov vectors (the correction xc accumulated since the last update,
// r, p, A p) are FP32, so an iteration costs an FP32 product instead of the
// df64 one.  Whenever the recursively updated ||r|| has fallen below
// ru_delta times its value at the last update, or below eps2 ||q||, or the
// iteration limit is reached, the correction is added to the df64 solution
// (x += xc, xc = 0) and r is recomputed from it in df64 (r = q - A x): the
// reliable updates of Sleijpen and van der Vorst ("Reliable updated
// residuals in hybrid Bi-CG methods", Computing 56, 1996), as mixed-precision
// lattice solvers use them.  The search direction is kept across an update.
// Convergence is decided on the recomputed residual, so the reported
// ||r|| / ||q|| is a df64 residual of the returned x.

// After an iteration: count it, flip the parity, and decide whether a
// reliable update is due: ||r|| <= eps2 ||q||, ||r|| <= delta ||r||_last
// update, cg_max iterations, or a non-finite ||r||.  Inside the graph the
// decision sets the IF node of the update (ru); the flag is also left in
// S_FLAG.  Run by one thread after ||r||^2 is in S_RR.
__device__ void ru_decide(double* dsc, double qnorm, double eps2, double delta, int cg_max,
                          cudaGraphConditionalHandle ru, int set) {
  const double rn = sqrt(dsc[S_RR]);
  const int it = (int)dsc[S_CGIT] + 1;
  dsc[S_CGIT] = (double)it;
  dsc[S_CGPAR] = (double)(((int)dsc[S_CGPAR]) ^ 1);
  dsc[S_CGFIRST] = 0.0;
  const bool upd = !(isfinite(rn) && rn > eps2 * qnorm && rn > delta * dsc[S_RMAX] && it < cg_max);
  dsc[S_FLAG] = upd ? 1.0 : 0.0;
  dsc[S_RREC] = rn;
  if (set) cudaGraphSetConditional(ru, upd ? 1u : 0u);
}

// alpha = rz / pAp; xc += alpha p; r -= alpha A p; ||r||^2 into dsc[S_RR],
// then the update decision (ru_decide) in the last block
__global__ void k_cg_xr32(float* __restrict__ xc, float* __restrict__ r, const float* __restrict__ p,
                          const float* __restrict__ p_alt, const double* parity,
                          const float* __restrict__ Ap, int n, const double* __restrict__ rz,
                          const double* __restrict__ pap, double* partials, unsigned int* counter,
                          double* dsc, double qnorm, double eps2, double delta, int cg_max,
                          cudaGraphConditionalHandle ru, int set) {
  pdl_wait();
  // every block reads the parity before the last one flips it
  if (parity && (((int)*parity) & 1)) p = p_alt;
  const float alpha = block_div_f(rz, pap);
  float acc = 0.f;
  const int stride = gridDim.x * blockDim.x;
  const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
  // four nodes per access (the vectors are 256-byte aligned allocations)
  const int n4 = n >> 2;
  float4* __restrict__ xc4 = reinterpret_cast<float4*>(xc);
  float4* __restrict__ r4 = reinterpret_cast<float4*>(r);
  const float4* __restrict__ p4 = reinterpret_cast<const float4*>(p);
  const float4* __restrict__ a4 = reinterpret_cast<const float4*>(Ap);
  for (int q = t0; q < n4; q += stride) {
    float4 xv = xc4[q], rv = r4[q];
    const float4 pv = p4[q], av = a4[q];
    xv.x = fmaf(alpha, pv.x, xv.x);
    xv.y = fmaf(alpha, pv.y, xv.y);
    xv.z = fmaf(alpha, pv.z, xv.z);
    xv.w = fmaf(alpha, pv.w, xv.w);
    rv.x = fmaf(-alpha, av.x, rv.x);
    rv.y = fmaf(-alpha, av.y, rv.y);
    rv.z = fmaf(-alpha, av.z, rv.z);
    rv.w = fmaf(-alpha, av.w, rv.w);
    xc4[q] = xv;
    r4[q] = rv;
    acc = fmaf(rv.x, rv.x, acc);
    acc = fmaf(rv.y, rv.y, acc);
    acc = fmaf(rv.z, rv.z, acc);
    acc = fmaf(rv.w, rv.w, acc);
  }
  for (int i = 4 * n4 + t0; i < n; i += stride) {
    xc[i] = fmaf(alpha, p[i], xc[i]);
    const float ri = fmaf(-alpha, Ap[i], r[i]);
    r[i] = ri;
    acc = fmaf(ri, ri, acc);
  }
  double t;
  if (block_sum_last_df(df{acc, 0.f}, partials, counter, t, threadIdx.x, blockDim.x, blockIdx.x,
                        gridDim.x) &&
      threadIdx.x == 0) {
    dsc[S_RR] = t;
    ru_decide(dsc, qnorm, eps2, delta, cg_max, ru, set);
  }
}

// iteration count, buffer parity, first-direction flag and the reference
// ||r|| after the initial residual
__global__ void k_ru_start(double* dsc) {
  dsc[S_CGIT] = 0.0;
  dsc[S_CGPAR] = 0.0;
  dsc[S_CGFIRST] = 1.0;
  dsc[S_RMAX] = sqrt(dsc[S_RR]);
  dsc[S_RUCOUNT] = 0.0;
  dsc[S_RUSTALL] = 0.0;
}

// x += xc in df64, xc = 0
__global__ void k_ru_update(float2* __restrict__ x, float* __restrict__ xc, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] = pack(df_add(unpack(x[i]), df{xc[i], 0.f}));
    xc[i] = 0.f;
  }
}

// After an update: the new reference ||r||.  Near the accuracy floor of the
// FP32 iterations the recursive residual drifts from the true one; an update
// that finds the true ||r|| above twice the recursive one restarts the
// direction (beta = 0), since beta's old r . z belongs to the drifted
// recursion, and updates that no longer halve the true ||r|| are counted so
// the loop can stop and leave the rest to the df64 CG.
__global__ void k_ru_mark(double* dsc) {
  const double rt = sqrt(dsc[S_RR]);
  if (rt > 2.0 * dsc[S_RREC]) dsc[S_CGFIRST] = 1.0;
  dsc[S_RUSTALL] = rt > 0.5 * dsc[S_RMAX] ? dsc[S_RUSTALL] + 1.0 : 0.0;
  dsc[S_RMAX] = rt;
  dsc[S_RUCOUNT] += 1.0;
}

// end of a pass of the graph's WHILE body: stop once an update has shown
// ||r|| <= eps2 ||q||, at cg_max iterations, on a non-finite ||r||, or after
// two updates in a row that did not halve the true ||r||
__global__ void k_ru_loop(double* dsc, double qnorm, double eps2, int cg_max,
                          cudaGraphConditionalHandle loop) {
  const double rn = sqrt(dsc[S_RR]);
  const int it = (int)dsc[S_CGIT];
  const bool conv = dsc[S_FLAG] != 0.0 && rn <= eps2 * qnorm;
  const bool go = !conv && isfinite(rn) && it < cg_max && dsc[S_RUSTALL] < 2.0;
  cudaGraphSetConditional(loop, go ? 1u : 0u);
}

// One FP32 iteration: V-cycle z = M r with r . z into RZ1, direction update
// and product (beta = RZ1 / RZ0, then RZ0 <- RZ1), update of xc and r, and
// the update decision.  set: inside the graph (the decision sets the IF
// handle ru); otherwise the V-cycle is replayed from its own graph and the
// host reads the decision.
static void ru_iteration(Ctx& c, cudaGraphConditionalHandle ru, bool set) {
  const int n = (int)c.n;
  if (set) {
    vcycle_dot(c, c.b32, c.x32, nullptr, c.dsc + S_RZ1);
  } else {
    const bool prof_inside = c.prof_class == MGAR_KC_SMOOTH0 || c.prof_class == MGAR_KC_RESID0;
    run_graph(c, 10, c.b32, c.x32, prof_inside,
              [&] { vcycle_dot(c, c.b32, c.x32, nullptr, c.dsc + S_RZ1); });
  }
  {
    ProfScope ps(c, MGAR_KC_APPLY32);
    fine3d_dir(c, c.x32, c.p32, c.p32b, c.dsc + S_RZ1, c.dsc + S_RZ0, c.dsc + S_CGFIRST,
               c.dsc + S_CGPAR, c.y32, c.dsc + S_PAP, c.dsc + S_RZ0);
  }
  // parity 0: the new p is in p32b
  launch_pdl(c.stream, c.use_pdl, k_cg_xr32, dim3(c.grid_blocks), dim3(kThreads), c.xc32, c.b32,
             (const float*)c.p32b, (const float*)c.p32, (const double*)(c.dsc + S_CGPAR),
             (const float*)c.y32, n, (const double*)(c.dsc + S_RZ0),
             (const double*)(c.dsc + S_PAP), c.partials, c.counter, c.dsc, c.qnorm, c.p.eps2,
             c.ru_delta, c.p.cg_max, ru, set ? 1 : 0);
  MGAR_LAUNCH_CHECK();
}

// Reliable update: x += xc, r = q - A x in df64 (only its FP32 copy and
// ||r||^2 are kept), reference ||r|| for the next decision.
static void ru_update(Ctx& c) {
  k_ru_update<<<c.grid_blocks, kThreads, 0, c.stream>>>(c.df_x, c.xc32, (int)c.n);
  MGAR_LAUNCH_CHECK();
  {
    ProfScope ps(c, MGAR_KC_RESID64);
    df3d_resid(c, c.df_q, c.df_x, nullptr, c.b32, c.dsc + S_RR);
  }
  k_ru_mark<<<1, 1, 0, c.stream>>>(c.dsc);
  MGAR_LAUNCH_CHECK();
}

// The graph of the whole FP32 iteration with its reliable updates: one
// WHILE node (condition 1 at every launch) whose body is an iteration, an
// IF node holding the update (condition set by the iteration's decision),
// and the loop test.  The host waits once per solve.  False if the device or
// driver refuses any part (the host loop is used then).
static bool build_ru_graph(Ctx& c) {
  cudaGraph_t g = nullptr;
  cudaGraphConditionalHandle loop = 0, ru = 0;
  cudaStream_t saved = c.stream;
  bool ok = false;
  const int64_t before = launches_so_far();
  int64_t upd_kernels = 0;
  do {
    if (cudaGraphCreate(&g, 0) != cudaSuccess) break;
    if (cudaGraphConditionalHandleCreate(&loop, g, 1, cudaGraphCondAssignDefault) != cudaSuccess)
      break;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = loop;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wnode = nullptr;
    if (cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &cp) != cudaSuccess) break;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if (cudaGraphConditionalHandleCreate(&ru, body, 0, cudaGraphCondAssignDefault) != cudaSuccess)
      break;
    if (cudaStreamBeginCaptureToGraph(c.cap_stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      break;
    c.stream = c.cap_stream;
    bool issued = true;
    try {
      ru_iteration(c, ru, true);
      // the IF node after the decision, its body captured on a second stream
      cudaStreamCaptureStatus st;
      cudaGraph_t bg = nullptr;
      const cudaGraphNode_t* deps = nullptr;
      const cudaGraphEdgeData* edges = nullptr;
      size_t ndeps = 0;
      MGAR_CUDA(cudaStreamGetCaptureInfo(c.stream, &st, nullptr, &bg, &deps, &edges, &ndeps));
      cudaGraphNodeParams ip = {};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = ru;
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      cudaGraphNode_t inode = nullptr;
      MGAR_CUDA(cudaGraphAddNode(&inode, bg, deps, nullptr, ndeps, &ip));
      cudaGraph_t ibody = ip.conditional.phGraph_out[0];
      MGAR_CUDA(cudaStreamBeginCaptureToGraph(c.cap_stream2, ibody, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal));
      c.stream = c.cap_stream2;
      const int64_t u0 = launches_so_far();
      bool upd_ok = true;
      try {
        ru_update(c);
      } catch (...) {
        upd_ok = false;
      }
      upd_kernels = launches_so_far() - u0;
      cudaGraph_t iout = nullptr;
      const cudaError_t ie = cudaStreamEndCapture(c.cap_stream2, &iout);
      c.stream = c.cap_stream;
      if (!upd_ok || ie != cudaSuccess) throw Error{MGAR_ERR_CUDA, "update capture failed"};
      MGAR_CUDA(cudaStreamUpdateCaptureDependencies(c.stream, &inode, nullptr, 1,
                                                    cudaStreamSetCaptureDependencies));
      k_ru_loop<<<1, 1, 0, c.stream>>>(c.dsc, c.qnorm, c.p.eps2, c.p.cg_max, loop);
      MGAR_LAUNCH_CHECK();
    } catch (...) {
      issued = false;
    }
    cudaGraph_t bout = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c.cap_stream, &bout);
    c.stream = saved;
    if (!issued || e != cudaSuccess) break;
    if (cudaGraphInstantiate(&c.ru_exec, g, 0) != cudaSuccess) {
      c.ru_exec = nullptr;
      break;
    }
    ok = true;
  } while (false);
  if (!ok) (void)cudaGetLastError();
  c.stream = saved;
  const int64_t captured = launches_so_far() - before;
  count_launches(-captured);  // captured, not executed
  c.ru_body_kernels = captured - upd_kernels;
  c.ru_update_kernels = upd_kernels;
  if (g) cudaGraphDestroy(g);
  return ok;
}

static int solve_mgcg_ru3(Ctx& c, double* T, int* iters, double* relres) {
  const int n = (int)c.n;
  k_d_to_df<<<blocks_for(n), kThreads, 0, c.stream>>>(T, c.df_x, n);
  MGAR_LAUNCH_CHECK();
  {
    ProfScope ps(c, MGAR_KC_RESID64);
    df3d_resid(c, c.df_q, c.df_x, nullptr, c.b32, c.dsc + S_RR);
  }
  fetch_scalars(c, S_RR, 1);
  double rel = std::sqrt(c.hsc[S_RR]) / c.qnorm;
  int it = 0;
  if (!(rel <= c.p.eps2)) {
    require(std::isfinite(rel), MGAR_ERR_NONFINITE, "non-finite initial residual");
    zero_async(c.xc32, n, c.stream);
    MGAR_LAUNCH_CHECK();
    k_ru_start<<<1, 1, 0, c.stream>>>(c.dsc);
    MGAR_LAUNCH_CHECK();
    // the graph while no kernel class is being timed with events
    const bool use_graph = c.cg_graph && c.prof_class == 0 && c.use_graphs &&
                           (c.ru_exec || build_ru_graph(c));
    if (use_graph) {
      join_coarse(c);
      MGAR_CUDA(cudaGraphLaunch(c.ru_exec, c.stream));
      fetch_scalars(c, S_RR, S_RUCOUNT - S_RR + 1);  // one fetch: RR..CGIT and RUCOUNT
      it = (int)c.hsc[S_CGIT];
      count_launches((int64_t)it * c.ru_body_kernels +
                     (int64_t)c.hsc[S_RUCOUNT] * c.ru_update_kernels);
      rel = std::sqrt(c.hsc[S_RR]) / c.qnorm;
    } else {
      double rmax = std::sqrt(c.hsc[S_RR]);  // ||r|| at the last reliable update
      while (true) {
        ru_iteration(c, 0, false);
        fetch_scalars(c, S_RR, S_CGIT - S_RR + 1);
        const double rn = std::sqrt(c.hsc[S_RR]);
        it = (int)c.hsc[S_CGIT];
        if (std::isfinite(rn) && rn > c.p.eps2 * c.qnorm && rn > c.ru_delta * rmax &&
            it < c.p.cg_max)
          continue;
        ru_update(c);
        fetch_scalars(c, S_RR, 1);
        rmax = std::sqrt(c.hsc[S_RR]);
        rel = rmax / c.qnorm;
        require(std::isfinite(rel), MGAR_ERR_NONFINITE, "CG breakdown (non-finite residual)");
        if (rel <= c.p.eps2 || it >= c.p.cg_max) break;
        fetch_scalars(c, S_RUSTALL, 1);
        if (c.hsc[S_RUSTALL] >= 2.0) break;
      }
    }
    require(std::isfinite(rel), MGAR_ERR_NONFINITE, "CG breakdown (non-finite residual)");
  }
  k_df_to_d<<<blocks_for(n), kThreads, 0, c.stream>>>(c.df_x, T, n);
  MGAR_LAUNCH_CHECK();
  if (!(rel <= c.p.eps2) && it < c.p.cg_max) {
    // the FP32 iterations stalled above eps2 (their accuracy floor): the
    // df64 CG continues from x with the iterations left
    const int cg_max = c.p.cg_max;
    int it2 = 0;
    c.p.cg_max = cg_max - it;
    int rc = MGAR_OK;
    try {
      rc = solve_mgcg_df3(c, T, &it2, &rel);
    } catch (...) {
      c.p.cg_max = cg_max;
      throw;
    }
    c.p.cg_max = cg_max;
    it += it2;
    if (iters) *iters = it;
    if (relres) *relres = rel;
    return rc;
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return rel <= c.p.eps2 ? MGAR_OK : MGAR_ERR_MAXIT;
}

int solve_mgcg_df(Ctx& c, double* T, int* iters, double* relres) {
  if (c.dim == 3 && !c.untiled)
    return c.ru_cg ? solve_mgcg_ru3(c, T, iters, relres) : solve_mgcg_df3(c, T, iters, relres);
  const int n = (int)c.n;
  const int rb = c.grid_blocks;
  const DfOp op = make_op(c);
  k_d_to_df<<<blocks_for(n), kThreads, 0, c.stream>>>(T, c.df_x, n);
  MGAR_LAUNCH_CHECK();
  {
    ProfScope ps(c, MGAR_KC_APPLY64);
    if (c.dim == 2)
      k_df_residual<2><<<blocks_for(n), kThreads, 0, c.stream>>>(op, c.df_q, c.df_x, c.df_r,
                                                                 c.partials, c.counter, c.dsc + S_RR);
    else
      k_df_residual<3><<<blocks_for(n), kThreads, 0, c.stream>>>(op, c.df_q, c.df_x, c.df_r,
                                                                 c.partials, c.counter, c.dsc + S_RR);
    MGAR_LAUNCH_CHECK();
  }
  fetch_scalars(c, S_RR, 1);
  double rel = std::sqrt(c.hsc[S_RR]) / c.qnorm;
  int it = 0;
  // 2D: the device-side loop while no kernel class is being timed with
  // events (event records cannot sit inside a conditional body)
  const bool graph = c.dim == 2 && c.cg_graph && c.prof_class == 0 && c.use_graphs;
  if (!(rel <= c.p.eps2) && graph) {
    require(std::isfinite(rel), MGAR_ERR_NONFINITE, "non-finite initial residual");
    drop_stale_cg_graph(c);
    if (!c.cg_exec && !build_cg_graph(c)) c.cg_graph = false;
  }
  if (!(rel <= c.p.eps2) && graph && c.cg_exec) {
    join_coarse(c);
    MGAR_CUDA(cudaGraphLaunch(c.cg_exec, c.stream));
    fetch_scalars(c, S_RR, S_CGIT - S_RR + 1);
    it = (int)c.hsc[S_CGIT];
    count_launches(c.prologue_kernels + (int64_t)std::max(it - 1, 0) * c.body_kernels);
    rel = std::sqrt(c.hsc[S_RR]) / c.qnorm;
    require(std::isfinite(rel), MGAR_ERR_NONFINITE, "CG breakdown (non-finite residual)");
  } else if (!(rel <= c.p.eps2)) {
    require(std::isfinite(rel), MGAR_ERR_NONFINITE, "non-finite initial residual");
    // 2D with the fused V-cycle: the FP32 copy of r comes from the update of x
    // and r, and r . z from the V-cycle's last sweep (the graph's arithmetic)
    const bool fused = c.dim == 2 && vcycle_dot_ok(c);
    int a = S_RZ0, b = S_RZ1;
    if (fused) {
      k_df_to_f32<<<blocks_for(n), kThreads, 0, c.stream>>>(c.df_r, c.b32, n);
      MGAR_LAUNCH_CHECK();
      precondition_f32(c, a);
    } else {
      precondition_df(c);
      k_df_dot_f<<<rb, kThreads, 0, c.stream>>>(c.df_r, c.x32, n, c.partials, c.counter, c.dsc + a);
      MGAR_LAUNCH_CHECK();
    }
    k_f32_to_df<<<blocks_for(n), kThreads, 0, c.stream>>>(c.x32, c.df_p, n);
    MGAR_LAUNCH_CHECK();
    while (it < c.p.cg_max) {
      {
        ProfScope ps(c, MGAR_KC_APPLY64);
        if (c.dim == 2)
          df_apply2_dot(op, c.df_p, c.df_Ap, c.partials, c.counter, c.dsc + S_PAP, c.stream);
        else
          k_df_apply<3, true><<<blocks_for(n), kThreads, 0, c.stream>>>(
              op, c.df_p, c.df_Ap, c.partials, c.counter, c.dsc + S_PAP);
        MGAR_LAUNCH_CHECK();
      }
      k_df_cg_xr<<<rb, kThreads, 0, c.stream>>>(c.df_x, c.df_r, c.df_p, c.df_Ap, n, c.dsc + a,
                                                c.dsc + S_PAP, c.partials, c.counter, c.dsc + S_RR,
                                                fused ? c.b32 : nullptr);
      MGAR_LAUNCH_CHECK();
      ++it;
      fetch_scalars(c, S_RR, 1);
      rel = std::sqrt(c.hsc[S_RR]) / c.qnorm;
      require(std::isfinite(rel), MGAR_ERR_NONFINITE, "CG breakdown (non-finite residual)");
      if (rel <= c.p.eps2) break;
      if (fused) {
        precondition_f32(c, b);
      } else {
        precondition_df(c);
        k_df_dot_f<<<rb, kThreads, 0, c.stream>>>(c.df_r, c.x32, n, c.partials, c.counter,
                                                  c.dsc + b);
        MGAR_LAUNCH_CHECK();
      }
      k_df_cg_p<<<rb, kThreads, 0, c.stream>>>(c.df_p, c.x32, n, c.dsc + b, c.dsc + a);
      MGAR_LAUNCH_CHECK();
      std::swap(a, b);
    }
  }
  k_df_to_d<<<blocks_for(n), kThreads, 0, c.stream>>>(c.df_x, T, n);
  MGAR_LAUNCH_CHECK();
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return rel <= c.p.eps2 ? MGAR_OK : MGAR_ERR_MAXIT;
}

}  // namespace mgar
