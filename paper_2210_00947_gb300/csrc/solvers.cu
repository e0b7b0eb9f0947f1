// MGCG and MGAR solves of A(rho~) t = q.
//
// MGCG (Sections 1 and 3.2): conjugate gradients in FP64 preconditioned by
// one V-cycle; stop when ||r|| / ||q|| <= eps2 (recursively updated residual)
// or after cg_max iterations.  The CG scalars stay in device memory; the host
// reads ||r||^2 once per iteration to decide convergence.
//
// MGAR (Eq. 17-21 and 28): r_1 = t_prev; r_i = one V-cycle on the reference
// hierarchy K0 with right-hand side -dK r_{i-1} and initial guess r_{i-1}
// (or zero); modified Gram-Schmidt twice in FP64 (vectors below 1e-12 ||r_1||
// are dropped); W = A R~; K_R = R~^T W, q_R = R~^T q; m x m Cholesky on the
// device; t~ = R~ y; Res = ||W y - q|| / ||q||.
#include "common.cuh"

#include <atomic>
#include <chrono>

namespace mgar {

// ----------------------------------------------------------------- kernels
__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                      double* partials, unsigned int* counter, double* out) {
  // four independent partial sums per thread: four loads in flight, and no
  // chain of dependent FP64 additions (fixed order, so still reproducible)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (; i + 3 * stride < n; i += 4 * stride) {
    s0 += a[i] * b[i];
    s1 += a[i + stride] * b[i + stride];
    s2 += a[i + 2 * stride] * b[i + 2 * stride];
    s3 += a[i + 3 * stride] * b[i + 3 * stride];
  }
  for (; i < n; i += stride) s0 += a[i] * b[i];
  double v[1] = {(s0 + s1) + (s2 + s3)};
  block_sum_finish<1>(v, partials, counter, out);
}

// The reduced system's products in one pass over R, W and q (Eq. 19-20):
// K_R[i][j] = R_i . W_j (j <= i) and q_R[i] = R_i . q, i < KEPT.
template <int KEPT>
__global__ void k_reduced_dots(const double* __restrict__ R, const double* __restrict__ W,
                               const double* __restrict__ q, int64_t n, double* partials,
                               unsigned int* counter, double* dsc) {
  constexpr int NP = KEPT * (KEPT + 1) / 2 + KEPT;
  double v[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) v[k] = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double r[KEPT], w[KEPT];
#pragma unroll
    for (int i = 0; i < KEPT; ++i) {
      r[i] = R[(int64_t)i * n + e];
      w[i] = W[(int64_t)i * n + e];
    }
    const double qe = q[e];
    int k = 0;
#pragma unroll
    for (int i = 0; i < KEPT; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) v[k++] += r[i] * w[j];
#pragma unroll
    for (int i = 0; i < KEPT; ++i) v[k++] += r[i] * qe;
  }
  double t[NP];
  if (block_sum_last<NP>(v, partials, counter, t) && threadIdx.x == 0) {
    int k = 0;
    for (int i = 0; i < KEPT; ++i)
      for (int j = 0; j <= i; ++j) dsc[S_KR + i * kMaxM + j] = t[k++];
    for (int i = 0; i < KEPT; ++i) dsc[S_QR + i] = t[k++];
  }
}

// r = q - A x with ||r||^2 (A from the current conductivities).
template <int DIM>
__global__ void k_residual_norm(FineOp<double> op, const double* __restrict__ q,
                                const double* __restrict__ x, double* __restrict__ r,
                                double* partials, unsigned int* counter, double* out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  double v[1] = {0.0};
  if (idx < op.n) {
    int i, j, k;
    coords(idx, op.fNX, op.fNXY, i, j, k);
    double d;
    const double ax = DIM == 2 ? fine_row2(op, x, i, j, d) : fine_row3(op, x, i, j, k, d);
    const double ri = q[idx] - ax;
    r[idx] = ri;
    v[0] = ri * ri;
  }
  block_sum_finish<1>(v, partials, counter, out);
}

// alpha = rz / pAp; x += alpha p; r -= alpha Ap; ||r||^2.
__global__ void k_cg_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                        const double* __restrict__ Ap, int64_t n, const double* __restrict__ rz,
                        const double* __restrict__ pap, double* partials, unsigned int* counter,
                        double* out) {
  const double alpha = block_div(rz, pap);
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * Ap[i];
    r[i] = ri;
    v[0] += ri * ri;
  }
  block_sum_finish<1>(v, partials, counter, out);
}

// p = z + (rz_new / rz_old) p
__global__ void k_cg_p(double* __restrict__ p, const double* __restrict__ z, int64_t n,
                       const double* __restrict__ rz_new, const double* __restrict__ rz_old) {
  const double beta = block_div(rz_new, rz_old);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// v -= coef * u, coef read from device memory
__global__ void k_axpy_dev(double* __restrict__ v, const double* __restrict__ u, int64_t n,
                           const double* __restrict__ coef) {
  const double a = *coef;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] -= a * u[i];
}

// y = a - y
__global__ void k_sub_from(double* __restrict__ y, const double* __restrict__ a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a[i] - y[i];
}

__global__ void k_scale(double* __restrict__ v, int64_t n, double s) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= s;
}

// Reduced m x m solve (Eq. 19-21): K_R y = q_R by Cholesky, one thread.
__global__ void k_reduced_solve(double* dsc, int m, int* err) {
  double L[kMaxM * kMaxM];
  const double* KR = dsc + S_KR;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j <= i; ++j) {
      double s = KR[i * kMaxM + j];
      for (int k = 0; k < j; ++k) s -= L[i * kMaxM + k] * L[j * kMaxM + k];
      if (i == j) {
        if (!(s > 0.0)) {
          *err = MGAR_ERR_NOT_SPD;
          return;
        }
        L[i * kMaxM + i] = sqrt(s);
      } else {
        L[i * kMaxM + j] = s / L[j * kMaxM + j];
      }
    }
  double y[kMaxM];
  for (int i = 0; i < m; ++i) {
    double s = dsc[S_QR + i];
    for (int k = 0; k < i; ++k) s -= L[i * kMaxM + k] * y[k];
    y[i] = s / L[i * kMaxM + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = y[i];
    for (int k = i + 1; k < m; ++k) s -= L[k * kMaxM + i] * y[k];
    y[i] = s / L[i * kMaxM + i];
  }
  // the reduced solution's compliance q . t~ = q . R~ y = q_R . y (Eq. 5, 21)
  double cred = 0.0;
  for (int i = 0; i < m; ++i) {
    dsc[S_Y + i] = y[i];
    cred += dsc[S_QR + i] * y[i];
  }
  dsc[S_CRED] = cred;
}

// t = sum_j y_j Q_j ; ||sum_j y_j W_j - q||^2
__global__ void k_reduced_combine(const double* __restrict__ Q, const double* __restrict__ W,
                                  const double* __restrict__ q, int64_t n, int m,
                                  const double* __restrict__ dsc, double* __restrict__ t,
                                  double* partials, unsigned int* counter, double* out) {
  double y[kMaxM];
  for (int j = 0; j < m; ++j) y[j] = dsc[S_Y + j];
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double ti = 0.0, wi = 0.0;
    for (int j = 0; j < m; ++j) {
      ti += y[j] * Q[(int64_t)j * n + i];
      wi += y[j] * W[(int64_t)j * n + i];
    }
    t[i] = ti;
    const double d = wi - q[i];
    v[0] += d * d;
  }
  block_sum_finish<1>(v, partials, counter, out);
}

// -------------------------------------------------------------------- host
static int red_blocks(Ctx& c) { return c.grid_blocks; }

void dot(Ctx& c, const double* a, const double* b, int64_t n, double* out_dev) {
  k_dot<<<red_blocks(c), kThreads, 0, c.stream>>>(a, b, n, c.partials, c.counter, out_dev);
  MGAR_LAUNCH_CHECK();
}

// Copies device scalars into the mapped pinned mirror, then bumps a
// sequence number there (after a system-scope fence).
__global__ void k_publish(const double* __restrict__ dsc, double* hmir, int first, int count,
                          volatile unsigned long long* seq, unsigned long long value,
                          const int* __restrict__ derr) {
  for (int k = threadIdx.x; k < count; k += blockDim.x) hmir[first + k] = dsc[first + k];
  if (threadIdx.x == 0) hmir[S_DERR] = (double)*derr;
  __threadfence_system();
  __syncwarp();
  if (threadIdx.x == 0) *seq = value;
}

// Device scalars to the host.  A one-warp kernel writes them straight into
// mapped pinned memory and the host spins on a sequence number: no copy
// engine round trip and no blocking stream synchronisation on the critical
// path between CG iterations.  The spin is bounded; after it (or if mapped
// memory is unavailable) the stream is synchronised, which also surfaces
// any device error.  The device error flag is published with the scalars
// (slot S_DERR of the mirror).
void fetch_scalars(Ctx& c, int first, int count) {
  if (!c.coarse_pending) c.derr_fresh = true;  // ordered after every factorisation
  if (!c.hseq) {
    int e = 0;
    MGAR_CUDA(cudaMemcpyAsync(c.hsc + first, c.dsc + first, count * sizeof(double),
                              cudaMemcpyDeviceToHost, c.stream));
    MGAR_CUDA(cudaMemcpyAsync(&e, c.derr, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    MGAR_CUDA(cudaStreamSynchronize(c.stream));
    c.hsc[S_DERR] = (double)e;
    return;
  }
  const unsigned long long want = ++c.seq_sent;
  k_publish<<<1, 32, 0, c.stream>>>(c.dsc, c.hsc_dev, first, count, c.hseq_dev, want, c.derr);
  MGAR_LAUNCH_CHECK();
  const auto t0 = std::chrono::steady_clock::now();
  for (uint64_t spins = 0;; ++spins) {
    if (*(volatile unsigned long long*)c.hseq >= want) {
      std::atomic_thread_fence(std::memory_order_acquire);
      return;
    }
    if ((spins & 1023) == 1023 &&
        std::chrono::steady_clock::now() - t0 > std::chrono::seconds(2)) {
      // slow or failed work: a blocking wait, which also reports a device error
      MGAR_CUDA(cudaStreamSynchronize(c.stream));
      require(*(volatile unsigned long long*)c.hseq >= want, MGAR_ERR_CUDA,
              "device scalars were not published");
      std::atomic_thread_fence(std::memory_order_acquire);
      return;
    }
  }
}

// The device error flag as published by the last fetch_scalars.
static void check_published_error(Ctx& c) {
  const int e = (int)c.hsc[S_DERR];
  if (e != 0) {
    MGAR_CUDA(cudaMemsetAsync(c.derr, 0, sizeof(int), c.stream));
    throw Error{e, e == MGAR_ERR_NOT_SPD ? "factorisation met a non-positive pivot"
                                         : "device error"};
  }
}

// z = M r (one V-cycle, zero initial guess) in the handle's precision.
static bool vcycle_profiled(Ctx& c) {
  return c.prof_class == MGAR_KC_SMOOTH0 || c.prof_class == MGAR_KC_RESID0;
}

void precondition(Ctx& c, const double* r, double* z) {
  run_graph(c, 1, r, z, vcycle_profiled(c), [&] {
    if (c.p.precision == MGAR_FP64) {
      vcycle<double>(c, r, z, true);
    } else {
      convert_d2f(c, r, c.b32, c.n);
      vcycle<float>(c, c.b32, c.x32, true);
      convert_f2d(c, c.x32, z, c.n);
    }
  });
}

template <int DIM>
static void residual_norm(Ctx& c, const double* x, double* r, double* out) {
  const Dims& d = c.L[0];
  FineOp<double> op{c.ke, nullptr, c.fixed, d.ex, d.ey, d.ez, d.NX, d.NY, d.NZ, (int)d.n,
                    d.fNX, d.fNXY};
  k_residual_norm<DIM><<<blocks_for(d.n), kThreads, 0, c.stream>>>(op, c.q, x, r, c.partials,
                                                                    c.counter, out);
  MGAR_LAUNCH_CHECK();
}

static int solve_mgcg_fp(Ctx& c, double* T, int* iters, double* relres);

// The factorisation's error flag is read with the solve's last scalar fetch
// (one more fetch only when none followed the factorisation); a failed
// factorisation is reported in place of any error it caused in the solve.
int solve_mgcg(Ctx& c, double* T, int* iters, double* relres) {
  build_hierarchy(c);
  int rc = MGAR_OK;
  try {
    rc = solve_mgcg_fp(c, T, iters, relres);
  } catch (const Error&) {
    join_coarse(c);
    fetch_scalars(c, S_RR, 1);
    check_published_error(c);
    throw;
  }
  join_coarse(c);
  if (!c.derr_fresh) fetch_scalars(c, S_RR, 1);
  check_published_error(c);
  return rc;
}

static int solve_mgcg_fp(Ctx& c, double* T, int* iters, double* relres) {
  if (c.p.precision == MGAR_MIXED) return solve_mgcg_df(c, T, iters, relres);
  const int64_t n = c.n;
  if (c.dim == 2) residual_norm<2>(c, T, c.r, c.dsc + S_RR);
  else residual_norm<3>(c, T, c.r, c.dsc + S_RR);
  fetch_scalars(c, S_RR, 1);
  double rel = std::sqrt(c.hsc[S_RR]) / c.qnorm;
  int it = 0;
  if (!(rel <= c.p.eps2)) {
    require(std::isfinite(rel), MGAR_ERR_NONFINITE, "non-finite initial residual");
    precondition(c, c.r, c.z);
    int a = S_RZ0, b = S_RZ1;
    dot(c, c.r, c.z, n, c.dsc + a);
    MGAR_CUDA(cudaMemcpyAsync(c.pv, c.z, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    while (it < c.p.cg_max) {
      apply_fine64(c, c.ke, c.pv, c.Ap, c.dsc + S_PAP);
      k_cg_xr<<<red_blocks(c), kThreads, 0, c.stream>>>(T, c.r, c.pv, c.Ap, n, c.dsc + a,
                                                        c.dsc + S_PAP, c.partials, c.counter,
                                                        c.dsc + S_RR);
      MGAR_LAUNCH_CHECK();
      ++it;
      fetch_scalars(c, S_RR, 1);
      rel = std::sqrt(c.hsc[S_RR]) / c.qnorm;
      require(std::isfinite(rel), MGAR_ERR_NONFINITE, "CG breakdown (non-finite residual)");
      if (rel <= c.p.eps2) break;
      precondition(c, c.r, c.z);
      dot(c, c.r, c.z, n, c.dsc + b);
      k_cg_p<<<red_blocks(c), kThreads, 0, c.stream>>>(c.pv, c.z, n, c.dsc + b, c.dsc + a);
      MGAR_LAUNCH_CHECK();
      std::swap(a, b);
    }
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return rel <= c.p.eps2 ? MGAR_OK : MGAR_ERR_MAXIT;
}

void solve_mgar(Ctx& c, const double* T_prev, double* T, double* res, int* accepted) {
  require(c.have_ref, MGAR_ERR_STATE, "MGAR needs a reference hierarchy (run MGCG first)");
  const int64_t n = c.n;
  const int m = c.p.m;
  const bool zero = c.p.basis_guess == MGAR_GUESS_ZERO;
  const int rb = red_blocks(c);
  MGAR_CUDA(cudaMemcpyAsync(c.R, T_prev, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  // Eq. 17: basis vectors by V-cycles on K0
  for (int i = 1; i < m; ++i) {
    const double* prev = c.R + (int64_t)(i - 1) * n;
    double* ri = c.R + (int64_t)i * n;
    if (c.p.precision == MGAR_FP64) {
      apply_dK64(c, prev, c.r);  // c.r = -dK r_{i-1}
      if (!zero)
        MGAR_CUDA(cudaMemcpyAsync(ri, prev, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
      run_graph(c, zero ? 2 : 3, c.r, ri, vcycle_profiled(c),
                [&] { vcycle<double>(c, c.r, ri, zero); });
    } else if (zero) {
      run_graph(c, 4, prev, ri, vcycle_profiled(c), [&] {
        convert_d2f(c, prev, c.x32, n);
        apply_dK32(c, c.x32, c.b32);  // b32 = -dK r_{i-1}
        vcycle<float>(c, c.b32, c.x32, true);
        convert_f2d(c, c.x32, ri, n);
      });
    } else {
      // One V-cycle from the guess r_{i-1} equals r_{i-1} + MG(-dK r_{i-1} - K0 r_{i-1}, 0)
      // = r_{i-1} - MG(K r_{i-1}, 0) (the V-cycle is affine in its guess).  In the
      // mixed path only the correction goes through FP32, so the large r_{i-1}
      // never cancels in single precision.
      // K r_0 goes straight to W_0: the first basis vector is r_0 / ||r_0||, so
      // the reduced system's W_0 = K R_0 is it scaled (Eq. 19)
      double* kprev = i == 1 ? c.W : c.r;
      apply_df64(c, prev, kprev);  // K r_{i-1}
      run_graph(c, 5, kprev, ri, vcycle_profiled(c), [&] {
        convert_d2f(c, kprev, c.b32, n);
        vcycle<float>(c, c.b32, c.x32, true);
        convert_f2d(c, c.x32, ri, n);
      });
      k_sub_from<<<rb, kThreads, 0, c.stream>>>(ri, prev, n);  // ri = r_{i-1} - ri
      MGAR_LAUNCH_CHECK();
    }
  }
  // Eq. 18: orthonormal basis (modified Gram-Schmidt, twice)
  dot(c, c.R, c.R, n, c.dsc + S_NORM);
  fetch_scalars(c, S_NORM, 1);
  const double ref = std::sqrt(c.hsc[S_NORM]);
  require(std::isfinite(ref), MGAR_ERR_NONFINITE, "non-finite MGAR basis");
  int kept = 0;
  for (int i = 0; i < m; ++i) {
    double* v = c.R + (int64_t)i * n;
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < kept; ++j) {
        const double* qj = c.R + (int64_t)j * n;
        dot(c, qj, v, n, c.dsc + S_GS);
        k_axpy_dev<<<rb, kThreads, 0, c.stream>>>(v, qj, n, c.dsc + S_GS);
        MGAR_LAUNCH_CHECK();
      }
    // the first vector's norm is the reference just fetched
    if (i > 0 || kept > 0) {
      dot(c, v, v, n, c.dsc + S_NORM);
      fetch_scalars(c, S_NORM, 1);
    }
    const double nv = (i > 0 || kept > 0) ? std::sqrt(c.hsc[S_NORM]) : ref;
    require(std::isfinite(nv), MGAR_ERR_NONFINITE, "non-finite MGAR basis");
    if (nv > 1e-12 * ref && nv > 0.0) {
      double* dst = c.R + (int64_t)kept * n;
      if (dst != v)
        MGAR_CUDA(cudaMemcpyAsync(dst, v, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
      k_scale<<<rb, kThreads, 0, c.stream>>>(dst, n, 1.0 / nv);
      MGAR_LAUNCH_CHECK();
      ++kept;
    }
  }
  require(kept > 0, MGAR_ERR_NONFINITE, "MGAR basis vanished");
  // Eq. 19-21: reduced system
  const bool w0_held = c.p.precision == MGAR_MIXED && !zero && m > 1;  // W_0 = K r_0 from Eq. 17
  for (int j = 0; j < kept; ++j) {
    if (j == 0 && w0_held) {
      k_scale<<<rb, kThreads, 0, c.stream>>>(c.W, n, 1.0 / ref);
      MGAR_LAUNCH_CHECK();
    } else if (c.p.precision == MGAR_MIXED) {
      apply_df64(c, c.R + (int64_t)j * n, c.W + (int64_t)j * n);
    } else {
      apply_fine64(c, c.ke, c.R + (int64_t)j * n, c.W + (int64_t)j * n, nullptr);
    }
  }
  if (kept <= 3) {
    switch (kept) {
      case 1: k_reduced_dots<1><<<rb, kThreads, 0, c.stream>>>(c.R, c.W, c.q, n, c.partials, c.counter, c.dsc); break;
      case 2: k_reduced_dots<2><<<rb, kThreads, 0, c.stream>>>(c.R, c.W, c.q, n, c.partials, c.counter, c.dsc); break;
      default: k_reduced_dots<3><<<rb, kThreads, 0, c.stream>>>(c.R, c.W, c.q, n, c.partials, c.counter, c.dsc); break;
    }
    MGAR_LAUNCH_CHECK();
  } else {
    for (int i = 0; i < kept; ++i) {
      for (int j = 0; j <= i; ++j) {
        dot(c, c.R + (int64_t)i * n, c.W + (int64_t)j * n, n, c.dsc + S_KR + i * kMaxM + j);
      }
      dot(c, c.R + (int64_t)i * n, c.q, n, c.dsc + S_QR + i);
    }
  }
  k_reduced_solve<<<1, 1, 0, c.stream>>>(c.dsc, kept, c.derr);
  MGAR_LAUNCH_CHECK();
  k_reduced_combine<<<rb, kThreads, 0, c.stream>>>(c.R, c.W, c.q, n, kept, c.dsc, T, c.partials,
                                                   c.counter, c.dsc + S_RES2);
  MGAR_LAUNCH_CHECK();
  fetch_scalars(c, S_RES2, S_CRED - S_RES2 + 1);
  check_published_error(c);
  c.mgar_cred = c.hsc[S_CRED];
  const double r = std::sqrt(c.hsc[S_RES2]) / c.qnorm;
  require(std::isfinite(r), MGAR_ERR_NONFINITE, "non-finite MGAR residual");
  if (res) *res = r;
  if (accepted) *accepted = (r <= c.p.eps1) ? 1 : 0;
}

}  // namespace mgar
