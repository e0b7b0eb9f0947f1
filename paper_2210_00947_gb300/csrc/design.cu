// Density filter (Eq. 6-8), SIMP conductivities (Eq. 4), compliance and
// sensitivities (Eq. 5, 9-11), and the optimality-criteria update.
#include "common.cuh"

#include <vector>

namespace mgar {

// ----------------------------------------------------------------- kernels
// out_e = inv_hs_e * sum_o w_o in_{e+o}            (forward, Eq. 6)
// out_j = sum_o w_o in_{j+o} inv_hs_{j+o}           (transpose, Eq. 9/11)
// over in-domain neighbours; the offset set is symmetric.
template <bool TRANSPOSE>
__global__ void k_filter(const double* __restrict__ in, double* __restrict__ out,
                         const double* __restrict__ inv_hs, const int4* __restrict__ offs,
                         const double* __restrict__ w, int noff, int ex, int ey, int ez) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ne = (int64_t)ex * ey * ez;
  if (e >= ne) return;
  const int i = (int)(e % ex), j = (int)((e / ex) % ey), k = (int)(e / ((int64_t)ex * ey));
  double acc = 0.0;
  for (int o = 0; o < noff; ++o) {
    const int4 d = offs[o];
    const int ii = i + d.x, jj = j + d.y, kk = k + d.z;
    if (ii < 0 || ii >= ex || jj < 0 || jj >= ey || kk < 0 || kk >= ez) continue;
    const int64_t nb = ii + (int64_t)ex * (jj + (int64_t)ey * kk);
    if (TRANSPOSE) acc += w[o] * (in[nb] * inv_hs[nb]);
    else acc += w[o] * in[nb];
  }
  out[e] = TRANSPOSE ? acc : acc * inv_hs[e];
}

__global__ void k_filter_norm(double* __restrict__ inv_hs, const int4* __restrict__ offs,
                              const double* __restrict__ w, int noff, int ex, int ey, int ez) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t ne = (int64_t)ex * ey * ez;
  if (e >= ne) return;
  const int i = (int)(e % ex), j = (int)((e / ex) % ey), k = (int)(e / ((int64_t)ex * ey));
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
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= d.ne) return;
  const int i = (int)(e % d.ex), j = (int)((e / d.ex) % d.ey);
  const int k = DIM == 3 ? (int)(e / ((int64_t)d.ex * d.ey)) : 0;
  double t[nen];
#pragma unroll
  for (int a = 0; a < nen; ++a)
    t[a] = T[(i + (a & 1)) + (int64_t)d.NX * ((j + ((a >> 1) & 1)) + (int64_t)d.NY * (k + ((a >> 2) & 1)))];
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

// OC preparation: s_e = rho_e sqrt(max(-dc_e, 0) / dv_e) and the move box.
__global__ void k_oc_prep(const double* __restrict__ rho, const double* __restrict__ dc,
                          const double* __restrict__ dv, double* __restrict__ s,
                          double* __restrict__ lo, double* __restrict__ hi, int64_t ne,
                          double move) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const double r = rho[e];
  s[e] = r * sqrt(fmax(-dc[e], 0.0) / dv[e]);
  lo[e] = fmax(0.0, r - move);
  hi[e] = fmin(1.0, r + move);
}

// One bisection step on lambda: volume sum_e dv_e clamp(s_e / sqrt(lambda))
// at the geometric midpoint of the bracket; the last block moves the
// bracket and raises the done flag once (hi - lo) / (hi + lo) <= tol.
__global__ void k_oc_pass(const double* __restrict__ s, const double* __restrict__ lo,
                          const double* __restrict__ hi, const double* __restrict__ dv, int64_t ne,
                          double volfrac, double tol, double* dsc, double* partials,
                          unsigned int* counter) {
  if (dsc[S_OC_DONE] != 0.0) return;
  const double blo = dsc[S_OC_LO], bhi = dsc[S_OC_HI];
  const double lam = sqrt(blo * bhi);
  const double mu = 1.0 / sqrt(lam);
  double v[1] = {0.0};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x)
    v[0] += dv[e] * fmin(fmax(s[e] * mu, lo[e]), hi[e]);
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

// rho <- clamp(s / sqrt(lambda)) with lambda the bracket's geometric
// midpoint; max |change| into dsc.
__global__ void k_oc_final(double* __restrict__ rho, const double* __restrict__ s,
                           const double* __restrict__ lo, const double* __restrict__ hi, int64_t ne,
                           double* dsc, double* partials, unsigned int* counter) {
  const double lam = sqrt(dsc[S_OC_LO] * dsc[S_OC_HI]);
  const double mu = 1.0 / sqrt(lam);
  double ch = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double rn = fmin(fmax(s[e] * mu, lo[e]), hi[e]);
    ch = fmax(ch, fabs(rn - rho[e]));
    rho[e] = rn;
  }
  block_max_finish(ch, partials, counter, dsc + S_OC_CHANGE);
  if (blockIdx.x == 0 && threadIdx.x == 0) dsc[S_OC_LAM] = lam;
}

__global__ void k_oc_init(double* dsc, double lo, double hi) {
  dsc[S_OC_LO] = lo;
  dsc[S_OC_HI] = hi;
  dsc[S_OC_DONE] = 0.0;
  dsc[S_OC_STEPS] = 0.0;
}

// ------------------------------------------------------------------- host
void setup_filter(Ctx& c) {
  const double r = c.p.rmin;
  const int reach = (int)std::ceil(r);
  std::vector<int4> offs;
  std::vector<double> w;
  const int zr = c.dim == 3 ? reach : 0;
  for (int dz = -zr; dz <= zr; ++dz)
    for (int dy = -reach; dy <= reach; ++dy)
      for (int dx = -reach; dx <= reach; ++dx) {
        const double wt = r - std::sqrt((double)(dx * dx + dy * dy + dz * dz));
        if (wt > 0.0) {
          offs.push_back(make_int4(dx, dy, dz, 0));
          w.push_back(wt);
        }
      }
  require((int)offs.size() <= kMaxFilterOffsets, MGAR_ERR_ARG, "filter radius too large");
  c.n_filter = (int)offs.size();
  MGAR_CUDA(cudaMalloc(&c.f_offs, offs.size() * sizeof(int4)));
  MGAR_CUDA(cudaMalloc(&c.f_w, w.size() * sizeof(double)));
  MGAR_CUDA(cudaMemcpy(c.f_offs, offs.data(), offs.size() * sizeof(int4), cudaMemcpyHostToDevice));
  MGAR_CUDA(cudaMemcpy(c.f_w, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
  const Dims& d = c.L[0];
  k_filter_norm<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(c.inv_hs, c.f_offs, c.f_w, c.n_filter,
                                                             d.ex, d.ey, d.ez);
  MGAR_LAUNCH_CHECK();
  // dv = F^T (1/E)
  std::vector<double> ones(c.ne, 1.0 / (double)c.ne);
  MGAR_CUDA(cudaMemcpyAsync(c.tmp_e, ones.data(), c.ne * sizeof(double), cudaMemcpyHostToDevice,
                            c.stream));
  filter(c, c.tmp_e, c.dv, true);
  MGAR_CUDA(cudaStreamSynchronize(c.stream));
}

void filter(Ctx& c, const double* in, double* out, bool transpose) {
  const Dims& d = c.L[0];
  ProfScope ps(c, MGAR_KC_FILTER);
  if (transpose)
    k_filter<true><<<blocks_for(c.ne), kThreads, 0, c.stream>>>(in, out, c.inv_hs, c.f_offs, c.f_w,
                                                                c.n_filter, d.ex, d.ey, d.ez);
  else
    k_filter<false><<<blocks_for(c.ne), kThreads, 0, c.stream>>>(in, out, c.inv_hs, c.f_offs, c.f_w,
                                                                 c.n_filter, d.ex, d.ey, d.ez);
  MGAR_LAUNCH_CHECK();
}

void set_density(Ctx& c, const double* rho, bool physical) {
  if (physical)
    MGAR_CUDA(cudaMemcpyAsync(c.rho_phys, rho, c.ne * sizeof(double), cudaMemcpyDeviceToDevice,
                              c.stream));
  else
    filter(c, rho, c.rho_phys, false);
  k_simp<<<blocks_for(c.ne), kThreads, 0, c.stream>>>(c.rho_phys, c.ke,
                                                      c.p.precision == MGAR_FP64 ? nullptr : c.ke_f,
                                                      c.ne, c.p.k0, c.p.kmin, c.p.penal);
  MGAR_LAUNCH_CHECK();
}

void sensitivity(Ctx& c, const double* T, double* dc, double* dv, double* compliance) {
  const Dims& d = c.L[0];
  const double coef = c.p.penal * (c.p.k0 - c.p.kmin);
  if (dc) {
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

void oc_update(Ctx& c, double* rho, const double* dc, double volfrac, double move, double* lambda,
               double* change) {
  const int64_t ne = c.ne;
  const int rb = c.grid_blocks_e;
  k_oc_prep<<<blocks_for(ne), kThreads, 0, c.stream>>>(rho, dc, c.dv, c.oc_s, c.oc_lo, c.oc_hi, ne,
                                                       move);
  MGAR_LAUNCH_CHECK();
  k_oc_init<<<1, 1, 0, c.stream>>>(c.dsc, 1e-40, 1e40);
  MGAR_LAUNCH_CHECK();
  const int max_steps = 200, batch = 16;
  for (int done = 0; done < max_steps; done += batch) {
    for (int b = 0; b < batch; ++b) {
      ProfScope ps(c, MGAR_KC_OC);
      k_oc_pass<<<rb, kThreads, 0, c.stream>>>(c.oc_s, c.oc_lo, c.oc_hi, c.dv, ne, volfrac, 1e-13,
                                               c.dsc, c.partials, c.counter);
      MGAR_LAUNCH_CHECK();
    }
    fetch_scalars(c, S_OC_DONE, 1);
    if (c.hsc[S_OC_DONE] != 0.0) break;
  }
  k_oc_final<<<rb, kThreads, 0, c.stream>>>(rho, c.oc_s, c.oc_lo, c.oc_hi, ne, c.dsc, c.partials,
                                            c.counter);
  MGAR_LAUNCH_CHECK();
  if (lambda || change) {
    fetch_scalars(c, S_OC_LAM, 3);
    if (lambda) *lambda = c.hsc[S_OC_LAM];
    if (change) *change = c.hsc[S_OC_CHANGE];
  }
}

}  // namespace mgar
