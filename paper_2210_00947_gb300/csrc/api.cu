// C ABI of libmgar (declared in include/mgar.h).
#include "common.cuh"

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include <atomic>

using namespace mgar;

namespace {
std::atomic<int64_t> g_launches{0};
}  // namespace

namespace mgar {
Ctx*& current_ctx() {
  static thread_local Ctx* cur = nullptr;
  return cur;
}
void prof_mark(const char* site) {
  Ctx* c = current_ctx();
  if (!c || c->prof_class != MGAR_KC_TIMELINE || c->stream == c->cap_stream ||
      c->stream == c->cap_stream2)
    return;
  if (c->prof_used >= 2 * kProfMax) return;
  cudaEventRecord(c->prof_ev[c->prof_used], c->stream);
  c->prof_sites[c->prof_used] = site;
  ++c->prof_used;
}
// The process-wide count (mgar_kernel_launches) and this thread's own, which
// the graph captures difference: handles may run in several host threads.
thread_local int64_t t_launches = 0;
void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
void count_launches(int64_t delta) {
  g_launches.fetch_add(delta, std::memory_order_relaxed);
  t_launches += delta;
}
int64_t launches_so_far() { return t_launches; }
}  // namespace mgar

namespace {

thread_local std::string g_create_error = "no error";

#ifdef MGAR_CHECKED
// Checked build: report the first out-of-bounds access recorded by CK().
int ck_report(Ctx& c) {
  cudaDeviceSynchronize();
  unsigned long long f[4] = {0, 0, 0, 0};
  cudaMemcpyFromSymbol(f, g_ck_fault, sizeof(f));
  if (f[0] == 0) return MGAR_OK;
  char buf[256];
  snprintf(buf, sizeof(buf), "bounds check failed at source line %llu: index %lld, bound %lld",
           f[0], (long long)f[1], (long long)f[2]);
  fprintf(stderr, "[libmgar checked] %s\n", buf);
  c.err = buf;
  const unsigned long long z[4] = {0, 0, 0, 0};
  cudaMemcpyToSymbol(g_ck_fault, z, sizeof(z));
  return MGAR_ERR_ARG;
}
#endif

// after a failed call: order the stream after a pending factorisation
// anyway (best effort; errors here are not reported)
static void release_side(Ctx& c) {
  if (c.coarse_pending && c.ev_join && c.stream != c.cap_stream && c.stream != c.cap_stream2 &&
      cudaStreamWaitEvent(c.stream, c.ev_join, 0) == cudaSuccess)
    c.coarse_pending = false;
}

template <class F>
int guarded(mgar_t h, F&& f) {
  Ctx* c = reinterpret_cast<Ctx*>(h);
  if (!c) return MGAR_ERR_ARG;
  struct CurGuard {
    Ctx* prev;
    explicit CurGuard(Ctx* c) : prev(current_ctx()) { current_ctx() = c; }
    ~CurGuard() { current_ctx() = prev; }
  } cur_guard(c);
  try {
    // every call returns with the handle's stream ordered after its work
#ifdef MGAR_CHECKED
    const int rc = f(*c);
    join_coarse(*c);
    const int ck = ck_report(*c);
    return ck != MGAR_OK ? ck : rc;
#else
    const int rc = f(*c);
    join_coarse(*c);
    return rc;
#endif
  } catch (const Error& e) {
    c->err = e.msg;
    release_side(*c);
    return e.code;
  } catch (const std::exception& e) {
    c->err = e.what();
    release_side(*c);
    return MGAR_ERR_CUDA;
  }
}

void free_ctx(Ctx& c) {
  for (auto& g : c.graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (c.cg_exec) cudaGraphExecDestroy(c.cg_exec);
  if (c.ru_exec) cudaGraphExecDestroy(c.ru_exec);
  if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
  if (c.cap_stream2) cudaStreamDestroy(c.cap_stream2);
  if (c.side_stream) cudaStreamDestroy(c.side_stream);
  if (c.ev_fork) cudaEventDestroy(c.ev_fork);
  if (c.ev_join) cudaEventDestroy(c.ev_join);
  free_hierarchy(c);
  if (c.prof_ev) {
    for (int i = 0; i < 2 * kProfMax; ++i)
      if (c.prof_ev[i]) cudaEventDestroy(c.prof_ev[i]);
    delete[] c.prof_ev;
    c.prof_ev = nullptr;
    delete[] c.prof_sites;
    c.prof_sites = nullptr;
  }
  cudaFree(c.run_rho);
  cudaFree(c.run_T);
  void* ptrs[] = {c.fixed, c.efix, c.gfix, c.q, c.rho_phys, c.ke, c.ke0, c.ke_f, c.ke0_f, c.inv_hs, c.inv_hs_df, c.rho_phys_df, c.f_offs, c.f_w,
                  c.dv, c.rsdv, c.dv_df, c.r, c.z, c.pv, c.Ap, c.tm, c.tmp_dc, c.R, c.W, c.b32, c.x32, c.ke_df, c.df_q, c.df_x, c.df_r, c.df_p, c.df_Ap, c.df_p2, c.df_e, c.kd_df, c.xc32, c.p32, c.p32b, c.y32, c.tmp_e, c.oc_s, c.oc_lo,
                  c.oc_hi, c.oc_rho, c.oc_s32, c.oc_lo32, c.oc_hi32, c.dv32, c.oc_amb, c.oc_namb, c.partials, c.counter, c.dsc, c.derr};
  for (void* p : ptrs) cudaFree(p);
  if (c.hsc) cudaFreeHost(c.hsc);
  if (c.f_offs_h) cudaFreeHost(c.f_offs_h);
  if (c.f_w_h) cudaFreeHost(c.f_w_h);
  if (c.hseq) cudaFreeHost(c.hseq);
}

// q = load with fixed nodes zeroed (Eq. 3: their rows are eliminated)
__global__ void k_masked_load(const double* __restrict__ src, const uint8_t* __restrict__ fixed,
                              double* __restrict__ q, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = fixed[i] ? 0.0 : src[i];
}

// One design cycle of Figure 5 on device arrays rho (design) and T.
mgar_step_info design_cycle(Ctx& c, double* rho, double* T, int cycle) {
  mgar_step_info inf{};
  inf.res = NAN;
  inf.relres = NAN;
  inf.compliance_mgar = NAN;
  int status = MGAR_OK;
  if (c.p.filter_alpha > 0.0) {
    const double r = filter_radius(c, cycle);
    if (r != c.filter_r) set_filter_radius(c, r);
  }
  set_density(c, rho, false);
  bool need_mgcg = cycle < c.p.n_on || !c.have_ref;
  if (!need_mgcg) {
    double res = 0.0;
    int acc = 0;
    solve_mgar(c, T, c.tm, &res, &acc);  // t_prev in T, t~ in tm
    inf.res = res;
    inf.accepted = acc;
    inf.compliance_mgar = c.mgar_cred;
    if (acc)
      MGAR_CUDA(cudaMemcpyAsync(T, c.tm, c.n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    else
      need_mgcg = true;  // Eq. 28 rejected: MGCG from t_prev, new reference
  }
  if (need_mgcg) {
    int it = 0;
    double rr = 0.0;
    status = solve_mgcg(c, T, &it, &rr);
    inf.used_mgcg = 1;
    inf.cg_iters = it;
    inf.relres = rr;
  }
  double comp = 0.0;
  // after a mixed MGCG solve the double-float pairs of T are still in df_x
  // (the 2D df64 CG and the tiled 3D path both end by converting df_x to T);
  // the mixed path hands dc to the OC update as double-float pairs
  const bool mixed = c.p.precision == MGAR_MIXED;
  const bool t_df = need_mgcg && mixed && (c.dim == 2 || !c.untiled);
  sensitivity(c, T, mixed ? nullptr : c.tmp_dc, nullptr, nullptr, t_df ? c.df_x : nullptr,
              mixed ? dc_pairs(c) : nullptr);
  // f = q^T T (Eq. 5), read with the OC update's first scalar fetch
  dot(c, c.q, T, c.n, c.dsc + S_COMPL);
  double lam = 0.0, change = 0.0;
  oc_update(c, rho, c.tmp_dc, c.p.volfrac, c.p.move, &lam, &change, mixed ? dc_pairs(c) : nullptr);
  comp = c.hsc[S_COMPL];
  inf.compliance = comp;
  inf.lambda = lam;
  inf.status = status;
  return inf;
}

}  // namespace

extern "C" {

void mgar_default_params(mgar_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->k0 = 1.0;
  p->kmin = 1e-3;
  p->penal = 3.0;
  p->rmin = 1.5;
  p->nl = 4;
  p->m = 2;
  p->eps1 = 0.5;
  p->eps2 = 1e-8;
  p->cg_max = 200;
  p->omega = 0.9;
  p->nu_pre = 1;
  p->nu_post = 1;
  p->precision = MGAR_FP64;
  p->basis_guess = MGAR_GUESS_PREVIOUS;
  p->n_on = 0;
  p->volfrac = 0.4;
  p->move = 0.2;
  p->filter_alpha = 0.0;
  p->filter_lp = 0;
  p->filter_L = 0.0;
}

const char* mgar_last_error(mgar_t h) {
  if (!h) return g_create_error.c_str();
  return reinterpret_cast<Ctx*>(h)->err.c_str();
}

int mgar_create(mgar_t* out, const mgar_params* p, const uint8_t* fixed_mask, const double* q,
                void* stream) {
  if (!out || !p || !fixed_mask || !q) {
    g_create_error = "mgar_create: null argument";
    return MGAR_ERR_ARG;
  }
  *out = nullptr;
  Ctx* c = new Ctx();
  try {
    c->p = *p;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    const mgar_params& P = c->p;
    require(P.nx >= 1 && P.ny >= 1 && P.nz >= 0, MGAR_ERR_ARG, "grid size must be positive");
    require(P.nl >= 2 && P.nl <= kMaxLevels, MGAR_ERR_ARG, "nl must be in [2, 14]");
    require(P.m >= 1 && P.m <= kMaxM, MGAR_ERR_ARG, "m must be in [1, 8]");
    require(P.cg_max >= 0 && P.nu_pre >= 0 && P.nu_post >= 0, MGAR_ERR_ARG, "negative count");
    require(P.precision == MGAR_FP64 || P.precision == MGAR_MIXED, MGAR_ERR_ARG, "bad precision");
    require(P.basis_guess == MGAR_GUESS_PREVIOUS || P.basis_guess == MGAR_GUESS_ZERO, MGAR_ERR_ARG,
            "bad basis_guess");
    require(P.rmin > 0.0 && P.k0 > P.kmin && P.kmin > 0.0, MGAR_ERR_ARG, "bad material/filter");
    c->dim = P.nz == 0 ? 2 : 3;
    c->nen = 1 << c->dim;
    c->S = c->dim == 2 ? 9 : 27;
    c->nl = P.nl;
    int ex = P.nx, ey = P.ny, ez = c->dim == 3 ? P.nz : 1;
    for (int l = 0; l < c->nl; ++l) {
      Dims& d = c->L[l];
      d.ex = ex;
      d.ey = ey;
      d.ez = ez;
      d.NX = ex + 1;
      d.NY = ey + 1;
      d.NZ = c->dim == 3 ? ez + 1 : 1;
      d.n = (int64_t)d.NX * d.NY * d.NZ;
      d.ne = (int64_t)ex * ey * ez;
      require(d.n < (int64_t(1) << 31) / 32, MGAR_ERR_ARG, "grid too large for 32-bit indexing");
      d.fNX = FastDiv((uint32_t)d.NX);
      d.fNXY = FastDiv((uint32_t)(d.NX * d.NY));
      d.fEX = FastDiv((uint32_t)ex);
      d.fEXY = FastDiv((uint32_t)(ex * ey));
      ex = (ex + 1) / 2;
      ey = (ey + 1) / 2;
      if (c->dim == 3) ez = (ez + 1) / 2;
    }
    const Dims& coarsest = c->L[c->nl - 1];
    require(coarsest.n <= 8192, MGAR_ERR_ARG,
            "coarsest grid too large for the direct solve (use more levels)");
    c->n = c->L[0].n;
    c->ne = c->L[0].ne;
    const int64_t n = c->n, ne = c->ne;
    // reduction partials: one per block of the widest launch (node/element
    // kernels, or the z-marching tiles, which stay below kMinPartialBlocks)
    const int64_t maxb = std::max<int64_t>(blocks_for(n > ne ? n : ne), kMinPartialBlocks);
    {
      int dev = 0;
      MGAR_CUDA(cudaGetDevice(&dev));
      MGAR_CUDA(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev));
    }
    c->grid_blocks = (int)std::min<int64_t>(blocks_for(n), (int64_t)c->sms * 8);
    c->grid_blocks_e = (int)std::min<int64_t>(blocks_for(ne), (int64_t)c->sms * 8);

    MGAR_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    MGAR_CUDA(cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking));
    MGAR_CUDA(cudaStreamCreateWithFlags(&c->side_stream, cudaStreamNonBlocking));
    MGAR_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    MGAR_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    MGAR_CUDA(cudaMalloc(&c->fixed, n));
    MGAR_CUDA(cudaMalloc(&c->q, n * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->rho_phys, ne * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->ke, ne * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->ke0, ne * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->inv_hs, ne * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->inv_hs_df, ne * sizeof(float2)));
    MGAR_CUDA(cudaMalloc(&c->rho_phys_df, ne * sizeof(float2)));
    MGAR_CUDA(cudaMalloc(&c->dv, ne * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->rsdv, ne * sizeof(float2)));
    MGAR_CUDA(cudaMalloc(&c->dv_df, ne * sizeof(float2)));
    MGAR_CUDA(cudaMalloc(&c->tmp_e, ne * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->oc_s, ne * sizeof(float2)));
    MGAR_CUDA(cudaMalloc(&c->oc_lo, ne * sizeof(float2)));
    MGAR_CUDA(cudaMalloc(&c->oc_hi, ne * sizeof(float2)));
    MGAR_CUDA(cudaMalloc(&c->oc_rho, ne * sizeof(float2)));
    MGAR_CUDA(cudaMalloc(&c->oc_s32, ne * sizeof(float)));
    MGAR_CUDA(cudaMalloc(&c->oc_lo32, ne * sizeof(float)));
    MGAR_CUDA(cudaMalloc(&c->oc_hi32, ne * sizeof(float)));
    MGAR_CUDA(cudaMalloc(&c->dv32, ne * sizeof(float)));
    MGAR_CUDA(cudaMalloc(&c->oc_amb, kOcAmbMax * sizeof(int)));
    MGAR_CUDA(cudaMalloc(&c->oc_namb, sizeof(int)));
    MGAR_CUDA(cudaMalloc(&c->r, n * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->z, n * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->pv, n * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->Ap, n * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->tm, n * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->tmp_dc, ne * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->R, (size_t)P.m * n * sizeof(double)));
    MGAR_CUDA(cudaMalloc(&c->W, (size_t)P.m * n * sizeof(double)));
    if (P.precision == MGAR_MIXED) {
      MGAR_CUDA(cudaMalloc(&c->ke_f, ne * sizeof(float)));
      MGAR_CUDA(cudaMalloc(&c->ke0_f, ne * sizeof(float)));
      MGAR_CUDA(cudaMalloc(&c->b32, n * sizeof(float)));
      MGAR_CUDA(cudaMalloc(&c->x32, n * sizeof(float)));
      MGAR_CUDA(cudaMalloc(&c->ke_df, ne * sizeof(float2)));
      MGAR_CUDA(cudaMalloc(&c->df_e, ne * sizeof(float2)));
      for (float2** v : {&c->df_q, &c->df_x, &c->df_r, &c->df_p, &c->df_Ap, &c->df_p2, &c->kd_df})
        MGAR_CUDA(cudaMalloc(v, n * sizeof(float2)));
      for (float** v : {&c->xc32, &c->p32, &c->p32b, &c->y32})
        MGAR_CUDA(cudaMalloc(v, n * sizeof(float)));
    }
    MGAR_CUDA(cudaMalloc(&c->partials, (size_t)32 * maxb * sizeof(double)));
#ifdef MGAR_CHECKED
    {
      const long long plen = (long long)32 * maxb;
      MGAR_CUDA(cudaMemcpyToSymbol(g_partials_len, &plen, sizeof(plen)));
    }
#endif
    MGAR_CUDA(cudaMalloc(&c->counter, 8 * sizeof(unsigned int)));
    MGAR_CUDA(cudaMemset(c->counter, 0, 8 * sizeof(unsigned int)));
    MGAR_CUDA(cudaMalloc(&c->dsc, S_COUNT * sizeof(double)));
    MGAR_CUDA(cudaMemset(c->dsc, 0, S_COUNT * sizeof(double)));
    MGAR_CUDA(cudaHostAlloc(&c->hsc, S_COUNT * sizeof(double), cudaHostAllocMapped));
    // mapped sequence number for fetch_scalars (blocking copies if unavailable)
    if (cudaHostAlloc(&c->hseq, sizeof(unsigned long long), cudaHostAllocMapped) == cudaSuccess &&
        cudaHostGetDevicePointer(&c->hsc_dev, c->hsc, 0) == cudaSuccess &&
        cudaHostGetDevicePointer(&c->hseq_dev, c->hseq, 0) == cudaSuccess) {
      *c->hseq = 0;
    } else {
      (void)cudaGetLastError();
      if (c->hseq) cudaFreeHost(c->hseq);
      c->hseq = nullptr;
    }
    MGAR_CUDA(cudaMalloc(&c->derr, sizeof(int)));
    MGAR_CUDA(cudaMemset(c->derr, 0, sizeof(int)));

    // problem data: q is zeroed on fixed nodes
    std::vector<double> qh(q, q + n);
    double qq = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      if (fixed_mask[i]) qh[i] = 0.0;
      qq += qh[i] * qh[i];
    }
    c->qnorm = std::sqrt(qq);
    require(c->qnorm > 0.0 && std::isfinite(c->qnorm), MGAR_ERR_ARG, "load vector is zero");
    std::vector<uint8_t> fh(fixed_mask, fixed_mask + n);
    for (auto& v : fh) v = v ? 1 : 0;
    MGAR_CUDA(cudaMemcpy(c->fixed, fh.data(), n, cudaMemcpyHostToDevice));
    {
      // per fine element: does any of its nodes carry T = 0?
      const Dims& d = c->L[0];
      std::vector<uint8_t> ef((size_t)ne, 0);
      for (int k = 0; k < d.ez; ++k)
        for (int j = 0; j < d.ey; ++j)
          for (int i = 0; i < d.ex; ++i) {
            uint8_t any = 0;
            for (int a = 0; a < c->nen; ++a) {
              const int64_t nd = (i + (a & 1)) + (int64_t)d.NX * ((j + ((a >> 1) & 1)) +
                                                                  (int64_t)d.NY * (k + ((a >> 2) & 1)));
              any |= fh[nd];
            }
            ef[i + (int64_t)d.ex * (j + (int64_t)d.ey * k)] = any;
          }
      MGAR_CUDA(cudaMalloc(&c->efix, ne));
      MGAR_CUDA(cudaMemcpy(c->efix, ef.data(), ne, cudaMemcpyHostToDevice));
      // level-1 (coarse) elements over fine elements with a fixed node
      if (c->nl > 1) {
        const Dims& cd = c->L[1];
        std::vector<uint8_t> cf((size_t)cd.ne, 0);
        for (int k = 0; k < d.ez; ++k)
          for (int j = 0; j < d.ey; ++j)
            for (int i = 0; i < d.ex; ++i)
              if (ef[i + (int64_t)d.ex * (j + (int64_t)d.ey * k)])
                cf[(i / 2) + (int64_t)cd.ex * ((j / 2) + (int64_t)cd.ey * (c->dim == 3 ? k / 2 : 0))] = 1;
        std::vector<int> list;
        for (int64_t e = 0; e < cd.ne; ++e)
          if (cf[e]) list.push_back((int)e);
        c->n_gfix = (int)list.size();
        if (!list.empty()) {
          MGAR_CUDA(cudaMalloc(&c->gfix, list.size() * sizeof(int)));
          MGAR_CUDA(cudaMemcpy(c->gfix, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice));
        }
      }
    }
    MGAR_CUDA(cudaMemcpy(c->q, qh.data(), n * sizeof(double), cudaMemcpyHostToDevice));
    alloc_hierarchy(*c);
    setup_filter(*c);
    if (P.precision == MGAR_MIXED) {
      q_to_df(*c);
      MGAR_CUDA(cudaStreamSynchronize(c->stream));
    }
    // debugging aid: MGAR_NO_GRAPHS=1 issues every V-cycle launch directly
    if (const char* ng = std::getenv("MGAR_NO_GRAPHS")) c->use_graphs = !(ng[0] == '1');
    if (const char* ut = std::getenv("MGAR_UNTILED")) c->untiled = (ut[0] == '1');
    bottom_prepare(*c);
    if (const char* np = std::getenv("MGAR_NO_PDL")) c->use_pdl = np[0] != '1';
    if (const char* ng = std::getenv("MGAR_NO_CG_GRAPH")) c->cg_graph = ng[0] != '1';
    if (const char* dc = std::getenv("MGAR_DF64_CG")) c->ru_cg = dc[0] != '1';
    if (const char* pp = std::getenv("MGAR_PROLONG_POINT")) c->prolong_col = pp[0] != '1';
    if (const char* rd = std::getenv("MGAR_RU_DELTA")) c->ru_delta = std::atof(rd);
    if (const char* fp = std::getenv("MGAR_FUSED_POST")) c->split_post = fp[0] != '1';
    if (const char* sc = std::getenv("MGAR_SPLIT_COARSE")) c->split_coarse_nodes = std::atoll(sc);
    if (const char* bn = std::getenv("MGAR_BOTTOM_NODES")) c->bottom_nodes = std::atoll(bn);
    // the bottom levels as one cluster launch: measured 2 % slower per design
    // cycle than their separate launches, so only on request
    {
      const char* cb = std::getenv("MGAR_CLUSTER_BOTTOM");
      c->bottom_ok = c->bottom_ok && cb && cb[0] == '1';
    }
    if (const char* fc = std::getenv("MGAR_FP64_COARSE")) c->df_coarse = fc[0] != '1';
    if (c->dim == 3) {
      fine3d_prepare(*c);
      if (P.precision == MGAR_MIXED) df3d_prepare(*c);
    }
  } catch (const Error& e) {
    g_create_error = e.msg;
    free_ctx(*c);
    delete c;
    return e.code;
  }
  *out = reinterpret_cast<mgar_t>(c);
  return MGAR_OK;
}

int mgar_destroy(mgar_t h) {
  if (!h) return MGAR_OK;
  Ctx* c = reinterpret_cast<Ctx*>(h);
  free_ctx(*c);
  delete c;
  return MGAR_OK;
}

int mgar_set_stream(mgar_t h, void* stream) {
  return guarded(h, [&](Ctx& c) {
    c.stream = reinterpret_cast<cudaStream_t>(stream);
    return MGAR_OK;
  });
}

int mgar_sizes(mgar_t h, int64_t* n_nodes, int64_t* n_elems) {
  return guarded(h, [&](Ctx& c) {
    if (n_nodes) *n_nodes = c.n;
    if (n_elems) *n_elems = c.ne;
    return MGAR_OK;
  });
}

int mgar_filter(mgar_t h, const double* in, double* out, int transpose) {
  return guarded(h, [&](Ctx& c) {
    require(in && out && in != out, MGAR_ERR_ARG, "filter: bad pointers");
    filter(c, in, out, transpose != 0);
    return MGAR_OK;
  });
}

int mgar_set_density(mgar_t h, const double* rho, int is_physical) {
  return guarded(h, [&](Ctx& c) {
    require(rho != nullptr, MGAR_ERR_ARG, "set_density: null rho");
    set_density(c, rho, is_physical != 0);
    return MGAR_OK;
  });
}

int mgar_set_load(mgar_t h, const double* q) {
  return guarded(h, [&](Ctx& c) {
    require(q != nullptr, MGAR_ERR_ARG, "set_load: null q");
    k_masked_load<<<blocks_for(c.n), kThreads, 0, c.stream>>>(q, c.fixed, c.q, c.n);
    MGAR_LAUNCH_CHECK();
    dot(c, c.q, c.q, c.n, c.dsc + S_TMP);
    fetch_scalars(c, S_TMP, 1);
    const double qnorm = std::sqrt(c.hsc[S_TMP]);
    require(qnorm > 0.0 && std::isfinite(qnorm), MGAR_ERR_ARG, "set_load: load vector is zero");
    c.qnorm = qnorm;
    if (c.p.precision == MGAR_MIXED) q_to_df(c);
    // the CG graphs carry ||q|| in their stopping tests: rebuilt on next use
    if (c.cg_exec) {
      MGAR_CUDA(cudaGraphExecDestroy(c.cg_exec));
      c.cg_exec = nullptr;
    }
    if (c.ru_exec) {
      MGAR_CUDA(cudaGraphExecDestroy(c.ru_exec));
      c.ru_exec = nullptr;
    }
    return MGAR_OK;
  });
}

int mgar_apply_K(mgar_t h, const double* x, double* y) {
  return guarded(h, [&](Ctx& c) {
    require(x && y && x != y, MGAR_ERR_ARG, "apply_K: bad pointers");
    apply_fine64(c, c.ke, x, y, nullptr);
    return MGAR_OK;
  });
}

int mgar_build_hierarchy(mgar_t h) {
  return guarded(h, [&](Ctx& c) {
    build_hierarchy(c);
    join_coarse(c);
    MGAR_CUDA(cudaStreamSynchronize(c.stream));
    int e = 0;
    MGAR_CUDA(cudaMemcpy(&e, c.derr, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
      MGAR_CUDA(cudaMemset(c.derr, 0, sizeof(int)));
      c.have_ref = false;
      throw Error{e, "coarsest factorisation met a non-positive pivot"};
    }
    return MGAR_OK;
  });
}

int mgar_vcycle(mgar_t h, const double* b, double* x) {
  return guarded(h, [&](Ctx& c) {
    require(c.have_ref, MGAR_ERR_STATE, "no hierarchy built");
    require(b && x && b != x, MGAR_ERR_ARG, "vcycle: bad pointers");
    if (c.p.precision == MGAR_FP64) {
      vcycle<double>(c, b, x, false);
    } else {
      convert_d2f(c, b, c.b32, c.n);
      convert_d2f(c, x, c.x32, c.n);
      vcycle<float>(c, c.b32, c.x32, false);
      convert_f2d(c, c.x32, x, c.n);
    }
    return MGAR_OK;
  });
}

int mgar_solve_mgcg(mgar_t h, double* T, int* iters, double* relres) {
  return guarded(h, [&](Ctx& c) {
    require(T != nullptr, MGAR_ERR_ARG, "solve_mgcg: null T");
    int it = 0;
    double rr = 0.0;
    const int rc = solve_mgcg(c, T, &it, &rr);
    if (iters) *iters = it;
    if (relres) *relres = rr;
    if (rc == MGAR_ERR_MAXIT) c.err = "MGCG reached cg_max";
    return rc;
  });
}

int mgar_solve_mgar(mgar_t h, const double* T_prev, double* T, double* res, int* accepted) {
  return guarded(h, [&](Ctx& c) {
    require(T_prev && T, MGAR_ERR_ARG, "solve_mgar: null pointer");
    solve_mgar(c, T_prev, T, res, accepted);
    return MGAR_OK;
  });
}

int mgar_sensitivity(mgar_t h, const double* T, double* dc, double* dv, double* compliance) {
  return guarded(h, [&](Ctx& c) {
    require(T != nullptr, MGAR_ERR_ARG, "sensitivity: null T");
    sensitivity(c, T, dc, dv, compliance);
    return MGAR_OK;
  });
}

int mgar_postprocess(mgar_t h, const double* rho, const double* T, double volfrac, double* rho_out,
                     double* level, double* volume) {
  return guarded(h, [&](Ctx& c) {
    require(rho && T && rho_out, MGAR_ERR_ARG, "postprocess: null pointer");
    require(volfrac > 0.0 && volfrac < 1.0, MGAR_ERR_ARG, "postprocess: volfrac outside (0, 1)");
    postprocess(c, rho, T, volfrac, rho_out, level, volume);
    return MGAR_OK;
  });
}

int mgar_oc_update(mgar_t h, double* rho, const double* dc, double volfrac, double move,
                   double* lambda, double* change) {
  return guarded(h, [&](Ctx& c) {
    require(rho && dc, MGAR_ERR_ARG, "oc_update: null pointer");
    require(volfrac > 0.0 && volfrac < 1.0 && move > 0.0, MGAR_ERR_ARG, "oc_update: bad volfrac/move");
    oc_update(c, rho, dc, volfrac, move, lambda, change);
    return MGAR_OK;
  });
}

int mgar_step(mgar_t h, double* rho, double* T, int cycle, mgar_step_info* info) {
  return guarded(h, [&](Ctx& c) {
    require(rho && T, MGAR_ERR_ARG, "step: null pointer");
    mgar_step_info inf = design_cycle(c, rho, T, cycle);
    if (info) *info = inf;
    if (inf.status == MGAR_ERR_MAXIT) c.err = "MGCG reached cg_max";
    return MGAR_OK;
  });
}

int mgar_run(mgar_t h, const double* rho_host, int cycles, double* rho_out_host,
             mgar_step_info* info_host) {
  return guarded(h, [&](Ctx& c) {
    require(rho_host && rho_out_host && cycles >= 0, MGAR_ERR_ARG, "run: bad arguments");
    if (!c.run_rho) {
      MGAR_CUDA(cudaMalloc(&c.run_rho, c.ne * sizeof(double)));
      MGAR_CUDA(cudaMalloc(&c.run_T, c.n * sizeof(double)));
    }
    MGAR_CUDA(cudaMemcpyAsync(c.run_rho, rho_host, c.ne * sizeof(double), cudaMemcpyHostToDevice,
                              c.stream));
    MGAR_CUDA(cudaMemsetAsync(c.run_T, 0, c.n * sizeof(double), c.stream));
    c.have_ref = false;
    for (int k = 1; k <= cycles; ++k) {
      mgar_step_info inf = design_cycle(c, c.run_rho, c.run_T, k);
      if (info_host) info_host[k - 1] = inf;
    }
    MGAR_CUDA(cudaMemcpyAsync(rho_out_host, c.run_rho, c.ne * sizeof(double),
                              cudaMemcpyDeviceToHost, c.stream));
    MGAR_CUDA(cudaStreamSynchronize(c.stream));
    return MGAR_OK;
  });
}

int mgar_profile_start(mgar_t h, int kernel_class) {
  return guarded(h, [&](Ctx& c) {
    if (!c.prof_ev) {
      c.prof_ev = new cudaEvent_t[2 * kProfMax]();
      c.prof_sites = new const char*[2 * kProfMax]();
      for (int i = 0; i < 2 * kProfMax; ++i) MGAR_CUDA(cudaEventCreate(&c.prof_ev[i]));
    }
    c.prof_class = kernel_class;
    c.prof_used = 0;
    c.prof_open = false;
    c.prof_report.clear();
    if (kernel_class == MGAR_KC_TIMELINE) {
      MGAR_CUDA(cudaEventRecord(c.prof_ev[0], c.stream));
      c.prof_sites[0] = "start";
      c.prof_used = 1;
    }
    return MGAR_OK;
  });
}

int mgar_profile_stop(mgar_t h, double* total_ms, int64_t* launches) {
  return guarded(h, [&](Ctx& c) {
    MGAR_CUDA(cudaStreamSynchronize(c.stream));
    double tot = 0.0;
    int64_t count = 0;
    if (c.prof_class == MGAR_KC_TIMELINE) {
      std::vector<std::pair<std::string, std::pair<int64_t, double>>> acc;
      for (int i = 1; i < c.prof_used; ++i) {
        float ms = 0.f;
        MGAR_CUDA(cudaEventElapsedTime(&ms, c.prof_ev[i - 1], c.prof_ev[i]));
        tot += ms;
        std::string site = c.prof_sites[i];
        const size_t slash = site.rfind('/');
        if (slash != std::string::npos) site = site.substr(slash + 1);
        bool found = false;
        for (auto& a : acc)
          if (a.first == site) {
            a.second.first += 1;
            a.second.second += ms;
            found = true;
          }
        if (!found) acc.push_back({site, {1, (double)ms}});
      }
      count = c.prof_used - 1;
      std::sort(acc.begin(), acc.end(),
                [](const auto& x, const auto& y) { return x.second.second > y.second.second; });
      char line[256];
      for (auto& a : acc) {
        snprintf(line, sizeof(line), "%-40s %8lld %10.3f ms %6.2f%%\n", a.first.c_str(),
                 (long long)a.second.first, a.second.second, 100.0 * a.second.second / tot);
        c.prof_report += line;
      }
    } else {
      for (int i = 0; i < c.prof_used; ++i) {
        float ms = 0.f;
        MGAR_CUDA(cudaEventElapsedTime(&ms, c.prof_ev[2 * i], c.prof_ev[2 * i + 1]));
        tot += ms;
      }
      count = c.prof_used;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = count;
    c.prof_class = 0;
    c.prof_used = 0;
    return MGAR_OK;
  });
}

int mgar_profile_report(mgar_t h, char* buf, int64_t len) {
  return guarded(h, [&](Ctx& c) {
    require(buf && len > 0, MGAR_ERR_ARG, "profile_report: bad buffer");
    const size_t n = std::min<size_t>((size_t)len - 1, c.prof_report.size());
    std::memcpy(buf, c.prof_report.data(), n);
    buf[n] = 0;
    return MGAR_OK;
  });
}

int64_t mgar_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
