// Internal definitions shared by the CUDA translation units of libmgar.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>

#include "../../include/mgar.h"
#include "df64.cuh"

namespace mgar {

// Bounds checks of computed indices.  In the checked build (MGAR_CHECKED,
// all units compiled as one) CK(i, n) verifies 0 <= i < n; a failure records
// the source line, index and bound of the first bad access, which is then
// skipped, and the API reports it.  In the normal build CK is `true`.
#ifdef MGAR_CHECKED
__device__ unsigned long long g_ck_fault[4];
__device__ __forceinline__ bool ck_fail(long long i, long long n, int line) {
  if (atomicCAS(&g_ck_fault[0], 0ull, (unsigned long long)line) == 0ull) {
    g_ck_fault[1] = (unsigned long long)i;
    g_ck_fault[2] = (unsigned long long)n;
  }
  return false;
}
#define CK(i, n) (((long long)(i) >= 0 && (long long)(i) < (long long)(n)) ? true : ::mgar::ck_fail((long long)(i), (long long)(n), __LINE__))
#else
#define CK(i, n) true
#endif
// length of the reduction scratch (checked build)
#ifdef MGAR_CHECKED
__device__ long long g_partials_len;
#else
constexpr long long g_partials_len = 0;
#endif

constexpr int kMaxLevels = 14;
constexpr int kThreads = 256;
constexpr int kMinPartialBlocks = 8192;
constexpr int64_t kBottomNodes = 8192;  // largest level handled by the V-cycle's cluster launch
constexpr int kMaxFilterOffsets = 3072;
constexpr int kMaxM = 8;
constexpr int kOcCand = 31;      // multisection candidates per pass (5 bits)
constexpr int kOcPasses = 6;     // FP32 passes at most: ln-bracket 92 -> 9e-8
constexpr double kOcTarget = 2e-5;  // passes stop once the ln-bracket is this narrow (the margin below)
constexpr int kOcAmbMax = 4096;  // ambiguous elements handled by the FP64 finish
constexpr double kOcMargin = 2e-5;  // ln-bracket widening that absorbs FP32 volume rounding
constexpr size_t kBandSmemMax = 160 * 1024;  // band factorised in shared memory up to this size

// Slots of the device scalar array.
enum Slot : int {
  S_RZ0 = 0, S_RZ1 = 1, S_PAP = 2, S_RR = 3, S_TMP = 4, S_NORM = 5,
  S_CGIT = 6, S_CGPAR = 7,  // device-side CG loop: iteration count, buffer parity
  S_OC_LO = 8, S_OC_HI = 9, S_OC_DONE = 10, S_OC_LAM = 11, S_OC_VOL = 12, S_OC_CHANGE = 13,
  S_OC_STEPS = 14, S_COMPL = 15,
  S_GS = 16,      // 16..31 Gram-Schmidt coefficients
  S_KR = 32,      // 32..95 reduced matrix (8x8)
  S_QR = 96,      // 96..103 reduced right-hand side
  S_Y = 104,      // 104..111 reduced solution
  S_RES2 = 112, S_FLAG = 113,
  S_CRED = 114,     // MGAR: compliance of the reduced solution, q_R . y = q . t~
  S_RUCOUNT = 115,  // FP32 CG: reliable updates so far
  S_OC_LA = 116, S_OC_LB = 117, S_OC_MUA = 118, S_OC_MUB = 119, S_OC_C = 120, S_OC_B = 121,
  S_OC_MU = 122, S_OC_FAIL = 123,
  S_OC_LPREV = 124, S_OC_HAVEPREV = 125,  // ln mu of the previous update (warm start)
  S_CGFIRST = 126,  // FP32 CG: nonzero until the first direction is formed
  S_RMAX = 127,     // FP32 CG: ||r|| at the last reliable update
  S_OC_CAND = 128,  // 128..158 multisection candidates mu
  S_OC_CANDL = 160, // 160..190 their ln mu
  S_DERR = 191,     // host mirror only: the device error flag, published with every fetch
  S_RREC = 192,     // FP32 CG: recursive ||r|| at the last update decision
  S_RUSTALL = 193,  // FP32 CG: successive updates that did not halve the true ||r||
  S_COUNT = 194
};

// 1 / sqrt(a) for a > 0: an FP32 seed refined by two Newton-Raphson steps
// y <- y (3 - a y^2) / 2 (each step doubles the correct bits: 24 -> 48 -> 96),
// so the pivot costs no FP64 square root or division chain.
__device__ __forceinline__ double rsqrt_nr(double a) {
  const float af = (float)a;
  if (!(af > 0.f) || isinf(af)) return 1.0 / sqrt(a);  // outside the FP32 range
  double y = (double)rsqrtf(af);
  y = y * (1.5 - 0.5 * a * y * y);
  y = y * (1.5 - 0.5 * a * y * y);
  return y;
}
__device__ __forceinline__ float rsqrt_nr(float a) {
  float y = rsqrtf(a);
  return y * (1.5f - 0.5f * a * y * y);
}

// Unsigned division by an invariant divisor d >= 1 for numerators below
// 2^31, by multiply-high and shift (Granlund and Montgomery, "Division by
// invariant integers using multiplication", 1994): with l = ceil(log2 d)
// and m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(m, n) + n) >> l.
struct FastDiv {
  uint32_t d = 1, m = 1, l = 0;
  FastDiv() = default;
  explicit FastDiv(uint32_t div) : d(div) {
    l = 0;
    while ((1ull << l) < div) ++l;
    m = (uint32_t)((((1ull << 32) * ((1ull << l) - div)) / div) + 1);
  }
  __host__ __device__ __forceinline__ uint32_t div(uint32_t n) const {
#ifdef __CUDA_ARCH__
    return (__umulhi(m, n) + n) >> l;
#else
    return (uint32_t)((((uint64_t)m * n) >> 32) + n) >> l;
#endif
  }
};

// Element/node counts of one multigrid level.  Indices are 32-bit: the
// library refuses grids with 2^31 / 32 nodes or more.
struct Dims {
  int ex, ey, ez;  // elements per axis (ez = 1 in 2D)
  int NX, NY, NZ;  // nodes per axis (NZ = 1 in 2D)
  int64_t n, ne;
  FastDiv fNX, fNXY, fEX, fEXY;  // node row / plane, element row / plane
};

template <typename Real>
struct LevelBuf {
  Real* st = nullptr;    // [S][n] assembled stencil, levels >= 1
  Real* dinv = nullptr;  // [n] 1/diag, levels >= 1
  Real* elem = nullptr;  // [ne][nen*nen] Galerkin element matrices, levels >= 1
  Real* x = nullptr;     // V-cycle iterate (levels >= 1; level 0 uses caller arrays)
  Real* b = nullptr;     // right-hand side (levels >= 1)
  Real* t = nullptr;     // smoothing double buffer
  Real* r = nullptr;     // residual
};

struct Ctx {
  mgar_params p{};
  int dim = 2, nen = 4, S = 9;
  cudaStream_t stream = nullptr;
  std::string err;
  int nl = 0;
  Dims L[kMaxLevels]{};
  int64_t n = 0, ne = 0;
  int sms = 152;          // multiprocessors of the device
  int grid_blocks = 0;    // blocks of grid-stride reduction kernels over nodes
  int grid_blocks_e = 0;  // ... over elements

  // fine level, problem data
  uint8_t* fixed = nullptr;
  uint8_t* efix = nullptr;   // per fine element: 1 if any of its nodes is fixed
  int* gfix = nullptr;       // level-1 elements containing a fine element with a fixed node
  int n_gfix = 0;
  double* q = nullptr;
  double qnorm = 0.0;
  double mgar_cred = 0.0;  // q . t~ of the last MGAR solve (Eq. 19-21)
  double* rho_phys = nullptr;
  double* ke = nullptr;     // current conductivities k_e(rho~)
  double* ke0 = nullptr;    // reference conductivities (K0)
  float* ke_f = nullptr;    // FP32 copies (mixed mode)
  float* ke0_f = nullptr;
  double* inv_hs = nullptr; // 1 / sum of filter weights
  float2* inv_hs_df = nullptr;  // the same as double-float pairs (mixed path)
  float2* rho_phys_df = nullptr; // rho~ as double-float pairs (mixed path)
  int4* f_offs = nullptr;   // filter offsets (dx, dy, dz)
  double* f_w = nullptr;    // filter weights max(0, r - |d|)
  double* dv = nullptr;     // F^T (1/E)
  float2* rsdv = nullptr;   // 1 / sqrt(dv), double-float
  float2* dv_df = nullptr;  // dv, double-float
  int n_filter = 0;
  double filter_r = 0.0;    // radius of the current tables
  int filter_cap = 0;       // offsets the tables have room for
  int4* f_offs_h = nullptr; // pinned staging of the tables (continuous filter)
  double* f_w_h = nullptr;

  // hierarchy
  LevelBuf<double> h64[kMaxLevels];
  LevelBuf<float> h32[kMaxLevels];
  bool have_ref = false;
  int nc = 0, bw = 0;
  double* band = nullptr;   // [nc][bw+1] Cholesky factor (lower band)
  double* rdiag = nullptr;  // [nc] reciprocals of the factor's diagonal
  double* cinv = nullptr;   // [nc][nc] inverse of the coarsest operator
  double* tables = nullptr;  // k0 (nen^2) then Galerkin sub-element tables G
  float* tables_f = nullptr; // G in FP32

  // Krylov / reanalysis vectors
  double *r = nullptr, *z = nullptr, *pv = nullptr, *Ap = nullptr, *tm = nullptr;
  double* tmp_dc = nullptr;
  double *R = nullptr, *W = nullptr;    // [m][n]
  float *b32 = nullptr, *x32 = nullptr; // mixed-mode level-0 buffers
  // mixed 3D CG with reliable updates: FP32 correction since the last update,
  // the two direction buffers and A p
  float *xc32 = nullptr, *p32 = nullptr, *p32b = nullptr, *y32 = nullptr;
  // mixed mode: double-float (hi, lo) copies for the outer CG
  float2 *ke_df = nullptr, *df_q = nullptr, *df_x = nullptr, *df_r = nullptr, *df_p = nullptr,
         *df_Ap = nullptr, *df_p2 = nullptr;
  float2* df_e = nullptr;  // mixed mode: df64 scratch over elements (filter input)
  float2* kd_df = nullptr; // mixed mode: 4 sum_e k_e per node (df64), the 3D operator's diagonal x 12
  double* tmp_e = nullptr;
  // OC update: s_e, the move limits and rho as double-float pairs, FP32 copies
  float2 *oc_s = nullptr, *oc_lo = nullptr, *oc_hi = nullptr, *oc_rho = nullptr;
  float *oc_s32 = nullptr, *oc_lo32 = nullptr, *oc_hi32 = nullptr, *dv32 = nullptr;
  int *oc_amb = nullptr, *oc_namb = nullptr;
  int64_t oc_fallbacks = 0;

  // reductions
  double* partials = nullptr;        // [8][max blocks]
  unsigned int* counter = nullptr;   // ticket counters [8]
  double* dsc = nullptr;             // device scalars [S_COUNT]
  double* hsc = nullptr;             // pinned host mirror [S_COUNT]
  double* hsc_dev = nullptr;         // its device-side address (mapped)
  unsigned long long* hseq = nullptr;      // mapped pinned sequence number
  unsigned long long* hseq_dev = nullptr;
  unsigned long long seq_sent = 0;
  int* derr = nullptr;               // device error flag

  // whole-run buffers (mgar_run)
  double *run_rho = nullptr, *run_T = nullptr;

  // CUDA graphs of fixed launch sequences (V-cycles), captured on cap_stream
  // once and replayed on stream; all buffers they touch live as long as the
  // handle, so a graph stays valid across hierarchy rebuilds.
  struct GraphEntry {
    int kind = -1;
    const void* a = nullptr;
    const void* b = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
  };
  static constexpr int kGraphs = 16;
  GraphEntry graphs[kGraphs];
  bool use_graphs = true;
  bool untiled = false;  // MGAR_UNTILED=1: generic finest-level kernels (debugging aid)
  int f3d_gz[5] = {};     // z runs of the tiled finest-level kernels [mode]
  int df3d_gz[3] = {};    // z runs of the tiled df64 operator kernels [mode]
  bool df3d_tile = false; // their tile: 32 x 8, or 43 x 11 when that leaves fewer lanes idle
  bool f3d_tile = false;  // FP32 finest-level tile: 32 x 8, or 43 x 5 when that leaves fewer lanes idle
  bool bottom_ok = false; // the V-cycle's bottom levels run as one cluster launch
  int bottom_cluster = 8; // CTAs in that cluster
  int64_t bottom_nodes = kBottomNodes;  // largest level it takes
  bool use_pdl = true;    // programmatic dependent launch of the V-cycle and CG kernels
  bool prolong_col = true;  // 3D interpolation by z-columns (MGAR_PROLONG_POINT=1: one node per thread)
  // device-side CG loop (3D mixed path): one graph with a conditional WHILE node
  bool cg_graph = true;
  cudaGraphExec_t cg_exec = nullptr;
  int cg_exec_cgmax = 0;   // the iteration cap captured in cg_exec
  int64_t prologue_kernels = 0, body_kernels = 0;
  // 3D mixed path: FP32 CG iterations with reliable updates of x and r in
  // df64 (MGAR_DF64_CG=1 selects the df64 CG); an update whenever ||r||
  // falls below ru_delta times its value at the previous update
  bool ru_cg = true;
  double ru_delta = 1e-3;
  cudaGraphExec_t ru_exec = nullptr;
  int64_t ru_body_kernels = 0, ru_update_kernels = 0;
  // finest post-smoothing as a thin interpolation pass + the tiled sweep
  // (faster than interpolating inside the tiled pass: 6.67 vs 6.83 ms per
  // design cycle at 128^3); MGAR_FUSED_POST=1 selects the fused pass
  bool split_post = true;
  // coarse levels above this many nodes post-smooth as interpolation + sweep
  // (the 65^3 level of a 128^3 grid: 6.60 vs 6.66 ms per design cycle)
  int64_t split_coarse_nodes = 100000;
  cudaStream_t cap_stream = nullptr;
  // the coarsest factorisation runs on a side stream while the solve starts
  // (it needs one SM for ~200 us); join_coarse orders the main stream after
  // it before the first V-cycle
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool coarse_pending = false;
  bool derr_fresh = true;  // the last published device error flag follows every factorisation
  cudaStream_t cap_stream2 = nullptr;  // captures the body of a graph's IF node
  // the FP32 V-cycle's coarsest factor and inverse in df64 on the FP32 pipe
  // (MGAR_FP64_COARSE=1: in FP64, as the FP64 V-cycle's)
  bool df_coarse = true;

  // instrumentation: CUDA-event timing of one kernel class
  int prof_class = 0;
  int prof_used = 0;
  bool prof_open = false;  // a scope of the timed class is open (inner ones are not timed)
  cudaEvent_t* prof_ev = nullptr;  // [2 * kProfMax]
  // timeline mode (prof_class == MGAR_KC_TIMELINE): an event after every
  // launch site; device time between consecutive marks goes to the later site
  const char** prof_sites = nullptr;  // [2 * kProfMax]
  std::string prof_report;
};

constexpr int kProfMax = 65536;

// Coarsest-level factor and inverse.  Both V-cycle precisions factorise
// and invert in FP64 and sum the coarse solve in FP64: an FP32 factor of the
// coarsest operator (condition number up to ~1e5 with the SIMP contrast)
// moves the V-cycle far enough to change the reanalysis basis of Eq. 17
// measurably.
template <typename Real>
struct CoarseT {
  using T = double;
  static double* band(Ctx& c) { return c.band; }
  static double* rdiag(Ctx& c) { return c.rdiag; }
  static double* inv(Ctx& c) { return c.cinv; }
};

// Programmatic dependent launch.  A kernel started by launch_pdl may begin
// while its predecessor on the stream is still running: it calls pdl_wait()
// first thing, a hardware wait until the predecessor has completed and its
// memory is visible, so only launch latency and block dispatch overlap.
// pdl_trigger() lets the successor be dispatched before this grid ends.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// handle whose API call is running on this host thread (set by the C ABI)
Ctx*& current_ctx();

// Brackets the launches issued in its scope with two events when the
// handle is timing kernel class `kc`.
struct ProfScope {
  Ctx& c;
  bool on;
  ProfScope(Ctx& ctx, int kc)
      : c(ctx), on(ctx.prof_class == kc && ctx.prof_used < kProfMax && !ctx.prof_open) {
    if (on) {
      cudaEventRecord(c.prof_ev[2 * c.prof_used], c.stream);
      c.prof_open = true;  // a nested scope of the same class is part of this one
    }
  }
  ~ProfScope() {
    if (on) {
      cudaEventRecord(c.prof_ev[2 * c.prof_used + 1], c.stream);
      ++c.prof_used;
      c.prof_open = false;
    }
  }
};

// ---------------------------------------------------------------- errors
struct Error {
  int code;
  std::string msg;
};

#define MGAR_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      throw ::mgar::Error{MGAR_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// Every kernel launch is followed by MGAR_LAUNCH_CHECK(), which also counts
// it and, while a handle records a device timeline, marks the launch site.
void count_launch();
void count_launches(int64_t delta);
int64_t launches_so_far();
void prof_mark(const char* site);
#define MGAR_STR2(x) #x
#define MGAR_STR(x) MGAR_STR2(x)
#define MGAR_LAUNCH_CHECK()                              \
  do {                                                   \
    ::mgar::count_launch();                              \
    ::mgar::prof_mark(__FILE__ ":" MGAR_STR(__LINE__));  \
    MGAR_CUDA(cudaGetLastError());                       \
  } while (0)
// as MGAR_LAUNCH_CHECK, with an explicit site name for the timeline
#define MGAR_LAUNCH_CHECK_AT(site)     \
  do {                                 \
    ::mgar::count_launch();            \
    ::mgar::prof_mark(site);           \
    MGAR_CUDA(cudaGetLastError());     \
  } while (0)
// "<kind> L<level>" site names (kind: 0 jacobi0, 1 sweep, 2 residual, 3 restrict,
// 4 prolong, 5 coarse, 6 pre3d, 7 post3d, 8 sweep3d, 9 resid3d)
const char* level_site(int kind, int level);

inline void require(bool ok, int code, const std::string& msg) {
  if (!ok) throw Error{code, msg};
}

inline int blocks_for(int64_t n, int threads = kThreads) {
  int64_t b = (n + threads - 1) / threads;
  return (int)(b < 1 ? 1 : b);
}

// Zero fill and device-to-device copy as kernels: in a graph they run on the
// SMs beside the other branches' kernels instead of queueing for a copy
// engine, and in a stream they follow a kernel without a switch of engine.
template <typename T>
__global__ void k_zero(T* __restrict__ a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = T(0);
}
template <typename T>
__global__ void k_copy(const T* __restrict__ src, T* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}
constexpr int kFillBlocksMax = 4096;
template <typename T>
inline void zero_async(T* a, int64_t n, cudaStream_t s) {
  k_zero<T><<<std::min(blocks_for(n), kFillBlocksMax), kThreads, 0, s>>>(a, n);
}
template <typename T>
inline void copy_async(const T* src, T* dst, int64_t n, cudaStream_t s) {
  k_copy<T><<<std::min(blocks_for(n), kFillBlocksMax), kThreads, 0, s>>>(src, dst, n);
}

// ------------------------------------------------------------ reductions
// Deterministic block sum of N values: each block's partial sums go to
// partials[k*gridDim.x + blockIdx.x]; the last block to arrive (ticket on
// *counter) adds them up, every thread accumulating all N sums over its
// share of the blocks (independent loads, no barrier per value), resets the
// ticket, and returns true with the totals in every thread.  Other blocks
// return false.  Every thread of every block must call it.  The summation
// order is fixed, so results are reproducible run to run.
// Block, thread and grid given as linear ids (tid < nthr <= 1024; a last
// partial warp is fine; bid < nblk), so multi-dimensional launches can use it.
// The ticket and cross-block stage, given each warp's sums in its lane 0
// (w; other lanes ignored).
template <int N>
__device__ __forceinline__ bool block_sum_last_core(const double (&w)[N], double* partials,
                                                    unsigned int* counter, double (&total)[N],
                                                    int tid, int nthr, int bid, int nblk) {
  __shared__ double sh[N][32];  // up to 1024 threads
  __shared__ double tot[N];
  __shared__ bool last;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k)
    if (lane == 0) sh[k][warp] = w[k];
  __syncthreads();
  for (int k = tid; k < N; k += nthr) {
    double s = 0.0;
    for (int q = 0; q < nw; ++q) s += sh[k][q];
    if (CK((int64_t)k * nblk + bid, g_partials_len)) partials[k * nblk + bid] = s;
    __threadfence();
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned int t = atomicAdd(counter, 1u);
    last = (t == (unsigned int)nblk - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // L2-coherent loads (ld.global.cg: the partials of other blocks, ordered
  // by their fences and the counter), U rows of blocks in flight together;
  // the adds keep the order b = tid, tid + nthr, ...
  constexpr int U = N <= 2 ? 4 : 1;
  double acc[N];
#pragma unroll
  for (int k = 0; k < N; ++k) acc[k] = 0.0;
  for (int b = tid; b < nblk; b += U * nthr) {
    double v[U][N];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < N; ++k)
        v[u][k] = b + u * nthr < nblk ? __ldcg(partials + k * nblk + b + u * nthr) : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < N; ++k) acc[k] += v[u][k];
  }
#pragma unroll
  for (int k = 0; k < N; ++k) {
    double s = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  for (int k = tid; k < N; k += nthr) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += sh[k][w];
    tot[k] = s;
  }
  if (tid == 0) *counter = 0u;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) total[k] = tot[k];
  return true;
}

template <int N>
__device__ __forceinline__ bool block_sum_last_ids(double (&v)[N], double* partials,
                                                   unsigned int* counter, double (&total)[N],
                                                   int tid, int nthr, int bid, int nblk) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
    double s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    v[k] = s;
  }
  return block_sum_last_core<N>(v, partials, counter, total, tid, nthr, bid, nblk);
}

// One double-float value per thread: the warp sums are formed in df64 on
// the FP32 pipe (GB300 runs FP64 at 1/58 of the FP32 rate, and an FP64
// shuffle tree over every warp of a wide grid costs microseconds), then
// FP64 across warps and blocks as in block_sum_last_ids.
__device__ __forceinline__ bool block_sum_last_df(df v, double* partials, unsigned int* counter,
                                                  double& total, int tid, int nthr, int bid,
                                                  int nblk) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_down_sync(0xffffffffu, v.hi, o);
    const float l = __shfl_down_sync(0xffffffffu, v.lo, o);
    v = df_add(v, df{h, l});
  }
  double w[1] = {0.0};
  if ((tid & 31) == 0) w[0] = df_to_double(v);
  double t[1];
  const bool last = block_sum_last_core<1>(w, partials, counter, t, tid, nthr, bid, nblk);
  total = t[0];
  return last;
}

template <int N>
__device__ __forceinline__ bool block_sum_last(double (&v)[N], double* partials,
                                               unsigned int* counter, double (&total)[N]) {
  return block_sum_last_ids<N>(v, partials, counter, total, threadIdx.x, blockDim.x, blockIdx.x,
                               gridDim.x);
}

// Many sums of FP32 per-thread values (N of them, e.g. candidate volumes):
// warp sums in FP32 (shuffles), then FP64 for the few cross-warp and
// cross-block additions.  FP64 runs at 1/58 of the FP32 rate here, so
// reducing N doubles through shuffles costs more than the data pass.  The
// last block sums each value's per-block partials with one warp, lanes
// striding over the blocks.  Same ticket protocol and fixed order as
// block_sum_last.
template <int N>
__device__ __forceinline__ bool block_sum_last_f32(float (&v)[N], double* partials,
                                                   unsigned int* counter, double (&total)[N]) {
  __shared__ float sh[N][kThreads / 32];
  __shared__ double tot[N];
  __shared__ bool last;
  const int tid = threadIdx.x, nthr = blockDim.x, bid = blockIdx.x, nblk = gridDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    float s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  for (int k = tid; k < N; k += nthr) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += (double)sh[k][w];
    if (CK((int64_t)k * nblk + bid, g_partials_len)) partials[k * nblk + bid] = s;
    __threadfence();
  }
  __syncthreads();
  if (tid == 0) {
    const unsigned int t = atomicAdd(counter, 1u);
    last = (t == (unsigned int)nblk - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  for (int k = warp; k < N; k += nw) {
    double s = 0.0;
    // four loads in flight per lane (L2-coherent), added in block order
    const double* pk = partials + (size_t)k * nblk;
    int b = lane;
    for (; b + 96 < nblk; b += 128) {
      const double v0 = __ldcg(pk + b), v1 = __ldcg(pk + b + 32), v2 = __ldcg(pk + b + 64),
                   v3 = __ldcg(pk + b + 96);
      s += v0;
      s += v1;
      s += v2;
      s += v3;
    }
    for (; b < nblk; b += 32) s += __ldcg(pk + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) tot[k] = s;
  }
  if (tid == 0) *counter = 0u;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) total[k] = tot[k];
  return true;
}

// As block_sum_last, storing the totals to out[0..N) from the last block.
template <int N>
__device__ __forceinline__ void block_sum_finish(double (&v)[N], double* partials,
                                                 unsigned int* counter, double* out) {
  double t[N];
  if (block_sum_last<N>(v, partials, counter, t) && threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = t[k];
  }
}

// As block_sum_last_df over a 1D grid, storing the total to *out.
__device__ __forceinline__ void block_sum_finish_df(df v, double* partials, unsigned int* counter,
                                                    double* out) {
  double t;
  if (block_sum_last_df(v, partials, counter, t, threadIdx.x, blockDim.x, blockIdx.x, gridDim.x) &&
      threadIdx.x == 0)
    *out = t;
}

// *a / *b for the whole block, computed once by thread 0: GB300's FP64
// division costs tens of FP64 operations at 1/58 of the FP32 rate, so one
// per thread of a wide grid costs microseconds.  Every thread of the block
// must call these, once per kernel.
__device__ __forceinline__ double block_div(const double* a, const double* b) {
  __shared__ double s;
  if (threadIdx.x == 0) s = *a / *b;
  __syncthreads();
  return s;
}
__device__ __forceinline__ float block_div_f(const double* a, const double* b) {
  __shared__ float s;
  if (threadIdx.x == 0) s = (float)(*a / *b);
  __syncthreads();
  return s;
}
__device__ __forceinline__ df block_div_df(const double* a, const double* b) {
  __shared__ float2 s;
  if (threadIdx.x == 0) {
    const df d = df_from_double(*a / *b);
    s = make_float2(d.hi, d.lo);
  }
  __syncthreads();
  return df{s.x, s.y};
}

// Deterministic block max (values >= 0) with the same last-block scheme.
__device__ __forceinline__ void block_max_finish(double v, double* partials, unsigned int* counter,
                                                 double* out) {
  __shared__ double sh[kThreads / 32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s = fmax(s, sh[w]);
    if (CK(blockIdx.x, g_partials_len)) partials[blockIdx.x] = s;
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
#pragma unroll 4
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s = fmax(s, __ldcg(partials + b));
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
  if (lane == 0) sh[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < nw; ++w) m = fmax(m, sh[w]);
    *out = m;
    *counter = 0u;
  }
}

// ------------------------------------------------------------- operators
// Matrix-free fine-level operator A = Z K Z + (I - Z) with element
// conductivities k_e (Eq. 3-4).  With ksub set, the coefficient is
// k_e - ksub_e and fixed rows give 0 (the operator dK = A - A0).
//
// Unit-element conductivity matrices (Galerkin integrals of the shape
// function gradients):
//   Q4: k0 = 1/6 * (4 on the diagonal, -1 between edge neighbours, -2
//       between opposite corners)
//   H8: k0 = 1/12 * (4 on the diagonal, 0 between edge neighbours, -1
//       between face- and body-diagonal corners)
// so the node-centred stencil of K at node i, with the (up to) 2^d
// elements e around it, is
//   2D: 4 sum k_e x_i - sum_edges (k_a + k_b) x_j - 2 sum_diag k_e x_j, / 6
//   3D: 4 sum k_e x_i - sum_facediag (k_a + k_b) x_j - sum_bodydiag k_e x_j, / 12
template <typename Real>
struct FineOp {
  const Real* ke;
  const Real* ksub;   // nullptr, or reference conductivities for dK
  const uint8_t* fixed;
  int ex, ey, ez, NX, NY, NZ;
  int n;
  FastDiv fNX, fNXY;
};

// Neighbour loads never form an out-of-range address, even speculatively:
// a neighbour outside the grid is read at a clamped valid index and its
// value discarded.
template <typename Real>
__device__ __forceinline__ Real ld_x(const Real* x, const uint8_t* fixed, int idx, bool ok, int n) {
  const int j = (ok && CK(idx, n)) ? idx : 0;
  const Real v = x[j];
  return (ok && !fixed[j]) ? v : Real(0);
}

template <typename Real>
__device__ __forceinline__ Real ld_k(const FineOp<Real>& op, int e, bool ok) {
  const int ee = (ok && CK(e, op.ex * op.ey * op.ez)) ? e : 0;
  Real k = op.ke[ee];
  if (op.ksub) k -= op.ksub[ee];
  return ok ? k : Real(0);
}

// (A x)_i and diag(A)_i for a 2D node (i, j).
template <typename Real>
__device__ __forceinline__ Real fine_row2(const FineOp<Real>& op, const Real* __restrict__ x,
                                          int i, int j, Real& diag) {
  const int idx = i + op.NX * j;
  if (!CK(idx, op.n)) return Real(0);
  if (op.fixed[idx]) {
    diag = Real(1);
    return op.ksub ? Real(0) : x[idx];
  }
  const bool xm = i > 0, xp = i < op.ex, ym = j > 0, yp = j < op.ey;
  // elements around the node: k[oy][ox], o = 0 -> element at -1, 1 -> at 0
  const int e00 = (i - 1) + op.ex * (j - 1);
  const Real k00 = ld_k(op, e00, xm && ym);
  const Real k01 = ld_k(op, e00 + 1, xp && ym);
  const Real k10 = ld_k(op, e00 + op.ex, xm && yp);
  const Real k11 = ld_k(op, e00 + op.ex + 1, xp && yp);
  const Real ksum = (k00 + k01) + (k10 + k11);
  const int NX = op.NX;
  const Real* xr = x;
  const uint8_t* fx = op.fixed;
  Real acc = Real(4) * ksum * xr[idx];
  acc -= (k00 + k10) * ld_x(xr, fx, idx - 1, xm, op.n);
  acc -= (k01 + k11) * ld_x(xr, fx, idx + 1, xp, op.n);
  acc -= (k00 + k01) * ld_x(xr, fx, idx - NX, ym, op.n);
  acc -= (k10 + k11) * ld_x(xr, fx, idx + NX, yp, op.n);
  acc -= Real(2) * k00 * ld_x(xr, fx, idx - NX - 1, xm && ym, op.n);
  acc -= Real(2) * k01 * ld_x(xr, fx, idx - NX + 1, xp && ym, op.n);
  acc -= Real(2) * k10 * ld_x(xr, fx, idx + NX - 1, xm && yp, op.n);
  acc -= Real(2) * k11 * ld_x(xr, fx, idx + NX + 1, xp && yp, op.n);
  diag = ksum * Real(4.0 / 6.0);
  return acc * Real(1.0 / 6.0);
}

// (A x)_i and diag(A)_i for a 3D node (i, j, k).
template <typename Real>
__device__ __forceinline__ Real fine_row3(const FineOp<Real>& op, const Real* __restrict__ x,
                                          int i, int j, int k, Real& diag) {
  const int NX = op.NX, NXY = op.NX * op.NY;
  const int idx = i + NX * j + NXY * k;
  if (!CK(idx, op.n)) return Real(0);
  if (op.fixed[idx]) {
    diag = Real(1);
    return op.ksub ? Real(0) : x[idx];
  }
  const bool xm = i > 0, xp = i < op.ex, ym = j > 0, yp = j < op.ey, zm = k > 0, zp = k < op.ez;
  const int EX = op.ex, EXY = op.ex * op.ey;
  const int e000 = (i - 1) + EX * (j - 1) + EXY * (k - 1);
  // kz y x ; index 0 = element on the minus side, 1 = plus side
  const Real k000 = ld_k(op, e000, xm && ym && zm);
  const Real k001 = ld_k(op, e000 + 1, xp && ym && zm);
  const Real k010 = ld_k(op, e000 + EX, xm && yp && zm);
  const Real k011 = ld_k(op, e000 + EX + 1, xp && yp && zm);
  const Real k100 = ld_k(op, e000 + EXY, xm && ym && zp);
  const Real k101 = ld_k(op, e000 + EXY + 1, xp && ym && zp);
  const Real k110 = ld_k(op, e000 + EXY + EX, xm && yp && zp);
  const Real k111 = ld_k(op, e000 + EXY + EX + 1, xp && yp && zp);
  const Real ksum = ((k000 + k001) + (k010 + k011)) + ((k100 + k101) + (k110 + k111));
  const Real* xr = x;
  const uint8_t* fx = op.fixed;
  Real acc = Real(4) * ksum * xr[idx];
  // face diagonals in the xy plane (dz = 0): shared by the two z-layers
  acc -= (k000 + k100) * ld_x(xr, fx, idx - 1 - NX, xm && ym, op.n);
  acc -= (k001 + k101) * ld_x(xr, fx, idx + 1 - NX, xp && ym, op.n);
  acc -= (k010 + k110) * ld_x(xr, fx, idx - 1 + NX, xm && yp, op.n);
  acc -= (k011 + k111) * ld_x(xr, fx, idx + 1 + NX, xp && yp, op.n);
  // xz plane (dy = 0)
  acc -= (k000 + k010) * ld_x(xr, fx, idx - 1 - NXY, xm && zm, op.n);
  acc -= (k001 + k011) * ld_x(xr, fx, idx + 1 - NXY, xp && zm, op.n);
  acc -= (k100 + k110) * ld_x(xr, fx, idx - 1 + NXY, xm && zp, op.n);
  acc -= (k101 + k111) * ld_x(xr, fx, idx + 1 + NXY, xp && zp, op.n);
  // yz plane (dx = 0)
  acc -= (k000 + k001) * ld_x(xr, fx, idx - NX - NXY, ym && zm, op.n);
  acc -= (k010 + k011) * ld_x(xr, fx, idx + NX - NXY, yp && zm, op.n);
  acc -= (k100 + k101) * ld_x(xr, fx, idx - NX + NXY, ym && zp, op.n);
  acc -= (k110 + k111) * ld_x(xr, fx, idx + NX + NXY, yp && zp, op.n);
  // body diagonals: one element each
  acc -= k000 * ld_x(xr, fx, idx - 1 - NX - NXY, xm && ym && zm, op.n);
  acc -= k001 * ld_x(xr, fx, idx + 1 - NX - NXY, xp && ym && zm, op.n);
  acc -= k010 * ld_x(xr, fx, idx - 1 + NX - NXY, xm && yp && zm, op.n);
  acc -= k011 * ld_x(xr, fx, idx + 1 + NX - NXY, xp && yp && zm, op.n);
  acc -= k100 * ld_x(xr, fx, idx - 1 - NX + NXY, xm && ym && zp, op.n);
  acc -= k101 * ld_x(xr, fx, idx + 1 - NX + NXY, xp && ym && zp, op.n);
  acc -= k110 * ld_x(xr, fx, idx - 1 + NX + NXY, xm && yp && zp, op.n);
  acc -= k111 * ld_x(xr, fx, idx + 1 + NX + NXY, xp && yp && zp, op.n);
  diag = ksum * Real(4.0 / 12.0);
  return acc * Real(1.0 / 12.0);
}

// Assembled (Galerkin) coarse operator: S = 3^d coefficients per node,
// s = (dx+1) + 3(dy+1) [+ 9(dz+1)], of which the operator's symmetry
// (A = P^T A_f P) leaves the upper half to store: slots s >= SH (the centre
// SH = S/2 and the neighbours after it in grid order) as st[(s-SH)*n + i];
// a lower slot's coefficient is the neighbour's mirror one, st[(SH-s)*n + j]
// with j = i + offset(s).  Half the bytes per pass and per build.
template <typename Real>
struct StencilOp {
  const Real* st;
  const Real* dinv;
  int NX, NY, NZ;
  int n;
  FastDiv fNX, fNXY;
};

// stored slots per node (upper half with the centre)
constexpr int stencil_slots(int dim) { return dim == 2 ? 5 : 14; }

// Coefficient of full slot s in row idx; nb is the neighbour's index and
// in_grid whether it lies in the grid (the assembled coefficient of a
// neighbour outside is zero; a lower slot reads the neighbour's storage, so
// it needs the test, an upper one holds the zero itself).
template <int DIM, typename Real>
__device__ __forceinline__ Real st_coef(const StencilOp<Real>& op, int s, int idx, int nb,
                                        bool in_grid) {
  constexpr int SH = DIM == 2 ? 4 : 13;
  if (s >= SH) return op.st[(s - SH) * op.n + idx];
  return in_grid ? op.st[(SH - s) * op.n + nb] : Real(0);
}

// A row in two halves: the coefficients (hierarchy data, so a kernel may
// gather them before it waits on its predecessor) and the product with x in
// slot order s = (dx+1) + 3 (dy+1) [+ 9 (dz+1)].  Clamped coordinates: the
// coefficient of a neighbour outside the grid is zero, so the clamped
// operand value it meets does not matter.
template <int DIM>
__host__ __device__ constexpr int stencil_size() { return DIM == 2 ? 9 : 27; }

template <int DIM, typename Real>
__device__ __forceinline__ void stencil_coefs(const StencilOp<Real>& op, int i, int j, int k,
                                              Real (&sv)[stencil_size<DIM>()]) {
  const int NX = op.NX, NXY = op.NX * op.NY;
  const int idx = i + NX * j + (DIM == 3 ? NXY * k : 0);
#pragma unroll
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz) {
    const int kk = DIM == 3 ? min(max(k + dz, 0), op.NZ - 1) : 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int jj = min(max(j + dy, 0), op.NY - 1);
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int ii = min(max(i + dx, 0), op.NX - 1);
        const int s = (dx + 1) + 3 * (dy + 1) + (DIM == 3 ? 9 * (dz + 1) : 0);
        const int nb = ii + NX * jj + (DIM == 3 ? NXY * kk : 0);
        const bool ok = CK(nb, op.n) && CK(idx, op.n);
        const bool in = ii == i + dx && jj == j + dy && (DIM == 2 || kk == k + dz);
        sv[s] = ok ? st_coef<DIM>(op, s, idx, nb, in) : Real(0);
      }
    }
  }
}

template <int DIM, typename Real, bool CG = false>
__device__ __forceinline__ Real stencil_apply(const StencilOp<Real>& op, const Real* __restrict__ x,
                                              int i, int j, int k,
                                              const Real (&sv)[stencil_size<DIM>()]) {
  const int NX = op.NX, NXY = op.NX * op.NY;
  const int idx = i + NX * j + (DIM == 3 ? NXY * k : 0);
  constexpr int S = stencil_size<DIM>();
  Real xv[S];
#pragma unroll
  for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz) {
    const int kk = DIM == 3 ? min(max(k + dz, 0), op.NZ - 1) : 0;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int jj = min(max(j + dy, 0), op.NY - 1);
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int ii = min(max(i + dx, 0), op.NX - 1);
        const int s = (dx + 1) + 3 * (dy + 1) + (DIM == 3 ? 9 * (dz + 1) : 0);
        const int nb = ii + NX * jj + (DIM == 3 ? NXY * kk : 0);
        const bool ok = CK(nb, op.n) && CK(idx, op.n);
        xv[s] = ok ? (CG ? __ldcg(x + nb) : x[nb]) : Real(0);
      }
    }
  }
  Real acc = Real(0);
#pragma unroll
  for (int s = 0; s < S; ++s) acc += sv[s] * xv[s];
  return acc;
}

// The whole row: coefficients and operand values loaded before the first
// product, so a row costs one memory round trip.
template <typename Real, bool CG = false>
__device__ __forceinline__ Real stencil_row2(const StencilOp<Real>& op, const Real* __restrict__ x,
                                             int i, int j) {
  Real sv[9];
  stencil_coefs<2>(op, i, j, 0, sv);
  return stencil_apply<2, Real, CG>(op, x, i, j, 0, sv);
}

template <typename Real, bool CG = false>
__device__ __forceinline__ Real stencil_row3(const StencilOp<Real>& op, const Real* __restrict__ x,
                                             int i, int j, int k) {
  Real sv[27];
  stencil_coefs<3>(op, i, j, k, sv);
  return stencil_apply<3, Real, CG>(op, x, i, j, k, sv);
}

// Coordinates of flat index idx on a row-major (x fastest) box whose rows
// and planes have the sizes behind fr (row) and fp (plane).
__device__ __forceinline__ void coords(int idx, const FastDiv& fr, const FastDiv& fp, int& i, int& j,
                                       int& k) {
  k = (int)fp.div((uint32_t)idx);
  const int rem = idx - k * (int)fp.d;
  j = (int)fr.div((uint32_t)rem);
  i = rem - j * (int)fr.d;
}

// ------------------------------------------------------- host interfaces
// hierarchy.cu
void alloc_hierarchy(Ctx& c);
void free_hierarchy(Ctx& c);
void build_hierarchy(Ctx& c);      // K0 <- K, all levels, coarsest factor
// vcycle.cu
template <typename Real>
void vcycle(Ctx& c, const Real* b, Real* x, bool zero_guess);
// fine3d.cu: tiled finest-level 3D passes (mode 0 pre, 1 post, 2 residual, 3 sweep)
void fine3d(Ctx& c, int mode, const float* ke, const float* b, const float* dinv, const float* x,
            const float* xc, float* out0, float* out1, const float2* rdot = nullptr,
            double* dout = nullptr);
// FP32 CG direction update and product: p = z + beta p_old (beta = *rz_new /
// *rz_old, 0 while *first is nonzero), y = A p with the current k_e, p . y
// into *dot; odd *parity swaps p_old and p; rz_set receives *rz_new
void fine3d_dir(Ctx& c, const float* z, const float* p_old, float* p, const double* rz_new,
                const double* rz_old, const double* first, const double* parity, float* y,
                double* dot, double* rz_set);
// zero-guess FP32 V-cycle x = M b that also leaves r . x in *dout (r in
// double-float pairs, or r = b when r is null; 3D tiled path)
// vcycle_dot applies: one pre- and one post-sweep, two levels or more, and
// (3D) the tiled finest kernels
inline bool vcycle_dot_ok(const Ctx& c) {
  return c.p.nu_pre == 1 && c.p.nu_post == 1 && c.nl >= 2 && !c.untiled;
}
void vcycle_dot(Ctx& c, const float* b, float* x, const float2* r, double* dout);
// launch shapes of the tiled kernels (occupancy query; call outside stream capture)
void fine3d_prepare(Ctx& c);
// vcycle.cu: can the bottom levels run as one thread-block cluster launch
void bottom_prepare(Ctx& c);
// df3d.cu: tiled df64 finest-level operator (3D)
void df3d_prepare(Ctx& c);
// kd_df from ke_df (after every change of the design)
void df3d_node_diag(Ctx& c);
void df3d_apply(Ctx& c, const double* x, double* y, double* dot);
// parity (device scalar, may be null): odd swaps the roles of p_old and p;
// rz_set (may be null) receives *rz_new after the launch has used it
void df3d_dir(Ctx& c, const float* z, const float2* p_old, float2* p, const double* rz_new,
              const double* rz_old, bool first, float2* y, double* dot,
              const double* parity = nullptr, double* rz_set = nullptr);
void df3d_resid(Ctx& c, const float2* q, const float2* x, float2* r, float* r32, double* rr);
void apply_fine64(Ctx& c, const double* ke, const double* x, double* y, double* dot_out);
void apply_fine32(Ctx& c, const float* ke, const float* x, float* y);
void apply_dK64(Ctx& c, const double* x, double* y);
void apply_dK32(Ctx& c, const float* x, float* y);
void convert_d2f(Ctx& c, const double* a, float* b, int64_t n);
void convert_f2d(Ctx& c, const float* a, double* b, int64_t n);
// cg_df.cu (mixed precision: df64 outer CG)
int solve_mgcg_df(Ctx& c, double* T, int* iters, double* relres);
void apply_df64(Ctx& c, const double* x, double* y);
void ke_to_df(Ctx& c);
void q_to_df(Ctx& c);
// solvers.cu
int solve_mgcg(Ctx& c, double* T, int* iters, double* relres);
void solve_mgar(Ctx& c, const double* T_prev, double* T, double* res, int* accepted);
void precondition(Ctx& c, const double* r, double* z);
// reductions
void dot(Ctx& c, const double* a, const double* b, int64_t n, double* out_dev);
void fetch_scalars(Ctx& c, int first, int count);
// design.cu
void setup_filter(Ctx& c);
// continuous filter (Eq. 22-23): radius of design cycle k, and new tables
// (offsets, weights, 1/Hs, dv and its copies) for radius r, stream-ordered
double filter_radius(const Ctx& c, int k);
void set_filter_radius(Ctx& c, double r);
void filter(Ctx& c, const double* in, double* out, bool transpose);
void set_density(Ctx& c, const double* rho, bool physical);
// T_df: the same temperatures as double-float pairs when the caller has them
// (mixed path), else null.  dc_df (mixed path only): dc as double-float pairs
// instead of FP64 (dc may then be null)
void sensitivity(Ctx& c, const double* T, double* dc, double* dv, double* compliance,
                 const float2* T_df = nullptr, float2* dc_df = nullptr);
void postprocess(Ctx& c, const double* rho, const double* T, double volfrac, double* rho_out,
                 double* level_out, double* volume_out);
// dc_df: dc as double-float pairs (then dc is not read)
void oc_update(Ctx& c, double* rho, const double* dc, double volfrac, double move, double* lambda,
               double* change, const float2* dc_df = nullptr);
// oc_update in two halves: the fast solve and its application queued without
// a host read, then the read of its outcome (and the plain bisection if it
// failed), so many handles' updates can be queued before any is read
void oc_issue(Ctx& c, double* rho, const double* dc, double volfrac, double move,
              const float2* dc_df = nullptr);
// The internal dc buffer as double-float pairs (the same bytes as its ne
// doubles): the mixed design cycle keeps dc in that form between the
// sensitivities and the OC update
inline float2* dc_pairs(Ctx& c) { return reinterpret_cast<float2*>(c.tmp_dc); }
void oc_complete(Ctx& c, double* rho, double volfrac, double* lambda, double* change);
// oc_complete without its read: the host mirror already holds S_OC_LAM,
// S_OC_CHANGE and S_OC_FAIL of the update
void oc_finish(Ctx& c, double* rho, double volfrac, double* lambda, double* change);

}  // namespace mgar

namespace mgar {
// Launch with the programmatic-dependent-launch attribute (see pdl_wait).
template <typename... KArgs, typename... Args>
inline void launch_pdl(cudaStream_t s, bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  MGAR_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

// Run `issue` (a fixed sequence of launches on c.stream) through a cached
// CUDA graph keyed by (kind, a, b); falls back to direct launches while a
// kernel class inside it is being timed.
// Orders the handle's stream after a pending coarsest factorisation (no-op
// otherwise, and never inside a stream capture).
inline void join_coarse(Ctx& c) {
  if (!c.coarse_pending || c.stream == c.cap_stream || c.stream == c.cap_stream2) return;
  MGAR_CUDA(cudaStreamWaitEvent(c.stream, c.ev_join, 0));
  c.coarse_pending = false;
}

template <class F>
void run_graph(Ctx& c, int kind, const void* a, const void* b, bool profiled_inside, F&& issue) {
  join_coarse(c);
  if (!c.use_graphs || profiled_inside) {
    issue();
    return;
  }
  Ctx::GraphEntry* hit = nullptr;
  for (auto& g : c.graphs)
    if (g.exec && g.kind == kind && g.a == a && g.b == b) hit = &g;
  if (!hit) {
    Ctx::GraphEntry* slot = nullptr;
    for (auto& g : c.graphs)
      if (!g.exec) {
        slot = &g;
        break;
      }
    if (!slot) {  // cache full: run directly
      issue();
      return;
    }
    const int64_t before = launches_so_far();
    MGAR_CUDA(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaStream_t saved = c.stream;
    c.stream = c.cap_stream;
    try {
      issue();
    } catch (...) {
      c.stream = saved;
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(c.cap_stream, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    c.stream = saved;
    cudaGraph_t g = nullptr;
    MGAR_CUDA(cudaStreamEndCapture(c.cap_stream, &g));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    MGAR_CUDA(e);
    slot->kind = kind;
    slot->a = a;
    slot->b = b;
    slot->exec = exec;
    slot->kernels = launches_so_far() - before;
    count_launches(-slot->kernels);  // captured, not executed
    hit = slot;
  }
  MGAR_CUDA(cudaGraphLaunch(hit->exec, c.stream));
  count_launches(hit->kernels);
  static const char* kGraphSites[] = {"graph:0", "graph:1 precondition", "graph:2 mgar-vcycle64-zero",
                                      "graph:3 mgar-vcycle64-guess", "graph:4 mgar-vcycle32-zero",
                                      "graph:5 mgar-vcycle32-guess", "graph:6 precondition-df",
                                      "graph:7", "graph:8 precondition-rz", "graph:9 precondition-rz",
                                      "graph:10 precondition-rz32"};
  prof_mark(kGraphSites[kind >= 0 && kind < 11 ? kind : 0]);
}
}  // namespace mgar
