// Design sensitivities (Eq. 9-11) for callers that cannot allocate device
// memory: code running where cudaMalloc is off limits, for instance inside
// a host framework that owns every device allocation through its own pool,
// or a plug-in that must not grow the process's device footprint after
// start-up.  It needs no handle, so nothing is allocated before or during
// the call: the per-element intermediate lives in a fixed static device array
// (kNoAllocMaxElems doubles, 8 MiB) that every GPU loading this library holds
// until the process exits.
#include "common.cuh"

#include <mutex>

namespace mgar {
namespace {

constexpr int64_t kNoAllocMaxElems = int64_t(1) << 20;

// Shared by every call of mgar_sensitivity_noalloc on a device: calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race on it.  Every entry a call reads is written by that call first, so
// nothing has to be cleared between calls.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxElems];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in, not an address).  The
// cached address belongs to the device's primary context as it was at the
// lookup: after cudaDeviceReset it is stale, so this entry point does not
// support a device reset during the life of the process.
int scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MGAR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return MGAR_ERR_CUDA;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return MGAR_OK;
}

// scratch_e = dc~_e / Hs_e with dc~_e = -p (k0-kmin) rho~_e^(p-1) t_e^T k0 t_e
// (Eq. 10) and Hs_e the sum of the in-domain cone weights of Eq. 8.
template <int DIM>
__global__ void k_sens_scaled(const double* __restrict__ rho, const double* __restrict__ T,
                              double* __restrict__ scratch, int ex, int ey, int ez, double coef,
                              double penal, double r, int reach) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int ne = ex * ey * ez;
  if (e >= ne) return;
  const int i = e % ex, j = (e / ex) % ey, k = e / (ex * ey);
  const int NX = ex + 1, NY = ey + 1;
  constexpr int nen = 1 << DIM;
  double t[nen];
#pragma unroll
  for (int a = 0; a < nen; ++a)
    t[a] = T[(i + (a & 1)) + NX * ((j + ((a >> 1) & 1)) + NY * (k + ((a >> 2) & 1)))];
  double energy = 0.0;  // t^T k0 t = -sum_{a<b} k0_ab (t_a - t_b)^2
#pragma unroll
  for (int a = 0; a < nen; ++a)
#pragma unroll
    for (int b = a + 1; b < nen; ++b) {
      const int bits = __popc(a ^ b);
      const double wgt = DIM == 2 ? (bits == 1 ? 1.0 / 6.0 : 2.0 / 6.0) : (bits >= 2 ? 1.0 / 12.0 : 0.0);
      const double dd = t[a] - t[b];
      energy += wgt * dd * dd;
    }
  double hs = 0.0;
  const int zr = DIM == 3 ? reach : 0;
  for (int dz = -zr; dz <= zr; ++dz)
    for (int dy = -reach; dy <= reach; ++dy)
      for (int dx = -reach; dx <= reach; ++dx) {
        const double w = r - sqrt((double)(dx * dx + dy * dy + dz * dz));
        const bool in = i + dx >= 0 && i + dx < ex && j + dy >= 0 && j + dy < ey && k + dz >= 0 &&
                        k + dz < ez;
        if (w > 0.0 && in) hs += w;
      }
  const double rr = rho[e];
  const double rp = penal == 3.0 ? rr * rr : pow(rr, penal - 1.0);
  scratch[e] = -coef * rp * energy / hs;
}

// dc_j = sum over in-domain e of w_ej scratch_e  (Eq. 9 with Eq. 11)
__global__ void k_sens_gather(const double* __restrict__ scratch, double* __restrict__ dc, int ex,
                              int ey, int ez, double r, int reach, int dim) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int ne = ex * ey * ez;
  if (e >= ne) return;
  const int i = e % ex, j = (e / ex) % ey, k = e / (ex * ey);
  const int zr = dim == 3 ? reach : 0;
  double acc = 0.0;
  for (int dz = -zr; dz <= zr; ++dz)
    for (int dy = -reach; dy <= reach; ++dy)
      for (int dx = -reach; dx <= reach; ++dx) {
        const double w = r - sqrt((double)(dx * dx + dy * dy + dz * dz));
        const bool in = i + dx >= 0 && i + dx < ex && j + dy >= 0 && j + dy < ey && k + dz >= 0 &&
                        k + dz < ez;
        const int nb = in ? (i + dx) + ex * ((j + dy) + ey * (k + dz)) : e;
        if (w > 0.0 && in) acc += w * scratch[nb];
      }
  dc[e] = acc;
}

}  // namespace
}  // namespace mgar

extern "C" int mgar_sensitivity_noalloc(const mgar_params* p, const double* rho_phys,
                                        const double* T, double* dc, void* stream) {
  using namespace mgar;
  if (!p || !rho_phys || !T || !dc) return MGAR_ERR_ARG;
  const int dim = p->nz == 0 ? 2 : 3;
  const int64_t ex = p->nx, ey = p->ny, ez = dim == 3 ? p->nz : 1;
  if (ex < 1 || ey < 1 || ez < 1 || !(p->rmin > 0.0) || p->rmin > 8.0) return MGAR_ERR_ARG;
  // the filter is the fixed-radius one of radius rmin: a continuation
  // schedule (filter_alpha > 0) belongs to a handle's loop and is refused
  if (p->filter_alpha > 0.0) return MGAR_ERR_ARG;
  const int64_t ne = ex * ey * ez;
  if (ne > kNoAllocMaxElems) return MGAR_ERR_TOO_LARGE;  // beyond the static scratch array
  double* scratch = nullptr;
  if (scratch_address(&scratch) != MGAR_OK) return MGAR_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int reach = (int)std::ceil(p->rmin);
  const double coef = p->penal * (p->k0 - p->kmin);
  const int blocks = (int)((ne + kThreads - 1) / kThreads);
  if (dim == 2)
    k_sens_scaled<2><<<blocks, kThreads, 0, s>>>(rho_phys, T, scratch, (int)ex, (int)ey, (int)ez,
                                                 coef, p->penal, p->rmin, reach);
  else
    k_sens_scaled<3><<<blocks, kThreads, 0, s>>>(rho_phys, T, scratch, (int)ex, (int)ey, (int)ez,
                                                 coef, p->penal, p->rmin, reach);
  k_sens_gather<<<blocks, kThreads, 0, s>>>(scratch, dc, (int)ex, (int)ey, (int)ez, p->rmin, reach,
                                            dim);
  if (cudaGetLastError() != cudaSuccess) return MGAR_ERR_CUDA;
  count_launches(2);
  return MGAR_OK;
}
