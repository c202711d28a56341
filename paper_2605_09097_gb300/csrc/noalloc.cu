// Energy-change reduction for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc or any allocating routine: code that
// runs inside a memory-capped sandbox or a host application whose allocator
// owns all device memory, and code that must not allocate while it holds
// a latency budget.  This file gives them osmpm_energy_change_noalloc: the
// line-search energy change E_h(u + alpha s) - E_h(u) of the library's
// Newton step, computed from caller-owned device arrays, with the
// reduction's scratch (block partials, counter and result) in a fixed
// file-scope device array instead of a buffer from an allocator.
//
// The array is allocated once per GPU when the library's module is loaded
// and stays allocated until the process exits.  Host code cannot use the
// array's name as a device address: the first call on each device looks
// the address up with cudaGetSymbolAddress while that device is current
// and reuses it afterwards.  All calls share the array, which keeps the
// last call's contents: every call clears the counter and the error word
// that must start at zero, and calls that overlap on the GPU (on different
// streams, or from several threads) race on it.  The cached address assumes
// the device's primary context lives as long as the process: after a
// cudaDeviceReset the address would be stale.
//
// The call waits for its stream before it returns, so that it can report a
// particle outside the grid box (OSMPM_E_OUT_OF_GRID) instead of a silently
// wrong sum.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/osmpm.h"
#include "osmpm_internal.h"

using namespace osmpm;

namespace {

constexpr int kNoallocHeader = 32;        // doubles reserved for the loop scalars
constexpr int kNoallocSlots = 4096;       // block partials: one per 256 work items
constexpr int kNoallocDevices = 64;

static_assert(sizeof(DevScalars) <= kNoallocHeader * sizeof(double), "scalar header too small");

// 4128 doubles (33 KB) per GPU that loads the library.
static __device__ __align__(256) double g_noalloc_scratch[kNoallocHeader + kNoallocSlots];

std::mutex g_setup_mutex;
double* g_scratch_addr[kNoallocDevices] = {nullptr};

osmpm_status scratch_for_current_device(double** out, const char** why) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoallocDevices) {
    *why = "no current CUDA device (or its ordinal is above 63)";
    return OSMPM_E_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      *why = cudaGetErrorString(e);
      return OSMPM_E_CUDA;
    }
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return OSMPM_OK;
}

}  // namespace

extern "C" osmpm_status osmpm_energy_change_noalloc(const osmpm_noalloc_grid* grid,
                                                    const osmpm_noalloc_particles* parts,
                                                    double dt, double alpha, double* dE,
                                                    void* cuda_stream) {
  if (!grid || !parts || !dE) return set_error(OSMPM_E_INVALID, "null argument");
  const int D = grid->dim;
  if (D != 2 && D != 3) return set_error(OSMPM_E_INVALID, "dim must be 2 or 3");
  if (!(grid->dx > 0.0) || !std::isfinite(grid->dx) || !(dt > 0.0) || !std::isfinite(dt) ||
      !std::isfinite(alpha) || !(grid->mass_eps >= 0.0))
    return set_error(OSMPM_E_INVALID, "dx, dt must be > 0; alpha finite; mass_eps >= 0");
  GridGeo g{};
  int64_t nn = 1;
  for (int a = 0; a < 3; ++a) {
    if (a < D && (grid->res[a] < 4 || grid->res[a] > (1 << 20)))
      return set_error(OSMPM_E_INVALID, "res[%d] out of range [4, 2^20]", a);
    g.o[a] = a < D ? grid->origin[a] : 0.0;
    g.res[a] = a < D ? grid->res[a] : 1;
    if (a < D) nn *= grid->res[a];
  }
  g.dx = grid->dx;
  g.inv_dx = 1.0 / grid->dx;
  g.nn = nn;
  g.mass_eps = grid->mass_eps;
  if (parts->n < 0) return set_error(OSMPM_E_INVALID, "negative particle count");
  const int64_t work = parts->n > nn * D ? parts->n : nn * D;
  const int64_t blocks = (work + 255) / 256;
  if (blocks > kNoallocSlots)
    return set_error(OSMPM_E_INVALID,
                           "problem too large for the fixed scratch: max(n_particles, n_nodes*dim) "
                           "= %lld exceeds %d", (long long)work, 256 * kNoallocSlots);
  if (!grid->m || !grid->vn || !grid->u || !grid->s ||
      (parts->n > 0 && (!parts->x || !parts->F || !parts->vol0 || !parts->mu || !parts->lam)))
    return set_error(OSMPM_E_INVALID, "null array");
  double* scratch = nullptr;
  const char* why = "";
  if (scratch_for_current_device(&scratch, &why) != OSMPM_OK)
    return set_error(OSMPM_E_CUDA, "scratch address lookup failed: %s", why);
  DevScalars* S = (DevScalars*)scratch;
  double* partials = scratch + kNoallocHeader;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the grid reduction's arrival counter and the error word start at zero
  cudaError_t e = cudaMemsetAsync(&S->counter, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&S->err, 0, sizeof(int), s);
  if (e != cudaSuccess) return set_error(OSMPM_E_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  PartPtrs P{};
  P.n = parts->n;
  P.x = const_cast<double*>(parts->x);
  P.F = const_cast<double*>(parts->F);
  P.vol0 = const_cast<double*>(parts->vol0);
  P.mu = const_cast<double*>(parts->mu);
  P.lam = const_cast<double*>(parts->lam);
  const double gravity[3] = {grid->gravity[0], grid->gravity[1], grid->gravity[2]};
  if (D == 2)
    Kernels<2, double>::energy_change_blocks(P, g, grid->m, grid->vn, grid->u, grid->s, gravity, dt, alpha,
                                     S, partials, (int)blocks, s);
  else
    Kernels<3, double>::energy_change_blocks(P, g, grid->m, grid->vn, grid->u, grid->s, gravity, dt, alpha,
                                     S, partials, (int)blocks, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(OSMPM_E_CUDA, "launch: %s", cudaGetErrorString(e));
  e = cudaMemcpyAsync(dE, &S->dE, sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return set_error(OSMPM_E_CUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(e));
  // the kernel flags a particle whose support leaves the grid box (its sum
  // is then NaN); reading the flag makes the call wait for the stream
  int err = 0;
  e = cudaMemcpyAsync(&err, &S->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return set_error(OSMPM_E_CUDA, "error word read-back: %s", cudaGetErrorString(e));
  if (err & kErrOutOfGrid)
    return set_error(OSMPM_E_OUT_OF_GRID, "a particle's B-spline support leaves the grid box");
  return OSMPM_OK;
}
