// boltz_relax_noalloc: forward-Euler relaxation that allocates no memory.
//
// boltz_relax keeps its scratch (one float64 row of moment targets per cell) in device
// memory that it allocates on first use and grows with cudaMalloc / cudaFree.  Some
// callers cannot allow that: a framework whose caching allocator already holds the
// device memory (a raw cudaMalloc then fails or fragments its pool), a time-stepping
// loop that must not stall on the device-wide synchronisation that cudaFree implies, or
// an embedding that forbids the library from owning device memory at all.  This entry
// point keeps the targets in a fixed array in the library's own device image instead:
// it exists from module load until process exit on every device that loads the library
// (kNoAllocMaxCells * 5 doubles = 2.5 MiB per device) and is never freed or resized.
//
// The caller still owns f.  Every call on a device shares the one array, and the array
// keeps whatever the last call wrote: each call first overwrites the targets of every
// cell it will use, so nothing needs to start at zero, but two calls whose work overlaps
// on the GPU (different streams, or different host threads) race on the array and give
// wrong results.  Serialise them (one stream, or events).
//
// Set-up: the first call on each device looks up the device address of the array with
// cudaGetSymbolAddress (the array's name in host code is only a host-side handle, not a
// device address) and caches it per device.  Make that first call before any stream
// capture begins.
#include <mutex>

#include "internal.h"

namespace {

constexpr int64_t kNoAllocMaxCells = 65536;
constexpr int kMaxDevices = 64;

// Moment targets Phi f (five float64 per cell) of the cells of the current call.
static __device__ __align__(256) double g_noalloc_targets[kNoAllocMaxCells * 5];

std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

boltz_status noalloc_targets(int device, double** out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_targets);
    if (e != cudaSuccess) {
      boltz::set_error(std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
      return BOLTZ_ECUDA;
    }
    g_noalloc_ptr[device] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[device];
  return BOLTZ_OK;
}

}  // namespace

extern "C" boltz_status boltz_relax_noalloc(const boltz_batch* b, void* f, double dt, int steps, void* stream) {
  if (!b || !b->grid) {
    boltz::set_error("null batch or grid");
    return BOLTZ_EINVAL;
  }
  if (b->n_cells < 0 || (b->f_is_fp64 != 0 && b->f_is_fp64 != 1)) {
    boltz::set_error("bad batch");
    return BOLTZ_EINVAL;
  }
  if (b->n_cells > kNoAllocMaxCells) {
    boltz::set_error("boltz_relax_noalloc: n_cells exceeds the static scratch limit of 65536 cells per call");
    return BOLTZ_EINVAL;
  }
  if (!boltz::collide_supported_grid(b->grid, b->prec)) {
    boltz::set_error("this precision has no kernel for this N in this library");
    return BOLTZ_EUNSUPPORTED;
  }
  if (!(dt > 0) || !(dt < 1e300)) {
    boltz::set_error("dt must be positive and finite");
    return BOLTZ_EINVAL;
  }
  if (steps < 0) {
    boltz::set_error("steps must be >= 0");
    return BOLTZ_EINVAL;
  }
  if (b->n_cells == 0 || steps == 0) return BOLTZ_OK;
  if (!f) {
    boltz::set_error("null f");
    return BOLTZ_EINVAL;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    boltz::set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return BOLTZ_ECUDA;
  }
  if (dev != b->grid->device) {
    boltz::set_error("the grid belongs to another device");
    return BOLTZ_EINVAL;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    boltz::set_error("device ordinal out of range");
    return BOLTZ_EINVAL;
  }
  double* targets = nullptr;
  boltz_status st = noalloc_targets(dev, &targets);
  if (st != BOLTZ_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  st = boltz::launch_phisums(b->grid, b->n_cells, b->f_is_fp64, f, targets, 1.0, s);
  if (st != BOLTZ_OK) return st;
  for (int it = 0; it < steps; ++it) {
    // groups = 1: a split launch would need the grid's scratch buffer
    st = boltz::launch_collide(b->grid, b->n_cells, b->prec, b->f_is_fp64, f, nullptr, f, 0.0, 1.0, dt, targets, 0,
                               1, s, nullptr, 0, 1);
    if (st != BOLTZ_OK) return st;
  }
  return BOLTZ_OK;
}
