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
// The launches are those of boltz_relax with rk_order 1 and one term group: the first
// step computes the targets from the f it loads and writes them to the array, the later
// steps read them back.  On a grid with term_groups = 1 (the default) the result is
// therefore bit for bit that of boltz_relax; with term_groups > 1 it differs by the
// rounding of the gain sum, since a split launch would need scratch the grid allocates.
//
// The caller still owns f.  Every call on a device shares the one array, and the array
// keeps whatever the last call wrote: each call's first launch overwrites the targets of
// every cell it will use, so nothing needs to start at zero, but two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on the array
// and give wrong results.  Serialise them (one stream, or events).
//
// Set-up: the array's name in host code is only a host-side handle, not a device
// address.  Each call looks the device address up with cudaGetSymbolAddress while the
// call's stream is not capturing (so a device reset, which reloads the module, cannot
// leave a stale address behind) and caches it per device; a call made while its stream
// is capturing uses the cached address, so the first call on a device must come before
// any stream capture.
#include <mutex>

#include "internal.h"

namespace {

constexpr int64_t kNoAllocMaxCells = 65536;
constexpr int kMaxDevices = 64;

// Moment targets Phi f (five float64 per cell) of the cells of the current call.
static __device__ __align__(256) double g_noalloc_targets[kNoAllocMaxCells * 5];

std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

boltz_status noalloc_targets(int device, cudaStream_t stream, double** out) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(stream, &cap);
  if (e != cudaSuccess) {
    boltz::set_error(std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
    return BOLTZ_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_targets);
    if (e != cudaSuccess) {
      boltz::set_error(std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
      return BOLTZ_ECUDA;
    }
    g_noalloc_ptr[device] = static_cast<double*>(p);
  } else if (!g_noalloc_ptr[device]) {
    boltz::set_error("boltz_relax_noalloc: the first call on a device must not be made during stream capture");
    return BOLTZ_EINVAL;
  }
  *out = g_noalloc_ptr[device];
  return BOLTZ_OK;
}

}  // namespace

extern "C" boltz_status boltz_relax_noalloc(const boltz_batch* b, void* f, double dt, int steps, void* stream) {
  boltz_status st = boltz::check_batch(b);
  if (st != BOLTZ_OK) return st;
  if (b->n_cells > kNoAllocMaxCells) {
    boltz::set_error("boltz_relax_noalloc: n_cells exceeds the static scratch limit of 65536 cells per call");
    return BOLTZ_EINVAL;
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
  if ((st = boltz::check_device(b->grid)) != BOLTZ_OK) return st;
  const int dev = b->grid->device;
  if (dev < 0 || dev >= kMaxDevices) {
    boltz::set_error("device ordinal out of range");
    return BOLTZ_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  double* targets = nullptr;
  if ((st = noalloc_targets(dev, s, &targets)) != BOLTZ_OK) return st;
  for (int it = 0; it < steps; ++it) {
    // the first launch takes the targets from f and stores them; groups = 1: a split
    // launch would need the grid's scratch buffer
    st = boltz::launch_collide(b->grid, b->n_cells, b->prec, b->f_is_fp64, f, nullptr, f, 0.0, 1.0, dt, targets,
                               it == 0 ? 1 : 0, 1, s, nullptr, 0, 1);
    if (st != BOLTZ_OK) return st;
  }
  return BOLTZ_OK;
}
