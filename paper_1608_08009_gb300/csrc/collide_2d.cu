// Kernel unit: two-dimensional (Maxwell-molecule) collision kernels.
#include "collide_kernels.cuh"

namespace boltz {

BOLTZ_UNIT_SERVICES(p2d)

template <typename T, typename TIO>
static boltz_status dispatch2d(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st) {
  switch (g->N) {
    case 8: return launch2d_impl<T, TIO, 8>(a, n_cells, st);
    case 16: return launch2d_impl<T, TIO, 16>(a, n_cells, st);
    case 32: return launch2d_impl<T, TIO, 32>(a, n_cells, st);
    case 64:
      if constexpr (sizeof(T) == 4) return launch2d_impl<T, TIO, 64>(a, n_cells, st);
      break;
    default: break;
  }
  set_error("no 2D collision kernel for this (N, precision)");
  return BOLTZ_EUNSUPPORTED;
}

boltz_status dispatch_2d(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st, int prec,
                         int f_is_fp64) {
  if (prec == BOLTZ_FP64)
    return f_is_fp64 ? dispatch2d<double, double>(g, a, n_cells, st) : dispatch2d<double, float>(g, a, n_cells, st);
  return f_is_fp64 ? dispatch2d<float, double>(g, a, n_cells, st) : dispatch2d<float, float>(g, a, n_cells, st);
}

}  // namespace boltz
