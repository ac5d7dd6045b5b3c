// Kernel unit: float32 register-FFT collision kernels for N = 8, 16, 24, 32 (all cluster sizes,
// with and without term groups; at 32^3 also one CTA per cell, collide_solo.cuh).
#include "collide_kernels.cuh"
#include "collide_solo.cuh"

namespace boltz {

BOLTZ_UNIT_SERVICES(f32)

template <typename T, typename TIO>
static boltz_status dispatch_n_impl(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st,
                               int cluster) {
  constexpr bool dbl = sizeof(T) == 8;
  int C = cluster > 0 ? cluster : default_cluster_for(g->N, dbl ? BOLTZ_FP64 : BOLTZ_FP32_FFT, a.groups);
  // f stored float64 at 32^3: the one-CTA-per-cell kernel spills at its 128 registers
  // there (float64 loads) and the clusters of 8 measured faster
  if (cluster <= 0 && sizeof(TIO) == 8 && g->N == 32 && C == 1) C = 8;
  if (g->N == 8 && C == 1) return launch_impl<T, TIO, 8, 1>(a, n_cells, st);
  if constexpr (dbl) {
    if (g->N == 16 && C == 2) return launch_impl<T, TIO, 16, 2>(a, n_cells, st);
    if (g->N == 24 && C == 3) return launch_impl<T, TIO, 24, 3>(a, n_cells, st);
    if (g->N == 32 && C == 8) return launch_impl<T, TIO, 32, 8>(a, n_cells, st);
  } else {
    if (g->N == 16 && C == 1) return launch_impl<T, TIO, 16, 1>(a, n_cells, st);
    if (g->N == 16 && C == 2) return launch_impl<T, TIO, 16, 2>(a, n_cells, st);
    if (g->N == 16 && C == 4) return launch_impl<T, TIO, 16, 4>(a, n_cells, st);
    if (g->N == 24 && C == 2) return launch_impl<T, TIO, 24, 2>(a, n_cells, st);
    if (g->N == 24 && C == 3) return launch_impl<T, TIO, 24, 3>(a, n_cells, st);
    if (g->N == 24 && C == 6) return launch_impl<T, TIO, 24, 6>(a, n_cells, st);
    if (g->N == 32 && C == 1) return launch_solo_impl<TIO>(a, n_cells, st);
    if (g->N == 32 && C == 4) return launch_impl<T, TIO, 32, 4>(a, n_cells, st);
    if (g->N == 32 && C == 8) return launch_impl<T, TIO, 32, 8>(a, n_cells, st);
    if (g->N == 32 && C == 16) return launch_impl<T, TIO, 32, 16>(a, n_cells, st);
  }
  set_error("no collision kernel for this (N, precision, cluster size)");
  return BOLTZ_EUNSUPPORTED;
}


boltz_status dispatch_3d_f32(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st,
                             int cluster, int f_is_fp64) {
  return f_is_fp64 ? dispatch_n_impl<float, double>(g, a, n_cells, st, cluster)
                   : dispatch_n_impl<float, float>(g, a, n_cells, st, cluster);
}

}  // namespace boltz
