// Kernel unit: tensor-core DFT collision kernels (N = 16, 32) and the N = 48, 64 kernels.
#include "collide_kernels.cuh"

namespace boltz {

BOLTZ_UNIT_SERVICES(tc)

// Tensor-core transforms (BOLTZ_TF32_DFT, BOLTZ_3XTF32_DFT): 128 pencils per CTA, i.e.
// N = 32 with clusters of 8 and N = 16 with clusters of 2.
template <typename TIO, int TC>
static boltz_status dispatch_tc(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st) {
  if (g->N == 32) return launch_impl<float, TIO, 32, 8, TC>(a, n_cells, st);
  if (g->N == 16) return launch_impl<float, TIO, 16, 2, TC>(a, n_cells, st);
  set_error("no tensor-core kernel for this N");
  return BOLTZ_EUNSUPPORTED;
}

boltz_status dispatch_3d_tc(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st, int prec,
                            int f_is_fp64) {
  if (prec == BOLTZ_TF32_DFT)
    return f_is_fp64 ? dispatch_tc<double, kTcTF32>(g, a, n_cells, st) : dispatch_tc<float, kTcTF32>(g, a, n_cells, st);
  if (prec == BOLTZ_3XBF16_DFT)
    return f_is_fp64 ? dispatch_tc<double, kTc3xBF16>(g, a, n_cells, st)
                     : dispatch_tc<float, kTc3xBF16>(g, a, n_cells, st);
  return f_is_fp64 ? dispatch_tc<double, kTc3xTF32>(g, a, n_cells, st) : dispatch_tc<float, kTc3xTF32>(g, a, n_cells, st);
}

// N = 48, 64 (float32 only)
boltz_status dispatch_3d_large(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st,
                               int cluster, int f_is_fp64) {
  const int C = cluster > 0 ? cluster : default_cluster(g->N, BOLTZ_FP32_FFT);
  if (g->N == 48 && C == 8)
    return f_is_fp64 ? launch_large_impl<double, 48, 8>(a, n_cells, st) : launch_large_impl<float, 48, 8>(a, n_cells, st);
  if (g->N == 48 && C == 12)
    return f_is_fp64 ? launch_large_impl<double, 48, 12>(a, n_cells, st)
                     : launch_large_impl<float, 48, 12>(a, n_cells, st);
  if (g->N == 64 && C == 16)
    return f_is_fp64 ? launch_large_impl<double, 64, 16>(a, n_cells, st)
                     : launch_large_impl<float, 64, 16>(a, n_cells, st);
  set_error("no large-N kernel for this (N, cluster size)");
  return BOLTZ_EUNSUPPORTED;
}

}  // namespace boltz
