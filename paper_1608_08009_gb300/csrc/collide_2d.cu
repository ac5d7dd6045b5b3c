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

// Self-check of the integer-pipe conversions the 2D kernel uses, against the hardware
// conversion: to_f64 on all 2^32 float bit patterns; from_f64 on 2^32 pseudo-random
// double bit patterns (splitmix64 of the index) and, for every finite float x with a
// finite neighbour y away from zero, on the double halfway between them (a tie) and the
// doubles one unit in the last place either side of it.  NaNs compare by class.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ bool same_f32(double d) {
  const float a = from_f64<float>(d), b = (float)d;
  return (a != a && b != b) || __float_as_uint(a) == __float_as_uint(b);
}
__global__ void conversion_check_kernel(unsigned long long* bad) {
  unsigned long long b0 = 0, b1 = 0;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < (1ull << 32);
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const float x = __uint_as_float((unsigned)i);
    const double a = to_f64(x), h = (double)x;
    b0 += ((a != a && h != h) || __double_as_longlong(a) == __double_as_longlong(h)) ? 0 : 1;
    b1 += same_f32(__longlong_as_double((long long)splitmix64(i))) ? 0 : 1;
    const float y = __uint_as_float((unsigned)i + 1u);
    if (isfinite(x) && isfinite(y)) {
      const double m = 0.5 * ((double)x + (double)y);  // exact: one bit more than a float
      const long long mb = __double_as_longlong(m);
      b1 += (same_f32(m) ? 0 : 1) + (same_f32(__longlong_as_double(mb + 1)) ? 0 : 1) +
            (same_f32(__longlong_as_double(mb - 1)) ? 0 : 1);
    }
  }
  if (b0) atomicAdd(bad, b0);
  if (b1) atomicAdd(bad + 1, b1);
}

boltz_status selftest_conversions(uint64_t* mismatches) {
  unsigned long long* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("conversion check: allocation failed");
    return BOLTZ_ENOMEM;
  }
  unsigned long long h[2] = {0, 0};
  if ((e = cudaMemset(d, 0, sizeof(h))) == cudaSuccess) {
    conversion_check_kernel<<<152 * 8, 256>>>(d);
    if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaDeviceSynchronize()) == cudaSuccess)
      e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  }
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "conversion check");
  mismatches[0] = h[0];
  mismatches[1] = h[1];
  return BOLTZ_OK;
}

boltz_status dispatch_2d(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st, int prec,
                         int f_is_fp64) {
  if (prec == BOLTZ_FP64)
    return f_is_fp64 ? dispatch2d<double, double>(g, a, n_cells, st) : dispatch2d<double, float>(g, a, n_cells, st);
  return f_is_fp64 ? dispatch2d<float, double>(g, a, n_cells, st) : dispatch2d<float, float>(g, a, n_cells, st);
}

}  // namespace boltz
