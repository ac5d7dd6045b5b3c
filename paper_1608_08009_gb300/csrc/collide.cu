// Fused per-cell kernels of the fast spectral collision operator (sm_103a).
//
// Paper: arxiv 1608.08009.  Per cell (Sec. 4.2): one forward 3D transform of f
// (Eq. FC), then for every separated quadrature term j the coefficients
// (alpha_j + i alpha'_j) fhat and one inverse 3D transform (Eq. FU) whose real and
// imaginary parts are the two factors of the gain term (Sec. 3.3, decoupling formula),
// accumulated as Q+ += w_j Re Im; then the loss term L = inverse(D fhat), Q = Q+ - f L,
// the conservation projection (Sec. 3.2, Eq. minim1) and optionally the collision step
// f <- f + dt Q (Eq. f_coll), all in one launch: f is read once and Q (or the new f)
// written once per cell.
//
// Work decomposition.  A cell is owned by a thread-block cluster of C CTAs.
//  * Spectrum: CTA c keeps fhat(kx, ky, kz) for the ky-slab [c N/C, (c+1) N/C), all kx
//    and kz: in registers (float32, thread (ky, kz) holds its kx pencil) or shared memory.
//  * Physical space: CTA q owns the x-slab [q N/C, (q+1) N/C); the gain accumulator of
//    its points lives in registers (thread (x, z) holds the N values along y).
//  * One inverse 3D transform = pass along kx (pencils of the CTA's ky-slab, in
//    registers) whose N outputs are scattered by x into the owners' shared memory through
//    distributed shared memory, a cluster barrier, then the passes along kz and ky inside
//    each x-plane of the owner.
//  * Every 1D pass is a fully unrolled radix-4/2 FFT of one pencil held by one thread.
// Twiddles, kernel tables and weights are float32 for the BOLTZ_FP32_FFT path and
// float64 for BOLTZ_FP64.  Moments, projection and the update are float64 in both.
//
// This unit holds the host side: table upload, the launch of the collision kernels
// (dispatched to the kernel units), the moment kernels and the status word.
#include <algorithm>
#include <climits>
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace boltz {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// U[c] = scale * (sum f, sum v_x f, sum v_y f, 0, sum |v|^2/2 f) of 2D cells; one warp per cell.
template <typename TIO>
__global__ void __launch_bounds__(256) phisums2d_kernel(const TIO* f, double* U, int N, double L, double dv,
                                                        double scale, long long n_cells) {
  const long long cell = (long long)blockIdx.x * 8 + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (cell >= n_cells) return;
  const TIO* fc = f + cell * (long long)N * N;
  double m[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int x = lane; x < N; x += 32) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int y = 0; y < N; ++y) {
      const double fv = (double)fc[x * N + y];
      s0 += fv;
      s1 += (double)y * fv;
      s2 += (double)(y * y) * fv;
    }
    const double vx = -L + x * dv;
    m[0] += s0;
    m[1] += vx * s0;
    m[2] += -L * s0 + dv * s1;
    m[4] += 0.5 * ((vx * vx + L * L) * s0 - 2.0 * L * dv * s1 + dv * dv * s2);
  }
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const double v = warp_sum_d(m[r]);
    if (lane == 0) U[cell * 5 + r] = scale * v;
  }
}

// Plain sums Phi f per cell, scaled: U[c][r] = scale * sum_v phi_r(v) f(v).  One thread
// per (x, y) row: sum f, sum z f and sum z^2 f along the row, then the row's share of the
// five moments from v_z = -L + z dv (float64 throughout; three float64 operations per
// value instead of one per moment).
template <typename TIO>
__global__ void __launch_bounds__(256) phisums_kernel(const TIO* f, double* U, int N, double L, double dv,
                                                      double scale) {
  const long long cell = blockIdx.x;
  const int n = N * N * N;
  const TIO* fc = f + cell * n;
  double m[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int row = threadIdx.x; row < N * N; row += blockDim.x) {
    const int x = row / N, y = row % N;
    const TIO* r = fc + (size_t)row * N;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int z = 0; z < N; ++z) {
      const double fv = (double)r[z];
      s0 += fv;
      s1 += (double)z * fv;
      s2 += (double)(z * z) * fv;
    }
    const double vx = -L + x * dv, vy = -L + y * dv;
    const double sz = -L * s0 + dv * s1;
    const double szz = L * L * s0 - 2.0 * L * dv * s1 + dv * dv * s2;
    m[0] += s0;
    m[1] += vx * s0;
    m[2] += vy * s0;
    m[3] += sz;
    m[4] += 0.5 * ((vx * vx + vy * vy) * s0 + szz);
  }
  __shared__ double red[8][5];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const double s = warp_sum_d(m[r]);
    if (lane == 0) red[warp][r] = s;
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
    U[cell * 5 + threadIdx.x] = scale * s;
  }
}

// ------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------

static boltz_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return BOLTZ_ECUDA;
}

boltz_status upload_tables(boltz_grid_s* g) {
  // twiddles of the register transforms, host libm in float64
  TwiddleTables tw;
  fill_twiddle_tables(tw);
  cudaError_t e;
  if ((e = unit_upload_twiddles_f32(tw)) != cudaSuccess || (e = unit_upload_twiddles_f64(tw)) != cudaSuccess ||
      (e = unit_upload_twiddles_tc(tw)) != cudaSuccess || (e = unit_upload_twiddles_p2d(tw)) != cudaSuccess)
    return cuda_fail(e, "twiddle upload");

  const size_t n = (g->dim == 2) ? (size_t)g->N * g->N : (size_t)g->N * g->N * g->N;
  const size_t entries = (size_t)(g->M_eff + 1) * n;
  std::vector<double2> h64;
  std::vector<float2> h32;
  const bool want64 = collide_supported_grid(g, BOLTZ_FP64);  // no float64 path at N = 48, 64
  try {
    if (want64) h64.resize(entries);
    h32.resize(entries);
  } catch (...) {
    set_error("host staging of the device tables failed");
    return BOLTZ_ENOMEM;
  }
  // device layout [i][ky][kx][kz]: the ky-slab of one direction is one contiguous block;
  // 2D grids keep the host order [i][kx][ky] (a cell's threads read along ky)
  const int N = g->N;
  if (g->dim == 2) {
    for (int i = 0; i <= g->M_eff; ++i)
      for (size_t k = 0; k < n; ++k) {
        const double a = (i < g->M_eff) ? g->alpha[(size_t)i * n + k] : g->D[k];
        const double b = (i < g->M_eff) ? g->alphap[(size_t)i * n + k] : 0.0;
        if (want64) h64[(size_t)i * n + k] = make_double2(a, b);
        h32[(size_t)i * n + k] = make_float2((float)a, (float)b);
      }
  }
  for (int i = 0; g->dim == 3 && i <= g->M_eff; ++i)
    for (int kx = 0; kx < N; ++kx)
      for (int ky = 0; ky < N; ++ky)
        for (int kz = 0; kz < N; ++kz) {
          const size_t src = ((size_t)kx * N + ky) * N + kz;
          const size_t dst = (size_t)i * n + ((size_t)ky * N + kx) * N + kz;
          const double a = (i < g->M_eff) ? g->alpha[(size_t)i * n + src] : g->D[src];
          const double b = (i < g->M_eff) ? g->alphap[(size_t)i * n + src] : 0.0;
          if (want64) h64[dst] = make_double2(a, b);
          h32[dst] = make_float2((float)a, (float)b);
        }
  if (want64 && (e = cudaMalloc(&g->tab64, entries * sizeof(double2))) != cudaSuccess) {
    cudaGetLastError();  // not sticky: clear it for later launches
    set_error(std::string("device tables: ") + cudaGetErrorString(e));
    return BOLTZ_ENOMEM;
  }
  if ((e = cudaMalloc(&g->tab32, entries * sizeof(float2))) != cudaSuccess) {
    cudaGetLastError();  // not sticky: clear it for later launches
    set_error(std::string("device tables: ") + cudaGetErrorString(e));
    return BOLTZ_ENOMEM;
  }
  if ((e = cudaMalloc(&g->w_dev, (size_t)std::max(1, g->M_eff) * sizeof(double))) != cudaSuccess) {
    cudaGetLastError();  // not sticky: clear it for later launches
    set_error(std::string("device tables: ") + cudaGetErrorString(e));
    return BOLTZ_ENOMEM;
  }
  if (want64 && (e = cudaMemcpy(g->tab64, h64.data(), entries * sizeof(double2), cudaMemcpyHostToDevice)) !=
                    cudaSuccess)
    return cuda_fail(e, "table upload");
  if ((e = cudaMemcpy(g->tab32, h32.data(), entries * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "table upload");
  if ((e = cudaMemcpy(g->w_dev, g->w.data(), g->M_eff * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(e, "table upload");
  return BOLTZ_OK;
}

bool collide_supported_grid(const boltz_grid_s* g, int prec) {
  if (g->dim == 2)
    return (g->N == 8 || g->N == 16 || g->N == 32) ? (prec == BOLTZ_FP64 || prec == BOLTZ_FP32_FFT)
                                                   : (g->N == 64 && prec == BOLTZ_FP32_FFT);
  return collide_supported(g->N, prec);
}

bool collide_supported(int N, int prec) {
  if (prec == BOLTZ_TF32_DFT || prec == BOLTZ_3XBF16_DFT || prec == BOLTZ_3XTF32_DFT) return N == 16 || N == 32;
  if (N == 8 || N == 16 || N == 24 || N == 32) return prec == BOLTZ_FP64 || prec == BOLTZ_FP32_FFT;
  if (N == 48 || N == 64) return prec == BOLTZ_FP32_FFT;  // float64 pencils of 48/64 do not fit
  return false;
}

// Cluster sizes.  float64: the smallest C whose per-CTA slab fits shared memory and
// registers.  float32: measured on GB300 -- at 32^3, C = 8 (128-thread CTAs, two clusters
// per SM whose barrier waits overlap) beats C = 4 (one 256-thread CTA per SM) by 8 % and
// C = 16 by 30 %; at 24^3 the autotuner prefers 3 to 2; at 48^3, C = 12 (two 192-thread
// CTAs per SM) beats C = 8 (one 288-thread CTA per SM) by 49 %.  The other built sizes are
// candidates for the autotuner of ragged plans and for boltz_grid_opts.cluster_size.
int default_cluster(int N, int prec) {
  const bool dbl = (prec == BOLTZ_FP64);
  switch (N) {
    case 8: return 1;
    case 16: return dbl ? 2 : 1;
    case 24: return 3;
    case 32: return dbl ? 8 : 1;  // float32: one CTA per cell (clusters of 8 with term groups)
    case 48: return dbl ? 0 : 12;
    case 64: return dbl ? 0 : 16;
    default: return 0;
  }
}

int default_cluster_for(int N, int prec, int groups) {
  const int c = default_cluster(N, prec);
  return (N == 32 && c == 1 && groups > 1) ? 8 : c;  // the one-CTA-per-cell kernel has no term groups
}

int cluster_choices(int N, int prec, int* out) {
  int k = 0;
  out[k++] = default_cluster(N, prec);
  if (prec != BOLTZ_FP64) {
    if (N == 16) {
      out[k++] = 2;
      out[k++] = 4;
    }
    if (N == 24) {
      out[k++] = 2;
      out[k++] = 6;
    }
    if (N == 32) {
      out[k++] = 8;  // clusters of 8 (also with term groups)
      out[k++] = 4;
      out[k++] = 16;
    }
    if (N == 48) out[k++] = 8;
  }
  return k;
}

int launch_groups(const boltz_grid_s* g, int prec, int groups) {
  const bool tc = (prec == BOLTZ_TF32_DFT || prec == BOLTZ_3XBF16_DFT || prec == BOLTZ_3XTF32_DFT);
  if (g->dim == 2 || tc) return 1;
  const int G = groups < 0 ? g->term_groups : groups;
  return std::max(1, std::min(G, g->M_eff));
}

size_t split_block_bytes(const boltz_grid_s* g, int G, int prec) {
  const size_t tsz = (prec == BOLTZ_FP64) ? sizeof(double) : sizeof(float);
  return ((size_t)(G + 1) * cell_points(g) * tsz + sizeof(unsigned) + kSplitUnit - 1) / kSplitUnit * kSplitUnit;
}

// Scratch of split launches: [cells] arrival counters (zeroed once; every launch leaves
// them at zero), then the partial gains [cells][G][n] and the loss multipliers [cells][n].
boltz_status ensure_split_scratch(const boltz_grid_s* g, int64_t n_cells, int G, int prec, cudaStream_t stream) {
  const size_t n = (size_t)g->N * g->N * g->N;
  const size_t tsz = (prec == BOLTZ_FP64) ? sizeof(double) : sizeof(float);
  const size_t cnt_bytes = ((size_t)n_cells * sizeof(unsigned) + 255) / 256 * 256;
  const size_t need = cnt_bytes + (size_t)n_cells * (G + 1) * n * tsz;
  if (need <= g->split_cap) return BOLTZ_OK;
  // the old buffer may still be read by work queued on this stream
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "split scratch sync");
  cudaFree(g->split_buf);
  g->split_buf = nullptr;
  g->split_cap = 0;
  if (cudaMalloc(&g->split_buf, need) != cudaSuccess) {
    cudaGetLastError();
    set_error("split scratch allocation failed");
    return BOLTZ_ENOMEM;
  }
  if ((e = cudaMemset(g->split_buf, 0, need)) != cudaSuccess) return cuda_fail(e, "split scratch clear");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "split scratch clear");
  g->split_cap = need;
  return BOLTZ_OK;
}

boltz_status launch_collide(const boltz_grid_s* g, int64_t n_cells, int prec, int f_is_fp64, const void* f_in,
                            const void* f_base, void* out, double a, double b, double s, double* Utgt,
                            int compute_targets, int project, cudaStream_t stream, const int64_t* cell_idx,
                            int64_t pool_cells, int groups, int cluster, const int64_t* split_idx,
                            void* split_base, const TransportArgs* tr) {
  if (n_cells == 0) return BOLTZ_OK;
  if (!collide_supported_grid(g, prec)) {
    set_error("unsupported (N, precision) combination");
    return BOLTZ_EUNSUPPORTED;
  }
  if (g->dim == 2) {
    CollideArgs a2 = {};
    a2.f_in = f_in;
    a2.f_base = f_base;
    a2.out = out;
    a2.w = g->w_dev;
    a2.Utgt = Utgt;
    a2.a = a;
    a2.b = b;
    a2.s = s;
    a2.M_eff = g->M_eff;
    a2.project = project;
    a2.compute_targets = compute_targets;
    a2.cell_idx = cell_idx;
    a2.pool_cells = pool_cells;
    a2.groups = 1;
    if (tr) a2.tr = *tr;
    a2.geom.L = g->L;
    a2.geom.dv = g->dv;
    for (int i = 0; i < 25; ++i) a2.geom.G[i] = g->proj.G[i];
    a2.tab = (prec == BOLTZ_FP64) ? (const void*)g->tab64 : (const void*)g->tab32;
    return dispatch_2d(g, a2, n_cells, stream, prec, f_is_fp64);
  }
  if (cluster == 0 && prec != BOLTZ_FP64) cluster = g->cluster_size;  // 0: the default of (N, prec)
  const bool tc = (prec == BOLTZ_TF32_DFT || prec == BOLTZ_3XBF16_DFT || prec == BOLTZ_3XTF32_DFT);
  const int G = launch_groups(g, prec, groups);
  if (n_cells * (int64_t)G * 16 > (int64_t)INT32_MAX) {
    set_error("n_cells * term_groups too large for one launch");
    return BOLTZ_EINVAL;
  }
  const size_t n = (size_t)g->N * g->N * g->N;
  const size_t tsz = (prec == BOLTZ_FP64) ? sizeof(double) : sizeof(float);
  const size_t cnt_bytes = ((size_t)n_cells * sizeof(unsigned) + 255) / 256 * 256;
  if (G > 1 && !split_idx) {
    boltz_status r = ensure_split_scratch(g, n_cells, G, prec, stream);
    if (r != BOLTZ_OK) return r;
  }
  CollideArgs args = {};
  args.f_in = f_in;
  args.f_base = f_base;
  args.out = out;
  args.w = g->w_dev;
  args.Utgt = Utgt;
  args.a = a;
  args.b = b;
  args.s = s;
  args.M_eff = g->M_eff;
  args.project = project;
  args.compute_targets = compute_targets;
  args.cell_idx = cell_idx;
  args.pool_cells = pool_cells;
  args.geom.L = g->L;
  args.geom.dv = g->dv;
  for (int i = 0; i < 25; ++i) args.geom.G[i] = g->proj.G[i];
  args.groups = G;
  if (tr) args.tr = *tr;
  args.split_idx = nullptr;
  args.split_unit = 0;
  if (G > 1 && split_idx) {
    args.split_idx = split_idx;
    args.split_unit = kSplitUnit;
    args.part = split_base;
    args.loss = nullptr;
    args.arrivals = nullptr;
  } else {
    char* sb = static_cast<char*>(g->split_buf);
    args.arrivals = (G > 1) ? reinterpret_cast<unsigned*>(sb) : nullptr;
    args.part = (G > 1) ? sb + cnt_bytes : nullptr;
    args.loss = (G > 1) ? sb + cnt_bytes + (size_t)n_cells * G * n * tsz : nullptr;
  }
  if (prec == BOLTZ_FP64) {
    args.tab = g->tab64;
    return dispatch_3d_f64(g, args, n_cells, stream, cluster, f_is_fp64);
  }
  args.tab = g->tab32;
  if (tc) return dispatch_3d_tc(g, args, n_cells, stream, prec, f_is_fp64);
  if (g->N > 32) return dispatch_3d_large(g, args, n_cells, stream, cluster, f_is_fp64);
  return dispatch_3d_f32(g, args, n_cells, stream, cluster, f_is_fp64);
}

boltz_status launch_phisums(const boltz_grid_s* g, int64_t n_cells, int f_is_fp64, const void* f, double* U,
                            double scale, cudaStream_t stream) {
  if (n_cells == 0) return BOLTZ_OK;
  if (g->dim == 2) {
    const unsigned blocks = (unsigned)((n_cells + 7) / 8);
    if (f_is_fp64)
      phisums2d_kernel<double><<<blocks, 256, 0, stream>>>((const double*)f, U, g->N, g->L, g->dv, scale, n_cells);
    else
      phisums2d_kernel<float><<<blocks, 256, 0, stream>>>((const float*)f, U, g->N, g->L, g->dv, scale, n_cells);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "moments launch");
    return BOLTZ_OK;
  }
  dim3 grid((unsigned)n_cells), block(256);
  if (f_is_fp64)
    phisums_kernel<double><<<grid, block, 0, stream>>>((const double*)f, U, g->N, g->L, g->dv, scale);
  else
    phisums_kernel<float><<<grid, block, 0, stream>>>((const float*)f, U, g->N, g->L, g->dv, scale);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "moments launch");
  return BOLTZ_OK;
}

boltz_status read_and_clear_status(cudaStream_t stream, unsigned* value) {
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  unsigned v = 0;
  if ((e = unit_read_clear_status_f32(&v)) != cudaSuccess || (e = unit_read_clear_status_f64(&v)) != cudaSuccess ||
      (e = unit_read_clear_status_tc(&v)) != cudaSuccess || (e = unit_read_clear_status_p2d(&v)) != cudaSuccess)
    return cuda_fail(e, "status read");
  *value = v;
  return BOLTZ_OK;
}

}  // namespace boltz
