// C ABI of libboltz (declared in include/boltz.h): argument checking, grid ownership,
// relaxation driver.  All compute happens in the kernels of the collide*.cu units.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

namespace boltz {

static thread_local std::string t_last_error;

void set_error(const std::string& msg) { t_last_error = msg; }

boltz_status read_and_clear_status(cudaStream_t stream, unsigned* value);

}  // namespace boltz

using boltz::set_error;

namespace boltz {

boltz_status check_batch(const boltz_batch* b) {
  if (!b || !b->grid) {
    set_error("null batch or grid");
    return BOLTZ_EINVAL;
  }
  if (b->n_cells < 0) {
    set_error("n_cells must be >= 0");
    return BOLTZ_EINVAL;
  }
  if (b->n_cells > (int64_t)1 << 24) {
    set_error("n_cells above 2^24 per call");
    return BOLTZ_EINVAL;
  }
  if (b->f_is_fp64 != 0 && b->f_is_fp64 != 1) {
    set_error("f_is_fp64 must be 0 or 1");
    return BOLTZ_EINVAL;
  }
  if (b->prec < BOLTZ_FP64 || b->prec > BOLTZ_3XTF32_DFT) {
    set_error("unknown precision");
    return BOLTZ_EINVAL;
  }
  if (!boltz::collide_supported_grid(b->grid, b->prec)) {
    set_error("this precision has no kernel for this N in this library");
    return BOLTZ_EUNSUPPORTED;
  }
  return BOLTZ_OK;
}

boltz_status check_device(const boltz_grid_s* g) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return BOLTZ_ECUDA;
  }
  if (dev != g->device) {
    set_error("the grid belongs to another device");
    return BOLTZ_EINVAL;
  }
  return BOLTZ_OK;
}

}  // namespace boltz

using boltz::check_batch;
using boltz::check_device;

extern "C" {

void boltz_default_opts(boltz_grid_opts* o) {
  if (!o) return;
  o->dirs_kind = 0;
  o->dirs_a1 = 0;
  o->R_trunc = 0.0;
  o->C_gamma = 1.0;
  o->radial_rank = 0;
  o->inner_nodes = 128;
  o->term_groups = 1;
  o->cluster_size = 0;
  o->project = 1;
}

boltz_status boltz_create_grid(int N_v, double L, double gamma, int M_dirs, const boltz_grid_opts* opts,
                               boltz_grid* out) {
  if (!out) {
    set_error("null output handle");
    return BOLTZ_EINVAL;
  }
  if (N_v != 8 && N_v != 16 && N_v != 24 && N_v != 32 && N_v != 48 && N_v != 64) {
    set_error("N_v must be 8, 16, 24, 32, 48 or 64 in this library");
    return (N_v > 0 && N_v % 2 == 0) ? BOLTZ_EUNSUPPORTED : BOLTZ_EINVAL;
  }
  if (!(L > 0) || !std::isfinite(L)) {
    set_error("L must be positive and finite");
    return BOLTZ_EINVAL;
  }
  if (!(gamma >= -3.0 && gamma <= 1.0)) {
    set_error("gamma must lie in [-3, 1]");
    return BOLTZ_EINVAL;
  }
  if (M_dirs < 1 || M_dirs > 4096) {
    set_error("M_dirs must lie in [1, 4096]");
    return BOLTZ_EINVAL;
  }
  boltz_grid_opts o;
  boltz_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.C_gamma > 0) || !std::isfinite(o.C_gamma)) {
    set_error("C_gamma must be positive");
    return BOLTZ_EINVAL;
  }
  if (o.inner_nodes <= 0) o.inner_nodes = 128;
  if (o.inner_nodes > 4096) {
    set_error("inner_nodes must be <= 4096");
    return BOLTZ_EINVAL;
  }
  int rank = o.radial_rank > 0 ? o.radial_rank : (gamma == 1.0 ? 1 : 16);
  if (rank * (long long)M_dirs > 65536) {
    set_error("M_dirs * radial_rank must be <= 65536");
    return BOLTZ_EINVAL;
  }
  if (rank == 1 && gamma != 1.0) {
    set_error("radial_rank 1 is exact only for gamma = 1");
    return BOLTZ_EINVAL;
  }
  if (o.term_groups < 0 || o.term_groups > 4096) {
    set_error("term_groups must lie in [0, 4096]");
    return BOLTZ_EINVAL;
  }
  if (o.cluster_size != 0) {
    int cl[4];
    const int k = boltz::cluster_choices(N_v, BOLTZ_FP32_FFT, cl);
    bool ok = false;
    for (int i = 0; i < k; ++i) ok |= (cl[i] == o.cluster_size);
    if (!ok) {
      set_error("no float32 kernel with this cluster size for this N");
      return BOLTZ_EUNSUPPORTED;
    }
  }
  boltz_grid_s* g = new (std::nothrow) boltz_grid_s();
  if (!g) {
    set_error("out of host memory");
    return BOLTZ_ENOMEM;
  }
  cudaError_t e = cudaGetDevice(&g->device);
  if (e != cudaSuccess) {
    delete g;
    set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return BOLTZ_ECUDA;
  }
  g->N = N_v;
  g->L = L;
  g->gamma = gamma;
  g->C_gamma = o.C_gamma;
  g->M = M_dirs;
  g->rank = rank;
  g->dirs_kind = o.dirs_kind;
  g->a1 = o.dirs_a1;
  g->inner_nodes = o.inner_nodes;
  g->project = o.project ? 1 : 0;
  g->term_groups = std::max(1, std::min(o.term_groups, M_dirs * rank));
  g->cluster_size = o.cluster_size;
  g->R = o.R_trunc > 0 ? o.R_trunc : 0.0;
  boltz_status st = boltz::build_tables(g);
  if (st == BOLTZ_OK) st = boltz::upload_tables(g);
  if (st != BOLTZ_OK) {
    boltz_destroy_grid(g);
    return st;
  }
  *out = g;
  return BOLTZ_OK;
}

boltz_status boltz_create_grid2d(int N_v, double L, int M_dirs, const boltz_grid_opts* opts, boltz_grid* out) {
  if (!out) {
    set_error("null output handle");
    return BOLTZ_EINVAL;
  }
  if (N_v != 8 && N_v != 16 && N_v != 32 && N_v != 64) {
    set_error("2D grids: N_v must be 8, 16, 32 or 64 in this library");
    return (N_v > 0 && N_v % 2 == 0) ? BOLTZ_EUNSUPPORTED : BOLTZ_EINVAL;
  }
  if (!(L > 0) || !std::isfinite(L)) {
    set_error("L must be positive and finite");
    return BOLTZ_EINVAL;
  }
  if (M_dirs < 1 || M_dirs > 4096) {
    set_error("M_dirs must lie in [1, 4096]");
    return BOLTZ_EINVAL;
  }
  boltz_grid_opts o;
  boltz_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.C_gamma > 0) || !std::isfinite(o.C_gamma)) {
    set_error("C_gamma must be positive");
    return BOLTZ_EINVAL;
  }
  boltz_grid_s* g = new (std::nothrow) boltz_grid_s();
  if (!g) {
    set_error("out of host memory");
    return BOLTZ_ENOMEM;
  }
  cudaError_t e = cudaGetDevice(&g->device);
  if (e != cudaSuccess) {
    delete g;
    set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    return BOLTZ_ECUDA;
  }
  g->dim = 2;
  g->N = N_v;
  g->L = L;
  g->gamma = 0.0;
  g->C_gamma = o.C_gamma;
  g->M = M_dirs;
  g->project = o.project ? 1 : 0;
  g->R = o.R_trunc > 0 ? o.R_trunc : 0.0;
  boltz_status st = boltz::build_tables2d(g);
  if (st == BOLTZ_OK) st = boltz::upload_tables(g);
  if (st != BOLTZ_OK) {
    boltz_destroy_grid(g);
    return st;
  }
  *out = g;
  return BOLTZ_OK;
}

boltz_status boltz_destroy_grid(boltz_grid g) {
  if (!g) return BOLTZ_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(g->device);
  cudaDeviceSynchronize();
  cudaFree(g->tab64);
  cudaFree(g->tab32);
  cudaFree(g->w_dev);
  cudaFree(g->U0);
  cudaFree(g->stage);
  cudaFree(g->split_buf);
  boltz::free_host_pipeline(g);
  if (prev >= 0) cudaSetDevice(prev);
  delete g;
  return BOLTZ_OK;
}

boltz_status boltz_collide(const boltz_batch* b, const void* f, void* Q, void* stream) {
  boltz_status st = check_batch(b);
  if (st != BOLTZ_OK) return st;
  if (b->n_cells == 0) return BOLTZ_OK;
  if (!f || !Q) {
    set_error("null f or Q");
    return BOLTZ_EINVAL;
  }
  if (f == Q) {
    set_error("f and Q must not overlap");
    return BOLTZ_EINVAL;
  }
  if ((st = check_device(b->grid)) != BOLTZ_OK) return st;
  return boltz::launch_collide(b->grid, b->n_cells, b->prec, b->f_is_fp64, f, nullptr, Q, 0.0, 0.0, 1.0, nullptr, 0,
                               b->grid->project, (cudaStream_t)stream);
}

boltz_status boltz_collide_indexed(const boltz_batch* b, const void* f, void* Q, const int64_t* cell_idx,
                                   int64_t pool_cells, void* stream) {
  boltz_status st = check_batch(b);
  if (st != BOLTZ_OK) return st;
  if (b->n_cells == 0) return BOLTZ_OK;
  if (!f || !Q || !cell_idx) {
    set_error("null f, Q or cell_idx");
    return BOLTZ_EINVAL;
  }
  if (f == Q) {
    set_error("f and Q must not overlap");
    return BOLTZ_EINVAL;
  }
  if (pool_cells < 1 || pool_cells > ((int64_t)1 << 31)) {
    set_error("pool_cells must lie in [1, 2^31]");
    return BOLTZ_EINVAL;
  }
  if ((st = check_device(b->grid)) != BOLTZ_OK) return st;
  return boltz::launch_collide(b->grid, b->n_cells, b->prec, b->f_is_fp64, f, nullptr, Q, 0.0, 0.0, 1.0, nullptr, 0,
                               b->grid->project, (cudaStream_t)stream, cell_idx, pool_cells);
}

boltz_status boltz_relax_indexed(const boltz_batch* b, void* f, const int64_t* cell_idx, int64_t pool_cells,
                                 double dt, int steps, void* stream) {
  boltz_status st = check_batch(b);
  if (st != BOLTZ_OK) return st;
  if (!(dt > 0) || !std::isfinite(dt)) {
    set_error("dt must be positive and finite");
    return BOLTZ_EINVAL;
  }
  if (steps < 0) {
    set_error("steps must be >= 0");
    return BOLTZ_EINVAL;
  }
  if (b->n_cells == 0 || steps == 0) return BOLTZ_OK;
  if (!f || !cell_idx) {
    set_error("null f or cell_idx");
    return BOLTZ_EINVAL;
  }
  if (pool_cells < 1 || pool_cells > ((int64_t)1 << 31)) {
    set_error("pool_cells must lie in [1, 2^31]");
    return BOLTZ_EINVAL;
  }
  if ((st = check_device(b->grid)) != BOLTZ_OK) return st;
  boltz_grid_s* g = b->grid;
  cudaStream_t s = (cudaStream_t)stream;
  // moment targets per slot: scratch sized for the pool, grown on demand
  if ((size_t)pool_cells > g->U0_cap) {
    cudaStreamSynchronize(s);
    cudaFree(g->U0);
    g->U0 = nullptr;
    g->U0_cap = 0;
    if (cudaMalloc(&g->U0, (size_t)pool_cells * 5 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();  // not sticky: clear it for later launches
      set_error("relax scratch allocation failed");
      return BOLTZ_ENOMEM;
    }
    g->U0_cap = (size_t)pool_cells;
  }
  for (int it = 0; it < steps; ++it) {
    st = boltz::launch_collide(g, b->n_cells, b->prec, b->f_is_fp64, f, nullptr, f, 0.0, 1.0, dt, g->U0,
                               it == 0 ? 1 : 0, 1, s, cell_idx, pool_cells);
    if (st != BOLTZ_OK) return st;
  }
  return BOLTZ_OK;
}

boltz_status boltz_moments(const boltz_batch* b, const void* f, double* U, void* stream) {
  if (!b || !b->grid || b->n_cells < 0 || (b->f_is_fp64 != 0 && b->f_is_fp64 != 1)) {
    set_error("bad batch");
    return BOLTZ_EINVAL;
  }
  if (b->n_cells == 0) return BOLTZ_OK;
  if (!f || !U) {
    set_error("null f or U");
    return BOLTZ_EINVAL;
  }
  boltz_status st = check_device(b->grid);
  if (st != BOLTZ_OK) return st;
  const double dv = b->grid->dv;
  const double vol = (b->grid->dim == 2) ? dv * dv : dv * dv * dv;  // dv^d
  return boltz::launch_phisums(b->grid, b->n_cells, b->f_is_fp64, f, U, vol, (cudaStream_t)stream);
}

boltz_status boltz_selftest_conversions(uint64_t* mismatches) {
  if (!mismatches) {
    set_error("null mismatches");
    return BOLTZ_EINVAL;
  }
  return boltz::selftest_conversions(mismatches);
}

boltz_status boltz_relax(const boltz_batch* b, void* f, double dt, int steps, int rk_order, void* stream) {
  boltz_status st = check_batch(b);
  if (st != BOLTZ_OK) return st;
  if (!(dt > 0) || !std::isfinite(dt)) {
    set_error("dt must be positive and finite");
    return BOLTZ_EINVAL;
  }
  if (steps < 0) {
    set_error("steps must be >= 0");
    return BOLTZ_EINVAL;
  }
  if (rk_order != 1 && rk_order != 2) {
    set_error("rk_order must be 1 or 2");
    return BOLTZ_EINVAL;
  }
  if (b->n_cells == 0 || steps == 0) return BOLTZ_OK;
  if (!f) {
    set_error("null f");
    return BOLTZ_EINVAL;
  }
  if ((st = check_device(b->grid)) != BOLTZ_OK) return st;
  boltz_grid_s* g = b->grid;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = boltz::cell_points(g);
  const size_t esz = b->f_is_fp64 ? 8 : 4;
  // scratch: moment targets (and the Heun stage), grown on demand, owned by the grid
  if ((size_t)b->n_cells > g->U0_cap) {
    cudaStreamSynchronize(s);
    cudaFree(g->U0);
    g->U0 = nullptr;
    g->U0_cap = 0;
    if (cudaMalloc(&g->U0, (size_t)b->n_cells * 5 * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();  // not sticky: clear it for later launches
      set_error("relax scratch allocation failed");
      return BOLTZ_ENOMEM;
    }
    g->U0_cap = (size_t)b->n_cells;
  }
  const size_t stage_bytes = (size_t)b->n_cells * n * esz;
  if (rk_order == 2 && stage_bytes > g->stage_cap) {
    cudaStreamSynchronize(s);
    cudaFree(g->stage);
    g->stage = nullptr;
    g->stage_cap = 0;
    if (cudaMalloc(&g->stage, stage_bytes) != cudaSuccess) {
      cudaGetLastError();  // not sticky: clear it for later launches
      set_error("relax scratch allocation failed");
      return BOLTZ_ENOMEM;
    }
    g->stage_cap = stage_bytes;
  }
  return boltz::relax_steps(g, b->n_cells, b->prec, b->f_is_fp64, f, dt, steps, rk_order, s, g->U0, g->stage);
}

}  // extern "C"

namespace boltz {

boltz_status relax_steps(const boltz_grid_s* g, int64_t n_cells, int prec, int f_is_fp64, void* f, double dt,
                         int steps, int rk_order, cudaStream_t s, double* U0, void* stage, int groups,
                         int cluster) {
  boltz_status st;
  // Targets: Phi-sums of the initial state (Eq. minim1 with U fixed), computed by the
  // first launch from the values it loads anyway and kept in U0 for the later ones.
  for (int it = 0; it < steps; ++it) {
    const int first = (it == 0) ? 1 : 0;
    if (rk_order == 1) {
      st = launch_collide(g, n_cells, prec, f_is_fp64, f, nullptr, f, 0.0, 1.0, dt, U0, first, 1, s, nullptr, 0,
                          groups, cluster);
      if (st != BOLTZ_OK) return st;
    } else {
      st = launch_collide(g, n_cells, prec, f_is_fp64, f, nullptr, stage, 0.0, 1.0, dt, U0, first, 1, s, nullptr,
                          0, groups, cluster);
      if (st != BOLTZ_OK) return st;
      st = launch_collide(g, n_cells, prec, f_is_fp64, stage, f, f, 0.5, 0.5, 0.5 * dt, U0, 0, 1, s, nullptr, 0,
                          groups, cluster);
      if (st != BOLTZ_OK) return st;
    }
  }
  return BOLTZ_OK;
}

}  // namespace boltz

extern "C" {

boltz_status boltz_stream_status(void* stream) {
  unsigned v = 0;
  boltz_status st = boltz::read_and_clear_status((cudaStream_t)stream, &v);
  if (st != BOLTZ_OK) return st;
  if (v & 8u) {
    set_error("a bounded mbarrier wait in a kernel gave up (results of that launch are invalid)");
    return BOLTZ_ETIMEOUT;
  }
  if (v & 4u) {
    set_error("a cell index was outside its pool (that cell was not written)");
    return BOLTZ_EINVAL;
  }
  if (v & 1u) {
    set_error("a non-finite value was produced on the device");
    return BOLTZ_ENONFINITE;
  }
  return BOLTZ_OK;
}

const char* boltz_last_error(void) { return boltz::t_last_error.c_str(); }

boltz_status boltz_grid_info(boltz_grid g, int* N_v, double* L, double* dv, double* S, double* R, int* M_eff) {
  if (!g) {
    set_error("null grid");
    return BOLTZ_EINVAL;
  }
  if (N_v) *N_v = g->N;
  if (L) *L = g->L;
  if (dv) *dv = g->dv;
  if (S) *S = g->S;
  if (R) *R = g->R;
  if (M_eff) *M_eff = g->M_eff;
  return BOLTZ_OK;
}

boltz_status boltz_grid_tables(boltz_grid g, double* e, double* w, double* alpha, double* alphap, double* D) {
  if (!g) {
    set_error("null grid");
    return BOLTZ_EINVAL;
  }
  if (e) std::memcpy(e, g->e.data(), g->e.size() * sizeof(double));
  if (w) std::memcpy(w, g->w.data(), g->w.size() * sizeof(double));
  if (alpha) std::memcpy(alpha, g->alpha.data(), g->alpha.size() * sizeof(double));
  if (alphap) std::memcpy(alphap, g->alphap.data(), g->alphap.size() * sizeof(double));
  if (D) std::memcpy(D, g->D.data(), g->D.size() * sizeof(double));
  return BOLTZ_OK;
}

const char* boltz_version(void) { return "libboltz 0.1 (sm_103a)"; }

}  // extern "C"
