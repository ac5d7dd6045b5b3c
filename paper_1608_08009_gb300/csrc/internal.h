// Internal declarations shared by the host table builder and the CUDA kernels of libboltz.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/boltz.h"
#include "twiddles.h"

namespace boltz {

// Projection data of one grid (Sec. 3.2, Eq. minim1): with Phi the 5 x n matrix of the
// rows (1, v_x, v_y, v_z, |v|^2/2) at the grid points, C = dv^3 Phi and
// C^T (C C^T)^-1 (U - C g) = Phi^T G (U / dv^3 - Phi g), G = (Phi Phi^T)^-1.
struct Projection {
  double G[25];
};

// Geometry and kernel parameters passed by value to every collision kernel.
struct KernelGeom {
  double L;
  double dv;
  double G[25];
};

// Transport stage of the Fast Kinetic Scheme in one space dimension (Sec. 3.1, Eq. f_bar),
// fused into the collision kernels' loads.  With nx > 0 the launch's cells are rows of nx
// cells along x (cell c is cell j = c % nx of row c / nx) and the thread that handles
// velocity-x index x reads cell j - d(x) of the same row, d(x) = +1 for the indices set in
// shift_pos, -1 for those in shift_neg, 0 otherwise: the exact shift of the piecewise-
// constant distribution sampled at the cell centres.  A source outside the row reads the
// row's state beyond that end, inflow_lo[row] (j - d < 0) or inflow_hi[row] (j - d >= nx),
// [rows][n] TIO each (the Dirichlet boundary states, or a neighbour's edge cells).
struct TransportArgs {
  int64_t nx;  // 0: no transport stage
  uint64_t shift_pos, shift_neg;
  const void* inflow_lo;
  const void* inflow_hi;
};

// Argument block of every collision kernel (passed by value).
struct CollideArgs {
  const void* f_in;    // [cells][N^3] TIO
  const void* f_base;  // [cells][N^3] TIO or null
  void* out;           // [cells][N^3] TIO
  const void* tab;     // [(M_eff + 1)][ky][kx][kz] (alpha, alpha') as Vec2<T>; entry M_eff = (D, 0)
  const double* w;     // [M_eff]
  double* Utgt;        // [cells][5] target Phi-sums, or null (target 0)
  double a, b, s;      // out = Pi(a f_base + b f_in + s Q)
  int M_eff;
  int project;
  int compute_targets; // 1: targets = Phi f_in, computed here and written to Utgt if non-null
  const int64_t* cell_idx;  // null: cell c of the launch is slot c; else slot cell_idx[c]
  int64_t pool_cells;       // number of slots behind f_in / f_base / out / Utgt (cell_idx)
  // Term groups.  groups = 1: one cluster per cell does every term and the epilogue.
  // groups = G > 1: cluster (c, g) does the terms [g M_eff / G, (g + 1) M_eff / G) (the
  // last group also the loss transform) and writes its partial gain to
  // part[(c G + g) n ...] and the loss multiplier to loss[c n ...] (c = cell of the
  // launch), then counts itself in arrivals[c]; the cluster that arrives last sums the
  // partials in group order and runs the epilogue (and resets arrivals[c] to 0).
  int groups;
  void* part;          // [cells][G][n] T
  void* loss;          // [cells][n] T
  unsigned* arrivals;  // [cells], zero between launches
  // Term-group scratch by block instead of by launch position (serving loop): when
  // split_idx is non-null, cell c of the launch uses the block at part + split_idx[c] *
  // split_unit bytes, laid out as [G][n] T partial gains, [n] T loss multipliers, one
  // unsigned arrival count (zero between launches); loss and arrivals are then unused.
  const int64_t* split_idx;
  size_t split_unit;
  TransportArgs tr;
  KernelGeom geom;
};

}  // namespace boltz

struct boltz_grid_s {
  int dim = 3;  // velocity dimension: 3, or 2 (Maxwell molecules, boltz_create_grid2d)
  int N = 0;
  double L = 0, dv = 0, S = 0, R = 0, gamma = 1, C_gamma = 1;
  int M = 0, rank = 1, M_eff = 0;
  int dirs_kind = 0, a1 = 0, inner_nodes = 128, project = 1;
  int term_groups = 1;  // clusters per cell sharing its separated terms (1 = no split)
  int cluster_size = 0; // cluster size of the float32 path (0 = default)
  int device = 0;
  // float64 host tables, mode storage order (kx, ky, kz), kz fastest
  std::vector<double> e, wdir, w, alpha, alphap, D;
  boltz::Projection proj{};
  // device tables: (M_eff + 1) * n pairs (alpha, alpha'); entry M_eff holds (D, 0)
  double2* tab64 = nullptr;
  float2* tab32 = nullptr;
  double* w_dev = nullptr;  // [M_eff]
  // scratch of boltz_relax, grown on demand
  double* U0 = nullptr;
  size_t U0_cap = 0;  // cells
  void* stage = nullptr;
  size_t stage_cap = 0;  // bytes
  // partial gains and loss of split launches (term_groups > 1), grown on demand
  mutable void* split_buf = nullptr;
  mutable size_t split_cap = 0;  // bytes
  // resources of boltz_relax_host (host_io.cpp), created on first use
  static constexpr int kHostBufs = 3;
  void* hbuf[kHostBufs] = {nullptr, nullptr, nullptr};  // device staging, one chunk each
  size_t hbuf_cap = 0;                                   // bytes per buffer
  double* hU0 = nullptr;                                 // [chunk][5]
  void* hstage = nullptr;                                // Heun stage of one chunk
  size_t hchunk_cap = 0;                                 // cells
  cudaStream_t up = nullptr, down = nullptr;
  cudaEvent_t ev_start = nullptr;
  cudaEvent_t ev_in[kHostBufs] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_done[kHostBufs] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_out[kHostBufs] = {nullptr, nullptr, nullptr};
};

namespace boltz {

// Velocity points per cell: N^3, or N^2 on a 2D grid.
inline size_t cell_points(const boltz_grid_s* g) {
  return g->dim == 2 ? (size_t)g->N * g->N : (size_t)g->N * g->N * g->N;
}

void set_error(const std::string& msg);

// Host table builder (tables.cpp): fills e, wdir, w, alpha, alphap, D, proj, S, R.
boltz_status build_tables(boltz_grid_s* g);
// Host table builder of the 2D Maxwell-molecule grids (tables.cpp).
boltz_status build_tables2d(boltz_grid_s* g);

// Kernel launchers (collide.cu, dispatching to the kernel units).
boltz_status upload_tables(boltz_grid_s* g);
// out = Pi(a f_base + b f_in + s Q(f_in)).  Pi projects onto the targets Utgt (Phi-sums,
// [cells][5]); compute_targets = 1 takes the targets from f_in itself (and stores them to
// Utgt when non-null), 0 reads Utgt (null: target 0, i.e. the projection of Q).
boltz_status launch_collide(const boltz_grid_s* g, int64_t n_cells, int prec, int f_is_fp64,
                            const void* f_in, const void* f_base, void* out, double a, double b,
                            double s, double* Utgt, int compute_targets, int project,
                            cudaStream_t stream, const int64_t* cell_idx = nullptr,
                            int64_t pool_cells = 0, int groups = -1, int cluster = 0,
                            const int64_t* split_idx = nullptr, void* split_base = nullptr,
                            const TransportArgs* tr = nullptr);
// Bytes of one term-group scratch block (CollideArgs::split_idx) of grid g with G groups:
// a multiple of kSplitUnit.  split_idx entries passed to launch_collide count kSplitUnit
// bytes from split_base.
constexpr size_t kSplitUnit = 16;
size_t split_block_bytes(const boltz_grid_s* g, int G, int prec);
// Term groups a launch of grid g in precision prec uses (groups < 0: the grid's setting).
int launch_groups(const boltz_grid_s* g, int prec, int groups);
// groups < 0: the grid's term_groups; cluster 0: the default cluster size of (N, prec)
int default_cluster(int N, int prec);
// The default cluster size of a launch with `groups` term groups (the one-CTA-per-cell
// 32^3 kernel runs without them; split launches take clusters of 8).
int default_cluster_for(int N, int prec, int groups);
// Grow the grid's scratch of split launches (term groups) to n_cells cells of G groups;
// synchronises `stream` when it has to reallocate.
boltz_status ensure_split_scratch(const boltz_grid_s* g, int64_t n_cells, int G, int prec, cudaStream_t stream);
// Cluster sizes with a kernel for (N, prec), the default first; returns the count (<= 4).
int cluster_choices(int N, int prec, int* out);
boltz_status launch_phisums(const boltz_grid_s* g, int64_t n_cells, int f_is_fp64, const void* f,
                            double* U, double scale, cudaStream_t stream);
bool collide_supported(int N, int prec);
// As collide_supported, for the grid's dimension (2D grids: 8, 16, 32 both precisions, 64 float32).
bool collide_supported_grid(const boltz_grid_s* g, int prec);
// `steps` Euler or Heun steps of n_cells cells of f in place (the body of boltz_relax);
// U0: [n_cells][5] scratch for the targets, stage: one copy of f (Heun only).
boltz_status relax_steps(const boltz_grid_s* g, int64_t n_cells, int prec, int f_is_fp64, void* f, double dt,
                         int steps, int rk_order, cudaStream_t s, double* U0, void* stage, int groups = -1,
                         int cluster = 0);
void free_host_pipeline(boltz_grid_s* g);
// Kernel units (collide_f32.cu, collide_f64.cu, collide_tc.cu, collide_2d.cu): launch of
// the collision kernels for one argument block, and each unit's twiddle upload and
// status word (every unit has its own copies).
boltz_status dispatch_3d_f32(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st,
                             int cluster, int f_is_fp64);
boltz_status dispatch_3d_f64(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st,
                             int cluster, int f_is_fp64);
boltz_status dispatch_3d_tc(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st, int prec,
                            int f_is_fp64);
boltz_status dispatch_3d_large(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st,
                               int cluster, int f_is_fp64);
boltz_status dispatch_2d(const boltz_grid_s* g, const CollideArgs& a, int64_t n_cells, cudaStream_t st, int prec,
                         int f_is_fp64);
boltz_status selftest_conversions(uint64_t* mismatches);
#define BOLTZ_DECLARE_UNIT(TAG)                                                                                    \
  cudaError_t unit_upload_twiddles_##TAG(const TwiddleTables& t);                                                 \
  cudaError_t unit_read_clear_status_##TAG(unsigned* value);
BOLTZ_DECLARE_UNIT(f32)
BOLTZ_DECLARE_UNIT(f64)
BOLTZ_DECLARE_UNIT(tc)
BOLTZ_DECLARE_UNIT(p2d)
#undef BOLTZ_DECLARE_UNIT
// Argument checks shared by the entry points (api.cpp): set the error message on failure.
boltz_status check_batch(const boltz_batch* b);
boltz_status check_device(const boltz_grid_s* g);

}  // namespace boltz
