// Ragged batches (boltz_plan_* in include/boltz.h): groups of cells on different grids
// (any mix of N_v, M_dirs, gamma, precision) advanced together by the relaxation of
// Sec. 3.1 (Eq. relax, Eq. f_coll; Heun for rk_order 2).
//
// The collision kernels are specialised per N (the register transforms have compile-time
// lengths), so a ragged step is one kernel launch per group.  The plan makes the whole
// step loop a single CUDA graph: every group's launches form one branch, branches run
// concurrently, and the host pays one graph launch per call.  Before capture an optional
// autotuner times every (term groups, cluster size) candidate of each group on a copy of
// its cells and keeps the fastest.
#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"

namespace {

struct PlanGroup {
  boltz_grid_s* grid = nullptr;
  int64_t n_cells = 0;
  int prec = 0, f_is_fp64 = 0;
  void* f = nullptr;
  int term_groups = 1, cluster = 0;
  double tuned_us = 0.0;
  double* U0 = nullptr;   // [n_cells][5]
  void* stage = nullptr;  // Heun stage, [n_cells][n]
  cudaStream_t stream = nullptr;
  cudaEvent_t join = nullptr;
};

}  // namespace

struct boltz_plan_s {
  std::vector<PlanGroup> groups;
  double dt = 0.0;
  int steps = 0, rk_order = 1, flags = 0;
  cudaStream_t cap = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

using boltz::set_error;

static boltz_status plan_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return BOLTZ_ECUDA;
}

static void free_plan(boltz_plan_s* p) {
  if (!p) return;
  cudaDeviceSynchronize();
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (auto& g : p->groups) {
    cudaFree(g.U0);
    cudaFree(g.stage);
    if (g.stream) cudaStreamDestroy(g.stream);
    if (g.join) cudaEventDestroy(g.join);
  }
  if (p->fork) cudaEventDestroy(p->fork);
  if (p->cap) cudaStreamDestroy(p->cap);
  delete p;
}

// Time one relaxation launch of every candidate on a copy of the group's cells (the
// user's f is not touched) and keep the fastest.  Term groups are only tried when the
// cells alone leave SMs idle.
static boltz_status autotune(PlanGroup& g, cudaStream_t s) {
  const size_t n = boltz::cell_points(g.grid);
  const size_t bytes = (size_t)g.n_cells * n * (g.f_is_fp64 ? 8 : 4);
  void *fa = nullptr, *qa = nullptr;
  cudaError_t e;
  if (cudaMalloc(&fa, bytes) != cudaSuccess || cudaMalloc(&qa, bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(fa);
    set_error("autotune scratch allocation failed");
    return BOLTZ_ENOMEM;
  }
  boltz_status st = BOLTZ_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int cl[4];
  const int ncl = boltz::cluster_choices(g.grid->N, g.prec, cl);
  double best = 1e300;
  if ((e = cudaMemcpyAsync(fa, g.f, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess ||
      (e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    st = plan_fail(e, "autotune setup");
    goto done;
  }
  for (int ci = 0; ci < ncl; ++ci) {
    for (int G = 1; G <= std::min(16, g.grid->M_eff); G *= 2) {
      if (G > 1 && g.n_cells * cl[ci] * (G / 2) >= 2 * (int64_t)sms) break;  // the GPU is already full
      float ms = 0.f, best_c = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {  // rep 0 warms up (and sizes the split scratch)
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
        st = boltz::launch_collide(g.grid, g.n_cells, g.prec, g.f_is_fp64, fa, nullptr, qa, 0.0, 1.0, 1e-3, g.U0, 1,
                                   1, s, nullptr, 0, G, cl[ci]);
        if (st == BOLTZ_EUNSUPPORTED) break;  // not schedulable here: skip the candidate
        if (st != BOLTZ_OK) goto done;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
          break;
        if (rep > 0) best_c = std::min(best_c, ms);
      }
      if (e != cudaSuccess) {
        st = plan_fail(e, "autotune timing");
        goto done;
      }
      if (st == BOLTZ_EUNSUPPORTED) {
        st = BOLTZ_OK;
        cudaEventSynchronize(e0);  // the skipped candidate recorded e0 only
        break;
      }
      if (best_c < best) {
        best = best_c;
        g.term_groups = G;
        g.cluster = cl[ci];
      }
    }
  }
  g.tuned_us = best * 1000.0;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(fa);
  cudaFree(qa);
  return st;
}

extern "C" {

boltz_status boltz_plan_create(const boltz_group* groups, int n_groups, double dt, int steps, int rk_order,
                               int flags, void* stream, boltz_plan* out) {
  if (!groups || !out || n_groups < 1 || n_groups > 256) {
    set_error("bad plan arguments (groups, n_groups in [1, 256], out)");
    return BOLTZ_EINVAL;
  }
  if (!(dt > 0) || !(dt < 1e300) || steps < 0 || (rk_order != 1 && rk_order != 2) ||
      (flags & ~(BOLTZ_PLAN_AUTOTUNE | BOLTZ_PLAN_SERIAL))) {
    set_error("dt must be positive and finite, steps >= 0, rk_order 1 or 2, flags known");
    return BOLTZ_EINVAL;
  }
  for (int i = 0; i < n_groups; ++i) {
    boltz_batch b{groups[i].grid, groups[i].n_cells, groups[i].prec, groups[i].f_is_fp64};
    boltz_status st = boltz::check_batch(&b);
    if (st != BOLTZ_OK) return st;
    if ((st = boltz::check_device(b.grid)) != BOLTZ_OK) return st;
    if (b.n_cells > 0 && !groups[i].f) {
      set_error("null f in a plan group");
      return BOLTZ_EINVAL;
    }
    for (int k = 0; k < i; ++k)
      if (groups[k].grid == groups[i].grid) {
        set_error("two plan groups share a grid (merge their cells into one group)");
        return BOLTZ_EINVAL;
      }
  }
  boltz_plan_s* p = new (std::nothrow) boltz_plan_s();
  if (!p) {
    set_error("out of host memory");
    return BOLTZ_ENOMEM;
  }
  p->dt = dt;
  p->steps = steps;
  p->rk_order = rk_order;
  p->flags = flags;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  boltz_status st = BOLTZ_OK;
  p->groups.resize(n_groups);
  for (int i = 0; i < n_groups; ++i) {
    PlanGroup& g = p->groups[i];
    g.grid = groups[i].grid;
    g.n_cells = groups[i].n_cells;
    g.prec = groups[i].prec;
    g.f_is_fp64 = groups[i].f_is_fp64;
    g.f = groups[i].f;
    g.term_groups = std::max(1, std::min(g.grid->term_groups, g.grid->M_eff));
    g.cluster = (g.prec != BOLTZ_FP64 && g.grid->cluster_size) ? g.grid->cluster_size
                                                                : boltz::default_cluster(g.grid->N, g.prec);
    const size_t n = boltz::cell_points(g.grid);
    const size_t cells = (size_t)std::max<int64_t>(1, g.n_cells);
    if (cudaMalloc(&g.U0, cells * 5 * sizeof(double)) != cudaSuccess ||
        (rk_order == 2 && cudaMalloc(&g.stage, cells * n * (g.f_is_fp64 ? 8 : 4)) != cudaSuccess)) {
      cudaGetLastError();
      free_plan(p);
      set_error("plan scratch allocation failed");
      return BOLTZ_ENOMEM;
    }
    if ((e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming)) != cudaSuccess) {
      free_plan(p);
      return plan_fail(e, "plan streams");
    }
  }
  if ((e = cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming)) != cudaSuccess) {
    free_plan(p);
    return plan_fail(e, "plan streams");
  }
  // tuning and scratch sizing happen outside the capture (they allocate and synchronise)
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
    free_plan(p);
    return plan_fail(e, "plan sync");
  }
  for (auto& g : p->groups) {
    if (g.n_cells == 0) continue;
    if ((flags & BOLTZ_PLAN_AUTOTUNE) && (st = autotune(g, p->cap)) != BOLTZ_OK) {
      free_plan(p);
      return st;
    }
    if (g.term_groups > 1 &&
        (st = boltz::ensure_split_scratch(g.grid, g.n_cells, g.term_groups, g.prec, p->cap)) != BOLTZ_OK) {
      free_plan(p);
      return st;
    }
  }
  // capture: fork every group's branch off the capture stream, join them at the end
  if ((e = cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
    free_plan(p);
    return plan_fail(e, "begin capture");
  }
  const bool serial = (flags & BOLTZ_PLAN_SERIAL) != 0;
  if ((e = cudaEventRecord(p->fork, p->cap)) != cudaSuccess) st = plan_fail(e, "fork");
  for (auto& g : p->groups) {
    if (st != BOLTZ_OK) break;
    if (g.n_cells == 0) continue;
    cudaStream_t gs = serial ? p->cap : g.stream;
    if (!serial && (e = cudaStreamWaitEvent(gs, p->fork, 0)) != cudaSuccess) {
      st = plan_fail(e, "fork");
      break;
    }
    st = boltz::relax_steps(g.grid, g.n_cells, g.prec, g.f_is_fp64, g.f, dt, steps, rk_order, gs, g.U0, g.stage,
                            g.term_groups, g.cluster);
    if (st != BOLTZ_OK) break;
    if (!serial && ((e = cudaEventRecord(g.join, gs)) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(p->cap, g.join, 0)) != cudaSuccess)) {
      st = plan_fail(e, "join");
      break;
    }
  }
  e = cudaStreamEndCapture(p->cap, &p->graph);
  if (st == BOLTZ_OK && e != cudaSuccess) st = plan_fail(e, "end capture");
  if (st == BOLTZ_OK && (e = cudaGraphInstantiate(&p->exec, p->graph, 0)) != cudaSuccess)
    st = plan_fail(e, "graph instantiate");
  if (st != BOLTZ_OK) {
    free_plan(p);
    return st;
  }
  *out = p;
  return BOLTZ_OK;
}

boltz_status boltz_plan_run(boltz_plan p, void* stream) {
  if (!p || !p->exec) {
    set_error("null plan");
    return BOLTZ_EINVAL;
  }
  cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return plan_fail(e, "graph launch");
  return BOLTZ_OK;
}

boltz_status boltz_plan_group_info(boltz_plan p, int group, int* term_groups, int* cluster, double* tuned_us) {
  if (!p || group < 0 || group >= (int)p->groups.size()) {
    set_error("bad plan group");
    return BOLTZ_EINVAL;
  }
  const PlanGroup& g = p->groups[group];
  if (term_groups) *term_groups = g.term_groups;
  if (cluster) *cluster = g.cluster;
  if (tuned_us) *tuned_us = g.tuned_us;
  return BOLTZ_OK;
}

boltz_status boltz_plan_destroy(boltz_plan p) {
  free_plan(p);
  return BOLTZ_OK;
}

}  // extern "C"
