// Ragged batches (boltz_plan_* in include/boltz.h): groups of cells on different grids
// (any mix of N_v, M_dirs, gamma, precision) advanced together by the relaxation of
// Sec. 3.1 (Eq. relax, Eq. f_coll; Heun for rk_order 2).
//
// The collision kernels are specialised per N (the register transforms have compile-time
// lengths), so a ragged step is one kernel launch per group.  The plan makes the whole
// step loop a single CUDA graph: every group's launches form one branch, branches run
// concurrently, and the host pays one graph launch per call.  Before capture an optional
// autotuner chooses each group's (term groups, cluster size) by timing the concurrent step
// (below).
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
  double tuned_step_us = 0.0;  // the autotuner's last whole-step time (0 without tuning)
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

// Autotuning.  A candidate is (term groups, cluster size) for one group.  Every group's
// candidates are first timed alone, one launch on a copy of its cells (the user's f is
// not touched; term groups only while the cells alone leave SMs idle), and the three
// fastest are kept.  Timing groups alone favours parallelism inside a group, but in the
// graph the groups run concurrently and share the SMs, so the choice is then refined on
// the step itself: starting from the grids' own settings, the groups are visited in
// order of their time alone (slowest first), each kept candidate is tried with the other
// groups fixed, and it is adopted only if the whole concurrent step gets faster by more
// than 1 %.  The result is never slower than the untuned plan beyond timing noise.
namespace {

struct Cand {
  int G = 1, cluster = 0;
  int prec = 0;    // the group's precision, or the tensor-core mode it may switch to
  float ms = 0.f;  // one launch of the group alone
};

struct TuneCopies {
  void* fa = nullptr;  // copy of the group's f (input of every timed launch)
  void* qa = nullptr;  // output of the timed launches
};

constexpr int kKeep = 3;          // candidates kept per group after timing alone
constexpr int kStepEvals = 48;    // whole-step timings at most
constexpr float kGain = 0.99f;    // adopt a candidate only if the step gets 1 % faster

boltz_status launch_candidate(const PlanGroup& g, const TuneCopies& c, const Cand& k, cudaStream_t s) {
  return boltz::launch_collide(g.grid, g.n_cells, k.prec, g.f_is_fp64, c.fa, nullptr, c.qa, 0.0, 1.0, 1e-3, g.U0, 1,
                               1, s, nullptr, 0, k.G, k.cluster);
}

boltz_status time_alone(const PlanGroup& g, const TuneCopies& c, int sms, bool tune_prec, cudaStream_t s,
                        cudaEvent_t e0, cudaEvent_t e1, std::vector<Cand>& out) {
  int cl[4];
  int ncl = boltz::cluster_choices(g.grid->N, g.prec, cl);
  // the tensor-core mode of the same N: one more candidate (default cluster, one group)
  const bool tc = tune_prec && g.prec == BOLTZ_FP32_FFT && boltz::collide_supported_grid(g.grid, BOLTZ_3XTF32_DFT);
  cudaError_t e = cudaSuccess;
  for (int ci = 0; ci < ncl + (tc ? 1 : 0); ++ci) {
    const bool tc_cand = (ci == ncl);
    for (int G = 1; G <= std::min(16, g.grid->M_eff); G *= 2) {
      if (G > 1 && (tc_cand || g.n_cells * cl[ci] * (G / 2) >= 2 * (int64_t)sms)) break;  // the GPU is full
      Cand k;
      k.G = G;
      k.cluster = tc_cand ? 0 : cl[ci];
      k.prec = tc_cand ? BOLTZ_3XTF32_DFT : g.prec;
      float best = 1e30f, ms = 0.f;
      boltz_status st = BOLTZ_OK;
      for (int rep = 0; rep < 3; ++rep) {  // rep 0 warms up (and sizes the split scratch)
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
        st = launch_candidate(g, c, k, s);
        if (st != BOLTZ_OK) break;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
            (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
          break;
        if (rep > 0) best = std::min(best, ms);
      }
      if (e != cudaSuccess) return plan_fail(e, "autotune timing");
      if (st == BOLTZ_EUNSUPPORTED) {  // not schedulable here: skip the cluster size
        cudaEventSynchronize(e0);        // the skipped candidate recorded e0 only
        break;
      }
      if (st != BOLTZ_OK) return st;
      k.ms = best;
      out.push_back(k);
    }
  }
  std::sort(out.begin(), out.end(), [](const Cand& x, const Cand& y) { return x.ms < y.ms; });
  return BOLTZ_OK;
}

// One step of every group concurrently (each on its own stream, forked from and joined to
// s), as the graph runs it; the faster of two runs.
boltz_status time_step(boltz_plan_s* p, const std::vector<TuneCopies>& copies, const std::vector<Cand>& pick,
                       cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float* out) {
  cudaError_t e;
  float best = 1e30f, ms = 0.f;
  for (int rep = 0; rep < 2; ++rep) {
    if ((e = cudaEventRecord(e0, s)) != cudaSuccess || (e = cudaEventRecord(p->fork, s)) != cudaSuccess)
      return plan_fail(e, "autotune fork");
    for (size_t i = 0; i < p->groups.size(); ++i) {
      PlanGroup& g = p->groups[i];
      if (g.n_cells == 0) continue;
      if ((e = cudaStreamWaitEvent(g.stream, p->fork, 0)) != cudaSuccess) return plan_fail(e, "autotune fork");
      boltz_status st = launch_candidate(g, copies[i], pick[i], g.stream);
      if (st != BOLTZ_OK) return st;
      if ((e = cudaEventRecord(g.join, g.stream)) != cudaSuccess || (e = cudaStreamWaitEvent(s, g.join, 0)) != cudaSuccess)
        return plan_fail(e, "autotune join");
    }
    if ((e = cudaEventRecord(e1, s)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
        (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess)
      return plan_fail(e, "autotune timing");
    best = std::min(best, ms);
  }
  *out = best;
  return BOLTZ_OK;
}

boltz_status autotune(boltz_plan_s* p, cudaStream_t s) {
  const size_t ng = p->groups.size();
  std::vector<TuneCopies> copies(ng);
  std::vector<std::vector<Cand>> cands(ng);
  std::vector<Cand> pick(ng);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e;
  boltz_status st = BOLTZ_OK;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
    st = plan_fail(e, "autotune setup");
    goto done;
  }
  for (size_t i = 0; i < ng; ++i) {
    PlanGroup& g = p->groups[i];
    pick[i].G = g.term_groups;
    pick[i].cluster = g.cluster;
    pick[i].prec = g.prec;
    if (g.n_cells == 0) continue;
    const size_t bytes = (size_t)g.n_cells * boltz::cell_points(g.grid) * (g.f_is_fp64 ? 8 : 4);
    if (cudaMalloc(&copies[i].fa, bytes) != cudaSuccess || cudaMalloc(&copies[i].qa, bytes) != cudaSuccess) {
      cudaGetLastError();
      set_error("autotune scratch allocation failed");
      st = BOLTZ_ENOMEM;
      goto done;
    }
    if ((e = cudaMemcpyAsync(copies[i].fa, g.f, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) {
      st = plan_fail(e, "autotune copy");
      goto done;
    }
    if ((st = time_alone(g, copies[i], sms, (p->flags & BOLTZ_PLAN_TUNE_PRECISION) != 0, s, e0, e1, cands[i])) !=
        BOLTZ_OK)
      goto done;
    if (cands[i].size() > (size_t)kKeep) cands[i].resize(kKeep);
    // the time alone of the grid's own setting orders the refinement
    pick[i].ms = 1e30f;
    for (const Cand& k : cands[i])
      if (k.G == pick[i].G && k.cluster == pick[i].cluster && k.prec == pick[i].prec) pick[i].ms = k.ms;
    if (pick[i].ms == 1e30f && !cands[i].empty()) pick[i].ms = cands[i].front().ms;
  }
  {
    float base = 0.f;
    if ((st = time_step(p, copies, pick, s, e0, e1, &base)) != BOLTZ_OK) goto done;  // warm-up
    if ((st = time_step(p, copies, pick, s, e0, e1, &base)) != BOLTZ_OK) goto done;
    std::vector<size_t> order;
    for (size_t i = 0; i < ng; ++i)
      if (p->groups[i].n_cells > 0) order.push_back(i);
    std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return pick[x].ms > pick[y].ms; });
    int evals = 0;
    for (size_t i : order) {
      for (const Cand& k : cands[i]) {
        if (evals >= kStepEvals) break;
        if (k.G == pick[i].G && k.cluster == pick[i].cluster && k.prec == pick[i].prec) continue;
        std::vector<Cand> trial = pick;
        trial[i] = k;
        float t = 0.f;
        if ((st = time_step(p, copies, trial, s, e0, e1, &t)) != BOLTZ_OK) goto done;
        ++evals;
        if (t < kGain * base) {
          base = t;
          pick[i] = k;
        }
      }
    }
    for (size_t i = 0; i < ng; ++i) {
      p->groups[i].term_groups = pick[i].G;
      p->groups[i].cluster = pick[i].cluster;
      p->groups[i].prec = pick[i].prec;
      p->groups[i].tuned_us = pick[i].ms * 1000.0;
    }
    p->tuned_step_us = base * 1000.0;
  }
done:
  cudaStreamSynchronize(s);
  for (auto& g : p->groups) cudaStreamSynchronize(g.stream);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (auto& c : copies) {
    cudaFree(c.fa);
    cudaFree(c.qa);
  }
  return st;
}

}  // namespace

extern "C" {

boltz_status boltz_plan_create(const boltz_group* groups, int n_groups, double dt, int steps, int rk_order,
                               int flags, void* stream, boltz_plan* out) {
  if (!groups || !out || n_groups < 1 || n_groups > 256) {
    set_error("bad plan arguments (groups, n_groups in [1, 256], out)");
    return BOLTZ_EINVAL;
  }
  if (!(dt > 0) || !(dt < 1e300) || steps < 0 || (rk_order != 1 && rk_order != 2) ||
      (flags & ~(BOLTZ_PLAN_AUTOTUNE | BOLTZ_PLAN_SERIAL | BOLTZ_PLAN_TUNE_PRECISION))) {
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
                                                                : boltz::default_cluster_for(g.grid->N, g.prec, g.term_groups);
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
  if ((flags & BOLTZ_PLAN_AUTOTUNE) && (st = autotune(p, p->cap)) != BOLTZ_OK) {
    free_plan(p);
    return st;
  }
  for (auto& g : p->groups) {
    if (g.n_cells == 0) continue;
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

boltz_status boltz_plan_group_precision(boltz_plan p, int group, int* prec) {
  if (!p || !prec || group < 0 || group >= (int)p->groups.size()) {
    set_error("bad plan group");
    return BOLTZ_EINVAL;
  }
  *prec = p->groups[group].prec;
  return BOLTZ_OK;
}

boltz_status boltz_plan_destroy(boltz_plan p) {
  free_plan(p);
  return BOLTZ_OK;
}

}  // extern "C"
