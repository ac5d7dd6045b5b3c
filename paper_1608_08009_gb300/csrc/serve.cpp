// Continuous-batching server for homogeneous relaxation jobs (boltz_server_* in
// include/boltz.h).
//
// A job is one spatial cell relaxing under df/dt = Q(f) (Sec. 3.1, Eq. relax) for a given
// number of forward-Euler collision steps (Eq. f_coll) with the conservation projection
// of Sec. 3.2 after every step.  Jobs of different grids (N, L, gamma, M) and step counts
// arrive at any time.  The server keeps every admitted job's distribution resident in a
// per-grid device pool of float32 slots, admits queued jobs as soon as the HBM budget
// and a slot allow, advances all resident jobs of a grid with one indexed launch per
// iteration (jobs admitted while others run join the next iteration), and retires
// finished jobs with an asynchronous copy back to the caller's host buffer.  Every job
// is computed by the same per-cell arithmetic whatever else is resident, so its result
// does not depend on the mix.
//
// Each grid has its own stream and at most kDepth iterations in flight, so grids advance
// at their own pace: cheap 16^3 steps do not wait behind 64^3 steps.  boltz_server_pump
// never blocks (a grid at full depth is skipped); boltz_server_step waits for room so that
// every resident job advances by exactly one step per call.
#include <cstring>
#include <deque>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace {

struct Job {
  int64_t id = 0;
  int grid = 0;
  int64_t slot = -1;
  int remaining = 0;
  const float* in = nullptr;
  float* out = nullptr;
  cudaEvent_t done = nullptr;  // recorded after the copy-out
  int state = 0;               // 0 queued, 1 resident, 2 copying out, 3 finished
};

constexpr int kDepth = 2;              // iterations in flight per grid
constexpr int kIdxBufs = kDepth + 1;   // pinned index lists: one more than the depth

struct Pool {
  boltz_grid_s* grid = nullptr;
  size_t n = 0;                 // N^3
  size_t slot_bytes = 0;
  int64_t capacity = 0;         // slots
  float* f = nullptr;           // [capacity][n]
  int64_t* idx_dev = nullptr;   // [capacity]
  int64_t* idx_host[kIdxBufs] = {};  // pinned, in rotation
  cudaEvent_t idx_ready[kIdxBufs] = {};
  int idx_turn = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t iter_done[kDepth] = {};  // completion of the iterations in flight, in a ring
  int iter_head = 0, in_flight = 0;
  std::vector<int64_t> free_slots;
  std::vector<int64_t> resident;  // job ids in admission order
};

}  // namespace

struct boltz_server_s {
  int prec = BOLTZ_FP32_FFT;
  double dt = 0.0;
  size_t budget = 0, used = 0;
  cudaStream_t stream = nullptr;
  std::vector<Pool> pools;
  std::deque<int64_t> queue;  // job ids waiting for admission
  std::vector<Job> jobs;      // indexed by id
};

using boltz::set_error;

static boltz_status cuda_err(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return BOLTZ_ECUDA;
}

static void free_server(boltz_server_s* s) {
  if (!s) return;
  for (auto& p : s->pools)
    if (p.stream) cudaStreamSynchronize(p.stream);
  for (auto& p : s->pools) {
    cudaFree(p.f);
    cudaFree(p.idx_dev);
    for (int b = 0; b < kIdxBufs; ++b) {
      cudaFreeHost(p.idx_host[b]);
      if (p.idx_ready[b]) cudaEventDestroy(p.idx_ready[b]);
    }
    for (int b = 0; b < kDepth; ++b)
      if (p.iter_done[b]) cudaEventDestroy(p.iter_done[b]);
    if (p.stream) cudaStreamDestroy(p.stream);
  }
  for (auto& j : s->jobs)
    if (j.done) cudaEventDestroy(j.done);
  delete s;
}

extern "C" {

boltz_status boltz_server_create(const boltz_grid* grids, int n_grids, int prec, double dt, size_t hbm_budget_bytes,
                                 void* stream, boltz_server* out) {
  if (!out || !grids || n_grids < 1 || n_grids > 64) {
    set_error("bad server arguments (grids, n_grids in [1, 64], out)");
    return BOLTZ_EINVAL;
  }
  if (!(dt > 0) || !(dt < 1e300) || hbm_budget_bytes == 0) {
    set_error("dt must be positive and finite, the budget positive");
    return BOLTZ_EINVAL;
  }
  for (int i = 0; i < n_grids; ++i) {
    if (!grids[i] || !boltz::collide_supported_grid(grids[i], prec)) {
      set_error("null grid or unsupported (N, precision)");
      return grids[i] ? BOLTZ_EUNSUPPORTED : BOLTZ_EINVAL;
    }
  }
  boltz_server_s* s = new (std::nothrow) boltz_server_s();
  if (!s) {
    set_error("out of host memory");
    return BOLTZ_ENOMEM;
  }
  s->prec = prec;
  s->dt = dt;
  s->budget = hbm_budget_bytes;
  s->stream = (cudaStream_t)stream;
  s->pools.resize(n_grids);
  for (int i = 0; i < n_grids; ++i) {
    Pool& p = s->pools[i];
    p.grid = grids[i];
    p.n = boltz::cell_points(grids[i]);
    p.slot_bytes = p.n * sizeof(float);
    p.capacity = (int64_t)(hbm_budget_bytes / p.slot_bytes);
    if (p.capacity < 1) {
      free_server(s);
      set_error("HBM budget smaller than one cell");
      return BOLTZ_EINVAL;
    }
    cudaError_t e;
    if ((e = cudaMalloc(&p.f, (size_t)p.capacity * p.slot_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&p.idx_dev, (size_t)p.capacity * sizeof(int64_t))) != cudaSuccess) {
      cudaGetLastError();  // an allocation failure is not sticky: clear it for later launches
      free_server(s);
      set_error(std::string("server pool allocation: ") + cudaGetErrorString(e));
      return BOLTZ_ENOMEM;
    }
    for (int b = 0; b < kIdxBufs; ++b) {
      if ((e = cudaMallocHost(&p.idx_host[b], (size_t)p.capacity * sizeof(int64_t))) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&p.idx_ready[b], cudaEventDisableTiming)) != cudaSuccess) {
        cudaGetLastError();
        free_server(s);
        set_error(std::string("server host buffers: ") + cudaGetErrorString(e));
        return BOLTZ_ENOMEM;
      }
    }
    if ((e = cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking)) != cudaSuccess) {
      free_server(s);
      return cuda_err(e, "server stream");
    }
    for (int b = 0; b < kDepth; ++b) {
      if ((e = cudaEventCreateWithFlags(&p.iter_done[b], cudaEventDisableTiming)) != cudaSuccess) {
        free_server(s);
        return cuda_err(e, "server events");
      }
    }
    // the grid's stream starts after the work already queued on the caller's stream
    cudaEvent_t start;
    if ((e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming)) != cudaSuccess) {
      free_server(s);
      return cuda_err(e, "server events");
    }
    e = cudaEventRecord(start, s->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p.stream, start, 0);
    cudaEventDestroy(start);
    if (e != cudaSuccess) {
      free_server(s);
      return cuda_err(e, "server stream order");
    }
    p.free_slots.reserve(p.capacity);
    for (int64_t k = p.capacity - 1; k >= 0; --k) p.free_slots.push_back(k);
  }
  *out = s;
  return BOLTZ_OK;
}

boltz_status boltz_server_destroy(boltz_server s) {
  free_server(s);
  return BOLTZ_OK;
}

boltz_status boltz_server_submit(boltz_server s, int grid_index, const float* f_host, float* out_host, int steps,
                                 int64_t* job_id) {
  if (!s || !f_host || !out_host || !job_id || grid_index < 0 || grid_index >= (int)s->pools.size() || steps < 1) {
    set_error("bad submit arguments");
    return BOLTZ_EINVAL;
  }
  Job j;
  j.id = (int64_t)s->jobs.size();
  j.grid = grid_index;
  j.remaining = steps;
  j.in = f_host;
  j.out = out_host;
  cudaError_t e = cudaEventCreateWithFlags(&j.done, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_err(e, "job event");
  s->jobs.push_back(j);
  s->queue.push_back(j.id);
  *job_id = j.id;
  return BOLTZ_OK;
}

}  // extern "C"

// Admission, then one iteration for every grid with resident jobs and room in its depth
// (blocking: wait for room; otherwise skip the grid).  *launched counts the iterations
// issued.
static boltz_status advance(boltz_server s, bool blocking, int* n_resident, int* n_queued, int* launched) {
  if (!s) {
    set_error("null server");
    return BOLTZ_EINVAL;
  }
  cudaError_t e;
  // admission, first come first served: a free slot of the job's grid and HBM budget
  while (!s->queue.empty()) {
    Job& j = s->jobs[s->queue.front()];
    Pool& p = s->pools[j.grid];
    if (p.free_slots.empty() || s->used + p.slot_bytes > s->budget) break;
    j.slot = p.free_slots.back();
    p.free_slots.pop_back();
    s->used += p.slot_bytes;
    if ((e = cudaMemcpyAsync(p.f + (size_t)j.slot * p.n, j.in, p.slot_bytes, cudaMemcpyHostToDevice, p.stream)) !=
        cudaSuccess)
      return cuda_err(e, "admission copy");
    j.state = 1;
    p.resident.push_back(j.id);
    s->queue.pop_front();
  }
  int issued = 0;
  for (auto& p : s->pools) {
    // iterations that have finished leave the ring
    while (p.in_flight > 0) {
      const int oldest = (p.iter_head - p.in_flight + kDepth) % kDepth;
      e = cudaEventQuery(p.iter_done[oldest]);
      if (e == cudaErrorNotReady) break;
      if (e != cudaSuccess) return cuda_err(e, "iteration event");
      --p.in_flight;
    }
    if (p.resident.empty()) continue;
    if (p.in_flight >= kDepth) {
      if (!blocking) continue;
      const int oldest = (p.iter_head - p.in_flight + kDepth) % kDepth;
      if ((e = cudaEventSynchronize(p.iter_done[oldest])) != cudaSuccess) return cuda_err(e, "iteration event");
      --p.in_flight;
    }
    // one collision step for every resident job of this grid: one indexed launch
    const int b = p.idx_turn;
    p.idx_turn = (p.idx_turn + 1) % kIdxBufs;
    if ((e = cudaEventSynchronize(p.idx_ready[b])) != cudaSuccess) return cuda_err(e, "index buffer");
    const int64_t m = (int64_t)p.resident.size();
    for (int64_t k = 0; k < m; ++k) p.idx_host[b][k] = s->jobs[p.resident[k]].slot;
    if ((e = cudaMemcpyAsync(p.idx_dev, p.idx_host[b], (size_t)m * sizeof(int64_t), cudaMemcpyHostToDevice,
                             p.stream)) != cudaSuccess)
      return cuda_err(e, "index copy");
    if ((e = cudaEventRecord(p.idx_ready[b], p.stream)) != cudaSuccess) return cuda_err(e, "index event");
    boltz_status st = boltz::launch_collide(p.grid, m, s->prec, 0, p.f, nullptr, p.f, 0.0, 1.0, s->dt, nullptr, 1, 1,
                                            p.stream, p.idx_dev, p.capacity);
    if (st != BOLTZ_OK) return st;
    // retire finished jobs: copy out, release the slot (later copies into it are ordered
    // after this copy on the same stream)
    std::vector<int64_t> keep;
    keep.reserve(p.resident.size());
    for (int64_t id : p.resident) {
      Job& j = s->jobs[id];
      if (--j.remaining > 0) {
        keep.push_back(id);
        continue;
      }
      if ((e = cudaMemcpyAsync(j.out, p.f + (size_t)j.slot * p.n, p.slot_bytes, cudaMemcpyDeviceToHost,
                               p.stream)) != cudaSuccess)
        return cuda_err(e, "result copy");
      if ((e = cudaEventRecord(j.done, p.stream)) != cudaSuccess) return cuda_err(e, "job event");
      j.state = 2;
      p.free_slots.push_back(j.slot);
      s->used -= p.slot_bytes;
    }
    p.resident.swap(keep);
    if ((e = cudaEventRecord(p.iter_done[p.iter_head], p.stream)) != cudaSuccess) return cuda_err(e, "iteration event");
    p.iter_head = (p.iter_head + 1) % kDepth;
    ++p.in_flight;
    ++issued;
  }
  if (n_resident) {
    int r = 0;
    for (auto& p : s->pools) r += (int)p.resident.size();
    *n_resident = r;
  }
  if (n_queued) *n_queued = (int)s->queue.size();
  if (launched) *launched = issued;
  return BOLTZ_OK;
}

extern "C" {

boltz_status boltz_server_step(boltz_server s, int* n_resident, int* n_queued) {
  return advance(s, true, n_resident, n_queued, nullptr);
}

boltz_status boltz_server_pump(boltz_server s, int* n_resident, int* n_queued, int* n_launched) {
  return advance(s, false, n_resident, n_queued, n_launched);
}

boltz_status boltz_server_checkpoint(boltz_server s, int64_t job_id, float* f_host, int* remaining_steps) {
  if (!s || !f_host || !remaining_steps || job_id < 0 || job_id >= (int64_t)s->jobs.size()) {
    set_error("bad checkpoint arguments");
    return BOLTZ_EINVAL;
  }
  Job& j = s->jobs[job_id];
  Pool& p = s->pools[j.grid];
  cudaError_t e;
  if (j.state == 0) {  // still queued: its state is the submitted one
    std::memcpy(f_host, j.in, p.slot_bytes);
  } else if (j.state == 1) {  // resident: the state after the iterations issued so far
    if ((e = cudaMemcpyAsync(f_host, p.f + (size_t)j.slot * p.n, p.slot_bytes, cudaMemcpyDeviceToHost, p.stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(p.stream)) != cudaSuccess)
      return cuda_err(e, "checkpoint copy");
  } else {  // finished or copying out: the result
    if ((e = cudaEventSynchronize(j.done)) != cudaSuccess) return cuda_err(e, "checkpoint wait");
    std::memcpy(f_host, j.out, p.slot_bytes);
  }
  *remaining_steps = (j.state >= 2) ? 0 : j.remaining;
  return BOLTZ_OK;
}

boltz_status boltz_server_poll(boltz_server s, int64_t job_id, int* done) {
  if (!s || !done || job_id < 0 || job_id >= (int64_t)s->jobs.size()) {
    set_error("bad poll arguments");
    return BOLTZ_EINVAL;
  }
  Job& j = s->jobs[job_id];
  if (j.state == 2) {
    cudaError_t e = cudaEventQuery(j.done);
    if (e == cudaSuccess) {
      j.state = 3;
    } else if (e != cudaErrorNotReady) {
      return cuda_err(e, "job completion");
    }
  }
  *done = (j.state == 3) ? 1 : 0;
  return BOLTZ_OK;
}

}  // extern "C"
