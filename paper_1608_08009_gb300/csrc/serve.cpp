// Continuous-batching server for homogeneous relaxation jobs (boltz_server_* in
// include/boltz.h).
//
// A job is a batch of one or more spatial cells of one grid relaxing under df/dt = Q(f)
// (Sec. 3.1, Eq. relax) for a given number of forward-Euler collision steps (Eq. f_coll)
// with the conservation projection of Sec. 3.2 after every step.  Jobs of different grids
// (N, L, gamma, M), sizes and step counts arrive at any time.
//
// Memory.  The server makes one device allocation, the HBM budget, and carves everything
// it uses on the device out of it: the index lists of every grid (at the end) and, per
// admitted job, its resident float32 distributions and, when the grid splits a cell's
// separated terms over several clusters (term_groups G > 1), the job's term-group scratch
// ((G + 1) N^3 values and an arrival count per cell), in one region.  A job is admitted
// when its region fits (first fit in the arena), so the reserved device memory never
// exceeds the budget and every byte a job needs is counted against it.  Regions are
// returned once the job's result has reached the host (its completion event), so no copy
// of another stream can overwrite memory still being read.
//
// Scheduling.  Each grid keeps its own first-come-first-served queue: a job that does not
// fit yet waits at the head of its grid's queue without holding back other grids (grids
// are visited round robin).  All resident cells of a grid advance with one indexed launch
// per iteration (jobs admitted while others run join the next iteration); the launch
// computes each cell's projection targets from its current f, so a cell's arithmetic does
// not depend on what else is resident and a job gives the same bits alone and in a mix.
// Each grid has its own stream and at most kDepth iterations in flight, so grids advance
// at their own pace: cheap 16^3 steps do not wait behind 64^3 steps.  boltz_server_pump
// never blocks (a grid at full depth is skipped); boltz_server_step waits for room so
// that every resident job advances by exactly one step per call.
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "internal.h"

namespace {

constexpr int kDepth = 2;             // iterations in flight per grid
constexpr int kIdxBufs = kDepth + 1;  // pinned index lists: one more than the depth

struct Job {
  int64_t id = 0;
  int grid = 0;
  int64_t cells = 1;
  int remaining = 0;
  const float* in = nullptr;
  float* out = nullptr;
  // arena region [off, off + bytes): the distributions of the job's cells, then their
  // term-group scratch blocks (none without term groups)
  size_t off = 0, bytes = 0;
  cudaEvent_t done = nullptr;     // recorded after the copy-out
  int state = 0;                  // 0 queued, 1 resident, 2 copying out, 3 finished
};

struct Pool {
  boltz_grid_s* grid = nullptr;
  size_t n = 0;           // points per cell
  size_t slot_bytes = 0;  // float32 distribution of one cell
  int G = 1;              // term groups of this grid's launches
  size_t blk_bytes = 0;   // term-group scratch of one cell (0 if G = 1)
  int64_t cap = 0;        // most cells that can be resident (index list length)
  int64_t* idx_dev = nullptr;        // [cap] slots, then [cap] scratch blocks (in the arena)
  int64_t* idx_host[kIdxBufs] = {};  // pinned, in rotation
  cudaEvent_t idx_ready[kIdxBufs] = {};
  int idx_turn = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t iter_done[kDepth] = {};  // completion of the iterations in flight, in a ring
  int iter_head = 0, in_flight = 0;
  std::deque<int64_t> queue;      // jobs of this grid waiting for admission
  std::vector<int64_t> resident;  // job ids in admission order
  int64_t resident_cells = 0;
};

// First-fit allocator over [0, limit) of the arena; offsets aligned to a multiple of the
// requested alignment (relative to the arena base, so slot = offset / slot_bytes).
class Arena {
 public:
  void init(size_t limit) {
    free_.clear();
    if (limit) free_[0] = limit;
  }
  bool alloc(size_t bytes, size_t align, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      const size_t a = it->first, sz = it->second;
      const size_t s = (a + align - 1) / align * align;
      if (s + bytes > a + sz) continue;
      const size_t tail = a + sz - (s + bytes);
      free_.erase(it);
      if (s > a) free_[a] = s - a;
      if (tail) free_[s + bytes] = tail;
      *off = s;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    if (!bytes) return;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

}  // namespace

struct boltz_server_s {
  int prec = BOLTZ_FP32_FFT;
  double dt = 0.0;
  size_t budget = 0;      // bytes of the arena (the whole device reservation)
  size_t jobs_limit = 0;  // [0, jobs_limit) holds job regions; the index lists follow
  size_t used = 0, peak = 0;
  char* arena = nullptr;
  Arena alloc;
  cudaStream_t stream = nullptr;
  std::vector<Pool> pools;
  std::vector<Job> jobs;  // indexed by id
  std::vector<int64_t> copying;  // jobs whose results are on their way to the host
  int rr = 0;                    // grid where the next admission round starts
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
    for (int b = 0; b < kIdxBufs; ++b) {
      cudaFreeHost(p.idx_host[b]);
      if (p.idx_ready[b]) cudaEventDestroy(p.idx_ready[b]);
    }
    for (int b = 0; b < kDepth; ++b)
      if (p.iter_done[b]) cudaEventDestroy(p.iter_done[b]);
    if (p.stream) cudaStreamDestroy(p.stream);
  }
  cudaFree(s->arena);
  for (auto& j : s->jobs)
    if (j.done) cudaEventDestroy(j.done);
  delete s;
}

// Return the arena regions of a job whose result has reached the host.
static void release_job(boltz_server_s* s, Job& j) {
  s->alloc.release(j.off, j.bytes);
  s->used -= j.bytes;
  j.bytes = 0;
  j.state = 3;
}

// Jobs copying out whose copy has completed give their regions back.
static boltz_status reap(boltz_server_s* s) {
  std::vector<int64_t> keep;
  for (int64_t id : s->copying) {
    Job& j = s->jobs[id];
    const cudaError_t e = cudaEventQuery(j.done);
    if (e == cudaSuccess) {
      release_job(s, j);
    } else if (e == cudaErrorNotReady) {
      keep.push_back(id);
    } else {
      return cuda_err(e, "job completion");
    }
  }
  s->copying.swap(keep);
  return BOLTZ_OK;
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
  if (prec < BOLTZ_FP64 || prec > BOLTZ_3XTF32_DFT) {
    set_error("unknown precision");
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
  // the footprint of one cell on each grid bounds its index lists; the lists sit at the
  // end of the arena, the job regions before them
  size_t idx_total = 0;
  for (int i = 0; i < n_grids; ++i) {
    Pool& p = s->pools[i];
    p.grid = grids[i];
    p.n = boltz::cell_points(grids[i]);
    p.slot_bytes = p.n * sizeof(float);
    p.G = boltz::launch_groups(grids[i], prec, -1);
    p.blk_bytes = p.G > 1 ? boltz::split_block_bytes(grids[i], p.G, prec) : 0;
    p.cap = (int64_t)(hbm_budget_bytes / (p.slot_bytes + p.blk_bytes));
    idx_total += ((size_t)p.cap * 2 * sizeof(int64_t) + 255) / 256 * 256;
  }
  if (idx_total >= hbm_budget_bytes) {
    free_server(s);
    set_error("HBM budget smaller than one cell");
    return BOLTZ_EINVAL;
  }
  s->jobs_limit = (hbm_budget_bytes - idx_total) / 256 * 256;
  for (int i = 0; i < n_grids; ++i) {
    const Pool& p = s->pools[i];
    if (p.cap < 1 || p.slot_bytes + p.blk_bytes > s->jobs_limit) {
      free_server(s);
      set_error("HBM budget smaller than one cell (with its term-group scratch) of grid " + std::to_string(i));
      return BOLTZ_EINVAL;
    }
  }
  cudaError_t e;
  if ((e = cudaMalloc(&s->arena, hbm_budget_bytes)) != cudaSuccess) {
    cudaGetLastError();  // an allocation failure is not sticky: clear it for later launches
    s->arena = nullptr;
    free_server(s);
    set_error(std::string("server arena allocation: ") + cudaGetErrorString(e));
    return BOLTZ_ENOMEM;
  }
  s->alloc.init(s->jobs_limit);
  s->used = hbm_budget_bytes - s->jobs_limit;  // the index lists
  s->peak = s->used;
  size_t idx_off = s->jobs_limit;
  for (int i = 0; i < n_grids; ++i) {
    Pool& p = s->pools[i];
    p.idx_dev = reinterpret_cast<int64_t*>(s->arena + idx_off);
    idx_off += ((size_t)p.cap * 2 * sizeof(int64_t) + 255) / 256 * 256;
    for (int b = 0; b < kIdxBufs; ++b) {
      if ((e = cudaMallocHost(&p.idx_host[b], (size_t)p.cap * 2 * sizeof(int64_t))) != cudaSuccess ||
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
  }
  *out = s;
  return BOLTZ_OK;
}

boltz_status boltz_server_destroy(boltz_server s) {
  free_server(s);
  return BOLTZ_OK;
}

boltz_status boltz_server_submit_batch(boltz_server s, int grid_index, const float* f_host, float* out_host,
                                       int64_t n_cells, int steps, int64_t* job_id) {
  if (!s || !f_host || !out_host || !job_id || grid_index < 0 || grid_index >= (int)s->pools.size() || steps < 1 ||
      n_cells < 1) {
    set_error("bad submit arguments");
    return BOLTZ_EINVAL;
  }
  const Pool& p = s->pools[grid_index];
  if (n_cells > p.cap || (size_t)n_cells * (p.slot_bytes + p.blk_bytes) > s->jobs_limit) {
    set_error("job larger than the server's HBM budget (distributions plus term-group scratch)");
    return BOLTZ_EINVAL;
  }
  Job j;
  j.id = (int64_t)s->jobs.size();
  j.grid = grid_index;
  j.cells = n_cells;
  j.remaining = steps;
  j.in = f_host;
  j.out = out_host;
  cudaError_t e = cudaEventCreateWithFlags(&j.done, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_err(e, "job event");
  s->jobs.push_back(j);
  s->pools[grid_index].queue.push_back(j.id);
  *job_id = j.id;
  return BOLTZ_OK;
}

boltz_status boltz_server_submit(boltz_server s, int grid_index, const float* f_host, float* out_host, int steps,
                                 int64_t* job_id) {
  return boltz_server_submit_batch(s, grid_index, f_host, out_host, 1, steps, job_id);
}

}  // extern "C"

// Admission of queued jobs into the arena: every grid's queue in turn (round robin), each
// first come first served while the head job's regions fit.  Returns whether a queue head
// is left waiting for memory.
static boltz_status admit(boltz_server_s* s, bool* blocked) {
  *blocked = false;
  cudaError_t e;
  const int ng = (int)s->pools.size();
  for (int k = 0; k < ng; ++k) {
    Pool& p = s->pools[(s->rr + k) % ng];
    while (!p.queue.empty()) {
      Job& j = s->jobs[p.queue.front()];
      // one region: the distributions (aligned so that slot = offset / slot bytes), then
      // the scratch blocks
      const size_t fb = (size_t)j.cells * p.slot_bytes, sb = (size_t)j.cells * p.blk_bytes;
      size_t off = 0;
      if (p.resident_cells + j.cells > p.cap || !s->alloc.alloc(fb + sb, p.slot_bytes, &off)) {
        *blocked = true;
        break;
      }
      j.off = off;
      j.bytes = fb + sb;
      s->used += j.bytes;
      if (s->used > s->peak) s->peak = s->used;
      if ((e = cudaMemcpyAsync(s->arena + off, j.in, fb, cudaMemcpyHostToDevice, p.stream)) != cudaSuccess)
        return cuda_err(e, "admission copy");
      // arrival counts start at zero (each launch leaves them at zero)
      if (sb && (e = cudaMemsetAsync(s->arena + off + fb, 0, sb, p.stream)) != cudaSuccess)
        return cuda_err(e, "scratch clear");
      j.state = 1;
      p.resident.push_back(j.id);
      p.resident_cells += j.cells;
      p.queue.pop_front();
    }
  }
  if (ng) s->rr = (s->rr + 1) % ng;
  return BOLTZ_OK;
}

// Admission, then one iteration for every grid with resident jobs and room in its depth
// (blocking: wait for room; otherwise skip the grid).  *launched counts the iterations
// issued.
static boltz_status advance(boltz_server s, bool blocking, int* n_resident, int* n_queued, int* launched) {
  if (!s) {
    set_error("null server");
    return BOLTZ_EINVAL;
  }
  cudaError_t e;
  boltz_status st = reap(s);
  if (st != BOLTZ_OK) return st;
  bool blocked = false;
  if ((st = admit(s, &blocked)) != BOLTZ_OK) return st;
  if (blocking && blocked && !s->copying.empty()) {
    // a queued job waits for memory that finished jobs return once their results have
    // reached the host: wait for those copies, then admit again
    for (int64_t id : s->copying)
      if ((e = cudaEventSynchronize(s->jobs[id].done)) != cudaSuccess) return cuda_err(e, "job completion");
    if ((st = reap(s)) != BOLTZ_OK) return st;
    if ((st = admit(s, &blocked)) != BOLTZ_OK) return st;
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
    // one collision step for every resident cell of this grid: one indexed launch; slots
    // are arena offsets over the slot size, scratch blocks arena offsets in split units
    const int b = p.idx_turn;
    p.idx_turn = (p.idx_turn + 1) % kIdxBufs;
    if ((e = cudaEventSynchronize(p.idx_ready[b])) != cudaSuccess) return cuda_err(e, "index buffer");
    const int64_t m = p.resident_cells;
    int64_t* slots = p.idx_host[b];
    int64_t* blks = p.idx_host[b] + p.cap;
    int64_t k = 0;
    for (int64_t id : p.resident) {
      const Job& j = s->jobs[id];
      const int64_t s0 = (int64_t)(j.off / p.slot_bytes);
      const size_t sbase = j.off + (size_t)j.cells * p.slot_bytes;  // the job's scratch blocks
      for (int64_t c = 0; c < j.cells; ++c, ++k) {
        slots[k] = s0 + c;
        blks[k] = (int64_t)((sbase + (size_t)c * p.blk_bytes) / boltz::kSplitUnit);
      }
    }
    if ((e = cudaMemcpyAsync(p.idx_dev, slots, (size_t)m * sizeof(int64_t), cudaMemcpyHostToDevice, p.stream)) !=
        cudaSuccess)
      return cuda_err(e, "index copy");
    if (p.blk_bytes &&
        (e = cudaMemcpyAsync(p.idx_dev + p.cap, blks, (size_t)m * sizeof(int64_t), cudaMemcpyHostToDevice,
                             p.stream)) != cudaSuccess)
      return cuda_err(e, "index copy");
    if ((e = cudaEventRecord(p.idx_ready[b], p.stream)) != cudaSuccess) return cuda_err(e, "index event");
    st = boltz::launch_collide(p.grid, m, s->prec, 0, s->arena, nullptr, s->arena, 0.0, 1.0, s->dt, nullptr, 1, 1,
                               p.stream, p.idx_dev, (int64_t)(s->jobs_limit / p.slot_bytes), p.G, 0,
                               p.blk_bytes ? p.idx_dev + p.cap : nullptr, s->arena);
    if (st != BOLTZ_OK) return st;
    // retire finished jobs: copy out; their regions return to the arena once the copy
    // has completed (reap)
    std::vector<int64_t> keep;
    keep.reserve(p.resident.size());
    for (int64_t id : p.resident) {
      Job& j = s->jobs[id];
      if (--j.remaining > 0) {
        keep.push_back(id);
        continue;
      }
      if ((e = cudaMemcpyAsync(j.out, s->arena + j.off, (size_t)j.cells * p.slot_bytes, cudaMemcpyDeviceToHost,
                               p.stream)) !=
          cudaSuccess)
        return cuda_err(e, "result copy");
      if ((e = cudaEventRecord(j.done, p.stream)) != cudaSuccess) return cuda_err(e, "job event");
      j.state = 2;
      p.resident_cells -= j.cells;
      s->copying.push_back(id);
    }
    p.resident.swap(keep);
    if ((e = cudaEventRecord(p.iter_done[p.iter_head], p.stream)) != cudaSuccess) return cuda_err(e, "iteration event");
    p.iter_head = (p.iter_head + 1) % kDepth;
    ++p.in_flight;
    ++issued;
  }
  if (n_resident) {
    int64_t r = 0;
    for (auto& p : s->pools) r += (int64_t)p.resident.size();
    *n_resident = (int)r;
  }
  if (n_queued) {
    int64_t q = 0;
    for (auto& p : s->pools) q += (int64_t)p.queue.size();
    *n_queued = (int)q;
  }
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
  const size_t bytes = (size_t)j.cells * p.slot_bytes;
  cudaError_t e;
  if (j.state == 0) {  // still queued: its state is the submitted one
    std::memcpy(f_host, j.in, bytes);
  } else if (j.state == 1) {  // resident: the state after the iterations issued so far
    if ((e = cudaMemcpyAsync(f_host, s->arena + j.off, bytes, cudaMemcpyDeviceToHost, p.stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(p.stream)) != cudaSuccess)
      return cuda_err(e, "checkpoint copy");
  } else {  // finished or copying out: the result
    if ((e = cudaEventSynchronize(j.done)) != cudaSuccess) return cuda_err(e, "checkpoint wait");
    std::memcpy(f_host, j.out, bytes);
  }
  *remaining_steps = (j.state >= 2) ? 0 : j.remaining;
  return BOLTZ_OK;
}

boltz_status boltz_server_poll(boltz_server s, int64_t job_id, int* done) {
  if (!s || !done || job_id < 0 || job_id >= (int64_t)s->jobs.size()) {
    set_error("bad poll arguments");
    return BOLTZ_EINVAL;
  }
  boltz_status st = reap(s);
  if (st != BOLTZ_OK) return st;
  *done = (s->jobs[job_id].state == 3) ? 1 : 0;
  return BOLTZ_OK;
}

boltz_status boltz_server_stats_get(boltz_server s, boltz_server_stats* out) {
  if (!s || !out) {
    set_error("bad stats arguments");
    return BOLTZ_EINVAL;
  }
  boltz_status st = reap(s);
  if (st != BOLTZ_OK) return st;
  out->reserved_bytes = s->budget;
  out->used_bytes = s->used;
  out->peak_used_bytes = s->peak;
  out->resident_cells = 0;
  out->resident_jobs = 0;
  out->queued_jobs = 0;
  for (const auto& p : s->pools) {
    out->resident_cells += p.resident_cells;
    out->resident_jobs += (int64_t)p.resident.size();
    out->queued_jobs += (int64_t)p.queue.size();
  }
  return BOLTZ_OK;
}

}  // extern "C"
