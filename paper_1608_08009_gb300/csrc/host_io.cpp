// boltz_relax_host (include/boltz.h): the relaxation of Sec. 3.1 (Eq. relax, Eq. f_coll)
// for distributions that live in host memory.
//
// The batch goes through the device in chunks of cells.  Three staging buffers rotate
// between three streams: the upload of chunk i (stream `up`), the collision steps of
// chunk i - 1 (the caller's stream) and the download of chunk i - 2 (stream `down`) run
// at the same time, so with page-locked host memory both copy directions hide behind the
// compute, except the upload of the first chunk and the download of the last.  The
// default schedule therefore starts and ends with small chunks and grows (shrinks) them
// by 3/2 per chunk towards the middle size: each upload still fits in the compute of the
// chunk before it as long as copies run at least 1.5 times faster per cell than the
// steps.  Each chunk runs exactly the launches boltz_relax would run on it, and cells are
// independent, so the result equals boltz_relax on the whole batch bit for bit.
#include <algorithm>
#include <string>

#include "internal.h"

namespace boltz {

static boltz_status fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return BOLTZ_ECUDA;
}

// Chunk sizes for n_cells cells of cell_bytes bytes (see boltz_host_chunks).
std::vector<int64_t> host_chunks(int64_t n_cells, int64_t cell_bytes, int64_t chunk_cells) {
  std::vector<int64_t> out;
  if (n_cells <= 0) return out;
  const int64_t cb = std::max<int64_t>(1, cell_bytes);
  const auto cells_of = [cb](int64_t bytes) { return std::max<int64_t>(1, bytes / cb); };
  const int64_t cap = cells_of((int64_t)1 << 30);  // at most 1 GiB of f per chunk
  if (chunk_cells > 0) {
    const int64_t c = std::min(chunk_cells, n_cells);
    for (int64_t c0 = 0; c0 < n_cells; c0 += c) out.push_back(std::min(c, n_cells - c0));
    return out;
  }
  // middle size: an eighth of the batch, at least 64 MiB of f; ramps from 32 MiB
  const int64_t mid = std::min(std::min(n_cells, cap), std::max((n_cells + 7) / 8, cells_of((int64_t)64 << 20)));
  std::vector<int64_t> ramp;
  int64_t ramp_sum = 0;
  for (int64_t c = std::min(cells_of((int64_t)32 << 20), mid); c < mid; c += std::max<int64_t>(1, c / 2)) {
    ramp.push_back(c);
    ramp_sum += c;
  }
  if (ramp.empty() || 2 * ramp_sum + mid > n_cells) {
    // too small for the ramps: about eight equal chunks of at least 64 MiB
    const int64_t c = std::min(cap, std::max((n_cells + 7) / 8, std::min(n_cells, cells_of((int64_t)64 << 20))));
    for (int64_t c0 = 0; c0 < n_cells; c0 += c) out.push_back(std::min(c, n_cells - c0));
    return out;
  }
  const int64_t rest = n_cells - 2 * ramp_sum;
  const int64_t k = (rest + mid - 1) / mid;  // middle chunks of equal size (within one cell)
  out = ramp;
  for (int64_t i = 0; i < k; ++i) out.push_back(rest / k + (i < rest % k ? 1 : 0));
  out.insert(out.end(), ramp.rbegin(), ramp.rend());
  return out;
}

void free_host_pipeline(boltz_grid_s* g) {
  for (int k = 0; k < boltz_grid_s::kHostBufs; ++k) {
    cudaFree(g->hbuf[k]);
    g->hbuf[k] = nullptr;
    if (g->ev_in[k]) cudaEventDestroy(g->ev_in[k]);
    if (g->ev_done[k]) cudaEventDestroy(g->ev_done[k]);
    if (g->ev_out[k]) cudaEventDestroy(g->ev_out[k]);
    g->ev_in[k] = g->ev_done[k] = g->ev_out[k] = nullptr;
  }
  cudaFree(g->hU0);
  cudaFree(g->hstage);
  g->hU0 = nullptr;
  g->hstage = nullptr;
  g->hbuf_cap = 0;
  g->hchunk_cap = 0;
  if (g->ev_start) cudaEventDestroy(g->ev_start);
  if (g->up) cudaStreamDestroy(g->up);
  if (g->down) cudaStreamDestroy(g->down);
  g->ev_start = nullptr;
  g->up = g->down = nullptr;
}

// Streams, events and buffers for chunks of `chunk` cells of `esz`-byte values.
static boltz_status ensure_pipeline(boltz_grid_s* g, int64_t chunk, size_t esz, cudaStream_t s) {
  cudaError_t e;
  if (!g->up) {
    if ((e = cudaStreamCreateWithFlags(&g->up, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&g->down, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&g->ev_start, cudaEventDisableTiming)) != cudaSuccess)
      return fail(e, "host pipeline streams");
    for (int k = 0; k < boltz_grid_s::kHostBufs; ++k) {
      if ((e = cudaEventCreateWithFlags(&g->ev_in[k], cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&g->ev_done[k], cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&g->ev_out[k], cudaEventDisableTiming)) != cudaSuccess)
        return fail(e, "host pipeline events");
    }
  }
  const size_t n = cell_points(g);
  const size_t bytes = (size_t)chunk * n * esz;
  if (bytes > g->hbuf_cap || (size_t)chunk > g->hchunk_cap) {
    // earlier work of this grid may still use the old buffers
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "host pipeline sync");
    if ((e = cudaStreamSynchronize(g->up)) != cudaSuccess || (e = cudaStreamSynchronize(g->down)) != cudaSuccess)
      return fail(e, "host pipeline sync");
    for (int k = 0; k < boltz_grid_s::kHostBufs; ++k) {
      cudaFree(g->hbuf[k]);
      g->hbuf[k] = nullptr;
    }
    cudaFree(g->hU0);
    cudaFree(g->hstage);
    g->hU0 = nullptr;
    g->hstage = nullptr;
    g->hbuf_cap = 0;
    g->hchunk_cap = 0;
    for (int k = 0; k < boltz_grid_s::kHostBufs; ++k)
      if (cudaMalloc(&g->hbuf[k], bytes) != cudaSuccess) goto oom;
    if (cudaMalloc(&g->hU0, (size_t)chunk * 5 * sizeof(double)) != cudaSuccess) goto oom;
    if (cudaMalloc(&g->hstage, bytes) != cudaSuccess) goto oom;
    g->hbuf_cap = bytes;
    g->hchunk_cap = (size_t)chunk;
  }
  return BOLTZ_OK;
oom:
  cudaGetLastError();
  set_error("host pipeline staging allocation failed");
  return BOLTZ_ENOMEM;
}

}  // namespace boltz

using boltz::set_error;

extern "C" {

boltz_status boltz_relax_host(const boltz_batch* b, const void* f_in, void* f_out, double dt, int steps,
                              int rk_order, int64_t chunk_cells, void* stream) {
  boltz_status st = boltz::check_batch(b);
  if (st != BOLTZ_OK) return st;
  if (!(dt > 0) || !(dt < 1e300)) {
    set_error("dt must be positive and finite");
    return BOLTZ_EINVAL;
  }
  if (steps < 0 || (rk_order != 1 && rk_order != 2) || chunk_cells < 0) {
    set_error("steps must be >= 0, rk_order 1 or 2, chunk_cells >= 0");
    return BOLTZ_EINVAL;
  }
  if (b->n_cells == 0) return BOLTZ_OK;
  if (!f_in || !f_out) {
    set_error("null host buffer");
    return BOLTZ_EINVAL;
  }
  if ((st = boltz::check_device(b->grid)) != BOLTZ_OK) return st;
  boltz_grid_s* g = b->grid;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = boltz::cell_points(g);
  const size_t esz = b->f_is_fp64 ? 8 : 4;
  std::vector<int64_t> chunks;
  try {
    chunks = boltz::host_chunks(b->n_cells, (int64_t)(n * esz), chunk_cells);
  } catch (...) {
    set_error("host chunk schedule: out of host memory");
    return BOLTZ_ENOMEM;
  }
  const int64_t chunk = *std::max_element(chunks.begin(), chunks.end());
  if ((st = boltz::ensure_pipeline(g, chunk, esz, s)) != BOLTZ_OK) return st;

  cudaError_t e;
  // the copy streams start after everything already on the caller's stream (which is
  // itself ordered after the previous call's last download)
  if ((e = cudaEventRecord(g->ev_start, s)) != cudaSuccess) return boltz::fail(e, "event");
  if ((e = cudaStreamWaitEvent(g->up, g->ev_start, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(g->down, g->ev_start, 0)) != cudaSuccess)
    return boltz::fail(e, "stream wait");
  const char* src = static_cast<const char*>(f_in);
  char* dst = static_cast<char*>(f_out);
  const int64_t n_chunks = (int64_t)chunks.size();
  int last = 0;
  int64_t c0 = 0;
  for (int64_t i = 0; i < n_chunks; c0 += chunks[(size_t)i], ++i) {
    const int k = (int)(i % boltz_grid_s::kHostBufs);
    const int64_t cells = chunks[(size_t)i];
    const size_t off = (size_t)c0 * n * esz, bytes = (size_t)cells * n * esz;
    if (i >= boltz_grid_s::kHostBufs && (e = cudaStreamWaitEvent(g->up, g->ev_out[k], 0)) != cudaSuccess)
      return boltz::fail(e, "stream wait");
    if ((e = cudaMemcpyAsync(g->hbuf[k], src + off, bytes, cudaMemcpyHostToDevice, g->up)) != cudaSuccess)
      return boltz::fail(e, "upload");
    if ((e = cudaEventRecord(g->ev_in[k], g->up)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(s, g->ev_in[k], 0)) != cudaSuccess)
      return boltz::fail(e, "upload event");
    st = boltz::relax_steps(g, cells, b->prec, b->f_is_fp64, g->hbuf[k], dt, steps, rk_order, s, g->hU0,
                            g->hstage);
    if (st != BOLTZ_OK) return st;
    if ((e = cudaEventRecord(g->ev_done[k], s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(g->down, g->ev_done[k], 0)) != cudaSuccess)
      return boltz::fail(e, "compute event");
    if ((e = cudaMemcpyAsync(dst + off, g->hbuf[k], bytes, cudaMemcpyDeviceToHost, g->down)) != cudaSuccess)
      return boltz::fail(e, "download");
    if ((e = cudaEventRecord(g->ev_out[k], g->down)) != cudaSuccess) return boltz::fail(e, "download event");
    last = k;
  }
  // downloads are in order on one stream: waiting for the last one covers them all
  if ((e = cudaStreamWaitEvent(s, g->ev_out[last], 0)) != cudaSuccess) return boltz::fail(e, "stream wait");
  return BOLTZ_OK;
}

int64_t boltz_host_chunks(int64_t n_cells, int64_t cell_bytes, int64_t chunk_cells, int64_t* sizes, int64_t cap) {
  if (n_cells < 0 || cell_bytes <= 0 || chunk_cells < 0 || cap < 0 || (cap > 0 && !sizes)) {
    set_error("boltz_host_chunks: n_cells, chunk_cells, cap >= 0, cell_bytes > 0, sizes non-null when cap > 0");
    return -1;
  }
  std::vector<int64_t> c;
  try {
    c = boltz::host_chunks(n_cells, cell_bytes, chunk_cells);
  } catch (...) {
    set_error("boltz_host_chunks: out of host memory");
    return -1;
  }
  for (int64_t i = 0; i < cap && i < (int64_t)c.size(); ++i) sizes[i] = c[(size_t)i];
  return (int64_t)c.size();
}

}  // extern "C"
