"""Throughput benchmark of the fast spectral Boltzmann collision step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload mixed32|fp64_32] [--cells C]

One step = one fused collision step of every cell of the batch: moments of f (float64),
forward transform, the angular loop over the M quadrature directions, loss term,
conservation projection and the update f <- f + dt Q (boltz_relax with steps = 1).
Metric: cell-collisions per second.

Workloads (synthetic, seeded two-Maxwellian cells; no dataset is involved):
  mixed32  -- 32768 cells x 32^3, VHS gamma = 1, M = 64 (8 x 8 product grid), L = 8,
              dt = 0.0025, f stored float32, transforms float32, moments / projection /
              update float64.  Default.
  fp64_32  -- 4096 cells x 32^3, same physics, float64 everywhere (the plain form).
  mixed32_f64 -- 16384 cells x 32^3, float32 transforms with f stored in float64.

The reference arm (--impl reference) times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# dt: forward Euler is stable while dt * max_v L(v) < 2; the densest cells of these inputs
# (rho = 4, T = 0.5) reach max L ~ 500 on [-8, 8)^3 and ~ 350 on [-6, 6)^3 (the loss
# rate grows with the truncation radius R = 4L / (3 + sqrt 2)), so dt = 0.0025 keeps
# dt * max L <= 1.25 for any number of steps.
WORKLOADS = {
    "mixed32": dict(cells=32768, N=32, L=8.0, M=64, gamma=1.0, dt=0.0025, prec="fp32_fft", f64=False, seed=20163),
    "fp64_32": dict(cells=4096, N=32, L=8.0, M=64, gamma=1.0, dt=0.0025, prec="fp64", f64=True, seed=20162),
    # the mixed path with f stored in float64 (float32 transforms): moment drift at the
    # float64 level instead of the float32 rounding of f
    "mixed32_f64": dict(cells=16384, N=32, L=8.0, M=64, gamma=1.0, dt=0.0025, prec="fp32_fft", f64=True,
                        seed=20163),
    # one cell, Maxwell molecules through the rank-16 radial expansion, 32 spherical-
    # Fibonacci directions, 3D BKW datum at K = 3/5 on the box of support radius 6,
    # one Heun step (two collision evaluations) per bench step
    # the N = 48, 64 kernels (float32 only): same physics as mixed32
    "mixed48": dict(cells=2048, N=48, L=8.0, M=64, gamma=1.0, dt=0.0025, prec="fp32_fft", f64=False, seed=20167),
    "mixed64": dict(cells=512, N=64, L=8.0, M=64, gamma=1.0, dt=0.0025, prec="fp32_fft", f64=False, seed=20168),
    # ragged batch: 10000 cells, N in {16: 40 %, 24: 30 %, 32: 25 %, 48: 5 %}, M in {32, 64},
    # gamma in {0, 0.5, 1} drawn per cell, half the cells two-Maxwellian and half 3D BKW
    # profiles; one group (grid) per (N, M, gamma)
    "ragged": dict(cells=10000, N=32, L=8.0, M=64, gamma=1.0, dt=0.0025, prec="fp32_fft", f64=False, seed=20164,
                   ragged=True),
    # 2D Maxwell molecules (Sec. 3.3 dimension two): 262144 cells of 32^2 on [-9, 9]^2,
    # eight angles (Test 1.1's grid), float32 transforms
    "plane32": dict(cells=262144, N=32, L=9.0, M=8, gamma=0.0, dt=0.02, prec="fp32_fft", f64=False, seed=20166,
                    dim=2, opts=dict(C_gamma=1.0 / (2.0 * math.pi))),
    # Fast Kinetic Scheme, 1D x 3D Sod-like problem of Test 2.3 (N = 32 on [-16, 16)^3,
    # M = 64, tau = 1e-2) on a fine mesh of 32768 cells per GPU over [0, 2] (x-slabs with
    # ghost-cell exchange between GPUs); dt = 0.9 dx / max|v|; one fused transport +
    # collision launch per step
    "sod32": dict(cells=32768, N=32, L=16.0, M=64, gamma=1.0, dt=None, prec="fp32_fft", f64=False, seed=20169,
                  fks=True, tau=1e-2),
    "bkw16": dict(cells=1, N=16, L=(3.0 + math.sqrt(2.0)) * 3.0, M=32, gamma=0.0, dt=0.01, prec="fp64", f64=True,
                  seed=20161, rk=2, init="bkw",
                  opts=dict(dirs_kind=1, C_gamma=1.0 / (4.0 * math.pi), radial_rank=16, term_groups=64)),
}
L2_BYTES = 126 << 20  # GB300 L2 as reported by the device; inputs below 2x this flush L2 between steps


def bkw_K(t: float) -> float:
    """Shape parameter of the 3D BKW solution at time t (K(t) = 1 - exp(-t / 6))."""
    return 1.0 - math.exp(-t / 6.0)


BKW_T0 = -6.0 * math.log(1.0 - 0.6)  # K(t0) = 3/5


def make_inputs(wl: dict, cells, total: int):
    """Seeded inputs of the workload for the listed cells of a batch of `total` cells."""
    from paper_1608_08009_gb300 import workloads as W

    if wl.get("dim") == 2:
        return W.two_maxwellians_2d(total, wl["N"], wl["L"], wl["seed"], cells=cells)
    if wl.get("init") == "bkw":
        return np.repeat(W.bkw(wl["N"], wl["L"], bkw_K(BKW_T0))[None], len(cells), axis=0)
    return W.two_maxwellians(total, wl["N"], wl["L"], wl["seed"], cells=cells)
NOMINAL_FP32_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x FMA x max SM clock
NOMINAL_FP64_TFLOPS = 1.25                            # GB300 FP64 (non-tensor), nominal
TF32_PER_BF16 = 1.1 / 2.25                            # nominal dense tensor-core rate ratio
# DRAM bytes (read + write) per cell of one collide_kernel launch, taken from one ncu
# capture (dram__bytes_read.sum + dram__bytes_write.sum) of the kernel as built, on 2048
# cells (float32 path) and 512 cells (float64 path) of the same workload, divided by the
# cells of that capture (traffic grows in proportion to the cells: one read of f and one
# write of the result per cell), keyed by (kernel, precision, f stored float64): the
# one-CTA-per-cell kernel of the float32 path and the 8-CTA cluster kernel of the float64
# path at 32^3.  None when the kernel or the storage type differs from the capture.
# The one-CTA-per-cell kernel changed after its capture (491.5 MB read + written per 2048
# cells: the loss pass now sums Q alone), so its entry is None until it is captured again.
NCU_DRAM_BYTES_PER_CELL = {("collide_solo_kernel", "fp32_fft", False): None,
                           ("collide_kernel", "fp64", True): (176.368896e6 + 97.058304e6) / 512}


def algorithmic_flops(N: int, M: int, dim: int = 3) -> float:
    """F(N, M) = (M + 2) 5 n log2 n + 8 M n + 40 n per cell-collision, n = N^dim.

    Complex-packed inverse transforms (one per direction plus the loss transform and the
    forward transform, 5 n log2 n each), the coefficient products and gain accumulation
    (8 n per direction) and the moment / projection / update work (40 n)."""
    n = N ** dim
    return (M + 2) * 5.0 * n * math.log2(n) + 8.0 * M * n + 40.0 * n


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in out.strip().splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        hi = max(sm)
        loaded = [s for s in sm if s >= 0.5 * hi] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def shard_cells(rank: int, cells_per_rank: int) -> range:
    """Cells of the global seeded batch owned by `rank` (weak scaling: a fixed number per
    rank; cells are independent, so no data is exchanged between ranks)."""
    return range(rank * cells_per_rank, (rank + 1) * cells_per_rank)


def fks_ghosts(f, lo_bc, hi_bc):
    """Boundary states of this rank's x-slab for the next step of the Fast Kinetic Scheme
    (Sec. 4.2, fig. mpi-decomp: the sub-domains' edge cells are exchanged after the
    collision step): the left neighbour's last cell and the right neighbour's first cell,
    or the domain's own boundary states at its ends.  The transport stage moves a column
    by at most one cell per step, so one ghost cell per side is all a step reads.  f:
    [cells][...] this rank's slab (CPU tensors over gloo, CUDA tensors over NCCL)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return lo_bc, hi_bc
    rank, ws = dist.get_rank(), dist.get_world_size()
    lo, hi, reqs = lo_bc, hi_bc, []
    if rank > 0:
        lo = torch.empty_like(f[:1])
        reqs += [dist.irecv(lo, rank - 1), dist.isend(f[:1].contiguous(), rank - 1)]
    if rank < ws - 1:
        hi = torch.empty_like(f[-1:])
        reqs += [dist.irecv(hi, rank + 1), dist.isend(f[-1:].contiguous(), rank + 1)]
    for r in reqs:
        r.wait()
    return lo, hi


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank scalar over the process group (identity without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _oracle_worker(job):
    """One host core's share of the oracle baseline: cells start, start + stride, ..."""
    wl, budget_s, start, stride = job
    return cpu_oracle_rate(wl, budget_s, first=start, stride=stride)


def cpu_oracle_rate_cores(wl: dict, budget_s: float, cores: int = 0):
    """The oracle on `cores` host cores (default: all this process may use), one process
    per core started with spawn and one BLAS / FFT thread each; every process times its
    own share for budget_s seconds.  Returns (cell-collisions/s, cell-collisions, seconds,
    cores)."""
    import multiprocessing as mp

    cores = cores or len(os.sched_getaffinity(0))
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(wl, budget_s, i, cores) for i in range(cores)])
    done = sum(r[1] for r in res)
    el = max(r[2] for r in res)
    return done / el, done, el, cores


def cpu_model() -> str:
    """Model name of the host CPU (lscpu, else /proc/cpuinfo), for the baseline record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_rate(wl: dict, budget_s: float, max_cells: int = 4096, first: int = 0, stride: int = 1):
    """Oracle (FP64 numpy, as it stands) collision steps on one host core: cells / second."""
    import oracle as O
    from paper_1608_08009_gb300 import workloads as W

    o = wl.get("opts", {})
    if wl.get("dim") == 2:
        from oracle import plane as P

        g = P.make_plane_grid(wl["N"], wl["L"], A=wl["M"], Btilde=2.0 * o.get("C_gamma", 1.0))
        mod = P
    else:
        g = O.make_grid(wl["N"], wl["L"], gamma=wl["gamma"], M=wl["M"], dirs_kind=o.get("dirs_kind", 0),
                        C_gamma=o.get("C_gamma", 1.0), rank=o.get("radial_rank") or None)
        mod = O
    rk = wl.get("rk", 1)
    U_done, t0 = 0, time.perf_counter()
    c = first
    while c < max_cells:
        f = make_inputs(wl, [c % wl["cells"]], wl["cells"])
        if rk == 1:
            U0 = mod.moments(f, g)
            Q = mod.collide(f, g, project=False)
            mod.project_f(f + wl["dt"] * Q, U0, g)
        else:
            mod.relax(f, g, wl["dt"], 1, rk_order=rk)
        c += stride
        U_done += rk
        if time.perf_counter() - t0 >= budget_s:
            break
    el = time.perf_counter() - t0
    return U_done / el, U_done, el


def run_serving(seconds: float, rate: float = 200.0, seed: int = 20165, budget_bytes: int = 2 << 30,
                term_groups=None, batch_frac: float = 0.2) -> dict:
    """Serving load (continuous batching through boltz_server_*): Poisson arrivals at
    `rate` req/s for `seconds`; each request relaxes for U{10..200} forward Euler steps on
    N in {16 (60 %), 32 (35 %), 64 (5 %)}, gamma = 1, M = 64, dt = 0.0025, float32 path;
    a fraction batch_frac of the requests are batches of U{2..8} cells, the others single
    cells; admission by an HBM budget that holds every job's distributions and term-group
    scratch.  Latency = completion seen by the host - arrival."""
    import torch

    from paper_1608_08009_gb300 import boltz as B
    from paper_1608_08009_gb300 import workloads as W

    term_groups = term_groups or {16: 4, 32: 8, 64: 4}
    rng = np.random.Generator(np.random.PCG64(seed))
    n_req = int(rng.poisson(rate * seconds))
    arrivals = np.sort(rng.uniform(0.0, seconds, n_req))
    sizes = rng.choice([16, 32, 64], size=n_req, p=[0.60, 0.35, 0.05])
    steps = rng.integers(10, 201, size=n_req)
    ncell = np.where(rng.uniform(size=n_req) < batch_frac, rng.integers(2, 9, size=n_req), 1)
    # 16^3 jobs on [-6, 6)^3 (dv = 0.75), 32^3 and 64^3 jobs on [-8, 8)^3 (dv = 0.5, 0.25)
    Ls = {16: 6.0, 32: 8.0, 64: 8.0}
    # term groups: a job's separated terms spread over several clusters, fixed per grid so
    # a job's arithmetic does not depend on what else is resident
    grids = {N: B.Grid(N, Ls[N], 1.0, 64, term_groups=term_groups[N]) for N in (16, 32, 64)}
    gidx = {16: 0, 32: 1, 64: 2}
    stream = torch.cuda.current_stream()
    server = B.Server([grids[16], grids[32], grids[64]], B.BOLTZ_FP32_FFT, 0.0025, budget_bytes, stream)
    reqs = []
    first = np.concatenate([[0], np.cumsum(ncell)[:-1]])
    total_cells = int(ncell.sum())
    for k in range(n_req):
        N = int(sizes[k])
        cells = range(int(first[k]), int(first[k] + ncell[k]))
        f = W.two_maxwellians(total_cells, N, Ls[N], seed, cells=cells).astype(np.float32).ravel()
        reqs.append((torch.from_numpy(f).pin_memory(), torch.empty(f.size, dtype=torch.float32).pin_memory()))
    # warm-up of every grid outside the measured window
    for N in (16, 32, 64):
        f = torch.zeros(N ** 3, dtype=torch.float32).pin_memory() + 1e-3
        o = torch.empty_like(f)
        j = server.submit(gidx[N], f, o, 2)
        while not server.poll(j):
            server.step()
    torch.cuda.synchronize()
    done_t = [None] * n_req
    ids = [None] * n_req
    nxt, n_steps, max_res, max_q, peak_used = 0, 0, 0, 0, 0
    t0 = time.perf_counter()
    pending = set()
    while True:
        now = time.perf_counter() - t0
        while nxt < n_req and arrivals[nxt] <= now:
            ids[nxt] = server.submit(gidx[int(sizes[nxt])], reqs[nxt][0], reqs[nxt][1], int(steps[nxt]),
                                     int(ncell[nxt]))
            pending.add(nxt)
            nxt += 1
        # non-blocking: every grid with room (two iterations in flight at most) advances
        res, q, launched = server.pump()
        n_steps += launched
        max_res, max_q = max(max_res, res), max(max_q, q)
        now = time.perf_counter() - t0
        for k in list(pending):
            if server.poll(ids[k]):
                done_t[k] = now
                pending.discard(k)
        if nxt >= n_req and not pending:
            break
        if res == 0 and q == 0 and not pending and nxt < n_req:
            time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
        elif launched == 0:
            time.sleep(2e-5)
        if now > seconds + 120.0:
            break
    wall = time.perf_counter() - t0
    stats = server.stats()
    B.boltz_stream_status(stream)

    def pct(sel):
        ln = np.array([done_t[k] - arrivals[k] for k in range(n_req) if done_t[k] is not None and sel(k)])
        if not ln.size:
            return None
        return {"jobs": int(ln.size), "p50_s": float(np.percentile(ln, 50)), "p99_s": float(np.percentile(ln, 99))}

    lat = np.array([done_t[k] - arrivals[k] for k in range(n_req) if done_t[k] is not None])
    by_n = {str(N): pct(lambda k, N=N: sizes[k] == N) for N in (16, 32, 64)}
    served = [k for k in range(n_req) if done_t[k] is not None]
    cell_steps = int(sum(int(steps[k]) * int(ncell[k]) for k in served))
    server.close()
    for g in grids.values():
        g.close()
    return {"p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_latency_s": float(lat.mean()) if lat.size else None,
            "completed": len(served), "by_size": by_n,
            "single_cell": pct(lambda k: ncell[k] == 1), "batch": pct(lambda k: ncell[k] > 1),
            "unfinished": int(sum(1 for k in range(n_req) if done_t[k] is None)),
            "offered_req_per_s": rate, "arrival_window_s": seconds, "wall_s": wall,
            "cell_collisions_per_s": cell_steps / wall, "grid_iterations": n_steps,
            "max_resident_jobs": max_res, "max_queued_jobs": max_q, "hbm_budget_bytes": budget_bytes,
            "server_reserved_bytes": stats["reserved_bytes"], "server_peak_used_bytes": stats["peak_used_bytes"],
            "mix": "N=16 (L=6): 60 %, N=32 (L=8): 35 %, N=64 (L=8): 5 %; steps U{10..200}; "
                   f"{int(round(100 * batch_frac))} % batches of U{{2..8}} cells; M=64; gamma=1; dt=0.0025; f32",
            "term_groups": {str(k): v for k, v in term_groups.items()}}


RAGGED_L = {16: 6.0, 24: 7.0, 32: 8.0, 48: 8.0}


def ragged_cells(wl: dict):
    """Seeded per-cell draws of the ragged batch, grouped by (N, M, gamma): for each cell
    of a group its initial datum, None for a two-Maxwellian cell, else the BKW shape
    parameter K in U[0.6, 0.95] (half the cells each; K >= 3/5 keeps the 3D BKW profile
    non-negative)."""
    rng = np.random.Generator(np.random.PCG64(wl["seed"]))
    n = wl["cells"]
    Ns = rng.choice([16, 24, 32, 48], size=n, p=[0.40, 0.30, 0.25, 0.05])
    Ms = rng.choice([32, 64], size=n)
    gs = rng.choice([0.0, 0.5, 1.0], size=n)
    is_bkw = rng.random(n) < 0.5
    Ks = rng.uniform(0.6, 0.95, size=n)
    groups = {}
    for N, M, g, b, K in zip(Ns.tolist(), Ms.tolist(), gs.tolist(), is_bkw.tolist(), Ks.tolist()):
        groups.setdefault((N, M, g), []).append(K if b else None)
    return dict(sorted(groups.items()))


def ragged_inputs(N: int, L: float, data: list, seed: int) -> np.ndarray:
    """The cells of one ragged group: two-Maxwellian cells (seeded) and BKW profiles."""
    from paper_1608_08009_gb300 import workloads as W

    f = W.two_maxwellians(len(data), N, L, seed)
    for c, K in enumerate(data):
        if K is not None:
            f[c] = W.bkw(N, L, K)
    return f


def run_ragged(args, wl):
    """Ragged batch through boltz_plan_*: per-shape launches (one boltz_relax per group,
    no graph) against one graph launch per step (groups as concurrent branches), with and
    without the autotuner.  value = cells of the supported groups x steps / time of the
    autotuned plan."""
    import torch

    from paper_1608_08009_gb300 import boltz as B

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    B.lib()
    spec = ragged_cells(wl)
    grids, fs, f0s, info = [], [], [], []
    for i, ((N, M, gamma), data) in enumerate(spec.items()):
        L = RAGGED_L[N]
        g = B.Grid(N, L, gamma, M, C_gamma=1.0 / (4.0 * math.pi) if gamma == 0.0 else 1.0)
        f = torch.from_numpy(ragged_inputs(N, L, data, wl["seed"] + 1000 + i)).float().cuda()
        grids.append(g)
        fs.append(f)
        f0s.append(f.clone())
        info.append({"N": N, "M": M, "gamma": gamma, "cells": len(data),
                     "bkw_cells": sum(K is not None for K in data), "M_eff": g.info["M_eff"]})
    cells_total = sum(x["cells"] for x in info)
    flops = sum(algorithmic_flops(x["N"], x["M_eff"]) * x["cells"] for x in info)
    stream = torch.cuda.current_stream()
    dt = wl["dt"]

    def reset():
        for f, f0 in zip(fs, f0s):
            f.copy_(f0)

    def timed(step_fn):
        reset()
        for _ in range(args.warmup):
            step_fn()
        torch.cuda.synchronize()
        reset()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step_fn()
        e1.record(stream)
        torch.cuda.synchronize()
        B.boltz_stream_status(stream)
        return e0.elapsed_time(e1) / args.steps  # ms per step

    def per_shape():
        for g, f, x in zip(grids, fs, info):
            B.boltz_relax(g.batch(x["cells"], B.BOLTZ_FP32_FFT, False), f, dt, 1, 1, stream)

    ms_shape = timed(per_shape)
    groups = [(g, f, B.BOLTZ_FP32_FFT) for g, f in zip(grids, fs)]
    with B.Plan(groups, dt, 1, 1, 0, stream) as p:
        ms_graph = timed(lambda: p.run(stream))
    t_tune = time.perf_counter()
    sampler = ClockSampler(local)
    with B.Plan(groups, dt, 1, 1, B.BOLTZ_PLAN_AUTOTUNE, stream) as p:
        tune_s = time.perf_counter() - t_tune
        for i, x in enumerate(info):
            x.update(p.info(i))
        sampler.start()
        time.sleep(0.3)
        ms_tuned = timed(lambda: p.run(stream))
        clocks = sampler.stop()
    value = cells_total / (ms_tuned / 1000.0)
    peak = NOMINAL_FP32_TFLOPS
    line = {
        "metric": "cell-collisions/s", "value": value, "unit": "cell-collisions/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_tuned, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ragged", "cells": wl["cells"], "cells_run": cells_total,
                   "mix": "N 16/24/32/48: 40/30/25/5 %; M 32/64; gamma 0/0.5/1 (rank-16 expansion for gamma != 1); "
                          "data: half two-Maxwellian, half 3D BKW profiles with K in U[0.6, 0.95]",
                   "L_by_N": RAGGED_L, "dt": dt, "precision": "fp32_fft", "f_storage": "f32",
                   "l2_policy": "inputs larger than L2 (f is %.2f GB)" % (sum(f.numel() * 4 for f in fs) / 1e9),
                   "parallelism": "1 GPU"},
        "roofline": {"bound": "alu", "achieved": flops / (ms_tuned / 1000.0) / 1e12, "peak": peak, "unit": "TFLOP/s",
                     "frac": flops / (ms_tuned / 1000.0) / 1e12 / peak, "traffic": None,
                     "kernel": "collide_kernel, one launch per group per step",
                     "peak_source": "FP32 ALU: 152 SMs x 128 lanes x 2 x 2.07 GHz"},
        "ragged": {"per_shape_launches_ms": ms_shape, "graph_plan_ms": ms_graph, "autotuned_graph_plan_ms": ms_tuned,
                   "autotune_seconds": tune_s, "groups": info},
        "gpu_launches": len(info) * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    for g in grids:
        g.close()
    return 0


def run_fks(args, wl):
    """Fast Kinetic Scheme steps (boltz_fks_step: transport fused into the collision
    launch) on the Sod-like data; x-slabs per rank with one ghost cell exchanged per side
    and step (fks_ghosts, NCCL under torchrun).  value = cells of all ranks x steps / time;
    the timed step includes the exchange."""
    import torch

    from paper_1608_08009_gb300 import boltz as B
    from paper_1608_08009_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.lib()
    N, L, M, cells, tau = wl["N"], wl["L"], wl["M"], wl["cells"], wl["tau"]
    grid = B.Grid(N, L, wl["gamma"], M)
    prec = {"fp64": B.BOLTZ_FP64, "fp32_fft": B.BOLTZ_FP32_FFT}[wl["prec"]]
    dtype = torch.float64 if wl["f64"] else torch.float32
    nx_all = cells * ws
    dx = 2.0 / nx_all
    dt = 0.9 * dx / L  # Eq. Time: |v_x| <= L on the grid
    fl, fr = (torch.from_numpy(a).to(device="cuda", dtype=dtype) for a in W.sod_states(N, L))
    xc = (torch.arange(rank * cells, (rank + 1) * cells, device="cuda", dtype=torch.float64) + 0.5) * dx
    f0 = torch.where((xc <= 1.0)[:, None, None, None], fl[None], fr[None]).contiguous()
    f, g2 = f0.clone(), torch.empty_like(f0)
    lo_bc, hi_bc = fl[None].contiguous(), fr[None].contiguous()
    batch = grid.batch(cells, prec, wl["f64"])
    stream = torch.cuda.current_stream()
    fks = B.Fks(grid, cells, dx)

    def step(a, b):
        lo, hi = fks_ghosts(a, lo_bc, hi_bc)
        fks.step(batch, a, b, lo, hi, dt, tau, stream)

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step(f, g2)
        f, g2 = g2, f
    B.boltz_stream_status(stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    t0.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        step(f, g2)
        ev[k][1].record(stream)
        f, g2 = g2, f
    t1.record(stream)
    barrier()
    clocks = sampler.stop()
    B.boltz_stream_status(stream)
    total_ms = max_over_ranks(t0.elapsed_time(t1), "cuda")
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value = cells * ws * args.steps / (total_ms / 1000.0)
    # end to end: every step uploads the slab from pinned host memory, steps it and reads
    # the result back
    host = f.cpu().pin_memory()
    out_host = torch.empty_like(host).pin_memory()
    nbytes = host.numel() * host.element_size()
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        f.copy_(host, non_blocking=True)
        step(f, g2)
        out_host.copy_(g2, non_blocking=True)
    e1.record(stream)
    barrier()
    B.boltz_stream_status(stream)
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), "cuda")
    if rank == 0:
        flops_cell = algorithmic_flops(N, grid.info["M_eff"])
        avg_s = statistics.mean(step_ms) / 1000.0
        achieved = flops_cell * cells / avg_s / 1e12
        peak = NOMINAL_FP32_TFLOPS if prec != B.BOLTZ_FP64 else NOMINAL_FP64_TFLOPS
        rho = None
        try:
            Ub = torch.empty(cells, 5, dtype=torch.float64, device="cuda")
            B.boltz_moments(batch, f, Ub, stream)
            B.boltz_stream_status(stream)
            rho = Ub[:, 0].cpu()
        except Exception:
            pass
        line = {
            "metric": "cell-collisions/s", "value": value, "unit": "cell-collisions/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if prec == B.BOLTZ_FP64 else "f32", "data": "synthetic",
            "config": {"workload": "sod32", "cells_per_gpu": cells, "cells_total": nx_all, "N_v": N, "L": L,
                       "M_dirs": M, "gamma": wl["gamma"], "tau": tau, "dx": dx, "dt": dt,
                       "domain": "[0, 2], Dirichlet states at both ends, x-slabs per GPU with one ghost cell",
                       "precision": wl["prec"], "f_storage": "f64" if wl["f64"] else "f32",
                       "l2_policy": "inputs larger than L2 (f is %.1f GB)" % (nbytes / 1e9),
                       "parallelism": f"x-slabs, {ws} GPU(s), ghost exchange per step"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "algorithmic_bytes": 2 * nbytes,
                         "kernel": kernel_name(wl, N, 3, grid) + ", the transport stage in its loads",
                         "flops_per_cell": flops_cell},
            "e2e": {"value": cells * ws * e2e_steps / (e2e_ms / 1000.0), "unit": "cell-collisions/s",
                    "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes},
            "gpu_launches": args.steps,
            "clocks": clocks,
            "density_range_after": [float(rho.min()), float(rho.max())] if rho is not None else None,
            "time_after": fks.time,
        }
        print(json.dumps(line), flush=True)
    fks.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    grid.close()
    return 0


def run_reference(args, wl):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    # every step: the oracle on all host cores, each core timing its share for ref_budget s
    rates, cells_total, secs_total, cores = [], 0, 0.0, 1
    for _ in range(args.warmup):
        cpu_oracle_rate(wl, budget_s=1.0, max_cells=1)
    for _ in range(args.steps):
        r, n, el, cores = cpu_oracle_rate_cores(wl, budget_s=args.ref_budget)
        rates.append(r)
        cells_total += n
        secs_total += el
    value = cells_total / secs_total
    line = {
        "impl": "reference", "metric": "cell-collisions/s", "value": value, "unit": "cell-collisions/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * wl["cells"] * wl.get("rk", 1) / value, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args, wl),
        "cpu_baseline": {"value": value, "unit": "cell-collisions/s", "cores": cores, "kind": "oracle",
                         "sample": f"{cells_total} cell-collisions of the workload over {args.steps} steps on "
                                   f"{cores} spawned processes, FP64 numpy oracle"},
        "e2e": {"value": value, "unit": "cell-collisions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def l2_policy(wl: dict) -> str:
    nbytes = wl["cells"] * wl["N"] ** wl.get("dim", 3) * (8 if wl["f64"] else 4)
    if nbytes >= 2 * L2_BYTES:
        return "inputs larger than L2 (f is %.1f GB)" % (nbytes / 1e9)
    return "L2 flushed between timed steps (f is %.1f MB)" % (nbytes / 1e6)


def config_of(args, wl):
    o = wl.get("opts", {})
    dirs = {0: "product grid of midpoints", 1: "spherical Fibonacci", 2: "Gauss x midpoint"}[o.get("dirs_kind", 0)]
    if wl.get("dim") == 2:
        dirs = "equally spaced angles pi p / A"
    extra = {}
    if wl.get("rk", 1) == 2:
        extra["integrator"] = "Heun (2 collision evaluations per step)"
    if o.get("term_groups", 1) > 1:
        extra["term_groups"] = o["term_groups"]
    if o.get("cluster_size"):
        extra["cluster_size"] = o["cluster_size"]
    if wl.get("init") == "bkw":
        extra["datum"] = "3D BKW at K = 3/5, Maxwell molecules, B = 1/(4 pi), radial rank %d" % o.get("radial_rank", 16)
    if wl.get("dim") == 2:
        extra["dimension"] = "2D Maxwell molecules, Btilde = 1/pi"
    return {"workload": args.workload, "cells_per_gpu": wl["cells"], "N_v": wl["N"], "L": wl["L"], "M_dirs": wl["M"],
            "gamma": wl["gamma"], "dirs": dirs, "dt": wl["dt"], "precision": wl["prec"], **extra,
            "f_storage": "f64" if wl["f64"] else "f32", "moments_projection_update": "f64",
            "l2_policy": l2_policy(wl),
            "parallelism": f"cells sharded, {args.gpus} GPU(s)"}


def run_targets(args, wl, grid, value, stream) -> dict:
    """The clauses of the mixed-precision target beside the headline number, measured in
    the same run (rank 0):

    * moment drift on a float64 master state: the headline batch (all its cells) stored
      in float64, 20 Euler steps of the same float32-transform kernel family; relative
      drift of mass, momentum (scaled by sqrt(2 rho E)) and energy per cell, max over cells;
    * the plain float64 form on its own configuration (4096 cells x 32^3, M = 64, float64
      everywhere): cell-collisions/s, event-timed, and the headline's factor over it."""
    import torch

    from paper_1608_08009_gb300 import boltz as B

    out = {}
    cells = wl["cells"]
    # ---- float64 master: same cells, f stored float64, float32 transforms --------------
    f = torch.empty((cells,) + (wl["N"],) * 3, dtype=torch.float64, device="cuda")
    for c0 in range(0, cells, 1024):
        c1 = min(cells, c0 + 1024)
        f[c0:c1] = torch.from_numpy(make_inputs(wl, range(c0, c1), cells)).cuda()
    batch = grid.batch(cells, B.BOLTZ_FP32_FFT, True)
    U0 = torch.empty(cells, 5, dtype=torch.float64, device="cuda")
    B.boltz_moments(batch, f, U0, stream)
    steps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    B.boltz_relax(batch, f, wl["dt"], steps, 1, stream)
    e1.record(stream)
    U1 = torch.empty_like(U0)
    B.boltz_moments(batch, f, U1, stream)
    B.boltz_stream_status(stream)
    scale = U0.abs().clone()
    scale[:, 1:4] = torch.sqrt(2.0 * U0[:, :1] * U0[:, 4:5]).expand(-1, 3)
    drift = ((U1 - U0).abs() / scale).max(dim=0).values.cpu().tolist()
    out["f64_master"] = {"cells": cells, "steps": steps, "moment_drift_rel": drift, "max_drift": max(drift),
                         "value": cells * steps / (e0.elapsed_time(e1) / 1000.0), "unit": "cell-collisions/s",
                         "storage": "f stored f64, transforms f32, moments/projection/update f64"}
    del f, U0, U1
    # ---- the plain float64 form on its configuration ----------------------------------
    w64 = WORKLOADS["fp64_32"]
    c64 = w64["cells"]
    f = torch.empty((c64,) + (w64["N"],) * 3, dtype=torch.float64, device="cuda")
    for c0 in range(0, c64, 1024):
        c1 = min(c64, c0 + 1024)
        f[c0:c1] = torch.from_numpy(make_inputs(w64, range(c0, c1), c64)).cuda()
    b64 = grid.batch(c64, B.BOLTZ_FP64, True)
    B.boltz_relax(b64, f, w64["dt"], 1, 1, stream)  # warm-up
    torch.cuda.synchronize()
    k = 3
    e0.record(stream)
    for _ in range(k):
        B.boltz_relax(b64, f, w64["dt"], 1, 1, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    B.boltz_stream_status(stream)
    r64 = c64 * k / (e0.elapsed_time(e1) / 1000.0)
    out["fp64_form"] = {"workload": "fp64_32", "cells": c64, "steps": k, "value": r64, "unit": "cell-collisions/s",
                        "flops_frac_of_nominal_fp64": algorithmic_flops(w64["N"], w64["M"]) * r64 / 1e12
                        / NOMINAL_FP64_TFLOPS}
    out["factor_vs_fp64_form"] = value / r64
    del f
    return out


def kernel_name(wl, N, dim, grid) -> str:
    """The collision kernel a launch of this workload runs (one launch per step)."""
    opts = wl.get("opts", {})
    if dim == 2:
        return "collide2d_kernel (one launch per step)"
    if N in (48, 64) and wl["prec"] == "fp32_fft":
        return "collide_large_kernel (one launch per step)"
    cs = opts.get("cluster_size", 0)
    if (N == 32 and wl["prec"] == "fp32_fft" and int(opts.get("term_groups", 1) or 1) <= 1
            and (cs == 1 or (cs == 0 and not wl["f64"]))):
        return "collide_solo_kernel (one CTA per cell, one launch per step)"
    return "collide_kernel (one launch per step)"


def run_ours(args, wl):
    import torch

    from paper_1608_08009_gb300 import boltz as B
    from paper_1608_08009_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.lib()
    N, L, M, cells = wl["N"], wl["L"], wl["M"], wl["cells"]
    prec = {"fp64": B.BOLTZ_FP64, "fp32_fft": B.BOLTZ_FP32_FFT, "tf32_dft": B.BOLTZ_TF32_DFT,
            "3xtf32_dft": B.BOLTZ_3XTF32_DFT, "3xbf16_dft": B.BOLTZ_3XBF16_DFT}[wl["prec"]]
    tc_split = {"tf32_dft": 1, "3xtf32_dft": 3, "3xbf16_dft": 3}.get(wl["prec"], 0)
    dtype = torch.float64 if wl["f64"] else torch.float32
    dim = wl.get("dim", 3)
    if dim == 2:
        grid = B.Grid2D(N, L, M, **wl.get("opts", {}))
    else:
        grid = B.Grid(N, L, wl["gamma"], M, **wl.get("opts", {}))
    batch = grid.batch(cells, prec, wl["f64"])
    rk = wl.get("rk", 1)
    # seeded inputs; rank r takes the cells [r * cells, (r+1) * cells) of one big batch
    host = torch.empty((cells,) + (N,) * dim, dtype=dtype).pin_memory()
    chunk = 1024
    for c0 in range(0, cells, chunk):
        c1 = min(cells, c0 + chunk)
        mine = shard_cells(rank, cells)
        host[c0:c1] = torch.from_numpy(make_inputs(wl, mine[c0:c1], cells * ws))
    f0 = host.cuda()
    f = f0.clone()
    stream = torch.cuda.current_stream()
    # inputs smaller than L2: flush it between timed steps (outside the step's events)
    nbytes = host.numel() * host.element_size()
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda") if nbytes < 2 * L2_BYTES else None

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    nvtx = torch.cuda.nvtx  # phase ranges for nsight timelines; no effect otherwise
    # ---- device-resident timing --------------------------------------------------------
    for _ in range(args.warmup):
        B.boltz_relax(batch, f, wl["dt"], 1, rk, stream)
    B.boltz_stream_status(stream)
    f.copy_(f0)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    barrier()
    nvtx.range_push("timed steps")
    t_start.record(stream)
    for k in range(args.steps):
        if flush is not None:
            flush.zero_()
        ev[k][0].record(stream)
        B.boltz_relax(batch, f, wl["dt"], 1, rk, stream)
        ev[k][1].record(stream)
    t_end.record(stream)
    barrier()
    nvtx.range_pop()
    clocks = sampler.stop()
    B.boltz_stream_status(stream)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # with L2 flushes between steps the timed region is the sum of the steps' own events
    total_ms = sum(step_ms) if flush is not None else t_start.elapsed_time(t_end)
    total_ms = max_over_ranks(total_ms, "cuda")
    value = cells * ws * args.steps * rk / (total_ms / 1000.0)

    # drift of the conserved moments over the timed steps, on the stored state
    U0 = torch.empty(cells, 5, dtype=torch.float64, device="cuda")
    U1 = torch.empty_like(U0)
    B.boltz_moments(batch, f0, U0, stream)
    B.boltz_moments(batch, f, U1, stream)
    B.boltz_stream_status(stream)
    # per cell, momentum is scaled by sqrt(2 rho E) >= |rho u| (a cell at rest has zero momentum)
    scale = U0.abs().clone()
    scale[:, 1:4] = torch.sqrt(2.0 * U0[:, :1] * U0[:, 4:5]).expand(-1, 3)
    drift = ((U1 - U0).abs() / scale).max(dim=0).values.cpu().tolist()

    # ---- end to end through the public API with host buffers ----------------------------
    nvtx.range_push("end to end")
    # boltz_relax_host: every step uploads f from pinned host memory, runs the step and
    # downloads the result, copies pipelined with the compute chunk by chunk
    out_host = torch.empty_like(host).pin_memory()
    e2e_steps = max(1, min(args.steps, 3))
    hc = args.host_chunk_cells
    B.boltz_relax_host(batch, host, out_host, wl["dt"], 1, rk, hc, stream)  # staging set up outside the timing
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        B.boltz_relax_host(batch, host, out_host, wl["dt"], 1, rk, hc, stream)
    e1.record(stream)
    barrier()
    B.boltz_stream_status(stream)
    nvtx.range_pop()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, "cuda")
    e2e_value = cells * ws * e2e_steps * rk / (e2e_ms / 1000.0)

    # accuracy of this path on the whole batch: Q(f0) against the float64 GPU path (itself
    # pinned to the oracle at ~1e-13), relative L2 over all cells and velocities
    err = None
    err_cells = None
    err_steps = None
    bkw_err = None
    if wl.get("init") == "bkw":
        # distance to the exact BKW solution after each of 10 Heun steps from t0
        from paper_1608_08009_gb300 import workloads as W

        fb = f0.clone()
        bkw_err = []
        for k in range(10):
            B.boltz_relax(batch, fb, wl["dt"], 1, rk, stream)
            ex = torch.from_numpy(W.bkw(N, L, bkw_K(BKW_T0 + wl["dt"] * (k + 1)))).to(fb)
            bkw_err.append(((fb[0] - ex).norm() / ex.norm()).item())
        B.boltz_stream_status(stream)
    # the float64 path exists up to N = 32; the accuracy checks compare against it
    if wl["prec"] != "fp64" and not args.no_accuracy and N <= 32:
        # 20 Euler steps of the float32 path and of the float64 path from the same f0 on a
        # 512-cell subset: relative L2 distance of the states after each step
        sub = min(cells, 512)
        a = f0[:sub].clone()
        b64 = f0[:sub].double()
        err_steps = []
        for _ in range(20):
            B.boltz_relax(grid.batch(sub, prec, wl["f64"]), a, wl["dt"], 1, 1, stream)
            B.boltz_relax(grid.batch(sub, B.BOLTZ_FP64, True), b64, wl["dt"], 1, 1, stream)
            err_steps.append(((a.double() - b64).norm() / b64.norm()).item())
        B.boltz_stream_status(stream)
        del a, b64
        Qx = torch.empty_like(f0)
        B.boltz_collide(batch, f0, Qx, stream)
        f64 = f0.double()
        Q64 = torch.empty_like(f64)
        B.boltz_collide(grid.batch(cells, B.BOLTZ_FP64, True), f64, Q64, stream)
        B.boltz_stream_status(stream)
        err = ((Qx.double() - Q64).norm() / Q64.norm()).item()
        # per cell the relative error scales with the cell's conditioning ||Q+|| / ||Q||
        # (near-equilibrium cells have a tiny Q); reported as quantiles beside the batch value
        pc = ((Qx.double() - Q64).flatten(1).norm(dim=1) / Q64.flatten(1).norm(dim=1)).cpu()
        err_cells = {"median": float(pc.median()), "p90": float(pc.quantile(0.9)),
                     "p99": float(pc.quantile(0.99)), "max": float(pc.max()),
                     "frac_above_1e-5": float((pc > 1e-5).double().mean())}
        del Qx, f64, Q64

    targets = None
    if (rank == 0 and args.workload == "mixed32" and not args.no_accuracy and not args.no_targets
            and wl["prec"] == "fp32_fft"):
        targets = run_targets(args, wl, grid, value, stream)
        targets["err_vs_fp64"] = err
        targets["spec"] = {"err_vs_fp64_max": 1e-5, "moment_drift_max": 1e-10, "roofline_frac_min": 0.5}

    if rank == 0:
        peaks = measured_peaks()
        flops_cell = algorithmic_flops(N, grid.info["M_eff"], dim)
        avg_s = statistics.mean(step_ms) / 1000.0 / rk  # one launch per collision evaluation
        achieved = flops_cell * cells / avg_s / 1e12
        bound = "alu"
        if wl["prec"] == "fp64":
            peak, peak_note = NOMINAL_FP64_TFLOPS, "nominal FP64 ALU 1.25 TFLOP/s"
        elif tc_split:
            # executed tensor FLOPs: every inverse 1D pass of every term is a dense
            # [N^2 pencils x 2N] x [2N x 2N] real contraction per cell (x3 for 3xTF32)
            bound = "tensor"
            sust = peaks.get("bf16_tflops_sustained") or 1700.0
            if wl["prec"] == "3xbf16_dft":
                peak, peak_note = sust, "measured sustained bf16 %.1f TFLOP/s (of measured)" % sust
            else:
                peak = sust * TF32_PER_BF16
                peak_note = "measured sustained bf16 %.1f TFLOP/s x nominal tf32/bf16 ratio 1.1/2.25 (of measured)" % sust
            achieved = ((grid.info["M_eff"] + 1) * 3 * N ** 2 * (2 * N) ** 2 * 2.0 * tc_split * cells
                        / avg_s / 1e12)
        else:
            peak, peak_note = NOMINAL_FP32_TFLOPS, "FP32 ALU: 152 SMs x 128 lanes x 2 x 2.07 GHz"
        line = {
            "metric": "cell-collisions/s", "value": value, "unit": "cell-collisions/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "tf32_dft": "tf32", "3xtf32_dft": "3xtf32", "3xbf16_dft": "3xbf16"}.get(
                wl["prec"], "f32"),
            "data": "synthetic",
            "config": config_of(args, wl),
            "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": ((NCU_DRAM_BYTES_PER_CELL.get((kernel_name(wl, N, dim, grid).split()[0], wl["prec"],
                                                                     bool(wl["f64"]))) or 0) * cells or None) if dim == 3
                         and N == 32 else None,
                         "traffic_unit": "bytes per launch (ncu dram read+write, scaled by cells)",
                         "algorithmic_bytes": 2 * N ** dim * (8 if wl["f64"] else 4) * cells,
                         "kernel": kernel_name(wl, N, dim, grid),
                         "flops_per_cell": flops_cell, "peak_source": peak_note,
                         "fft_equivalent_tflops": flops_cell * cells / avg_s / 1e12},
            "e2e": {"value": e2e_value, "unit": "cell-collisions/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes},
            "gpu_launches": args.steps * rk,
            "err_vs_fp64": err,
            "err_vs_fp64_per_cell": err_cells,
            "err_vs_fp64_per_step": err_steps,
            "err_vs_bkw_exact_per_step": bkw_err,
            "clocks": clocks,
            "moment_drift_rel": drift,
            "hbm_peak_gbs": peaks.get("hbm_gbs"),
        }
        if targets is not None:
            targets["roofline_frac"] = achieved / peak
            line["targets"] = targets
        if args.serve_seconds > 0 and ws == 1:
            line["serve"] = run_serving(args.serve_seconds, term_groups=args.serve_groups)
        if not args.no_cpu_baseline and ws == 1:
            r, ncell, el, cores = cpu_oracle_rate_cores(wl, budget_s=args.cpu_budget)
            r1, n1, el1 = cpu_oracle_rate(wl, budget_s=min(10.0, args.cpu_budget))
            line["cpu_baseline"] = {"value": r, "unit": "cell-collisions/s", "cores": cores, "kind": "oracle",
                                    "sample": f"{ncell} cell-collisions of the same workload (cells strided over "
                                              f"{cores} spawned processes, one FP64 numpy oracle step each), "
                                              f"{el:.1f} s",
                                    "cpu_model": cpu_model(), "hardware_threads": os.cpu_count(),
                                    "one_core": {"value": r1, "unit": "cell-collisions/s", "cores": 1,
                                                 "sample": f"{n1} cell-collisions in {el1:.1f} s, this process"}}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    grid.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed32", choices=sorted(WORKLOADS))
    ap.add_argument("--cells", type=int, default=0, help="override cells per GPU")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-budget", type=float, default=20.0)
    ap.add_argument("--host-chunk-cells", type=int, default=0,
                    help="chunk size of the end-to-end boltz_relax_host run (0: the library's default schedule)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the float64 comparison of the batch")
    ap.add_argument("--no-targets", action="store_true",
                    help="skip the float64-master drift and plain float64 form legs of the default workload")
    ap.add_argument("--serve-seconds", type=float, default=5.0, help="serving-load window (0: skip)")
    ap.add_argument("--serve-groups", type=str, default="",
                    help="term groups of the serving grids, e.g. 16:4,32:8 (default)")
    ap.add_argument("--term-groups", type=int, default=0, help="override the workload grid's term_groups")
    ap.add_argument("--cluster-size", type=int, default=0, help="override the float32 cluster size")
    ap.add_argument("--prec", default="", choices=["", "fp32_fft", "tf32_dft", "3xtf32_dft", "3xbf16_dft", "fp64"],
                    help="override the workload's precision mode")
    args = ap.parse_args()
    wl = dict(WORKLOADS[args.workload])
    if args.cells > 0:
        wl["cells"] = args.cells
    if args.term_groups > 0:
        wl["opts"] = dict(wl.get("opts", {}), term_groups=args.term_groups)
    if args.cluster_size > 0:
        wl["opts"] = dict(wl.get("opts", {}), cluster_size=args.cluster_size)
    if args.prec:
        wl["prec"] = args.prec
        wl["f64"] = args.prec == "fp64"
    args.serve_groups = ({int(a): int(b) for a, b in (kv.split(":") for kv in args.serve_groups.split(","))}
                         if args.serve_groups else None)
    if args.impl == "reference":
        return run_reference(args, wl)
    if wl.get("ragged"):
        return run_ragged(args, wl)
    if wl.get("fks"):
        return run_fks(args, wl)
    return run_ours(args, wl)


if __name__ == "__main__":
    sys.exit(main())
