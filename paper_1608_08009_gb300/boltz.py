"""Thin Python binding of libboltz (include/boltz.h), argument marshalling only.

Every computation runs in the CUDA kernels of ``libboltz.so``; this module converts
torch tensors (or raw integers) into device pointers and status codes into
exceptions.  There is no fallback: if the in-tree library is missing the first call
raises ``BoltzError``.  Build it with ``python -m paper_1608_08009_gb300.build``.
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libboltz.so")

BOLTZ_OK = 0
BOLTZ_EINVAL = 1
BOLTZ_ENOMEM = 2
BOLTZ_ECUDA = 3
BOLTZ_EUNSUPPORTED = 4
BOLTZ_ENONFINITE = 5
BOLTZ_ETIMEOUT = 6

BOLTZ_FP64 = 0
BOLTZ_FP32_FFT = 1
BOLTZ_TF32_DFT = 2
BOLTZ_3XBF16_DFT = 3
BOLTZ_3XTF32_DFT = 4

_STATUS_NAMES = {0: "BOLTZ_OK", 1: "BOLTZ_EINVAL", 2: "BOLTZ_ENOMEM", 3: "BOLTZ_ECUDA",
                 4: "BOLTZ_EUNSUPPORTED", 5: "BOLTZ_ENONFINITE", 6: "BOLTZ_ETIMEOUT"}

EXPORTED = ("boltz_default_opts", "boltz_create_grid", "boltz_destroy_grid", "boltz_collide",
            "boltz_relax", "boltz_moments", "boltz_stream_status", "boltz_last_error",
            "boltz_grid_info", "boltz_grid_tables", "boltz_version", "boltz_relax_noalloc",
            "boltz_collide_indexed", "boltz_relax_indexed", "boltz_server_create", "boltz_server_submit",
            "boltz_server_step", "boltz_server_poll", "boltz_server_destroy", "boltz_relax_host",
            "boltz_plan_create", "boltz_plan_run", "boltz_plan_group_info", "boltz_plan_destroy",
            "boltz_server_pump", "boltz_create_grid2d", "boltz_server_checkpoint", "boltz_host_chunks",
            "boltz_server_submit_batch", "boltz_server_stats_get", "boltz_fks_create", "boltz_fks_step",
            "boltz_fks_time", "boltz_fks_set_time", "boltz_fks_shifts", "boltz_fks_destroy",
            "boltz_plan_group_precision", "boltz_selftest_conversions")


class BoltzError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class boltz_grid_opts(ctypes.Structure):
    _fields_ = [("dirs_kind", ctypes.c_int), ("dirs_a1", ctypes.c_int), ("R_trunc", ctypes.c_double),
                ("C_gamma", ctypes.c_double), ("radial_rank", ctypes.c_int), ("inner_nodes", ctypes.c_int),
                ("project", ctypes.c_int), ("term_groups", ctypes.c_int), ("cluster_size", ctypes.c_int)]


class boltz_batch(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_void_p), ("n_cells", ctypes.c_int64), ("prec", ctypes.c_int),
                ("f_is_fp64", ctypes.c_int)]


class boltz_server_stats(ctypes.Structure):
    _fields_ = [("reserved_bytes", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t),
                ("peak_used_bytes", ctypes.c_size_t), ("resident_cells", ctypes.c_int64),
                ("resident_jobs", ctypes.c_int64), ("queued_jobs", ctypes.c_int64)]


class boltz_group(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_void_p), ("n_cells", ctypes.c_int64), ("prec", ctypes.c_int),
                ("f_is_fp64", ctypes.c_int), ("f", ctypes.c_void_p)]


BOLTZ_PLAN_AUTOTUNE = 1
BOLTZ_PLAN_SERIAL = 2
BOLTZ_PLAN_TUNE_PRECISION = 4

_lib = None


def lib() -> ctypes.CDLL:
    """Load the in-tree libboltz.so once (raises BoltzError if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise BoltzError(BOLTZ_ECUDA, f"libboltz.so not built ({LIB_PATH}); run the build first")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        P = ctypes.POINTER
        L.boltz_default_opts.argtypes = [P(boltz_grid_opts)]
        L.boltz_default_opts.restype = None
        L.boltz_create_grid.argtypes = [i32, f64, f64, i32, P(boltz_grid_opts), P(vp)]
        L.boltz_create_grid2d.argtypes = [i32, f64, i32, P(boltz_grid_opts), P(vp)]
        L.boltz_destroy_grid.argtypes = [vp]
        L.boltz_collide.argtypes = [P(boltz_batch), vp, vp, vp]
        L.boltz_relax.argtypes = [P(boltz_batch), vp, f64, i32, i32, vp]
        L.boltz_moments.argtypes = [P(boltz_batch), vp, vp, vp]
        L.boltz_relax_noalloc.argtypes = [P(boltz_batch), vp, f64, i32, vp]
        L.boltz_relax_host.argtypes = [P(boltz_batch), vp, vp, f64, i32, i32, i64, vp]
        L.boltz_host_chunks.argtypes = [i64, i64, i64, P(i64), i64]
        L.boltz_host_chunks.restype = i64
        L.boltz_plan_create.argtypes = [P(boltz_group), i32, f64, i32, i32, i32, vp, P(vp)]
        L.boltz_plan_run.argtypes = [vp, vp]
        L.boltz_plan_group_info.argtypes = [vp, i32, P(i32), P(i32), P(f64)]
        L.boltz_plan_destroy.argtypes = [vp]
        L.boltz_collide_indexed.argtypes = [P(boltz_batch), vp, vp, vp, i64, vp]
        L.boltz_relax_indexed.argtypes = [P(boltz_batch), vp, vp, i64, f64, i32, vp]
        L.boltz_server_create.argtypes = [P(vp), i32, i32, f64, ctypes.c_size_t, vp, P(vp)]
        L.boltz_server_submit.argtypes = [vp, i32, vp, vp, i32, P(i64)]
        L.boltz_server_submit_batch.argtypes = [vp, i32, vp, vp, i64, i32, P(i64)]
        L.boltz_server_stats_get.argtypes = [vp, P(boltz_server_stats)]
        L.boltz_fks_create.argtypes = [vp, i64, f64, P(vp)]
        L.boltz_fks_step.argtypes = [vp, P(boltz_batch), vp, vp, vp, vp, f64, f64, vp]
        L.boltz_fks_time.argtypes = [vp, P(f64)]
        L.boltz_fks_set_time.argtypes = [vp, f64]
        L.boltz_fks_shifts.argtypes = [vp, f64, P(i32)]
        L.boltz_fks_destroy.argtypes = [vp]
        L.boltz_plan_group_precision.argtypes = [vp, i32, P(i32)]
        L.boltz_selftest_conversions.argtypes = [P(ctypes.c_uint64)]
        L.boltz_server_step.argtypes = [vp, P(i32), P(i32)]
        L.boltz_server_pump.argtypes = [vp, P(i32), P(i32), P(i32)]
        L.boltz_server_checkpoint.argtypes = [vp, i64, vp, P(i32)]
        L.boltz_server_poll.argtypes = [vp, i64, P(i32)]
        L.boltz_server_destroy.argtypes = [vp]
        L.boltz_stream_status.argtypes = [vp]
        L.boltz_last_error.argtypes = []
        L.boltz_last_error.restype = ctypes.c_char_p
        L.boltz_grid_info.argtypes = [vp, P(i32), P(f64), P(f64), P(f64), P(f64), P(i32)]
        L.boltz_grid_tables.argtypes = [vp, vp, vp, vp, vp, vp]
        L.boltz_version.argtypes = []
        L.boltz_version.restype = ctypes.c_char_p
        for name in ("boltz_create_grid", "boltz_destroy_grid", "boltz_collide", "boltz_relax",
                     "boltz_moments", "boltz_stream_status", "boltz_grid_info", "boltz_grid_tables",
                     "boltz_relax_noalloc", "boltz_collide_indexed", "boltz_relax_indexed",
                     "boltz_server_create", "boltz_server_submit", "boltz_server_step", "boltz_server_poll",
                     "boltz_server_destroy", "boltz_relax_host", "boltz_plan_create", "boltz_plan_run",
                     "boltz_plan_group_info", "boltz_plan_destroy", "boltz_server_pump",
                     "boltz_create_grid2d", "boltz_server_checkpoint", "boltz_server_submit_batch",
                     "boltz_server_stats_get", "boltz_fks_create", "boltz_fks_step", "boltz_fks_time",
                     "boltz_fks_set_time", "boltz_fks_shifts", "boltz_fks_destroy", "boltz_plan_group_precision",
                     "boltz_selftest_conversions"):
            getattr(L, name).restype = i32
        _lib = L
    return _lib


def _check(status: int) -> None:
    if status != BOLTZ_OK:
        raise BoltzError(status, lib().boltz_last_error().decode())


def _ptr(x) -> int | None:
    """Device (or host) address of a tensor / integer / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def boltz_default_opts() -> boltz_grid_opts:
    o = boltz_grid_opts()
    lib().boltz_default_opts(ctypes.byref(o))
    return o


def boltz_create_grid(N_v: int, L: float, gamma: float, M_dirs: int, opts: boltz_grid_opts | None = None) -> int:
    h = ctypes.c_void_p()
    _check(lib().boltz_create_grid(N_v, L, gamma, M_dirs, ctypes.byref(opts) if opts is not None else None,
                                   ctypes.byref(h)))
    return h.value


def boltz_destroy_grid(grid: int) -> None:
    _check(lib().boltz_destroy_grid(grid))


def make_batch(grid: int, n_cells: int, prec: int, f_is_fp64: bool) -> boltz_batch:
    return boltz_batch(grid, n_cells, prec, 1 if f_is_fp64 else 0)


def boltz_collide(batch: boltz_batch, f, Q, stream=None) -> None:
    _check(lib().boltz_collide(ctypes.byref(batch), _ptr(f), _ptr(Q), _stream(stream)))


def boltz_relax(batch: boltz_batch, f, dt: float, steps: int, rk_order: int = 1, stream=None) -> None:
    _check(lib().boltz_relax(ctypes.byref(batch), _ptr(f), dt, steps, rk_order, _stream(stream)))


def boltz_relax_noalloc(batch: boltz_batch, f, dt: float, steps: int, stream=None) -> None:
    """Forward-Euler relaxation with no allocation (scratch in a fixed device array)."""
    _check(lib().boltz_relax_noalloc(ctypes.byref(batch), _ptr(f), dt, steps, _stream(stream)))


def boltz_relax_host(batch: boltz_batch, f_in, f_out, dt: float, steps: int, rk_order: int = 1,
                     chunk_cells: int = 0, stream=None) -> None:
    """boltz_relax on host (preferably pinned) buffers; copies pipelined with the compute.
    Enqueued only: synchronise `stream` before reading f_out."""
    _check(lib().boltz_relax_host(ctypes.byref(batch), _ptr(f_in), _ptr(f_out), dt, steps, rk_order, chunk_cells,
                                  _stream(stream)))


def boltz_host_chunks(n_cells: int, cell_bytes: int, chunk_cells: int = 0) -> list:
    """The chunk sizes boltz_relax_host uses for this batch (host only)."""
    n = lib().boltz_host_chunks(n_cells, cell_bytes, chunk_cells, None, 0)
    if n < 0:
        raise BoltzError(BOLTZ_EINVAL, lib().boltz_last_error().decode())
    out = (ctypes.c_int64 * max(1, n))()
    lib().boltz_host_chunks(n_cells, cell_bytes, chunk_cells, out, n)
    return list(out[:n])


def boltz_collide_indexed(batch: boltz_batch, f, Q, cell_idx, pool_cells: int, stream=None) -> None:
    _check(lib().boltz_collide_indexed(ctypes.byref(batch), _ptr(f), _ptr(Q), _ptr(cell_idx), pool_cells,
                                       _stream(stream)))


def boltz_relax_indexed(batch: boltz_batch, f, cell_idx, pool_cells: int, dt: float, steps: int,
                        stream=None) -> None:
    _check(lib().boltz_relax_indexed(ctypes.byref(batch), _ptr(f), _ptr(cell_idx), pool_cells, dt, steps,
                                     _stream(stream)))


def boltz_moments(batch: boltz_batch, f, U, stream=None) -> None:
    _check(lib().boltz_moments(ctypes.byref(batch), _ptr(f), _ptr(U), _stream(stream)))


def boltz_stream_status(stream=None) -> None:
    _check(lib().boltz_stream_status(_stream(stream)))


def boltz_last_error() -> str:
    return lib().boltz_last_error().decode()


def boltz_selftest_conversions() -> tuple:
    """(float->double mismatches, double->float mismatches) of the library's integer-pipe
    conversions against the hardware ones on the current device."""
    out = (ctypes.c_uint64 * 2)()
    _check(lib().boltz_selftest_conversions(out))
    return int(out[0]), int(out[1])


def boltz_version() -> str:
    return lib().boltz_version().decode()


def boltz_grid_info(grid: int) -> dict:
    N = ctypes.c_int()
    M = ctypes.c_int()
    L, dv, S, R = (ctypes.c_double() for _ in range(4))
    _check(lib().boltz_grid_info(grid, ctypes.byref(N), ctypes.byref(L), ctypes.byref(dv), ctypes.byref(S),
                                 ctypes.byref(R), ctypes.byref(M)))
    return {"N": N.value, "L": L.value, "dv": dv.value, "S": S.value, "R": R.value, "M_eff": M.value}


def boltz_grid_tables(grid: int, M_dirs: int, dim: int = 3):
    """Host float64 tables (e, w, alpha, alphap, D) as numpy arrays (for parity tests)."""
    import numpy as np

    info = boltz_grid_info(grid)
    N, Me = info["N"], info["M_eff"]
    shape = (N,) * dim
    n = N ** dim
    e = np.empty(M_dirs * 3)
    w = np.empty(Me)
    al = np.empty(Me * n)
    ap = np.empty(Me * n)
    D = np.empty(n)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(lib().boltz_grid_tables(grid, p(e), p(w), p(al), p(ap), p(D)))
    return e.reshape(M_dirs, 3), w, al.reshape((Me,) + shape), ap.reshape((Me,) + shape), D.reshape(shape)


class Server:
    """Continuous-batching relaxation server (boltz_server_*): one device arena of the HBM
    budget holds every admitted job's state and scratch."""

    def __init__(self, grids, prec: int, dt: float, hbm_budget_bytes: int, stream=None):
        arr = (ctypes.c_void_p * len(grids))(*[g.handle for g in grids])
        h = ctypes.c_void_p()
        _check(lib().boltz_server_create(arr, len(grids), prec, dt, hbm_budget_bytes, _stream(stream),
                                         ctypes.byref(h)))
        self.handle = h.value
        self._keep = []  # host buffers stay alive until their job is done

    def submit(self, grid_index: int, f_host, out_host, steps: int, n_cells: int = 1) -> int:
        """Queue a job of n_cells cells (f_host, out_host: n_cells * N^3 floats)."""
        jid = ctypes.c_int64()
        _check(lib().boltz_server_submit_batch(self.handle, grid_index, _ptr(f_host), _ptr(out_host), n_cells,
                                               steps, ctypes.byref(jid)))
        self._keep.append((f_host, out_host))
        return jid.value

    def stats(self) -> dict:
        st = boltz_server_stats()
        _check(lib().boltz_server_stats_get(self.handle, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in boltz_server_stats._fields_}

    def step(self):
        r, q = ctypes.c_int(), ctypes.c_int()
        _check(lib().boltz_server_step(self.handle, ctypes.byref(r), ctypes.byref(q)))
        return r.value, q.value

    def pump(self):
        """Non-blocking step: (resident, queued, iterations launched)."""
        r, q, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().boltz_server_pump(self.handle, ctypes.byref(r), ctypes.byref(q), ctypes.byref(n)))
        return r.value, q.value, n.value

    def checkpoint(self, job_id: int, f_host) -> int:
        """Copy the job's current state into f_host; returns the steps still to run."""
        r = ctypes.c_int()
        _check(lib().boltz_server_checkpoint(self.handle, job_id, _ptr(f_host), ctypes.byref(r)))
        return r.value

    def poll(self, job_id: int) -> bool:
        d = ctypes.c_int()
        _check(lib().boltz_server_poll(self.handle, job_id, ctypes.byref(d)))
        return bool(d.value)

    def close(self) -> None:
        if getattr(self, "handle", None):
            boltz_destroy_server = lib().boltz_server_destroy
            _check(boltz_destroy_server(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Fks:
    """Fast Kinetic Scheme in one space dimension (boltz_fks_*): rows of n_x cells of
    width dx on `grid`; step() transports and collides f_in into f_out."""

    def __init__(self, grid, n_x: int, dx: float):
        h = ctypes.c_void_p()
        _check(lib().boltz_fks_create(grid.handle, n_x, dx, ctypes.byref(h)))
        self.handle = h.value
        self.grid = grid

    def step(self, batch: boltz_batch, f_in, f_out, inflow_lo, inflow_hi, dt: float, tau: float,
             stream=None) -> None:
        _check(lib().boltz_fks_step(self.handle, ctypes.byref(batch), _ptr(f_in), _ptr(f_out), _ptr(inflow_lo),
                                    _ptr(inflow_hi), dt, tau, _stream(stream)))

    @property
    def time(self) -> float:
        t = ctypes.c_double()
        _check(lib().boltz_fks_time(self.handle, ctypes.byref(t)))
        return t.value

    @time.setter
    def time(self, t: float) -> None:
        _check(lib().boltz_fks_set_time(self.handle, t))

    def shifts(self, dt: float):
        d = (ctypes.c_int * self.grid.info["N"])()
        _check(lib().boltz_fks_shifts(self.handle, dt, d))
        return list(d)

    def close(self) -> None:
        if getattr(self, "handle", None):
            _check(lib().boltz_fks_destroy(self.handle))
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grid:
    """Owning handle of a boltz grid (destroyed on close / garbage collection)."""

    def __init__(self, N_v: int, L: float, gamma: float = 1.0, M_dirs: int = 64, **opts):
        o = boltz_default_opts()
        for k, v in opts.items():
            setattr(o, k, v)
        self.M_dirs = M_dirs
        self.handle = boltz_create_grid(N_v, L, gamma, M_dirs, o)
        self.info = boltz_grid_info(self.handle)

    def batch(self, n_cells: int, prec: int = BOLTZ_FP64, f_is_fp64: bool = True) -> boltz_batch:
        return make_batch(self.handle, n_cells, prec, f_is_fp64)

    def tables(self):
        return boltz_grid_tables(self.handle, self.M_dirs)

    def close(self) -> None:
        if getattr(self, "handle", None):
            boltz_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Grid2D(Grid):
    """2D Maxwell-molecule grid (boltz_create_grid2d); same batch/close interface as Grid."""

    def __init__(self, N_v: int, L: float, A: int = 8, **opts):
        o = boltz_default_opts()
        for k, v in opts.items():
            setattr(o, k, v)
        self.M_dirs = A
        h = ctypes.c_void_p()
        _check(lib().boltz_create_grid2d(N_v, L, A, ctypes.byref(o), ctypes.byref(h)))
        self.handle = h.value
        self.info = boltz_grid_info(self.handle)

    def tables(self):
        return boltz_grid_tables(self.handle, self.M_dirs, dim=2)


class Plan:
    """Owning handle of a ragged-batch plan.  `groups`: list of (Grid, f tensor, prec);
    the tensors must stay alive and in place while the plan exists."""

    def __init__(self, groups, dt: float, steps: int, rk_order: int = 1, flags: int = 0, stream=None):
        arr = (boltz_group * len(groups))()
        self._keep = []
        for i, (grid, f, prec) in enumerate(groups):
            fp64 = str(f.dtype) == "torch.float64"
            arr[i] = boltz_group(grid.handle, f.shape[0], prec, 1 if fp64 else 0, _ptr(f))
            self._keep.append(f)
        h = ctypes.c_void_p()
        _check(lib().boltz_plan_create(arr, len(groups), dt, steps, rk_order, flags, _stream(stream),
                                       ctypes.byref(h)))
        self.handle = h.value
        self.n_groups = len(groups)

    def run(self, stream=None) -> None:
        _check(lib().boltz_plan_run(self.handle, _stream(stream)))

    def info(self, group: int) -> dict:
        G, C, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _check(lib().boltz_plan_group_info(self.handle, group, ctypes.byref(G), ctypes.byref(C), ctypes.byref(us)))
        pr = ctypes.c_int()
        _check(lib().boltz_plan_group_precision(self.handle, group, ctypes.byref(pr)))
        return {"term_groups": G.value, "cluster": C.value, "tuned_us": us.value, "prec": pr.value}

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().boltz_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
