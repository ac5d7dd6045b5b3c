"""The C-ABI library loads and exports every entry point include/boltz.h declares.

CPU only: no compute call is made; argument errors are checked before any CUDA call.
"""

import ctypes
import os
import re

import pytest

from paper_1608_08009_gb300 import boltz as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libboltz():
    if not os.path.exists(B.LIB_PATH):
        from paper_1608_08009_gb300 import build
        build.build()
    return B.lib()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(boltz_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(libboltz):
    decl = declared_functions()
    assert "boltz_collide" in decl and "boltz_relax" in decl and "boltz_moments" in decl
    for name in decl:
        assert hasattr(libboltz, name), name
    assert set(B.EXPORTED) <= set(decl)


def test_version_string(libboltz):
    assert "sm_103a" in B.boltz_version()


def test_default_opts(libboltz):
    o = B.boltz_default_opts()
    assert o.dirs_kind == 0 and o.project == 1 and o.C_gamma == 1.0 and o.inner_nodes == 128


def test_argument_errors_without_device(libboltz):
    L = libboltz
    assert L.boltz_collide(None, None, None, None) == B.BOLTZ_EINVAL
    assert L.boltz_relax(None, None, 0.1, 1, 1, None) == B.BOLTZ_EINVAL
    assert L.boltz_moments(None, None, None, None) == B.BOLTZ_EINVAL
    h = ctypes.c_void_p()
    assert L.boltz_create_grid(15, 8.0, 1.0, 64, None, ctypes.byref(h)) == B.BOLTZ_EINVAL
    assert L.boltz_create_grid(96, 8.0, 1.0, 64, None, ctypes.byref(h)) == B.BOLTZ_EUNSUPPORTED
    assert L.boltz_create_grid(32, -1.0, 1.0, 64, None, ctypes.byref(h)) == B.BOLTZ_EINVAL
    assert L.boltz_create_grid(32, 8.0, 2.0, 64, None, ctypes.byref(h)) == B.BOLTZ_EINVAL
    assert L.boltz_create_grid(32, 8.0, 1.0, 0, None, ctypes.byref(h)) == B.BOLTZ_EINVAL
    assert L.boltz_create_grid(32, 8.0, 1.0, 64, None, None) == B.BOLTZ_EINVAL
    assert h.value is None
    assert "L must be" in B.boltz_last_error() or len(B.boltz_last_error()) > 0
    assert L.boltz_destroy_grid(None) == B.BOLTZ_OK
    assert L.boltz_grid_info(None, None, None, None, None, None, None) == B.BOLTZ_EINVAL


def test_host_chunk_schedule(libboltz):
    """boltz_relax_host's chunks: they tile the batch, stay within 1 GiB of f, and the
    default ramps (32 MiB first and last chunks, growth 3/2) hold for large batches."""
    cb = 32 ** 3 * 4  # one 32^3 float32 cell
    c = B.boltz_host_chunks(32768, cb)
    assert sum(c) == 32768 and min(c) > 0
    assert c[0] == (32 << 20) // cb and c[-1] == c[0]
    # ramp up by 3/2 until the middle size, about an eighth of the batch
    up = [c[0]]
    while c[len(up)] > up[-1] and c[len(up)] == up[-1] + up[-1] // 2:
        up.append(c[len(up)])
    assert len(up) >= 3
    middle = c[len(up):len(c) - len(up)]
    assert max(middle) - min(middle) <= 1 and abs(max(middle) - 32768 // 8) <= 32768 // 64
    assert c[len(c) - len(up):] == up[::-1]
    # explicit chunk size: equal chunks, last one shorter
    assert B.boltz_host_chunks(1000, cb, 300) == [300, 300, 300, 100]
    # small batch: one chunk; large cells are capped at 1 GiB per chunk
    assert B.boltz_host_chunks(100, cb) == [100]
    big = 64 ** 3 * 8
    c = B.boltz_host_chunks(5000, big)
    assert sum(c) == 5000 and max(c) * big <= (1 << 30)
    assert B.boltz_host_chunks(0, cb) == []
    with pytest.raises(B.BoltzError):
        B.boltz_host_chunks(10, 0)
    assert libboltz.boltz_host_chunks(-1, cb, 0, None, 0) == -1


def test_argument_errors_of_the_other_entry_points(libboltz):
    """Every entry point rejects missing handles and arguments with a status before any
    CUDA call (no device needed); destroying a null grid is a no-op."""
    L = libboltz
    h = ctypes.c_void_p()
    assert L.boltz_create_grid2d(12, 8.0, 8, None, ctypes.byref(h)) == B.BOLTZ_EUNSUPPORTED
    assert L.boltz_create_grid2d(32, -1.0, 8, None, ctypes.byref(h)) == B.BOLTZ_EINVAL
    assert L.boltz_create_grid2d(32, 8.0, 0, None, ctypes.byref(h)) == B.BOLTZ_EINVAL
    assert L.boltz_create_grid2d(32, 8.0, 8, None, None) == B.BOLTZ_EINVAL
    assert L.boltz_relax_host(None, None, None, 0.1, 1, 1, 0, None) == B.BOLTZ_EINVAL
    assert L.boltz_relax_noalloc(None, None, 0.1, 1, None) == B.BOLTZ_EINVAL
    assert L.boltz_collide_indexed(None, None, None, None, 0, None) == B.BOLTZ_EINVAL
    assert L.boltz_relax_indexed(None, None, None, 0, 0.1, 1, None) == B.BOLTZ_EINVAL
    assert L.boltz_plan_create(None, 0, 0.1, 1, 1, 0, None, None) == B.BOLTZ_EINVAL
    assert L.boltz_plan_run(None, None) == B.BOLTZ_EINVAL
    assert L.boltz_server_create(None, 0, 1, 0.1, 0, None, None) == B.BOLTZ_EINVAL
    assert L.boltz_server_submit(None, 0, None, None, 1, None) == B.BOLTZ_EINVAL
    assert L.boltz_server_step(None, None, None) == B.BOLTZ_EINVAL
    assert L.boltz_server_poll(None, 0, None) == B.BOLTZ_EINVAL
    assert L.boltz_grid_info(None, None, None, None, None, None, None) == B.BOLTZ_EINVAL
    assert L.boltz_last_error()  # the message of the last failure
    assert L.boltz_destroy_grid(None) == B.BOLTZ_OK
