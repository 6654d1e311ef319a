"""Python binding of the B300 Gribov-copy enumerator (C ABI in include/gribov.h).

Argument marshalling only: every step of the enumeration runs in the CUDA
kernels of ``libgribov.so``.  PyTorch supplies device memory (its caching
allocator, through the library's allocator hooks) and streams.  There is no
CPU fallback: if the library cannot be loaded, importing the binding's entry
points raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

GC_OK = 0
GC_EINVAL = -1
GC_ENOMEM = -2
GC_ECUDA = -3
GC_ETIMEDOUT = -4
GC_ESTATE = -5

GC_FP64 = 0
GC_MIXED = 1

GC_FP_AUTO = 0
GC_FP_LANCZOS = 1
GC_FP_DENSE = 2
GC_FP_NONE = 3

GC_RELAX_AUTO = 0
GC_RELAX_GENERIC = 1

GC_DEDUP_CONFIG = 0
GC_DEDUP_F8 = 1

GC_START_CONVERGED = 1
GC_START_NOT_CONVERGED = 2
GC_START_DEDUP_FAILED = 3

GC_REGION_UNTESTED = -1
GC_REGION_OUT = 0
GC_REGION_IN = 1
GC_REGION_MARGINAL = 2

GC_PEAK_FFMA = 0
GC_PEAK_FFMA2 = 1
GC_PEAK_DFMA = 2
GC_PEAK_RSQ = 3
GC_PEAK_DFMA_LANE1 = 4


class GribovError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class gc_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("check_every", ctypes.c_int),
        ("max_sweeps", ctypes.c_int),
        ("eps32", ctypes.c_double),
        ("dedup_delta", ctypes.c_double),
        ("fp_tau", ctypes.c_double),
        ("fp_mode", ctypes.c_int),
        ("lanczos_k", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("keep_per_start", ctypes.c_int),
        ("newton_inner", ctypes.c_int),
        ("newton_max", ctypes.c_int),
        ("batch_starts", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("relax_variant", ctypes.c_int),
        ("async_", ctypes.c_int),
        ("use_graph", ctypes.c_int),
        ("autotune", ctypes.c_int),
        ("dedup_mode", ctypes.c_int),
    ]


class gc_server_info(ctypes.Structure):
    _fields_ = [("loop_status", ctypes.c_int), ("loop_running", ctypes.c_int),
                ("loop_launches", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("released", ctypes.c_uint64), ("waiting", ctypes.c_uint64),
                ("bytes_in_use", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64),
                ("regions", ctypes.c_uint32)]


class gc_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "n_starts", "n_converged", "n_not_converged", "n_dedup_failed", "n_distinct",
        "n_distinct_F8", "n_in", "n_marginal", "n_out", "n_untested", "sweeps_fp32",
        "sweeps_fp64", "site_updates_fp32", "site_updates_fp64", "newton_steps",
        "newton_inner_sweeps", "polish_fallbacks", "fp64_residual_passes", "fp_tests", "fp_tests_fp64",
        "lanczos_steps")] + [(n, ctypes.c_double) for n in (
        "ms_relax", "ms_polish", "ms_dedup", "ms_fptest")] + [
        ("kernel_launches", ctypes.c_uint64), ("df_residual_passes", ctypes.c_uint64),
        ("ms_polish_redo", ctypes.c_double), ("polish_redo_starts", ctypes.c_uint64),
        ("lanczos_steps_fp64", ctypes.c_uint64), ("ms_starts", ctypes.c_double)]


EXPORTED = ("gc_set_allocator", "gc_options_default", "gc_create_orbit", "gc_enumerate_copies",
            "gc_fetch_copies", "gc_fetch_copies_async", "gc_fetch_wait", "gc_fetch_minima_f8", "gc_load_copies",
            "gc_fetch_starts", "gc_orbit_stats", "gc_destroy_orbit",
            "gc_last_error", "gc_version", "gc_fp_test_static", "gc_enumerate_batch",
            "gc_autotune", "gc_autotune_ex", "gc_server_create", "gc_server_submit",
            "gc_server_wait", "gc_server_destroy", "gc_peak_probe", "gc_test_dedup_locks", "gc_server_state")

_lib = None
_lock = threading.Lock()
_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_hooks = []


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Load libgribov.so (compiling it first when stale and nvcc is present)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_stale and not _build.up_to_date():
            if os.path.exists("/usr/local/cuda/bin/nvcc") or os.environ.get("NVCC"):
                _build.build()
        if not os.path.exists(_build.LIB):
            raise ImportError(f"libgribov.so not built at {_build.LIB}; run "
                              "python -m paper_1403_0555_b300.build")
        L = ctypes.CDLL(_build.LIB)
        p_d = ctypes.POINTER(ctypes.c_double)
        p_u64 = ctypes.POINTER(ctypes.c_uint64)
        p_i = ctypes.POINTER(ctypes.c_int)
        L.gc_set_allocator.argtypes = [_ALLOC_FN, _FREE_FN, ctypes.c_void_p]
        L.gc_options_default.argtypes = [ctypes.POINTER(gc_options)]
        L.gc_create_orbit.argtypes = [ctypes.c_int, ctypes.c_int, p_d, ctypes.c_uint64,
                                      ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]
        L.gc_enumerate_copies.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double,
                                          ctypes.c_double, ctypes.POINTER(gc_options)]
        L.gc_fetch_copies.argtypes = [ctypes.c_void_p, ctypes.c_size_t,
                                      ctypes.POINTER(ctypes.c_size_t), p_d, p_d, p_u64, p_u64,
                                      p_d, p_i]
        L.gc_fetch_copies_async.argtypes = L.gc_fetch_copies.argtypes
        L.gc_fetch_wait.argtypes = [ctypes.c_void_p]
        L.gc_fetch_minima_f8.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t),
                                         p_d, p_u64]
        L.gc_load_copies.argtypes = [ctypes.c_void_p, ctypes.c_size_t, p_d, p_d, p_u64, p_u64, p_d, p_i,
                                     ctypes.c_size_t, p_d, p_u64, ctypes.c_uint64]
        L.gc_fetch_starts.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, p_i,
                                      p_i, p_d, ctypes.POINTER(ctypes.c_int64)]
        L.gc_orbit_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(gc_stats)]
        L.gc_destroy_orbit.argtypes = [ctypes.c_void_p]
        L.gc_fp_test_static.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_uint64, ctypes.c_double, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]
        L.gc_enumerate_batch.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_uint64), ctypes.c_double,
                                         ctypes.c_double, ctypes.POINTER(gc_options)]
        L.gc_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int, p_i, p_i, p_i]
        L.gc_autotune_ex.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, p_i, p_i, p_i, p_i]
        L.gc_server_create.argtypes = [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(gc_options),
                                       ctypes.POINTER(ctypes.c_void_p)]
        L.gc_server_submit.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, p_d, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_uint64)]
        L.gc_server_wait.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_double, p_i,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p)]
        L.gc_server_destroy.argtypes = [ctypes.c_void_p]
        L.gc_server_state.argtypes = [ctypes.c_void_p, ctypes.POINTER(gc_server_info)]
        L.gc_peak_probe.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]
        L.gc_test_dedup_locks.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong]
        L.gc_last_error.restype = ctypes.c_char_p
        L.gc_version.restype = ctypes.c_char_p
        _lib = L
        return L


def _check(rc):
    if rc != GC_OK:
        raise GribovError(rc, load().gc_last_error().decode())
    return rc


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ct))


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    import torch
    live = {}

    def _alloc(n, stream, ctx):
        try:
            p = torch.cuda.caching_allocator_alloc(int(n), stream=int(stream or 0))
        except Exception:
            return None
        live[p] = True
        return p

    def _free(p, stream, ctx):
        if p in live:
            live.pop(p)
            torch.cuda.caching_allocator_delete(p)

    a, f = _ALLOC_FN(_alloc), _FREE_FN(_free)
    _hooks[:] = [a, f, live]
    _check(load().gc_set_allocator(a, f, None))


def use_cuda_allocator():
    _check(load().gc_set_allocator(_ALLOC_FN(), _FREE_FN(), None))
    _hooks.clear()


# ---------------------------------------------------------------------------
# the C ABI, one wrapper per entry point
# ---------------------------------------------------------------------------

def gc_set_allocator(alloc=None, free_fn=None, ctx=None):
    """Install device-memory hooks (Python callables alloc(n, stream, ctx) -> ptr
    and free_fn(ptr, stream, ctx)); no arguments restores cudaMalloc/cudaFree."""
    if alloc is None and free_fn is None:
        _hooks.clear()
        _check(load().gc_set_allocator(_ALLOC_FN(), _FREE_FN(), None))
        return
    a, f = _ALLOC_FN(alloc), _FREE_FN(free_fn)
    _hooks[:] = [a, f]
    _check(load().gc_set_allocator(a, f, ctx))


def gc_version() -> str:
    return load().gc_version().decode()


def gc_last_error() -> str:
    return load().gc_last_error().decode()


def gc_options_default(**overrides) -> gc_options:
    opt = gc_options()
    _check(load().gc_options_default(ctypes.byref(opt)))
    for k, v in overrides.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = int(v.cuda_stream)
        if k == "async":
            k = "async_"
        setattr(opt, k, v)
    return opt


def gc_create_orbit(dim: int, L: int, link_angles, orbit_id: int = 0, max_copies: int = 0):
    phi = np.ascontiguousarray(link_angles, dtype=np.float64)
    if phi.size != L ** dim * dim:
        raise ValueError(f"link_angles has {phi.size} entries, expected {L ** dim * dim}")
    h = ctypes.c_void_p()
    _check(load().gc_create_orbit(dim, L, _ptr(phi, ctypes.c_double), orbit_id, max_copies,
                                  ctypes.byref(h)))
    return h


def gc_enumerate_copies(orbit, n_starts: int, omega: float, eps: float, opt: gc_options | None = None):
    _check(load().gc_enumerate_copies(orbit, n_starts, omega, eps,
                                      None if opt is None else ctypes.byref(opt)))


def gc_enumerate_batch(orbits, n_starts, omega: float, eps: float, opt: gc_options | None = None):
    k = len(orbits)
    arr = (ctypes.c_void_p * k)(*[o.value if isinstance(o, ctypes.c_void_p) else o for o in orbits])
    ns = (ctypes.c_uint64 * k)(*[int(n) for n in n_starts])
    _check(load().gc_enumerate_batch(arr, k, ns, omega, eps,
                                     None if opt is None else ctypes.byref(opt)))


def gc_autotune_ex(orbit, precision: int, mode: int) -> dict:
    """Launch shapes (mode 1) and, in mode 2 with GC_MIXED, the sweep-unroll depth."""
    r, p, f, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().gc_autotune_ex(orbit, precision, mode, ctypes.byref(r), ctypes.byref(p),
                                 ctypes.byref(f), ctypes.byref(c)))
    return {"r_warps": r.value, "p_warps": p.value, "f_warps": f.value, "check_every": c.value}


def gc_autotune(orbit, precision: int, mode: int = 1) -> dict:
    return gc_autotune_ex(orbit, precision, mode)


def gc_fetch_minima_f8(orbit, capacity: int | None = None) -> dict:
    """The paper's distinct minima: F/(dV) quantised at 1e-8 (each the bin's
    lower edge), increasing, with the number of starts that reached each."""
    lib = load()
    n = ctypes.c_size_t()
    _check(lib.gc_fetch_minima_f8(orbit, 0, ctypes.byref(n), None, None))
    m = n.value if capacity is None else min(capacity, n.value)
    F = np.empty(m)
    count = np.empty(m, np.uint64)
    if m:
        _check(lib.gc_fetch_minima_f8(orbit, m, ctypes.byref(n), _ptr(F, ctypes.c_double),
                                      _ptr(count, ctypes.c_uint64)))
    return {"n_minima": n.value, "F_norm": F, "count": count}


def gc_fetch_copies(orbit, V: int, capacity: int | None = None, theta: bool = True,
                    out: dict | None = None, async_: bool = False) -> dict:
    """Distinct copies sorted by (F, first start).  `out` may hold preallocated
    arrays (for example in pinned host memory) named like the result's keys,
    each with at least as many rows as are fetched; the result then holds views
    of them.  With async_ the device-to-host copies are only enqueued
    (gc_fetch_copies_async): the arrays, which should then be pinned, hold the
    copies once gc_fetch_wait(orbit) returns."""
    lib = load()
    n = ctypes.c_size_t()
    _check(lib.gc_fetch_copies(orbit, 0, ctypes.byref(n), None, None, None, None, None, None))
    m = n.value if capacity is None else min(capacity, n.value)
    if out is not None:
        for k_, a_ in out.items():
            if a_ is not None and len(a_) < m:
                raise ValueError(f"out[{k_!r}] holds {len(a_)} rows, {m} needed")
        F = out["F"][:m]
        th = out["theta"][:m] if theta else None
        first = out["first_start"][:m]
        count = out["count"][:m]
        lam = out["lambda2"][:m]
        reg = out["region"][:m]
    else:
        F = np.empty(m)
        th = np.empty((m, V)) if theta else None
        first = np.empty(m, np.uint64)
        count = np.empty(m, np.uint64)
        lam = np.empty(m)
        reg = np.empty(m, np.int32)
    if m:
        fetch = lib.gc_fetch_copies_async if async_ else lib.gc_fetch_copies
        _check(fetch(orbit, m, ctypes.byref(n), _ptr(F, ctypes.c_double),
                                   _ptr(th, ctypes.c_double), _ptr(first, ctypes.c_uint64),
                                   _ptr(count, ctypes.c_uint64), _ptr(lam, ctypes.c_double),
                                   _ptr(reg, ctypes.c_int)))
    return {"n_distinct": n.value, "F": F, "theta": th, "first_start": first, "count": count,
            "lambda2": lam, "region": reg}


def gc_fetch_copies_async(orbit, V: int, capacity: int | None = None, theta: bool = True,
                          out: dict | None = None) -> dict:
    """gc_fetch_copies with the device-to-host copies left in flight (read-back stream)."""
    return gc_fetch_copies(orbit, V, capacity, theta, out, async_=True)


def gc_fetch_wait(orbit) -> None:
    _check(load().gc_fetch_wait(orbit))


def gc_load_copies(orbit, copies: dict, minima: dict, next_start: int) -> None:
    """Restore a run's state into a new orbit (checkpoint / resume): `copies` as
    gc_fetch_copies returned them (angles included), `minima` as
    gc_fetch_minima_f8 returned them, next_start the number of starts the run
    had taken.  Later calls continue from start next_start."""
    n = int(copies["n_distinct"])
    if len(copies["F"]) < n or copies["theta"] is None:
        raise ValueError("copies must hold every distinct copy with its angles")
    c = lambda a, dt: np.ascontiguousarray(np.asarray(a)[:n], dtype=dt)
    F, th = c(copies["F"], np.float64), c(copies["theta"], np.float64)
    first, count = c(copies["first_start"], np.uint64), c(copies["count"], np.uint64)
    lam, reg = c(copies["lambda2"], np.float64), c(copies["region"], np.int32)
    m = int(minima["n_minima"])
    Fn = np.ascontiguousarray(np.asarray(minima["F_norm"])[:m], dtype=np.float64)
    mc = np.ascontiguousarray(np.asarray(minima["count"])[:m], dtype=np.uint64)
    _check(load().gc_load_copies(orbit, n, _ptr(F, ctypes.c_double), _ptr(th, ctypes.c_double),
                                 _ptr(first, ctypes.c_uint64), _ptr(count, ctypes.c_uint64),
                                 _ptr(lam, ctypes.c_double), _ptr(reg, ctypes.c_int), m,
                                 _ptr(Fn, ctypes.c_double), _ptr(mc, ctypes.c_uint64), int(next_start)))


def gc_fetch_starts(orbit, first: int, n: int) -> dict:
    st = np.zeros(n, np.int32)
    sw = np.zeros(n, np.int32)
    F = np.zeros(n)
    ci = np.zeros(n, np.int64)
    _check(load().gc_fetch_starts(orbit, first, n, _ptr(st, ctypes.c_int), _ptr(sw, ctypes.c_int),
                                  _ptr(F, ctypes.c_double), _ptr(ci, ctypes.c_int64)))
    return {"status": st, "sweeps": sw, "F": F, "copy_idx": ci}


def gc_orbit_stats(orbit) -> dict:
    s = gc_stats()
    _check(load().gc_orbit_stats(orbit, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in gc_stats._fields_}


def gc_destroy_orbit(orbit):
    _check(load().gc_destroy_orbit(orbit))


def gc_fp_test_static(dim: int, L: int, d_links: int, d_configs: int, n: int, fp_tau: float,
                      d_lambda2: int, d_region: int, stream: int = 0):
    """Allocation-free first-region test on device buffers (raw device pointers)."""
    _check(load().gc_fp_test_static(dim, L, d_links, d_configs, n, fp_tau, d_lambda2, d_region,
                                    stream))


def gc_server_create(workers: int = 8, mem_budget_bytes: int = 0, opt: gc_options | None = None):
    h = ctypes.c_void_p()
    _check(load().gc_server_create(workers, mem_budget_bytes, None if opt is None else ctypes.byref(opt),
                                   ctypes.byref(h)))
    return h


def gc_server_submit(server, dim: int, L: int, link_angles, orbit_id: int, n_starts: int,
                     omega: float = 1.7, eps: float = 1e-24) -> int:
    phi = np.ascontiguousarray(link_angles, dtype=np.float64)
    t = ctypes.c_uint64()
    _check(load().gc_server_submit(server, dim, L, _ptr(phi, ctypes.c_double), orbit_id, n_starts,
                                   omega, eps, ctypes.byref(t)))
    return t.value


def gc_server_wait(server, ticket: int, timeout_s: float = -1.0, keep_orbit: bool = True):
    """Returns (status, latency_s, orbit or None)."""
    st = ctypes.c_int()
    lat = ctypes.c_double()
    orb = ctypes.c_void_p()
    _check(load().gc_server_wait(server, ticket, timeout_s, ctypes.byref(st), ctypes.byref(lat),
                                 ctypes.byref(orb) if keep_orbit else None))
    return st.value, lat.value, (orb if orb.value else None)


def gc_server_destroy(server):
    _check(load().gc_server_destroy(server))


def gc_peak_probe(kind: int, stream=None) -> float:
    """Measured throughput of one arithmetic unit (GC_PEAK_*), lane operations per second."""
    if stream is not None and not isinstance(stream, int):
        stream = int(stream.cuda_stream)
    v = ctypes.c_double()
    _check(load().gc_peak_probe(kind, stream, ctypes.byref(v)))
    return v.value


def gc_test_dedup_locks(orbit, hold: bool, spin_budget: int = 0):
    """Test hook: hold (or free) every lock of the orbit's copy table and set the
    lock-wait budget (0 = default)."""
    _check(load().gc_test_dedup_locks(orbit, 1 if hold else 0, spin_budget))


def gc_server_state(server) -> dict:
    """Snapshot of the device-resident request loop and its admission counters."""
    info = gc_server_info()
    _check(load().gc_server_state(server, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in gc_server_info._fields_}
