"""Python binding of libslr (include/slr.h): argument marshalling only.

Every function here has the name of the C entry point it wraps and does no
numerical work: arrays are converted to contiguous FP64/int64 numpy buffers
and passed by pointer; every step of the method runs in the CUDA library.
PyTorch supplies the device memory (its caching allocator, injected through
the slr_allocator callbacks) and the CUDA stream.

There is no CPU fallback: if libslr.so is missing or fails to load,
:func:`lib` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libslr.so")
_lock = threading.Lock()
_lib = None

SLR_OK, SLR_E_INVALID, SLR_E_NOMEM, SLR_E_CUDA, SLR_E_TIMEOUT, SLR_E_STATE, SLR_E_CAPACITY = range(7)
STATUS_NAMES = ["SLR_OK", "SLR_E_INVALID", "SLR_E_NOMEM", "SLR_E_CUDA", "SLR_E_TIMEOUT", "SLR_E_STATE",
                "SLR_E_CAPACITY"]
SLR_FIELD_U, SLR_FIELD_D, SLR_FIELD_ARGMIN = 0, 1, 2

# every entry point declared in include/slr.h
EXPORTS = [
    "slr_config_default", "slr_create", "slr_load_cloud", "slr_build_distance", "slr_build_distance_fsm",
    "slr_set_distance", "slr_init_u",
    "slr_step", "slr_step_async", "slr_evolve", "slr_batch_evolve", "slr_batch_chunk", "slr_batch_run", "slr_batch_run_info", "slr_extract", "slr_get_field", "slr_get_band", "slr_energy", "slr_diagnostics",
    "slr_export_state", "slr_import_state", "slr_set_profiling", "slr_last_iteration_times",
    "slr_last_iteration_phases", "slr_kernel_launches", "slr_brick_shape", "slr_brick_shape_set", "slr_probe_fma",
    "slr_last_error", "slr_destroy", "slr_distance_grid_noalloc", "slr_cloud_spacing", "slr_l1_error", "slr_selftest_barrier",
    "slr_server_create", "slr_server_set_policy", "slr_server_submit", "slr_server_poll", "slr_server_timing", "slr_server_release",
    "slr_server_last_error",
    "slr_server_destroy", "slr_multirun_default", "slr_reconstruct",
]


class SlrError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


class slr_config(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("n", C.c_int64 * 3),
        ("lo", C.c_double * 3),
        ("hi", C.c_double * 3),
        ("precision", C.c_int),
        ("interp", C.c_int),
        ("p", C.c_double),
        ("delta", C.c_double),
        ("dt", C.c_double),
        ("band", C.c_int),
        ("gamma", C.c_double),
        ("beta", C.c_double),
        ("c_sing", C.c_double),
        ("alpha", C.c_double),
        ("energy_R", C.c_int),
        ("stop_tol", C.c_double),
        ("stop_k", C.c_int),
        ("min_iters", C.c_int),
        ("max_iters", C.c_int),
        ("reinit", C.c_int),
        ("reinit_sweeps", C.c_int),
        ("reinit_dtau", C.c_double),
        ("step_kind", C.c_int),
    ]


class slr_multirun_config(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("precision", C.c_int),
        ("interp", C.c_int),
        ("runs", C.c_int),
        ("K_s", C.c_double),
        ("sample_frac", C.c_double),
        ("seed", C.c_uint64),
        ("max_nodes", C.c_int64),
        ("max_iters", C.c_int),
        ("distance_fsm", C.c_int),
        ("exact_sphere", C.c_int),
        ("sphere", C.c_double * 4),
    ]


SLR_MAX_RUNS = 8


class slr_multirun_report(C.Structure):
    _fields_ = [
        ("h_s", C.c_double),
        ("sample_size", C.c_int64),
        ("runs_done", C.c_int),
        ("coarsened", C.c_int),
        ("run_dx", C.c_double * SLR_MAX_RUNS),
        ("run_n", (C.c_int64 * 3) * SLR_MAX_RUNS),
        ("run_lo", (C.c_double * 3) * SLR_MAX_RUNS),
        ("run_iters", C.c_int * SLR_MAX_RUNS),
        ("run_converged", C.c_int * SLR_MAX_RUNS),
        ("run_energy", C.c_double * SLR_MAX_RUNS),
        ("run_err_cloud", C.c_double * SLR_MAX_RUNS),
        ("run_l1_err", C.c_double * SLR_MAX_RUNS),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class slr_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", C.c_void_p)]


_vp, _dp, _i64p, _ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int)


def lib():
    """Load libslr.so (raises if it is absent: there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libslr.so not built ({LIB_PATH}); run paper_2410_22205_gb300/build.py first")
            L = C.CDLL(LIB_PATH)
            P = C.POINTER(slr_config)
            sig = {
                "slr_config_default": (None, [P]),
                "slr_create": (C.c_int, [P, C.POINTER(slr_allocator), _vp, C.POINTER(_vp)]),
                "slr_load_cloud": (C.c_int, [_vp, _dp, C.c_int64]),
                "slr_build_distance": (C.c_int, [_vp]),
                "slr_build_distance_fsm": (C.c_int, [_vp]),
                "slr_set_distance": (C.c_int, [_vp, _dp]),
                "slr_init_u": (C.c_int, [_vp, C.c_int, _dp, _dp]),
                "slr_step": (C.c_int, [_vp, C.c_int, C.c_double]),
                "slr_step_async": (C.c_int, [_vp, C.c_int, C.c_double]),
                "slr_evolve": (C.c_int, [_vp, _ip, _ip]),
                "slr_batch_evolve": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, _vp, _ip, _ip]),
                "slr_batch_chunk": (C.c_int, [_vp]),
                "slr_batch_run": (C.c_int, [C.POINTER(_vp), C.c_int, C.c_int, _vp, _ip, _ip]),
                "slr_batch_run_info": (C.c_int, [_vp, _ip, _ip, _ip, _ip, C.POINTER(C.c_float)]),
                "slr_extract": (C.c_int, [_vp, C.c_double, _i64p, _dp, C.c_int64, _i64p]),
                "slr_get_field": (C.c_int, [_vp, C.c_int, _vp, C.c_int64]),
                "slr_get_band": (C.c_int, [_vp, _i64p, C.c_int64, _i64p]),
                "slr_energy": (C.c_int, [_vp, C.c_double, _dp, _dp]),
                "slr_diagnostics": (C.c_int, [_vp, _dp, _dp, _i64p, C.c_int, _ip, _dp]),
                "slr_export_state": (C.c_int, [_vp, _vp, C.c_int64, _i64p]),
                "slr_import_state": (C.c_int, [_vp, _vp, C.c_int64]),
                "slr_set_profiling": (C.c_int, [_vp, C.c_int]),
                "slr_last_iteration_times": (C.c_int, [_vp, C.POINTER(C.c_float)]),
                "slr_last_iteration_phases": (C.c_int, [_vp, C.POINTER(C.c_float)]),
                "slr_kernel_launches": (C.c_int64, [_vp]),
                "slr_brick_shape": (C.c_int, [_vp, _ip, _ip, C.POINTER(C.c_float)]),
                "slr_brick_shape_set": (C.c_int, [_vp, C.c_int, C.c_int]),
                "slr_probe_fma": (C.c_int, [C.c_int, C.c_int64, _dp, _dp]),
                "slr_cloud_spacing": (C.c_int, [_vp, _i64p, C.c_int64, _dp]),
                "slr_l1_error": (C.c_int, [_vp, C.c_int, _dp, _dp, _dp]),
                "slr_selftest_barrier": (C.c_int, [C.c_int]),
                "slr_last_error": (C.c_char_p, [_vp]),
                "slr_destroy": (None, [_vp]),
                "slr_distance_grid_noalloc": (C.c_int, [C.c_int, _i64p, _dp, C.c_double, C.c_int, _vp, C.c_int64,
                                                        _vp, _vp, _vp]),
            }
            sig.update({
                "slr_multirun_default": (None, [C.POINTER(slr_multirun_config)]),
                "slr_reconstruct": (C.c_int, [C.POINTER(slr_multirun_config), _dp, C.c_int64, C.POINTER(slr_allocator),
                                              _vp, C.POINTER(_vp), C.POINTER(slr_multirun_report)]),
                "slr_server_set_policy": (C.c_int, [_vp, C.c_int]),
                "slr_server_create": (C.c_int, [C.c_size_t, C.c_int, C.c_int, C.POINTER(slr_allocator),
                                                C.POINTER(_vp)]),
                "slr_server_timing": (C.c_int, [_vp, C.c_uint64, _dp, _dp, _dp]),
                "slr_server_submit": (C.c_int, [_vp, P, _dp, C.c_int64, _dp, C.POINTER(C.c_uint64)]),
                "slr_server_poll": (C.c_int, [_vp, C.c_uint64, _ip, C.POINTER(_vp), _dp]),
                "slr_server_release": (C.c_int, [_vp, C.c_uint64]),
                "slr_server_last_error": (C.c_char_p, [_vp]),
                "slr_server_destroy": (None, [_vp]),
            })
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(ctx, status):
    if status != SLR_OK:
        msg = lib().slr_last_error(ctx)
        raise SlrError(status, msg.decode() if msg else "")


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t)


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

_CFG_FIELDS = {f[0] for f in slr_config._fields_}


def slr_config_default(**overrides) -> slr_config:
    cfg = slr_config()
    lib().slr_config_default(C.byref(cfg))
    for k, v in overrides.items():
        if k in ("n", "lo", "hi"):
            v = list(v) + [1 if k == "n" else 0.0] * (3 - len(v))
            arr = getattr(cfg, k)
            for a in range(3):
                arr[a] = v[a]
        elif k in _CFG_FIELDS:
            setattr(cfg, k, v)
        else:
            raise TypeError(f"slr_config has no field {k!r}")
    return cfg


class _TorchAllocator:
    """slr_allocator backed by torch's CUDA caching allocator."""

    def __init__(self, device: int, stream: int):
        import torch

        self._torch = torch
        self.device = device
        self.stream = stream

        def _alloc(nbytes, _user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream))
            except Exception:
                return None

        def _free(ptr, _user):
            if ptr:
                torch.cuda.caching_allocator_delete(int(ptr))

        self.c_alloc = ALLOC_FN(_alloc)
        self.c_free = FREE_FN(_free)
        self.struct = slr_allocator(self.c_alloc, self.c_free, None)


def slr_create(cfg: slr_config, allocator=None, stream=None):
    """Returns an opaque context handle (int). ``allocator`` is an
    slr_allocator (or an object with a ``.struct``), ``stream`` a raw
    cudaStream_t value (int) or None."""
    h = C.c_void_p()
    al = None
    if allocator is not None:
        al = C.byref(allocator.struct if hasattr(allocator, "struct") else allocator)
    st = C.c_void_p(stream) if stream else None
    s = lib().slr_create(C.byref(cfg), al, st, C.byref(h))
    _check(None, s)
    return h.value


def slr_load_cloud(ctx, xyz):
    xyz = _f64(xyz)
    _check(ctx, lib().slr_load_cloud(ctx, _ptr(xyz), xyz.shape[0]))


def slr_build_distance(ctx):
    _check(ctx, lib().slr_build_distance(ctx))


def slr_build_distance_fsm(ctx):
    _check(ctx, lib().slr_build_distance_fsm(ctx))


def slr_set_distance(ctx, d):
    d = _f64(d)
    _check(ctx, lib().slr_set_distance(ctx, _ptr(d)))


def slr_init_u(ctx, kind, params=None, u0=None):
    p = _f64(params) if params is not None else None
    u = _f64(u0) if u0 is not None else None
    _check(ctx, lib().slr_init_u(ctx, int(kind), _ptr(p) if p is not None else None,
                                 _ptr(u) if u is not None else None))


def slr_cloud_spacing(ctx, sample):
    s = np.ascontiguousarray(sample, dtype=np.int64)
    out = C.c_double(0.0)
    _check(ctx, lib().slr_cloud_spacing(ctx, _ptr(s, _i64p), int(s.size), C.byref(out)))
    return out.value


def slr_l1_error(ctx, sphere=None, exact=None):
    """§4 L^1 error against |x - c| - r (sphere = (cx, cy, cz, r)) or an
    exact array of every node."""
    out = C.c_double(0.0)
    if sphere is not None:
        prm = _f64(sphere)
        _check(ctx, lib().slr_l1_error(ctx, 0, _ptr(prm), None, C.byref(out)))
    else:
        ex = _f64(exact)
        _check(ctx, lib().slr_l1_error(ctx, 1, None, _ptr(ex), C.byref(out)))
    return out.value


def slr_selftest_barrier(unreachable):
    """Status of the bounded grid barrier's self-test (see include/slr.h)."""
    return int(lib().slr_selftest_barrier(int(unreachable)))


def slr_step(ctx, n_steps=1, energy_override=-1.0):
    _check(ctx, lib().slr_step(ctx, int(n_steps), float(energy_override)))


def slr_step_async(ctx, n_steps=1, energy_override=-1.0):
    _check(ctx, lib().slr_step_async(ctx, int(n_steps), float(energy_override)))


def slr_set_profiling(ctx, on=True):
    _check(ctx, lib().slr_set_profiling(ctx, 1 if on else 0))


def slr_last_iteration_times(ctx):
    ms = (C.c_float * 3)()
    _check(ctx, lib().slr_last_iteration_times(ctx, ms))
    return list(ms)


def slr_last_iteration_phases(ctx):
    ms = (C.c_float * 4)()
    _check(ctx, lib().slr_last_iteration_phases(ctx, ms))
    return list(ms)


def slr_evolve(ctx):
    it, conv = C.c_int(0), C.c_int(0)
    _check(ctx, lib().slr_evolve(ctx, C.byref(it), C.byref(conv)))
    return it.value, bool(conv.value)


def slr_batch_evolve(ctxs, chunk=8, stream=None):
    """Evolve several contexts together (one graph launch advances all of
    them by `chunk` iterations; chunk < 0: autotuned); returns (iters,
    converged) per context."""
    n = len(ctxs)
    arr = (_vp * n)(*ctxs)
    it = (C.c_int * n)()
    cv = (C.c_int * n)()
    s = lib().slr_batch_evolve(arr, n, int(chunk), C.c_void_p(stream) if stream else None, it, cv)
    _check(ctxs[0] if n else None, s)
    return list(it), [bool(x) for x in cv]


def slr_batch_run(ctxs, autotune=True, stream=None):
    """Evolve several narrow-band contexts together in one persistent kernel
    launch (graph-captured); returns (iters, converged) per context."""
    n = len(ctxs)
    arr = (_vp * n)(*ctxs)
    it = (C.c_int * n)()
    cv = (C.c_int * n)()
    s = lib().slr_batch_run(arr, n, 1 if autotune else 0, C.c_void_p(stream) if stream else None, it, cv)
    _check(ctxs[0] if n else None, s)
    return list(it), [bool(x) for x in cv]


def slr_batch_run_info(ctx):
    """Launch shape of the last slr_batch_run that ctx led: dict of threads
    per block, resident blocks per SM, bricks per item, graph capture and
    the autotuner's best trial time (ms)."""
    th, bl, bp, gr, ms = C.c_int(0), C.c_int(0), C.c_int(0), C.c_int(0), C.c_float(0.0)
    _check(ctx, lib().slr_batch_run_info(ctx, C.byref(th), C.byref(bl), C.byref(bp), C.byref(gr), C.byref(ms)))
    return {"threads_per_block": th.value, "blocks_per_sm": bl.value, "bricks_per_item": bp.value,
            "graph_captured": bool(gr.value), "autotune_trial_ms": ms.value}


def slr_batch_chunk(ctx):
    """Chunk used by the last slr_batch_evolve that ctx led (ctx = its first job)."""
    return int(lib().slr_batch_chunk(ctx))


def slr_extract(ctx, width):
    n = C.c_int64(0)
    _check(ctx, lib().slr_extract(ctx, float(width), None, None, 0, C.byref(n)))
    idx = np.empty(max(n.value, 1), np.int64)
    val = np.empty(max(n.value, 1), np.float64)
    _check(ctx, lib().slr_extract(ctx, float(width), _ptr(idx, _i64p), _ptr(val), idx.size, C.byref(n)))
    return idx[: n.value], val[: n.value]


def slr_get_field(ctx, which, num_nodes):
    if which == SLR_FIELD_ARGMIN:
        out = np.empty(num_nodes, np.int32)
    else:
        out = np.empty(num_nodes, np.float64)
    _check(ctx, lib().slr_get_field(ctx, int(which), out.ctypes.data_as(_vp), num_nodes))
    return out


def slr_get_band(ctx):
    n = C.c_int64(0)
    _check(ctx, lib().slr_get_band(ctx, None, 0, C.byref(n)))
    out = np.empty(max(n.value, 1), np.int64)
    _check(ctx, lib().slr_get_band(ctx, _ptr(out, _i64p), out.size, C.byref(n)))
    return out[: n.value]


def slr_energy(ctx, p=2.0):
    E, S = C.c_double(0), C.c_double(0)
    _check(ctx, lib().slr_energy(ctx, float(p), C.byref(E), C.byref(S)))
    return E.value, S.value


def slr_diagnostics(ctx, cap=4096, err_cloud=False):
    e2 = np.zeros(cap)
    dphi = np.zeros(cap)
    band = np.zeros(cap, np.int64)
    n = C.c_int(0)
    ec = C.c_double(0)
    _check(ctx, lib().slr_diagnostics(ctx, _ptr(e2), _ptr(dphi), _ptr(band, _i64p), cap, C.byref(n),
                                      C.byref(ec) if err_cloud else None))
    k = n.value
    return dict(iters=k, e2=e2[: min(k + 1, cap)], dphi=dphi[: min(k, cap)], band=band[: min(k, cap)],
                err_cloud=ec.value if err_cloud else None)


def slr_export_state(ctx) -> bytes:
    n = C.c_int64(0)
    lib().slr_export_state(ctx, None, 0, C.byref(n))
    buf = C.create_string_buffer(n.value)
    _check(ctx, lib().slr_export_state(ctx, C.cast(buf, _vp), n.value, C.byref(n)))
    return buf.raw


def slr_import_state(ctx, data: bytes):
    buf = C.create_string_buffer(data, len(data))
    _check(ctx, lib().slr_import_state(ctx, C.cast(buf, _vp), len(data)))


def slr_kernel_launches(ctx) -> int:
    return int(lib().slr_kernel_launches(ctx))


def slr_brick_shape(ctx):
    """(threads per block, stages, trial ms) of the brick-staged 3-D step."""
    t, s = C.c_int(0), C.c_int(0)
    ms = C.c_float(0.0)
    _check(ctx, lib().slr_brick_shape(ctx, C.byref(t), C.byref(s), C.byref(ms)))
    return t.value, s.value, ms.value


def slr_brick_shape_set(ctx, threads, stages):
    _check(ctx, lib().slr_brick_shape_set(ctx, int(threads), int(stages)))


def slr_probe_fma(precision=32, trips=None):
    """Measured FMA throughput of the current device: (TFLOP/s, ms of the timed launch)."""
    if trips is None:
        trips = 50_000 if precision == 32 else 1_000
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    st = lib().slr_probe_fma(int(precision), int(trips), C.byref(tf), C.byref(ms))
    if st != SLR_OK:
        raise SlrError(st, "probe_fma failed")
    return tf.value, ms.value


def slr_last_error(ctx) -> str:
    m = lib().slr_last_error(ctx)
    return m.decode() if m else ""


def slr_distance_grid_noalloc(dim, n, lo, h, precision, pts_dev, n_points, d_dev, argmin_dev, stream=None):
    """Distance grid from caller-owned device buffers with no device
    allocation (see include/slr.h): pts_dev, d_dev and argmin_dev are raw
    device addresses (ints), stream a raw cudaStream_t value or None."""
    nn = (C.c_int64 * 3)(*(list(n) + [1] * (3 - len(n))))
    ll = (C.c_double * 3)(*(list(lo) + [0.0] * (3 - len(lo))))
    s = lib().slr_distance_grid_noalloc(int(dim), nn, ll, float(h), int(precision), C.c_void_p(pts_dev),
                                        int(n_points), C.c_void_p(d_dev), C.c_void_p(argmin_dev),
                                        C.c_void_p(stream) if stream else None)
    _check(None, s)


def slr_destroy(ctx):
    if ctx:
        lib().slr_destroy(ctx)


def _check_srv(srv, status):
    if status != SLR_OK:
        msg = lib().slr_server_last_error(srv)
        raise SlrError(status, msg.decode() if msg else "")


def slr_server_create(hbm_budget, max_active=16, allocator=None, setup_threads=1, policy=0):
    """A continuous-batching server; policy 0 admits the oldest request first,
    1 the least estimated set-up time less its waiting time."""
    h = C.c_void_p()
    al = C.byref(allocator.struct if hasattr(allocator, "struct") else allocator) if allocator is not None else None
    s = lib().slr_server_create(int(hbm_budget), int(max_active), int(setup_threads), al, C.byref(h))
    if s != SLR_OK:
        raise SlrError(s, "server creation failed")
    if policy:
        s = lib().slr_server_set_policy(h.value, int(policy))
        if s != SLR_OK:
            lib().slr_server_destroy(h.value)
            raise SlrError(s, "invalid server policy")
    return h.value


def slr_server_submit(srv, cfg, xyz, sphere):
    xyz = _f64(xyz)
    sp = _f64(list(sphere) + [0.0] * (4 - len(sphere)))
    t = C.c_uint64(0)
    _check_srv(srv, lib().slr_server_submit(srv, C.byref(cfg), _ptr(xyz), xyz.shape[0], _ptr(sp), C.byref(t)))
    return t.value


def slr_server_poll(srv, ticket):
    """Returns (state, ctx or None, latency_ms or None); state 0 queued,
    1 running, 2 done, 3 failed (raises for failed)."""
    st = C.c_int(0)
    res = C.c_void_p()
    lat = C.c_double(-1.0)
    _check_srv(srv, lib().slr_server_poll(srv, C.c_uint64(ticket), C.byref(st), C.byref(res), C.byref(lat)))
    return st.value, res.value, (lat.value if lat.value >= 0 else None)


def slr_server_timing(srv, ticket):
    """(queue_ms, setup_ms, iterate_ms) of a finished job."""
    q, su, it = C.c_double(0), C.c_double(0), C.c_double(0)
    _check_srv(srv, lib().slr_server_timing(srv, C.c_uint64(ticket), C.byref(q), C.byref(su), C.byref(it)))
    return q.value, su.value, it.value


def slr_server_release(srv, ticket):
    _check_srv(srv, lib().slr_server_release(srv, C.c_uint64(ticket)))


def slr_server_last_error(srv):
    m = lib().slr_server_last_error(srv)
    return m.decode() if m else ""


def slr_server_destroy(srv):
    if srv:
        lib().slr_server_destroy(srv)


# ---------------------------------------------------------------------------
# convenience wrapper: one reconstruction job
# ---------------------------------------------------------------------------

def slr_multirun_default(**overrides) -> slr_multirun_config:
    mc = slr_multirun_config()
    lib().slr_multirun_default(C.byref(mc))
    names = {f[0] for f in slr_multirun_config._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError(f"slr_multirun_config has no field {k!r}")
        setattr(mc, k, v)
    return mc


def slr_reconstruct(mc, xyz, allocator=None, stream=None):
    """Runs from coarse to fine (§4); returns (context handle, report dict)."""
    pts = _f64(xyz)
    h = C.c_void_p()
    rep = slr_multirun_report()
    al = C.byref(allocator.struct) if allocator is not None else None
    st = C.c_void_p(stream) if stream else None
    status = lib().slr_reconstruct(C.byref(mc), _ptr(pts), int(pts.shape[0]), al, st, C.byref(h), C.byref(rep))
    if status != SLR_OK:
        msg = lib().slr_last_error(None)
        raise SlrError(status, msg.decode() if msg else "")
    k = rep.runs_done
    report = dict(h_s=rep.h_s, sample_size=rep.sample_size, runs_done=k, coarsened=bool(rep.coarsened),
                  run_dx=list(rep.run_dx[:k]), run_n=[tuple(rep.run_n[r][:]) for r in range(k)],
                  run_lo=[tuple(rep.run_lo[r][:]) for r in range(k)],
                  run_iters=list(rep.run_iters[:k]), run_converged=[bool(x) for x in rep.run_converged[:k]],
                  run_energy=list(rep.run_energy[:k]), run_err_cloud=list(rep.run_err_cloud[:k]),
                  run_l1_err=list(rep.run_l1_err[:k]))
    return h.value, report


def reconstruct(xyz, dim=3, precision=32, interp=1, runs=3, K_s=2.0, sample_frac=0.1, seed=1, max_nodes=1 << 27,
                max_iters=100, distance="exact", sphere=None, stream=None):
    """The paper's pipeline from a cloud (§4): h_S, the §3.6 initial data, then
    `runs` runs of Algorithm 1 from coarse to fine. distance: "exact" or
    "fsm" (the §3.4 construction). sphere = (cx, cy, cz, r): report the L^1
    error of every run against its signed distance. Returns (Reconstruction of
    the last run, report)."""
    import torch

    if distance not in ("exact", "fsm"):
        raise ValueError(f"unknown distance method {distance!r}")
    mc = slr_multirun_default(dim=dim, precision=precision, interp=interp, runs=runs, K_s=K_s,
                              sample_frac=sample_frac, seed=seed, max_nodes=max_nodes, max_iters=max_iters,
                              distance_fsm=int(distance == "fsm"), exact_sphere=int(sphere is not None))
    if sphere is not None:
        for i in range(4):
            mc.sphere[i] = float(sphere[i])
    dev = torch.cuda.current_device()
    s = stream if stream is not None else torch.cuda.Stream(dev)
    al = _TorchAllocator(dev, s.cuda_stream)
    ctx, rep = slr_reconstruct(mc, xyz, al, s.cuda_stream)
    n = rep["run_n"][-1]
    rec = Reconstruction.__new__(Reconstruction)
    rec.dim = dim
    rec.shape = tuple(int(x) for x in n)
    rec.num_nodes = int(np.prod(rec.shape))
    rec.stream = s
    rec._alloc = al
    rec.ctx = ctx
    rec.cfg = None
    return rec, rep


class Reconstruction:
    """One reconstruction job on the current CUDA device.

    Device memory comes from torch's caching allocator; work is queued on
    ``stream`` (a torch.cuda.Stream; default: a new stream owned by the job,
    so that the allocator and the kernels agree on the stream).
    """

    def __init__(self, dim=3, n=64, lo=-1.0, hi=1.0, precision=32, interp=1, band=1, stream=None, allocator="torch",
                 **cfg):
        import torch

        if isinstance(n, int):
            n = (n,) * dim + ((1,) if dim == 2 else ())
        if isinstance(lo, (int, float)):
            lo = (lo,) * dim
        if isinstance(hi, (int, float)):
            hi = (hi,) * dim
        self.cfg = slr_config_default(dim=dim, n=n, lo=lo, hi=hi, precision=precision, interp=interp, band=band,
                                      **cfg)
        self.dim = dim
        self.shape = tuple(int(x) for x in n)
        self.num_nodes = int(np.prod(self.shape))
        dev = torch.cuda.current_device()
        s = stream if stream is not None else torch.cuda.Stream(dev)
        self.stream = s
        self._alloc = _TorchAllocator(dev, s.cuda_stream) if allocator == "torch" else None
        self.ctx = slr_create(self.cfg, self._alloc, s.cuda_stream)

    # Algorithm 1 calls
    def load_cloud(self, xyz):
        slr_load_cloud(self.ctx, xyz)

    def build_distance(self, method="exact"):
        """d on every node: "exact" (slr_build_distance) or "fsm", the §3.4
        construction (exact near the cloud, fast sweeping elsewhere)."""
        if method == "exact":
            slr_build_distance(self.ctx)
        elif method == "fsm":
            slr_build_distance_fsm(self.ctx)
        else:
            raise ValueError(f"unknown distance method {method!r}")

    def set_distance(self, d):
        slr_set_distance(self.ctx, d)

    def init_sphere(self, radius, center=(0.0, 0.0, 0.0)):
        c = list(center) + [0.0] * (3 - len(center))
        slr_init_u(self.ctx, 0, params=[c[0], c[1], c[2], radius])

    def init_array(self, u0):
        slr_init_u(self.ctx, 1, u0=u0)

    def cloud_spacing(self, sample):
        """h_S of §4: mean nearest-other-point distance over the sampled points."""
        return slr_cloud_spacing(self.ctx, sample)

    def l1_error(self, sphere=None, exact=None):
        """§4 L^1 error of the current state against an exact signed distance."""
        return slr_l1_error(self.ctx, sphere=sphere, exact=exact)

    def init_marking(self, gamma_s):
        """§3.6 initial data from the cloud: external marking and fast sweeping."""
        slr_init_u(self.ctx, 2, params=[float(gamma_s), 0.0, 0.0, 0.0])

    def step(self, n=1, energy_override=-1.0):
        slr_step(self.ctx, n, energy_override)

    def step_async(self, n=1, energy_override=-1.0):
        slr_step_async(self.ctx, n, energy_override)

    def set_profiling(self, on=True):
        slr_set_profiling(self.ctx, on)

    def last_iteration_times(self):
        return slr_last_iteration_times(self.ctx)

    def last_iteration_phases(self):
        """[SL step, reinitialisation, energy, record] of the last iteration, in ms."""
        return slr_last_iteration_phases(self.ctx)

    def evolve(self):
        return slr_evolve(self.ctx)

    def extract(self, width):
        return slr_extract(self.ctx, width)

    def u(self):
        return slr_get_field(self.ctx, SLR_FIELD_U, self.num_nodes)

    def d(self):
        return slr_get_field(self.ctx, SLR_FIELD_D, self.num_nodes)

    def argmin(self):
        return slr_get_field(self.ctx, SLR_FIELD_ARGMIN, self.num_nodes)

    def band(self):
        return slr_get_band(self.ctx)

    def energy(self, p=2.0):
        return slr_energy(self.ctx, p)

    def diagnostics(self, err_cloud=False):
        return slr_diagnostics(self.ctx, err_cloud=err_cloud)

    def export_state(self):
        return slr_export_state(self.ctx)

    def import_state(self, data):
        slr_import_state(self.ctx, data)

    @property
    def kernel_launches(self):
        return slr_kernel_launches(self.ctx)

    def brick_shape(self):
        return slr_brick_shape(self.ctx)

    def set_brick_shape(self, threads, stages):
        slr_brick_shape_set(self.ctx, threads, stages)

    def close(self):
        if getattr(self, "ctx", None):
            slr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
