"""FP64 CPU oracle of the semi-Lagrangian level-set step (arXiv 2410.22205).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product
(``paper_2410_22205_gb300``) never does, and the two share no code.

The arithmetic lives in ``slr_oracle.c`` (plain C99, FP64,
``-ffp-contract=off``); this module compiles it with gcc on first use and
wraps it with ctypes, converting numpy arrays to FP64.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slr_oracle.c")
_HDR = os.path.join(_HERE, "slr_oracle.h")
_LIB = os.path.join(_HERE, "libslr_oracle.so")
_lock = threading.Lock()
_lib = None

FLAG_FALLBACK = 1
FLAG_MARGIN = 2
FLAG_REGULAR = 4


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libslr_oracle.so`` (gcc, OpenMP)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class MultirunReport(C.Structure):
    _fields_ = [
        ("h_s", C.c_double),
        ("sample_size", C.c_longlong),
        ("runs_done", C.c_int),
        ("run_dx", C.c_double * 8),
        ("run_n", (C.c_longlong * 3) * 8),
        ("run_lo", (C.c_double * 3) * 8),
        ("run_iters", C.c_int * 8),
        ("run_converged", C.c_int * 8),
        ("run_energy", C.c_double * 8),
        ("run_err_cloud", C.c_double * 8),
        ("run_l1_err", C.c_double * 8),
    ]


class Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("n", C.c_longlong * 3),
        ("lo", C.c_double * 3),
        ("h", C.c_double),
        ("interp", C.c_int),
        ("p", C.c_double),
        ("delta", C.c_double),
        ("dt", C.c_double),
        ("band", C.c_int),
        ("gamma", C.c_double),
        ("beta", C.c_double),
        ("c_sing", C.c_double),
        ("alpha", C.c_double),
        ("prec", C.c_int),
    ]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_lp = C.POINTER(C.c_longlong)
_P = C.POINTER(Params)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            sig = {
                "or_num_nodes": (C.c_longlong, [_P]),
                "or_node_coord": (None, [_P, C.c_longlong, _dp]),
                "or_distance": (None, [_P, _dp, C.c_longlong, _lp, C.c_longlong, _dp, _ip]),
                "or_distance_kd": (None, [_P, _dp, C.c_longlong, _lp, C.c_longlong, _dp, _ip]),
                "or_gradient": (None, [_P, _dp, C.c_longlong, _dp]),
                "or_interp_q1": (C.c_double, [_P, _dp, _dp]),
                "or_weno1d": (C.c_double, [_dp, C.c_double, C.c_double]),
                "or_weno1d_weights": (C.c_double, [_dp, C.c_double, C.c_double, _dp]),
                "or_interp_weno": (C.c_double, [_P, _dp, _dp]),
                "or_interp": (C.c_double, [_P, _dp, _dp]),
                "or_cutoff": (C.c_double, [_P, C.c_double]),
                "or_in_band": (C.c_int, [_P, C.c_double]),
                "or_cut": (C.c_double, [_P, C.c_double]),
                "or_cut_all": (None, [_P, _dp]),
                "or_band": (C.c_longlong, [_P, _dp, _lp]),
                "or_sigma2d": (None, [_dp, _dp]),
                "or_tangent_basis": (C.c_int, [_dp, _dp, _dp]),
                "or_feet": (C.c_int, [_P, _dp, _dp, _dp, C.c_double, C.c_double, _dp]),
                "or_scale_factor": (C.c_double, [_P, C.c_double, C.c_double]),
                "or_sl_node": (C.c_double, [_P, _dp, _dp, C.c_double, C.c_longlong, _ip]),
                "or_sl_step": (C.c_double, [_P, _dp, _dp, C.c_double, _dp, _ip]),
                "or_sl_nodes": (None, [_P, _dp, _dp, C.c_double, _lp, C.c_longlong, _dp, _ip]),
                "or_energy": (None, [_P, _dp, _dp, C.c_double, C.c_int, C.c_double, _dp]),
                "or_stop": (C.c_int, [_dp, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, _dp]),
                "or_evolve": (C.c_int, [_P, _dp, _dp, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, _dp, _dp,
                                        _ip]),
                "or_evolve_reinit": (C.c_int, [_P, _dp, _dp, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int,
                                               C.c_int, C.c_double, _dp, _dp, _ip]),
                "or_reinit": (C.c_longlong, [_P, _dp, _dp, C.c_int, C.c_double, _dp, C.POINTER(C.c_ubyte)]),
                "or_reinit_sweeps": (C.c_int, [_P]),
                "or_init_marking": (C.c_longlong, [_P, _dp, C.c_double, _dp, C.POINTER(C.c_ubyte)]),
                "or_fsm_solve": (C.c_double, [_dp, C.c_int, C.c_double]),
                "or_cloud_spacing": (C.c_double, [C.c_int, _dp, C.c_longlong, _lp, C.c_longlong]),
                "or_distance_fsm": (C.c_longlong, [C.POINTER(Params), _dp, C.c_longlong, _dp, C.POINTER(C.c_ubyte)]),
                "or_splitmix64": (C.c_ulonglong, [C.c_ulonglong, C.c_ulonglong]),
                "or_reconstruct": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_ulonglong,
                                             C.c_longlong, C.c_int, C.c_int, C.c_int, _dp, _dp, C.c_longlong, _dp,
                                             C.c_longlong, C.POINTER(MultirunReport)]),
                "or_l1_error": (C.c_double, [_P, _dp, _dp]),
                "or_sdf_sphere": (None, [_P, _dp, _dp]),
                "or_extract": (C.c_longlong, [_P, _dp, C.c_double, _lp, _dp]),
                "or_err_cloud": (C.c_double, [_P, _dp, _dp, C.c_longlong]),
                "or_set_threads": (C.c_int, [C.c_int]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _l(a):
    a = np.ascontiguousarray(a, dtype=np.int64)
    return a, a.ctypes.data_as(_lp)


def params(dim, n, lo, hi=None, h=None, interp=0, p=2.0, delta=1.0, dt=None, band=0, gamma=None, beta=None,
           c_sing=1e-3, alpha=1.0, prec=64) -> Params:
    """Build the parameter block with the paper's defaults: Δt = Δx/4
    (eq. dxdt), γ = 4Δx / 6Δx and β = 2Δx / 3Δx in 2-D / 3-D (§3.8),
    C = 1e-3 and α = 1 for the singular test (§3.1)."""
    n = list(n) + [1] * (3 - len(n))
    lo = list(lo) + [0.0] * (3 - len(lo))
    if h is None:
        h = (hi[0] - lo[0]) / (n[0] - 1)
    if dt is None:
        dt = h / 4.0
    if gamma is None:
        gamma = (4.0 if dim == 2 else 6.0) * h
    if beta is None:
        beta = (2.0 if dim == 2 else 3.0) * h
    P = Params()
    P.dim = dim
    for a in range(3):
        P.n[a] = int(n[a])
        P.lo[a] = float(lo[a])
    P.h, P.interp, P.p, P.delta, P.dt = float(h), int(interp), float(p), float(delta), float(dt)
    P.band, P.gamma, P.beta, P.c_sing, P.alpha, P.prec = int(band), float(gamma), float(beta), float(c_sing), \
        float(alpha), int(prec)
    return P


def params_for_grid(grid, **kw) -> Params:
    return params(grid.dim, grid.n, grid.lo, grid.hi, **kw)


def num_nodes(P):
    return int(P.n[0] * P.n[1] * P.n[2])


def distance(P, pts, nodes=None, method="brute"):
    """d and argmin on all nodes (or the listed ones). method "brute" scans
    every point; "kd" uses the k-d tree with identical decisions."""
    pts, pp = _d(pts)
    if nodes is None:
        m = num_nodes(P)
        np_ = None
        lp = None
    else:
        np_, lp = _l(nodes)
        m = np_.size
    d = np.empty(m, np.float64)
    arg = np.empty(m, np.int32)
    f = lib().or_distance_kd if method == "kd" else lib().or_distance
    f(C.byref(P), pp, pts.shape[0], lp, m, d.ctypes.data_as(_dp), arg.ctypes.data_as(_ip))
    return d, arg


def gradient(P, v, idx):
    v, vp = _d(v)
    out = np.zeros(3)
    lib().or_gradient(C.byref(P), vp, int(idx), out.ctypes.data_as(_dp))
    return out


def interp(P, v, x, kind=None):
    v, vp = _d(v)
    x = np.asarray(x, dtype=np.float64)
    pts = np.atleast_2d(x)
    out = np.empty(pts.shape[0])
    f = {None: lib().or_interp, "q1": lib().or_interp_q1, "weno": lib().or_interp_weno}[kind]
    for i, q in enumerate(pts):
        q3 = np.zeros(3)
        q3[: q.size] = q
        out[i] = f(C.byref(P), vp, q3.ctypes.data_as(_dp))
    return out if x.ndim > 1 else out[0]


def weno1d(v, theta, h, with_weights=False):
    v, vp = _d(v)
    if with_weights:
        w = np.zeros(2)
        r = lib().or_weno1d_weights(vp, float(theta), float(h), w.ctypes.data_as(_dp))
        return r, w
    return lib().or_weno1d(vp, float(theta), float(h))


def cutoff(P, u):
    return lib().or_cutoff(C.byref(P), float(u))


def in_band(P, u):
    return bool(lib().or_in_band(C.byref(P), float(u)))


def cut(P, u):
    u = np.array(u, dtype=np.float64, copy=True)
    lib().or_cut_all(C.byref(P), u.ctypes.data_as(_dp))
    return u


def band(P, u):
    u, up = _d(u)
    m = lib().or_band(C.byref(P), up, None)
    out = np.empty(max(m, 1), np.int64)
    lib().or_band(C.byref(P), up, out.ctypes.data_as(_lp))
    return out[:m]


def sigma2d(grad):
    g = np.zeros(3)
    g[:2] = grad[:2]
    s = np.zeros(3)
    lib().or_sigma2d(g.ctypes.data_as(_dp), s.ctypes.data_as(_dp))
    return s[:2]


def tangent_basis(grad):
    g = np.asarray(grad, dtype=np.float64).copy()
    n1 = np.zeros(3)
    n2 = np.zeros(3)
    reg = lib().or_tangent_basis(g.ctypes.data_as(_dp), n1.ctypes.data_as(_dp), n2.ctypes.data_as(_dp))
    return n1, n2, bool(reg)


def feet(P, xj, grad_u, grad_d, dj, ct):
    a = [np.zeros(3) for _ in range(3)]
    for dst, src in zip(a, (xj, grad_u, grad_d)):
        dst[: len(src)] = src
    out = np.zeros((4, 3))
    k = lib().or_feet(C.byref(P), a[0].ctypes.data_as(_dp), a[1].ctypes.data_as(_dp), a[2].ctypes.data_as(_dp),
                      float(dj), float(ct), out.ctypes.data_as(_dp))
    return out[:k, : P.dim]


def scale_factor(P, dj, Ep):
    return lib().or_scale_factor(C.byref(P), float(dj), float(Ep))


def sl_step(P, u, d, Ep):
    """One SL step of every node (band + cut in band mode); returns
    (u_next, flags, dphi)."""
    u, up = _d(u)
    d, dp = _d(d)
    out = np.empty_like(u)
    flags = np.zeros(u.size, np.int32)
    dphi = lib().or_sl_step(C.byref(P), up, dp, float(Ep), out.ctypes.data_as(_dp), flags.ctypes.data_as(_ip))
    return out, flags, dphi


def sl_nodes(P, u, d, Ep, nodes):
    u, up = _d(u)
    d, dp = _d(d)
    nodes, lp = _l(nodes)
    out = np.empty(nodes.size)
    flags = np.zeros(nodes.size, np.int32)
    lib().or_sl_nodes(C.byref(P), up, dp, float(Ep), lp, nodes.size, out.ctypes.data_as(_dp),
                      flags.ctypes.data_as(_ip))
    return out, flags


def energy(P, u, d, p=2.0, R=5, amb_tol=0.0):
    """Returns dict(sum=Σ|d|^p·measure, E=E_p, amb=ambiguous part, cells=front cells)."""
    u, up = _d(u)
    d, dp = _d(d)
    out = np.zeros(4)
    lib().or_energy(C.byref(P), up, dp, float(p), int(R), float(amb_tol), out.ctypes.data_as(_dp))
    return dict(sum=out[0], E=out[1], amb=out[2], cells=int(out[3]))


def stop(E2, n, kmax=10, tol=1e-4, min_iters=10, max_iters=100):
    E2, ep = _d(E2)
    delta = C.c_double(0.0)
    s = lib().or_stop(ep, int(n), int(kmax), float(tol), int(min_iters), int(max_iters), C.byref(delta))
    return bool(s), delta.value


def evolve(P, u0, d, R=5, tol=1e-4, kmax=10, min_iters=10, max_iters=100, reinit=False, sweeps=0, dtau=0.0):
    """Algorithm 1 loop (§4 stop rule); with reinit, the reinitialisation (§3.7) after every SL step."""
    u = np.array(u0, dtype=np.float64, copy=True)
    d, dp = _d(d)
    E2 = np.zeros(max_iters + 1)
    dphi = np.zeros(max(max_iters, 1))
    conv = C.c_int(0)
    n = lib().or_evolve_reinit(C.byref(P), u.ctypes.data_as(_dp), dp, int(R), float(tol), int(kmax), int(min_iters),
                               int(max_iters), int(bool(reinit)), int(sweeps), float(dtau), E2.ctypes.data_as(_dp),
                               dphi.ctypes.data_as(_dp), C.byref(conv))
    return dict(u=u, iters=n, converged=bool(conv.value), E2=E2[: n + 1], dphi=dphi[:n])


def reinit(P, phi_band, phi_tilde, sweeps=0, dtau=0.0):
    """§3.7 reinitialisation of phi_tilde on the band {|phi_band| < γ} and its
    face neighbours, then eq. cut. Returns (out, flags, |Ḡ|); flags bit 0 =
    node in Ḡ, bit 1 = interface node (explicit step)."""
    pb, pbp = _d(phi_band)
    pt, ptp = _d(phi_tilde)
    out = np.empty_like(pt)
    flags = np.zeros(pt.shape[0], dtype=np.uint8)
    m = lib().or_reinit(C.byref(P), pbp, ptp, int(sweeps), float(dtau), out.ctypes.data_as(_dp),
                        flags.ctypes.data_as(C.POINTER(C.c_ubyte)))
    return out, flags, int(m)


def init_marking(P, d, gamma_s):
    """§3.6 initial data from the distance field: returns (φ0, external flags)."""
    d, dp = _d(d)
    out = np.empty_like(d)
    ext = np.zeros(d.shape[0], dtype=np.uint8)
    lib().or_init_marking(C.byref(P), dp, float(gamma_s), out.ctypes.data_as(_dp),
                          ext.ctypes.data_as(C.POINTER(C.c_ubyte)))
    return out, ext


def cloud_spacing(pts, sample):
    """h_S of §4: mean distance from each sampled point to its nearest other point."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    smp = np.ascontiguousarray(sample, dtype=np.int64)
    return float(lib().or_cloud_spacing(int(pts.shape[1]), pts.ctypes.data_as(_dp), int(pts.shape[0]),
                                        smp.ctypes.data_as(_lp), int(smp.size)))


def distance_fsm(P, pts):
    """§3.4 distance grid: exact on the box of 4^dim nodes around each point,
    fast sweeping elsewhere. Returns (d, fixed mask)."""
    pts, pp = _d(pts)
    N = num_nodes(P)
    d = np.empty(N)
    fix = np.zeros(N, np.uint8)
    m = lib().or_distance_fsm(C.byref(P), pp, pts.shape[0], d.ctypes.data_as(_dp),
                              fix.ctypes.data_as(C.POINTER(C.c_ubyte)))
    if m == 0:
        raise ValueError("no point of the cloud lies within one cell of the grid")
    return d, fix


def splitmix64(seed, i):
    return int(lib().or_splitmix64(int(seed), int(i)))


def reconstruct(pts, dim, prec=64, interp=0, runs=2, K_s=2.0, sample_frac=0.1, seed=1, max_nodes=1 << 20,
                max_iters=100, distance="exact", sphere=None):
    """§4 runs from coarse to fine; returns (φ of the last run, report dict).
    sphere = (cx, cy, cz, r): also report the L^1 error against its signed
    distance."""
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    out = np.empty(max_nodes)
    rep = MultirunReport()
    sph = np.zeros(4) if sphere is None else np.asarray(sphere, dtype=np.float64)
    rc = lib().or_reconstruct(int(dim), int(prec), int(interp), int(runs), float(K_s), float(sample_frac), int(seed),
                              int(max_nodes), int(max_iters), int(distance == "fsm"), int(sphere is not None),
                              sph.ctypes.data_as(_dp), pts.ctypes.data_as(_dp), int(pts.shape[0]),
                              out.ctypes.data_as(_dp), int(max_nodes), C.byref(rep))
    if rc != 0:
        raise ValueError("or_reconstruct failed")
    k = rep.runs_done
    n = tuple(rep.run_n[k - 1][:])
    return out[: int(np.prod(n))].copy(), dict(
        h_s=rep.h_s, sample_size=rep.sample_size, runs_done=k, run_dx=list(rep.run_dx[:k]),
        run_n=[tuple(rep.run_n[r][:]) for r in range(k)], run_lo=[tuple(rep.run_lo[r][:]) for r in range(k)],
        run_iters=list(rep.run_iters[:k]), run_converged=[bool(x) for x in rep.run_converged[:k]],
        run_energy=list(rep.run_energy[:k]), run_err_cloud=list(rep.run_err_cloud[:k]),
        run_l1_err=list(rep.run_l1_err[:k]))


def l1_error(P, u, exact):
    """§4 L^1 error Δx^dim Σ|c(u) - c(φ*)| (c: the cut at γ in band mode)."""
    u, up = _d(u)
    exact, ep = _d(exact)
    return float(lib().or_l1_error(C.byref(P), up, ep))


def sdf_sphere(P, sphere):
    out = np.empty(num_nodes(P))
    s = np.asarray(sphere, dtype=np.float64)
    lib().or_sdf_sphere(C.byref(P), s.ctypes.data_as(_dp), out.ctypes.data_as(_dp))
    return out


def fsm_solve(a, h):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return float(lib().or_fsm_solve(a.ctypes.data_as(_dp), int(a.size), float(h)))


def reinit_sweeps(P):
    return int(lib().or_reinit_sweeps(C.byref(P)))


def extract(P, u, width):
    u, up = _d(u)
    m = lib().or_extract(C.byref(P), up, float(width), None, None)
    idx = np.empty(max(m, 1), np.int64)
    val = np.empty(max(m, 1))
    lib().or_extract(C.byref(P), up, float(width), idx.ctypes.data_as(_lp), val.ctypes.data_as(_dp))
    return idx[:m], val[:m]


def err_cloud(P, u, pts):
    u, up = _d(u)
    pts, pp = _d(pts)
    return lib().or_err_cloud(C.byref(P), up, pp, pts.shape[0])


def set_threads(n: int) -> int:
    return lib().or_set_threads(int(n))


def node_coords(P):
    """All node coordinates (N, dim) as lo + i*h."""
    ax = [P.lo[a] + np.arange(P.n[a], dtype=np.float64) * P.h for a in range(P.dim)]
    if P.dim == 2:
        y, x = np.meshgrid(ax[1], ax[0], indexing="ij")
        return np.stack([x.ravel(), y.ravel()], axis=1)
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


SQRT3_2 = math.sqrt(3.0) / 2.0
