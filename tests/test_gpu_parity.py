"""GPU parity: every kernel through the C ABI against the FP64 oracle.

Bars (written in each test):
  - distance argmin and band / extract index lists: bit-exact;
  - d: bit-exact (same FP64 arithmetic, same rounding to the storage type);
  - u after one SL step from identical inputs: max-abs <= 1e-12 (FP64 mode),
    <= 1e-5 * h (FP32 mode; the FP32 input is widened exactly for the
    oracle), excluding the nodes the oracle flags as within 1e-6 of the
    singular-gradient threshold (a discontinuous branch);
  - energy: relative 1e-12 (FP64) or within the ambiguous mass the oracle
    reports for subcells near the inclusion threshold plus relative 1e-5
    (FP32).
"""
import numpy as np
import pytest

import oracle as O
from paper_2410_22205_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _slr():
    from paper_2410_22205_gb300 import slr

    return slr


def tol_u(prec, h):
    return 1e-12 if prec == 64 else 1e-5 * h


def make(dim, n, prec, interp, band, lo=-1.0, hi=1.0, **kw):
    slr = _slr()
    shape = (n,) * dim if isinstance(n, int) else tuple(n)
    if dim == 2:
        shape = shape[:2] + (1,)
    los = (lo,) * dim
    his = tuple(lo + (hi - lo) * (shape[a] - 1) / (shape[0] - 1) for a in range(dim))
    rec = slr.Reconstruction(dim=dim, n=shape, lo=los, hi=his, precision=prec, interp=interp, band=band, **kw)
    okw = {k: v for k, v in kw.items() if k in ("p", "delta", "dt", "gamma", "beta", "c_sing", "alpha")}
    P = O.params(dim, shape[:dim], los, his, interp=interp, band=band, prec=prec, **okw)
    return rec, P


def step_parity(rec, P, Ep, prec):
    """One GPU step from the current GPU state vs the oracle from the same input."""
    u0 = rec.u()
    d = rec.d()
    rec.step(1, energy_override=Ep)
    u1 = rec.u()
    ref, flags, _ = O.sl_step(P, u0, d, Ep)
    ok = (flags & O.FLAG_MARGIN) == 0
    err = np.abs(u1 - ref)
    return float(err[ok].max()), int((~ok).sum()), u0, u1, ref


# ---------------------------------------------------------------- distance

@pytest.mark.parametrize("dim,n,npts", [(2, 64, 200), (3, 33, 500), (2, (37, 29), 57), (3, (19, 23, 17), 300)])
@pytest.mark.parametrize("prec", [32, 64])
def test_distance_grid_bit_exact(dim, n, npts, prec):
    rng = np.random.default_rng(npts)
    rec, P = make(dim, n, prec, 0, 1)
    pts = rng.uniform(-1.2, 1.2, (npts, dim))
    rec.load_cloud(pts)
    rec.build_distance()
    d_o, a_o = O.distance(P, pts)
    d_o = d_o.astype(np.float32).astype(np.float64) if prec == 32 else d_o
    assert np.array_equal(rec.argmin(), a_o)
    assert np.array_equal(rec.d(), d_o)


def test_distance_ties_and_duplicates_lowest_index():
    """Symmetric and duplicated points give exact ties; the lowest index wins."""
    rec, P = make(3, 21, 64, 0, 1)
    base = np.array([[0.3, 0.0, 0.0], [-0.3, 0.0, 0.0], [0.0, 0.3, 0.0], [0.0, -0.3, 0.0], [0.0, 0.0, 0.3],
                     [0.0, 0.0, -0.3], [0.5, 0.5, 0.5], [-0.5, -0.5, -0.5]])
    pts = np.concatenate([base, base[::-1], base])  # duplicates at several indices
    rec.load_cloud(pts)
    rec.build_distance()
    d_o, a_o = O.distance(P, pts)
    assert np.array_equal(rec.argmin(), a_o)
    assert np.array_equal(rec.d(), d_o)


def test_distance_single_point_and_far_cloud():
    rec, P = make(3, 17, 64, 0, 1)
    pts = np.array([[5.0, -3.0, 7.0]])
    rec.load_cloud(pts)
    rec.build_distance()
    d_o, a_o = O.distance(P, pts)
    assert np.array_equal(rec.argmin(), a_o) and np.array_equal(rec.d(), d_o)


def _leaf_shape_clouds(dim):
    """Clouds whose 32-point leaves are degenerate for the leaves' bounding
    cylinders: collinear points, points on a grid-aligned plane or line (zero
    half-height, with nodes exactly on it), coincident points, a leaf of one
    point, and clusters far apart (leaves spanning a gap)."""
    rng = np.random.default_rng(5)
    t = np.linspace(-0.9, 0.9, 300)
    if dim == 3:
        line = np.stack([t, 0.5 * t + 0.1, -0.25 * t], 1)
        plane = np.stack([rng.uniform(-0.9, 0.9, 600), rng.uniform(-0.9, 0.9, 600), np.full(600, 0.25)], 1)
        lattice = np.stack(np.meshgrid(np.linspace(-1, 1, 9), np.linspace(-1, 1, 9), [0.0]), -1).reshape(-1, 3)
        same = np.tile([[0.2, -0.3, 0.4]], (70, 1))
        clusters = np.concatenate([rng.normal(0, 0.01, (40, 3)) + c for c in
                                   ([-0.8, -0.8, -0.8], [0.8, 0.7, -0.6], [0.0, 0.9, 0.9])])
        one = np.array([[0.31, 0.47, -0.53]])
    else:
        line = np.stack([t, 0.5 * t + 0.1], 1)
        plane = np.stack([rng.uniform(-0.9, 0.9, 600), np.full(600, 0.25)], 1)
        lattice = np.stack(np.meshgrid(np.linspace(-1, 1, 17), [0.0]), -1).reshape(-1, 2)
        same = np.tile([[0.2, -0.3]], (70, 1))
        clusters = np.concatenate([rng.normal(0, 0.01, (40, 2)) + c for c in ([-0.8, -0.8], [0.8, 0.7], [0.0, 0.9])])
        one = np.array([[0.31, 0.47]])
    return {"line": line, "plane": plane, "lattice": lattice, "same": same, "clusters": clusters,
            "one_extra": np.concatenate([same[:32], one])}


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", [32, 64])
def test_distance_degenerate_leaves_bit_exact(dim, prec):
    """Leaves of degenerate shape (see _leaf_shape_clouds) prune with their
    bounding cylinders exactly as the oracle's brute force decides: argmin and
    d bit-exact on every node."""
    n = 25 if dim == 3 else 65
    for name, pts in _leaf_shape_clouds(dim).items():
        rec, P = make(dim, n, prec, 0, 1)
        rec.load_cloud(pts)
        rec.build_distance()
        d_o, a_o = O.distance(P, pts)
        d_o = d_o.astype(np.float32).astype(np.float64) if prec == 32 else d_o
        assert np.array_equal(rec.argmin(), a_o), name
        assert np.array_equal(rec.d(), d_o), name
        rec.close()


def test_distance_torus_128_sampled():
    """Torus workload size (20k points, 128^3): sampled nodes vs brute force."""
    g = synth.cube_grid(3, 128)
    pts = synth.torus_cloud(20000, 0.5, 0.2, 0.002, 1)
    rec, P = make(3, 128, 32, 1, 1)
    rec.load_cloud(pts)
    rec.build_distance()
    nodes = np.random.default_rng(0).choice(g.num_nodes, 3000, replace=False)
    d_o, a_o = O.distance(P, pts, nodes)
    assert np.array_equal(rec.argmin()[nodes], a_o)
    assert np.array_equal(rec.d()[nodes], d_o.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("dim,n,npts", [(3, (45, 38, 29), 6000), (2, (203, 157), 4000)])
def test_distance_surface_cloud_ragged_whole_grid(dim, n, npts):
    """A surface cloud deep enough for three hierarchy levels on a grid whose
    sizes are no multiple of the search's warp tile (4x4x4 nodes in 3-D, 8x8
    in 2-D): every node, d and argmin, against the oracle's k-d search."""
    rec, P = make(dim, n, 32, 1, 1)
    pts = synth.torus_cloud(npts, 0.5, 0.2, 0.002, 3) if dim == 3 else synth.circle_noisy(npts, 0.6, 0.003, 3)
    rec.load_cloud(pts)
    rec.build_distance()
    d_o, a_o = O.distance(P, pts, method="kd")
    assert np.array_equal(rec.argmin(), a_o)
    assert np.array_equal(rec.d(), d_o.astype(np.float32).astype(np.float64))


# ---------------------------------------------------------------- init, band

@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("dim", [2, 3])
def test_init_sphere_and_band_bit_exact(prec, dim):
    n = 48 if dim == 3 else 96
    rec, P = make(dim, n, prec, 1, 1)
    g = synth.cube_grid(dim, n)
    rec.set_distance(np.full(g.num_nodes, 0.3))
    rec.init_sphere(0.7)
    ref = synth.sphere_sdf(g, 0.7)
    if prec == 32:
        ref = ref.astype(np.float32).astype(np.float64)
    ref = O.cut(P, ref)
    assert np.array_equal(rec.u(), ref)
    assert np.array_equal(rec.band(), O.band(P, ref))


def test_empty_band_steps_are_no_ops():
    rec, P = make(3, 24, 32, 0, 1)
    rec.set_distance(np.full(24 ** 3, 0.2))
    rec.init_sphere(5.0)  # front far outside the grid: every node cut to -γ
    assert rec.band().size == 0
    u0 = rec.u()
    rec.step(3, energy_override=1.0)
    assert np.array_equal(rec.u(), u0)
    assert rec.band().size == 0


# ---------------------------------------------------------------- SL step

@pytest.mark.parametrize("interp", [0, 1])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("dim,n", [(2, 64), (3, 40), (3, (33, 41, 29))])
def test_sl_step_band_parity(dim, n, prec, interp):
    rec, P = make(dim, n, prec, interp, 1)
    pts = (synth.sphere_cloud(800, 0.5, 0.01, 2) if dim == 3 else synth.circle_noisy(300, 0.5, 0.01, 2))
    rec.load_cloud(pts)
    rec.build_distance()
    rec.init_sphere(0.62)
    for s in range(3):
        band_gpu_before = rec.band()
        err, nflag, u0, u1, ref = step_parity(rec, P, 0.37, prec)
        assert err <= tol_u(prec, P.h), (s, err)
        assert nflag < 5
        # the band used by this step is G^n of the state it started from
        assert np.array_equal(rec.band(), O.band(P, u0))
        assert set(rec.band()) <= set(band_gpu_before)


@pytest.mark.parametrize("interp", [0, 1])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("dim", [2, 3])
def test_sl_step_full_grid_parity(dim, prec, interp):
    n = 48 if dim == 2 else 26
    rec, P = make(dim, n, prec, interp, 0)
    pts = synth.sphere_cloud(300, 0.45, 0.0, 5) if dim == 3 else synth.circle_noisy(200, 0.5, 0.005, 0)
    rec.load_cloud(pts)
    rec.build_distance()
    rec.init_sphere(0.9)
    for s in range(2):
        err, nflag, *_ = step_parity(rec, P, 0.21, prec)
        assert err <= tol_u(prec, P.h), (s, err)


@pytest.mark.parametrize("p,delta", [(1.0, 0.0), (1.0, 1.0), (3.0, 0.5), (2.0, 0.0)])
def test_sl_step_parameters(p, delta):
    rec, P = make(3, 30, 64, 1, 1, p=p, delta=delta)
    rec.load_cloud(synth.torus_cloud(3000, 0.5, 0.2, 0.002, 4))
    rec.build_distance()
    rec.init_sphere(0.7)
    err, *_ = step_parity(rec, P, 0.8, 64)
    assert err <= 1e-12


def test_singular_fallback_node_at_centre():
    """Odd n puts a node at the sphere centre: eq. SL:2 on both sides."""
    rec, P = make(3, 9, 64, 1, 0, p=1.0)
    rec.set_distance(np.full(9 ** 3, 0.2))
    rec.init_sphere(0.5)
    err, nflag, u0, u1, ref = step_parity(rec, P, 1.0, 64)
    c = 4 + 9 * (4 + 9 * 4)
    assert err <= 1e-12 and u1[c] == pytest.approx(P.h - 0.5, abs=1e-15)


def test_step_is_deterministic():
    outs = []
    for _ in range(2):
        rec, P = make(3, 40, 32, 1, 1)
        rec.load_cloud(synth.sphere_cloud(2000, 0.5, 0.01, 9))
        rec.build_distance()
        rec.init_sphere(0.62)
        rec.step(4)
        outs.append((rec.u(), rec.band(), rec.diagnostics()["e2"]))
        rec.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert np.array_equal(outs[0][2], outs[1][2])


# ---------------------------------------------------------------- energy

@pytest.mark.parametrize("interp", [0, 1])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("band", [0, 1])
def test_energy_parity(dim, prec, interp, band):
    n = 64 if dim == 2 else 36
    rec, P = make(dim, n, prec, interp, band)
    pts = synth.sphere_cloud(1500, 0.5, 0.01, 3) if dim == 3 else synth.circle_noisy(200, 0.5, 0.005, 0)
    rec.load_cloud(pts)
    rec.build_distance()
    rec.init_sphere(0.61)
    if band:
        rec.step(2, energy_override=0.4)
    u, d = rec.u(), rec.d()
    for p in (2.0, 1.0, 3.0):
        E, S = rec.energy(p)
        amb_tol = 0.0 if prec == 64 else 1e-5 * P.h / 5
        ref = O.energy(P, u, d, p, 5, amb_tol)
        if prec == 64:
            assert S == pytest.approx(ref["sum"], rel=1e-12, abs=1e-300)
        else:
            assert abs(S - ref["sum"]) <= ref["amb"] + 1e-5 * ref["sum"]


def test_energy_2d_paper_circle():
    """The paper's 64-point unit circle with the exact SDF: GPU E_2 matches
    the oracle to 1e-12 and approaches 7.1035e-2."""
    n = 201
    rec, P = make(2, n, 64, 1, 0, lo=-1.3, hi=1.3)
    pts = synth.circle_uniform(64, 1.0)
    rec.load_cloud(pts)
    rec.build_distance()
    g = synth.cube_grid(2, n, -1.3, 1.3)
    rec.init_array(synth.sphere_sdf(g, 1.0))
    E, S = rec.energy(2.0)
    ref = O.energy(P, rec.u(), rec.d(), 2.0)
    assert S == pytest.approx(ref["sum"], rel=1e-12)
    assert E == pytest.approx(7.103510780002126e-02, rel=2e-2)


# ---------------------------------------------------------------- evolve, extract, diagnostics

def test_circle64_workload_100_steps_fp64_q1():
    """Small 2-D workload: 200 noisy circle points, 64^2 on [-1,1]^2,
    u0 = circle r = 0.9, 100 SL steps, whole grid, FP64 Q1, each step with
    the GPU's own E_2. Every step is compared with the oracle from the same
    input state and energy (<= 1e-12); the GPU energies match the oracle's
    energy of the same state (rel 1e-12). Free-running drift is not gated:
    in whole-grid mode a one-ulp change of u0 already grows to 1e-3 by step
    85 in the oracle alone (boundary rows, one-sided differences)."""
    wl = synth.workload_circle64()
    rec, P = make(2, 64, 64, 0, 0)
    rec.load_cloud(wl["cloud"])
    rec.build_distance()
    rec.init_sphere(0.9)
    d = rec.d()
    worst = 0.0
    for s in range(100):
        u = rec.u()
        E = rec.diagnostics()["e2"][s]
        assert E == pytest.approx(O.energy(P, u, d, 2.0)["E"], rel=1e-12)
        rec.step(1)
        ref, flags, _ = O.sl_step(P, u, d, E)
        ok = (flags & O.FLAG_MARGIN) == 0
        worst = max(worst, float(np.abs(rec.u() - ref)[ok].max()))
    assert worst <= 1e-12, worst
    assert rec.diagnostics()["iters"] == 100


@pytest.mark.parametrize("interp", [0, 1])
def test_plane_front_moves_at_unit_speed_toward_a_line_cloud(interp):
    """The closed form the oracle is pinned to, through the C ABI: FP64, whole
    grid, p = 1, δ = 0, a line cloud y = c with one point above every node
    column, the plane front y = y0; 8 steps. Every node equals the oracle's
    loop (<= 1e-12), and the rows beyond the reach of the line and the grid
    edge equal y - (y0 - 8Δt) (<= 1e-12)."""
    n, steps = 64, 8
    rec, P = make(2, n, 64, interp, 0, p=1.0, delta=0.0)
    h, dt = P.h, P.dt
    x = -1.0 + h * np.arange(n)
    c = -1.0 + 10.5 * h
    rec.load_cloud(np.stack([x, np.full(n, c)], 1))
    rec.build_distance()
    X, Y = np.meshgrid(x, x)
    y0 = -1.0 + 40.3 * h
    u0 = (Y - y0).reshape(-1)
    rec.init_array(u0)
    rec.step(steps)
    u = rec.u()
    ref = O.evolve(P, u0, rec.d(), min_iters=steps, max_iters=steps)
    assert ref["iters"] == steps
    assert np.abs(u - ref["u"]).max() <= 1e-12
    reach = (1 if interp == 0 else 2) * (steps + 1)
    rows = np.arange(n)
    clean = (rows > 10.5 + reach) & (rows < n - 1 - reach)
    err = np.abs(u.reshape(n, n) - (Y - (y0 - steps * dt)))[clean]
    assert err.max() <= 1e-12


@pytest.mark.parametrize("interp", [0, 1])
def test_plane_front_moves_at_unit_speed_toward_a_plane_cloud_3d(interp):
    """The 3-D closed form through the C ABI: FP64, whole grid, p = 1, δ = 0,
    a plane cloud z = c with one point above every (x, y) node column, the
    front z = z0; 6 steps. Every node equals the oracle's loop (<= 1e-12); the
    planes beyond the reach of the cloud and the grid edge equal
    z - (z0 - 6Δt) (<= 1e-12)."""
    n, steps = 40, 6
    rec, P = make(3, n, 64, interp, 0, p=1.0, delta=0.0)
    h, dt = P.h, P.dt
    x = -1.0 + h * np.arange(n)
    c = -1.0 + 6.5 * h
    Xp, Yp = np.meshgrid(x, x, indexing="ij")
    rec.load_cloud(np.stack([Xp.ravel(), Yp.ravel(), np.full(n * n, c)], 1))
    rec.build_distance()
    Z = np.broadcast_to(x[:, None, None], (n, n, n))
    z0 = -1.0 + 24.3 * h
    u0 = np.ascontiguousarray(Z - z0).reshape(-1)
    rec.init_array(u0)
    rec.step(steps)
    u = rec.u()
    ref = O.evolve(P, u0, rec.d(), min_iters=steps, max_iters=steps)
    assert ref["iters"] == steps
    assert np.abs(u - ref["u"]).max() <= 1e-12
    reach = (1 if interp == 0 else 2) * (steps + 1)
    planes = np.arange(n)
    clean = (planes > 6.5 + reach) & (planes < n - 1 - reach)
    err = np.abs(u.reshape(n, n, n) - (Z - (z0 - steps * dt)))[clean]
    assert err.max() <= 1e-12


@pytest.mark.parametrize("kmax,min_iters,tol", [(10, 10, 1e-4), (3, 2, 1e-3), (25, 5, 1e-3)])
def test_evolve_matches_oracle_stop_rule(kmax, min_iters, tol):
    rec, P = make(2, 48, 64, 1, 1, p=1.0, delta=0.0, stop_k=kmax, min_iters=min_iters, stop_tol=tol)
    pts = synth.circle_noisy(150, 0.5, 0.0, 0)
    rec.load_cloud(pts)
    rec.build_distance()
    rec.init_sphere(0.8)
    u0, d = rec.u(), rec.d()
    iters, conv = rec.evolve()
    ref = O.evolve(P, u0, d, kmax=kmax, min_iters=min_iters, tol=tol)
    assert iters == ref["iters"] and conv == ref["converged"]
    assert np.abs(rec.u() - ref["u"]).max() <= 1e-10
    np.testing.assert_allclose(rec.diagnostics()["e2"], ref["E2"], rtol=1e-10)


@pytest.mark.parametrize("prec", [32, 64])
def test_extract_and_err_cloud(prec):
    rec, P = make(3, 40, prec, 1, 1)
    pts = synth.sphere_cloud(1000, 0.5, 0.0, 1)
    rec.load_cloud(pts)
    rec.build_distance()
    rec.init_sphere(0.55)
    rec.step(2, energy_override=0.5)
    u = rec.u()
    idx, val = rec.extract(2 * P.h)
    ridx, rval = O.extract(P, u, 2 * P.h)
    assert np.array_equal(idx, ridx) and np.array_equal(val, rval)
    es = rec.diagnostics(err_cloud=True)["err_cloud"]
    assert es == pytest.approx(O.err_cloud(P, u, pts), rel=1e-12 if prec == 64 else 1e-5, abs=1e-7 * P.h)


def test_checkpoint_resume_bit_identical():
    rec, P = make(3, 36, 32, 1, 1)
    pts = synth.torus_cloud(5000, 0.5, 0.2, 0.002, 1)
    rec.load_cloud(pts)
    rec.build_distance()
    rec.init_sphere(0.7)
    rec.step(3)
    blob = rec.export_state()
    rec.step(4)
    u_ref, diag_ref = rec.u(), rec.diagnostics()
    rec2, _ = make(3, 36, 32, 1, 1)
    rec2.import_state(blob)
    rec2.step(4)
    assert np.array_equal(rec2.u(), u_ref)
    assert np.array_equal(rec2.diagnostics()["e2"], diag_ref["e2"])


def test_invalid_inputs_and_order():
    slr = _slr()
    rec, P = make(3, 16, 32, 0, 1)
    with pytest.raises(slr.SlrError) as e:
        rec.step(1)
    assert e.value.status == slr.SLR_E_STATE
    with pytest.raises(slr.SlrError) as e:
        rec.build_distance()
    assert e.value.status == slr.SLR_E_STATE
    with pytest.raises(slr.SlrError) as e:
        rec.load_cloud(np.array([[np.nan, 0.0, 0.0]]))
        rec.build_distance()
    assert e.value.status == slr.SLR_E_INVALID
    with pytest.raises(slr.SlrError):
        slr.Reconstruction(dim=3, n=(16, 16, 16), lo=(-1, -1, -1), hi=(1, 1, 2))


def test_profiling_times_and_async_steps():
    rec, P = make(3, 32, 32, 1, 1)
    rec.load_cloud(synth.sphere_cloud(1000, 0.5, 0.01, 3))
    rec.build_distance()
    rec.init_sphere(0.6)
    rec.set_profiling(True)
    rec.step_async(2)
    ms = rec.last_iteration_times()
    assert len(ms) == 3 and all(m > 0 for m in ms)
    u_async = rec.u()
    rec2, _ = make(3, 32, 32, 1, 1)
    rec2.load_cloud(synth.sphere_cloud(1000, 0.5, 0.01, 3))
    rec2.build_distance()
    rec2.init_sphere(0.6)
    rec2.step(2)
    assert np.array_equal(rec2.u(), u_async)


def _small_job(kind, seed):
    """A small mixed job: (dim, n, prec, interp, band) by kind."""
    dim, n, prec, interp, band = kind
    rec, P = make(dim, n, prec, interp, band, max_iters=40)
    pts = (synth.sphere_cloud(800, 0.5, 0.01, seed) if dim == 3 else synth.circle_noisy(300, 0.5, 0.01, seed))
    rec.load_cloud(pts)
    rec.build_distance()
    rec.init_sphere(0.75)
    return rec


KINDS = [(2, 64, 32, 0, 1), (2, 96, 64, 1, 1), (3, 32, 32, 1, 1), (3, 40, 32, 0, 1), (3, 24, 64, 1, 0),
         (2, 48, 32, 1, 0)]


@pytest.mark.parametrize("chunk", [4, -1])
def test_batch_evolve_equals_solo_runs(chunk):
    """Jobs advanced together in one graph per chunk give the same states,
    iteration counts and energies as each job evolved alone; with chunk -1
    the chunk is autotuned (one of 4, 8, 16, 32) and the results are the
    same."""
    slr = _slr()
    solo = []
    for i, k in enumerate(KINDS):
        r = _small_job(k, i)
        it, conv = r.evolve()
        solo.append((it, conv, r.u(), r.diagnostics()["e2"]))
        r.close()
    jobs = [_small_job(k, i) for i, k in enumerate(KINDS)]
    its, convs = slr.slr_batch_evolve([j.ctx for j in jobs], chunk=chunk)
    used = slr.slr_batch_chunk(jobs[0].ctx)
    assert used == chunk if chunk > 0 else used in (4, 8, 16, 32)
    for idx, (j, (it, conv, u, e2)) in enumerate(zip(jobs, solo)):
        assert its[idx] == it and convs[idx] == conv
        assert np.array_equal(j.u(), u)
        assert np.array_equal(j.diagnostics()["e2"], e2)


@pytest.mark.parametrize("policy", [0, 1])
def test_server_results_equal_solo_runs(policy):
    """Continuous batching: jobs submitted into a running mix (at most 3
    admitted at once, a tight memory budget) finish with exactly the state,
    iteration count and energies of the same job run alone, whether the
    server admits the oldest request first (policy 0) or the least estimated
    set-up first (policy 1)."""
    import time

    slr = _slr()
    specs = []
    for i, k in enumerate(KINDS):
        dim, n, prec, interp, band = k
        shape = (n,) * dim + ((1,) if dim == 2 else ())
        cfg = slr.slr_config_default(dim=dim, n=shape, lo=(-1.0,) * dim, hi=(1.0,) * dim, precision=prec,
                                     interp=interp, band=band, max_iters=40)
        pts = (synth.sphere_cloud(800, 0.5, 0.01, i) if dim == 3 else synth.circle_noisy(300, 0.5, 0.01, i))
        specs.append((cfg, pts))
    solo = []
    for i, k in enumerate(KINDS):
        r = _small_job(k, i)
        it, conv = r.evolve()
        solo.append((it, r.u(), r.diagnostics()["e2"]))
        r.close()
    srv = slr.slr_server_create(64 << 20, max_active=3, setup_threads=2, policy=policy)
    try:
        tickets = []
        for cfg, pts in specs:
            tickets.append(slr.slr_server_submit(srv, cfg, pts, (0.0, 0.0, 0.0, 0.75)))
            time.sleep(0.002)
        results = {}
        t0 = time.time()
        while len(results) < len(tickets) and time.time() - t0 < 120:
            for t in tickets:
                if t in results:
                    continue
                st, ctx, lat = slr.slr_server_poll(srv, t)
                if st == 2:
                    n_nodes = int(np.prod([specs[tickets.index(t)][0].n[a] for a in range(3)]))
                    u = slr.slr_get_field(ctx, slr.SLR_FIELD_U, n_nodes)
                    d = slr.slr_diagnostics(ctx)
                    q, su, itm = slr.slr_server_timing(srv, t)
                    # the three parts of the latency: queue, set-up, iterations
                    assert min(q, su, itm) >= 0.0 and abs(q + su + itm - lat) <= 1e-6 * max(lat, 1.0)
                    results[t] = (d["iters"], u, d["e2"], lat)
                    slr.slr_server_release(srv, t)
                    with pytest.raises(slr.SlrError):
                        slr.slr_server_timing(srv, t)  # released
            time.sleep(0.005)
        assert len(results) == len(tickets)
        for t, (it, u, e2) in zip(tickets, solo):
            rit, ru, re2, lat = results[t]
            assert rit == it and np.array_equal(ru, u) and np.array_equal(re2, e2)
            assert lat is not None and lat > 0
    finally:
        slr.slr_server_destroy(srv)
