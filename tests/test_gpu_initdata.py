"""GPU parity of the §3.6 initial data (external marking and fast sweeping)
through the C ABI against the oracle.

Bar: φ^0 bit-exact. Both sides decide the marking on the same stored d (the
GPU's d equals the oracle's exact distance rounded to the storage type),
compute the FP64 field with the same correctly rounded operations in the same
order (the GPU's plane-by-plane sweeps see the same values as the oracle's
lexicographic ones), and round and cut it the same way.
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


def expected_u0(P, d_stored, gamma_s, prec, band):
    phi, ext = O.init_marking(P, d_stored, gamma_s)
    if prec == 32:
        u = phi.astype(np.float32)
        if band:
            g = np.float32(P.gamma)
            u = np.minimum(np.maximum(u, -g), g)
        return u.astype(np.float64), ext
    if band:
        phi = np.minimum(np.maximum(phi, -P.gamma), P.gamma)
    return phi, ext


@pytest.mark.parametrize("dim,n,prec,band", [(2, 96, 64, 1), (2, 77, 32, 1), (3, 40, 32, 1), (3, 33, 64, 0),
                                             (3, 48, 32, 0)])
def test_initial_data_bit_exact(dim, n, prec, band):
    slr = _slr()
    shape = (n,) * dim + ((1,) if dim == 2 else ())
    rec = slr.Reconstruction(dim=dim, n=shape, precision=prec, interp=1, band=band)
    P = O.params(dim, (n,) * dim, (-1.0,) * dim, (1.0,) * dim, band=band, prec=prec)
    if dim == 3:
        pts = synth.superquadric_union_cloud(30000, 3, 5)
    else:
        pts = synth.circle_noisy(800, 0.5, 0.01, 2)
    rec.load_cloud(pts)
    rec.build_distance()
    d = rec.d()
    d_ref, _ = O.distance(P, pts, method="kd")
    if prec == 32:
        d_ref = d_ref.astype(np.float32).astype(np.float64)
    assert np.array_equal(d, d_ref)
    gamma_s = 2.5 * P.h
    rec.init_marking(gamma_s)
    u = rec.u()
    ref, ext = expected_u0(P, d, gamma_s, prec, band)
    assert ext.sum() > 0 and (ext == 0).sum() > 0
    assert np.array_equal(u, ref)
    # a signed distance around the cloud: non-negative exactly on the marked nodes
    assert np.array_equal(u >= 0, ext == 1)


def test_initial_data_rejects_bad_threshold():
    slr = _slr()
    rec = slr.Reconstruction(dim=3, n=24, precision=32, interp=1, band=1)
    rec.load_cloud(synth.sphere_cloud(500, 0.5, 0.0, 1))
    rec.build_distance()
    with pytest.raises(slr.SlrError) as e:
        rec.init_marking(0.0)
    assert e.value.status == slr.SLR_E_INVALID


def test_evolution_from_the_initial_data_stays_on_the_cloud():
    """Started from the §3.6 initial data (zero set at about γ_S from the
    cloud), a short evolution with the reinitialisation brings the zero set
    onto the cloud: error on the cloud (eq. errCloud) below h/2."""
    slr = _slr()
    n = 64
    h = 2.0 / (n - 1)
    pts = synth.sphere_cloud(20000, 0.55, 0.0, 4)
    rec = slr.Reconstruction(dim=3, n=n, precision=32, interp=1, band=1, reinit=1, p=1.0, delta=0.0,
                             max_iters=40, min_iters=40)
    rec.load_cloud(pts)
    rec.build_distance()
    rec.init_marking(2.0 * h)
    e0 = rec.diagnostics(err_cloud=True)["err_cloud"]
    rec.evolve()
    e1 = rec.diagnostics(err_cloud=True)["err_cloud"]
    assert 1.5 * h < e0 < 2.5 * h
    assert e1 < 0.5 * h


@pytest.mark.parametrize("dim,npts", [(3, 40000), (2, 5000), (3, 3)])
def test_cloud_spacing_parity(dim, npts):
    """h_S of §4 on the GPU equals the oracle's (exact nearest-other-point
    distances; only the order of the mean's additions differs), with
    duplicated points in the cloud."""
    slr = _slr()
    rng = np.random.default_rng(dim + npts)
    pts = synth.superquadric_union_cloud(npts, 3, 6) if (dim == 3 and npts > 100) else (
        synth.circle_noisy(npts, 0.5, 0.01, 1) if dim == 2 else rng.uniform(-0.5, 0.5, (npts, 3)))
    pts = np.concatenate([pts, pts[: max(1, npts // 50)]])
    n = 16
    rec = slr.Reconstruction(dim=dim, n=n, precision=32, interp=1, band=1)
    rec.load_cloud(pts)
    sample = rng.choice(len(pts), max(2, len(pts) // 10), replace=False)
    h = rec.cloud_spacing(sample)
    assert h == pytest.approx(O.cloud_spacing(pts, sample), rel=1e-12)
    with pytest.raises(slr.SlrError):
        rec.cloud_spacing(np.array([0, 0]))


def _ragged(dim, shape, prec, band):
    slr = _slr()
    shape = tuple(shape) + ((1,) if dim == 2 else ())
    los = (-1.0,) * dim
    his = tuple(-1.0 + 2.0 * (shape[a] - 1) / (shape[0] - 1) for a in range(dim))
    rec = slr.Reconstruction(dim=dim, n=shape, lo=los, hi=his, precision=prec, interp=1, band=band)
    P = O.params(dim, shape[:dim], los, his, band=band, prec=prec)
    return rec, P


@pytest.mark.parametrize("dim,shape,prec", [(3, (33, 41, 29), 64), (3, (29, 23, 37), 32), (2, (37, 29), 64),
                                            (2, (29, 45), 32)])
def test_initial_data_bit_exact_on_ragged_grids(dim, shape, prec):
    """The plane-by-plane sweeps on grids with a different node count per
    axis (every plane bound differs): φ^0 bit-exact against the oracle."""
    rec, P = _ragged(dim, shape, prec, 1)
    pts = synth.sphere_even(4000, 0.45) if dim == 3 else synth.circle_even_noisy(600, 0.45, 0.003, 3)
    rec.load_cloud(pts)
    rec.build_distance()
    d = rec.d()
    gamma_s = 2.0 * P.h
    rec.init_marking(gamma_s)
    ref, ext = expected_u0(P, d, gamma_s, prec, 1)
    assert ext.sum() > 0 and (ext == 0).sum() > 0
    assert np.array_equal(rec.u(), ref)
