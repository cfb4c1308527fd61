"""GPU parity of the reinitialisation of Algorithm 1, §3.7 (SL step,
then reinitialisation on the band and its first neighbours, then eq. cut),
through the C ABI against the FP64 oracle.

Bars (each written in its test):
  - the next step's scan list Ḡ^n (the step's band and its face
    neighbours): bit-exact;
  - φ after one iteration from identical inputs: FP64 max-abs <= 1e-12; FP32
    <= 1e-5·h (the SL step's own bars: the sweeps do not expand differences
    in the max norm, and measured errors are ~1e-14·h and ~1e-6·h). Nodes within two cells of a node whose sign class (φ̃ < 0 versus
    φ̃ >= 0) could differ between the two sides (|φ̃| within the SL step's
    tolerance of 0) or of a node the SL step flags near its singular threshold
    are excluded: the interface set of the explicit step is decided there;
  - Δ_φ of the iteration: relative 1e-10 (FP64), 1e-4 (FP32).
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


def make(dim, n, prec, interp, **kw):
    slr = _slr()
    shape = (n,) * dim + ((1,) if dim == 2 else ())
    rec = slr.Reconstruction(dim=dim, n=shape, lo=-1.0, hi=1.0, precision=prec, interp=interp, band=1, reinit=1, **kw)
    okw = {k: v for k, v in kw.items() if k in ("p", "delta", "dt", "gamma", "beta", "c_sing", "alpha")}
    P = O.params(dim, (n,) * dim, (-1.0,) * dim, (1.0,) * dim, interp=interp, band=1, prec=prec, **okw)
    return rec, P


def cloud(dim, seed=0):
    return synth.sphere_cloud(3000, 0.45, 0.002, seed) if dim == 3 else synth.circle_noisy(500, 0.45, 0.002, seed)


def dilate(mask, shape, times):
    m = mask.reshape(shape)
    for _ in range(times):
        out = m.copy()
        for ax in range(m.ndim):
            a = [slice(None)] * m.ndim
            b = [slice(None)] * m.ndim
            a[ax], b[ax] = slice(1, None), slice(None, -1)
            out[tuple(a)] |= m[tuple(b)]
            out[tuple(b)] |= m[tuple(a)]
        m = out
    return m.reshape(-1)


@pytest.mark.parametrize("dim,n", [(2, 64), (3, 40)])
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("interp", [0, 1])
def test_reinit_iteration_parity(dim, n, prec, interp):
    rec, P = make(dim, n, prec, interp, p=2.0, delta=1.0)
    rec.load_cloud(cloud(dim, 1))
    rec.build_distance()
    rec.init_sphere(0.8)
    Ep = 0.4
    rec.step(3, energy_override=Ep)  # a front that has moved, with sharpened gradients
    u0, d = rec.u(), rec.d()
    rec.step(1, energy_override=Ep)
    u1 = rec.u()
    nxt, flags, _ = O.sl_step(P, u0, d, Ep)
    ref, rfl, m = O.reinit(P, u0, nxt)
    # the next scan list: Ḡ^n, bit-exact
    assert np.array_equal(rec.band(), np.flatnonzero(rfl & 1))
    tol_sl = 1e-12 if prec == 64 else 1e-5 * P.h
    shape = (n,) * dim
    risky = ((flags & O.FLAG_MARGIN) != 0) | (((rfl & 1) != 0) & (np.abs(nxt) <= tol_sl))
    ok = ~dilate(risky, shape, 2)
    tol = 1e-12 if prec == 64 else 1e-5 * P.h
    err = np.abs(u1 - ref)[ok]
    assert err.max() <= tol, (err.max(), tol, int((~ok).sum()))
    assert np.all(np.abs(u1) <= np.float32(P.gamma) if prec == 32 else np.abs(u1) <= P.gamma)
    dphi = rec.diagnostics()["dphi"][-1]
    dref = np.abs(ref - u0).sum() * P.h ** dim
    assert dphi == pytest.approx(dref, rel=1e-10 if prec == 64 else 1e-4)


def test_evolve_with_reinit_matches_oracle_fp64():
    """Algorithm 1 with the reinitialisation, 2-D, FP64 Q1, p = 1, 60 iterations: the GPU
    trajectory follows the oracle's; E_2 history within 1e-9 relative."""
    rec, P = make(2, 64, 64, 0, p=1.0, delta=0.0, max_iters=60, min_iters=60)
    pts = synth.circle_uniform(400, 0.45)
    rec.load_cloud(pts)
    rec.build_distance()
    rec.init_sphere(0.8)
    u0, d = rec.u(), rec.d()
    it, conv = rec.evolve()
    ref = O.evolve(P, u0, d, max_iters=60, min_iters=60, reinit=True)
    assert it == ref["iters"] == 60
    np.testing.assert_allclose(rec.diagnostics()["e2"], ref["E2"], rtol=1e-9)
    assert np.abs(rec.u() - ref["u"]).max() <= 1e-9


@pytest.mark.parametrize("prec,interp", [(32, 1), (64, 0)])
def test_band_follows_the_front_to_a_far_cloud(prec, interp):
    """§3.8 last paragraph, on the GPU: started from a sphere whose band does
    not reach the cloud, the zero level set reaches it with the
    reinitialisation (error on the cloud below h) and stays at the band
    edge without it."""
    slr = _slr()
    pts = synth.sphere_cloud(4000, 0.45, 0.0, 3)
    errs = []
    for reinit in (0, 1):
        r = slr.Reconstruction(dim=3, n=48, precision=prec, interp=interp, band=1, reinit=reinit, p=1.0, delta=0.0,
                               max_iters=90, min_iters=90)
        r.load_cloud(pts)
        r.build_distance()
        r.init_sphere(0.8)
        r.evolve()
        errs.append(r.diagnostics(err_cloud=True)["err_cloud"])
        r.close()
    h = 2.0 / 47
    assert errs[0] > 0.99 * 6 * h * (1 - 1e-6)
    assert errs[1] < h


def test_batch_and_checkpoint_with_reinit():
    """Batched evolve and checkpoint/resume give bit-identical states with
    the reinitialisation on."""
    slr = _slr()

    def job(seed):
        r, _ = make(3, 32, 32, 1, max_iters=30, min_iters=30)
        r.load_cloud(cloud(3, seed))
        r.build_distance()
        r.init_sphere(0.75)
        return r

    solo = []
    for s in range(3):
        r = job(s)
        r.evolve()
        solo.append(r.u())
        r.close()
    jobs = [job(s) for s in range(3)]
    slr.slr_batch_evolve([j.ctx for j in jobs], chunk=4)
    for j, u in zip(jobs, solo):
        assert np.array_equal(j.u(), u)
        j.close()
    r = job(7)
    r.step(5)
    blob = r.export_state()
    r.step(6)
    u_ref, e_ref = r.u(), r.diagnostics()["e2"]
    r2 = job(7)
    r2.import_state(blob)
    r2.step(6)
    assert np.array_equal(r2.u(), u_ref)
    assert np.array_equal(r2.diagnostics()["e2"], e_ref)
