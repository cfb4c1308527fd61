"""GPU checks of the brick-staged 3-D SL step (§3.1 eq. SL3d on 8x8x8-node
bricks staged in shared memory) beyond the oracle parity of
test_gpu_parity.py, which every 3-D context without the reinitialisation
already runs through it:

  - every launch shape (threads per block x pipeline stages) gives the same
    u, band and Δ_φ history bit for bit, on a grid whose rows are 16-byte
    aligned (TMA staging) and on a ragged one (cp.async staging), in the band
    and on the whole grid; and each matches the oracle step by step;
  - the autotuner's choice is one of the candidate shapes;
  - feet that leave the staged box (a large diffusive offset) take the
    global-memory interpolators and still match the oracle.
"""
import numpy as np
import pytest

import oracle as O
from paper_2410_22205_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = [(256, 1), (128, 1), (256, 2), (128, 2)]


def _make(n, prec, interp, band, **kw):
    from paper_2410_22205_gb300 import slr

    shape = (n,) * 3 if isinstance(n, int) else tuple(n)
    lo = (-1.0,) * 3
    hi = tuple(-1.0 + 2.0 * (shape[a] - 1) / (shape[0] - 1) for a in range(3))
    kw.setdefault("step_kind", 1)  # the brick step on every grid (by rule, Q1 band runs on ragged rows take the list step)
    rec = slr.Reconstruction(dim=3, n=shape, lo=lo, hi=hi, precision=prec, interp=interp, band=band, **kw)
    okw = {k: v for k, v in kw.items() if k in ("p", "delta")}
    P = O.params(3, shape, lo, hi, interp=interp, band=band, prec=prec, **okw)
    return rec, P


def _run(n, prec, interp, band, shape, steps=3):
    rec, P = _make(n, prec, interp, band)
    rec.load_cloud(synth.torus_cloud(6000, 0.5, 0.2, 0.002, 3))
    rec.build_distance()
    rec.init_sphere(0.7)
    if shape is not None:
        rec.set_brick_shape(*shape)
    bands, errs = [], []
    for _ in range(steps):
        u0 = rec.u()
        Ep = float(rec.energy(2.0)[0])
        rec.step(1, energy_override=Ep)
        u1 = rec.u()
        ref, flags, _ = O.sl_step(P, u0, rec.d(), Ep)
        ok = (flags & O.FLAG_MARGIN) == 0
        errs.append(float(np.abs(u1 - ref)[ok].max()))
        bands.append(rec.band())
    out = (rec.u(), bands, rec.diagnostics(), errs, rec.brick_shape(), P.h)
    rec.close()
    return out


@pytest.mark.parametrize("interp", [0, 1])
@pytest.mark.parametrize("n,band", [(40, 1), ((33, 41, 29), 1), (24, 0), ((25, 22, 23), 0)])
def test_every_launch_shape_gives_identical_results(n, band, interp):
    runs = [_run(n, 32, interp, band, sh) for sh in SHAPES]
    u_ref, bands_ref, diag_ref = runs[0][:3]
    for (u, bands, diag, errs, got, h), sh in zip(runs, SHAPES):
        assert got[0] == sh[0]
        assert np.array_equal(u, u_ref), sh
        for a, b in zip(bands, bands_ref):
            assert np.array_equal(a, b), sh
        assert np.array_equal(diag["dphi"], diag_ref["dphi"]), sh
        assert np.array_equal(diag["band"], diag_ref["band"]), sh
        assert max(errs) <= 1e-5 * h, (sh, errs)


@pytest.mark.parametrize("prec", [32, 64])
def test_autotuned_shape_is_a_candidate(prec):
    rec, _ = _make(40, prec, 1, 1)
    rec.load_cloud(synth.torus_cloud(4000, 0.5, 0.2, 0.002, 1))
    rec.build_distance()
    rec.init_sphere(0.7)
    threads, stages, ms = rec.brick_shape()
    assert (threads, stages) in SHAPES
    assert ms > 0.0
    rec.close()


@pytest.mark.parametrize("interp", [0, 1])
def test_far_feet_take_the_global_path(interp):
    """A constant distance d0 = 2.5 with p = 1 and δ = 1 gives a diffusive
    offset sqrt(d0 Δt / p) / h = 3.5 cells at n = 40, and |λ1 ν1 + λ2 ν2| = √2,
    so feet land up to about 5 cells from their node: beyond the staged halo
    of 4 for many of them, which then take the global-memory interpolators.
    The whole-grid step still matches the oracle."""
    n = 40
    rec, P = _make(n, 64, interp, 0, p=1.0, delta=1.0)
    rec.set_distance(np.full(n ** 3, 2.5))
    rec.init_sphere(0.6)
    u0 = rec.u()
    rec.step(1, energy_override=1.0)
    ref, flags, _ = O.sl_step(P, u0, rec.d(), 1.0)
    ok = (flags & O.FLAG_MARGIN) == 0
    assert float(np.abs(rec.u() - ref)[ok].max()) <= 1e-12
    rec.close()


def test_shape_setter_rejects_unknown_shapes():
    from paper_2410_22205_gb300 import slr

    rec, _ = _make(24, 32, 0, 1)
    rec.load_cloud(synth.torus_cloud(2000, 0.5, 0.2, 0.002, 1))
    rec.build_distance()
    rec.init_sphere(0.7)
    with pytest.raises(slr.SlrError) as e:
        rec.set_brick_shape(64, 1)
    with pytest.raises(slr.SlrError):
        rec.set_brick_shape(256, 3)
    assert e.value.status == slr.SLR_E_INVALID
    rec.close()


def test_fma_probe_measures_a_plausible_rate():
    """The FMA probe behind the ALU roofline: FP32 between 20% and 110% of the
    unit-count peak (SMs x 128 lanes x 2 flops x the maximum SM clock, 2.07 GHz
    on GB300), and FP64 below FP32."""
    from paper_2410_22205_gb300 import slr

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    derived = sms * 128 * 2 * 2.07e9 / 1e12
    f32, ms32 = slr.slr_probe_fma(32, 20_000)
    f64, ms64 = slr.slr_probe_fma(64, 500)
    assert 0.2 * derived < f32 < 1.1 * derived, (f32, derived)
    assert 0.0 < f64 < f32
