"""GPU parity of the §3.4 distance grid as the paper builds it (exact on the
4^dim node box around each point, fast sweeping elsewhere) through the C ABI
(slr_build_distance_fsm) against the oracle's or_distance_fsm.

Bar: d bit-exact (both sides take the exact FP64 distance on the same box
nodes, sweep with the same correctly rounded FP64 operations in an order that
sees the same values, and round to the storage type once); argmin bit-exact on
the box nodes and -1 elsewhere.
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


@pytest.mark.parametrize("dim,n,prec,cloud", [(2, 96, 64, "circle"), (2, 77, 32, "edge"), (3, 40, 32, "squ"),
                                              (3, 33, 64, "sphere"), (3, 48, 32, "edge"), (2, 16, 64, "one")])
def test_distance_fsm_bit_exact(dim, n, prec, cloud):
    slr = _slr()
    shape = (n,) * dim + ((1,) if dim == 2 else ())
    rec = slr.Reconstruction(dim=dim, n=shape, precision=prec, interp=1, band=1)
    P = O.params(dim, (n,) * dim, (-1.0,) * dim, (1.0,) * dim, band=1, prec=prec)
    rng = np.random.default_rng(n)
    if cloud == "circle":
        pts = synth.circle_noisy(800, 0.5, 0.01, 2)
    elif cloud == "squ":
        pts = synth.superquadric_union_cloud(20000, 3, 5)
    elif cloud == "sphere":
        pts = synth.sphere_even(3000, 0.6)
    elif cloud == "one":
        pts = rng.uniform(-0.9, 0.9, (1, dim))
    else:
        # points near and beyond the faces: partial boxes, and points with none
        pts = rng.uniform(-1.15, 1.15, (500, dim))
    rec.load_cloud(pts)
    rec.build_distance("fsm")
    d, arg = rec.d(), rec.argmin()
    ref, fix = O.distance_fsm(P, pts)
    if prec == 32:
        ref = ref.astype(np.float32).astype(np.float64)
    assert np.array_equal(d, ref)
    _, aref = O.distance(P, pts, method="kd")
    assert np.array_equal(arg[fix == 1], aref[fix == 1])
    assert np.all(arg[fix == 0] == -1)


def test_distance_fsm_without_a_box_node_is_invalid():
    slr = _slr()
    rec = slr.Reconstruction(dim=3, n=16, precision=32, interp=1, band=1)
    rec.load_cloud(np.array([[5.0, 5.0, 5.0], [-4.0, 0.0, 0.0]]))
    with pytest.raises(slr.SlrError) as e:
        rec.build_distance("fsm")
    assert e.value.status == slr.SLR_E_INVALID


def test_evolution_on_the_swept_distance_reaches_the_cloud():
    """§3.4 reading check end to end: Algorithm 1 driven by the swept d (exact
    near the cloud) from the §3.6 initial data ends on the cloud, as with the
    exact d (eq. errCloud below h/2)."""
    slr = _slr()
    n = 64
    h = 2.0 / (n - 1)
    pts = synth.sphere_even(20000, 0.55)
    errs = []
    for method in ("exact", "fsm"):
        rec = slr.Reconstruction(dim=3, n=n, precision=32, interp=1, band=1, reinit=1, p=1.0, delta=0.0,
                                 max_iters=40, min_iters=40)
        rec.load_cloud(pts)
        rec.build_distance(method)
        rec.init_marking(2.0 * h)
        rec.evolve()
        errs.append(rec.diagnostics(err_cloud=True)["err_cloud"])
        rec.close()
    assert errs[0] < 0.5 * h and errs[1] < 0.5 * h


def test_multirun_with_the_swept_distance_matches_the_oracle():
    slr = _slr()
    pts = synth.circle_even_noisy(600, 0.45, 0.002, 4)
    kw = dict(runs=2, K_s=2.0, sample_frac=0.5, seed=5, max_nodes=1 << 22, max_iters=100, distance="fsm")
    rec, rep = slr.reconstruct(pts, dim=2, precision=64, interp=0, **kw)
    ref_phi, ref = O.reconstruct(pts, 2, prec=64, interp=0, **kw)
    assert rep["run_n"] == ref["run_n"] and rep["run_iters"] == ref["run_iters"]
    assert np.abs(rec.u() - ref_phi).max() <= 1e-9
    assert rec.diagnostics(err_cloud=True)["err_cloud"] < 0.5 * rep["run_dx"][-1]
    rec.close()


@pytest.mark.parametrize("dim,shape,prec", [(3, (33, 41, 29), 32), (3, (21, 17, 26), 64), (2, (37, 29), 32)])
def test_distance_fsm_bit_exact_on_ragged_grids(dim, shape, prec):
    slr = _slr()
    shape = tuple(shape) + ((1,) if dim == 2 else ())
    los = (-1.0,) * dim
    his = tuple(-1.0 + 2.0 * (shape[a] - 1) / (shape[0] - 1) for a in range(dim))
    rec = slr.Reconstruction(dim=dim, n=shape, lo=los, hi=his, precision=prec, interp=1, band=1)
    P = O.params(dim, shape[:dim], los, his, band=1, prec=prec)
    pts = synth.sphere_even(3000, 0.45) if dim == 3 else synth.circle_even_noisy(500, 0.45, 0.003, 5)
    rec.load_cloud(pts)
    rec.build_distance("fsm")
    ref, fix = O.distance_fsm(P, pts)
    if prec == 32:
        ref = ref.astype(np.float32).astype(np.float64)
    assert np.array_equal(rec.d(), ref)
