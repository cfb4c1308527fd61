"""The persistent batched kernel (slr_batch_run) through the C ABI.

Each job of a batch must end in exactly the state of the same job evolved
alone (slr_evolve, itself checked against the FP64 oracle step by step in
test_gpu_parity.py): the same iteration count and stop reason, u bit for
bit and the E_2 history bit for bit. The mix covers 2-D (list step) and 3-D
(brick step) jobs, Q1 and WENO, FP32 and FP64, grids whose rows suit TMA
staging (n_x a multiple of 4 in FP32, of 2 in FP64) and ragged grids staged
by cp.async, and both block sizes of the autotuner.
"""
import numpy as np
import pytest

from paper_2410_22205_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _slr():
    from paper_2410_22205_gb300 import slr

    return slr


# (dim, n, precision, interp): band mode, p = 2, δ = 1 (the defaults)
KINDS = [(2, 64, 32, 0), (2, 96, 64, 1), (3, 32, 32, 1), (3, 40, 32, 0), (3, (37, 29, 33), 32, 1),
         (3, 24, 64, 1), (2, (53, 47), 32, 1), (3, (33, 35, 31), 64, 0)]


def _job(kind, seed, max_iters=40, u0=0.75):
    slr = _slr()
    dim, n, prec, interp = kind
    shape = (n,) * dim if isinstance(n, int) else tuple(n)
    if dim == 2:
        shape = shape[:2] + (1,)
    h = 2.0 / (shape[0] - 1)
    hi = tuple(-1.0 + h * (shape[a] - 1) for a in range(dim))
    rec = slr.Reconstruction(dim=dim, n=shape, lo=(-1.0,) * dim, hi=hi, precision=prec, interp=interp, band=1,
                             max_iters=max_iters)
    pts = (synth.sphere_cloud(800, 0.5, 0.01, seed) if dim == 3 else synth.circle_noisy(300, 0.5, 0.01, seed))
    rec.load_cloud(pts)
    rec.build_distance()
    rec.init_sphere(u0)
    return rec


def _solo(kinds, **kw):
    out = []
    for i, k in enumerate(kinds):
        r = _job(k, i, **kw)
        it, conv = r.evolve()
        out.append((it, conv, r.u(), r.diagnostics()["e2"]))
        r.close()
    return out


def _solo_one(kind, seed, max_iters):
    r = _job(kind, seed, max_iters=max_iters)
    it, conv = r.evolve()
    out = (it, conv, r.u(), r.diagnostics()["e2"])
    r.close()
    return out


def _check(jobs, its, convs, solo):
    for idx, (j, (it, conv, u, e2)) in enumerate(zip(jobs, solo)):
        assert its[idx] == it and convs[idx] == conv, (idx, its[idx], it)
        assert np.array_equal(j.u(), u), idx
        assert np.array_equal(j.diagnostics()["e2"], e2), idx


@pytest.mark.parametrize("autotune", [0, 1])
def test_batch_run_equals_solo_runs(autotune):
    """One persistent launch (graph-captured) over a mixed batch ends every
    job in the state of its solo run, bit for bit; with autotuning the
    block size is one of the two candidates and the results do not change."""
    slr = _slr()
    solo = _solo(KINDS)
    jobs = [_job(k, i) for i, k in enumerate(KINDS)]
    its, convs = slr.slr_batch_run([j.ctx for j in jobs], autotune=bool(autotune))
    info = slr.slr_batch_run_info(jobs[0].ctx)
    if autotune:
        assert info["threads_per_block"] in (128, 256) and info["bricks_per_item"] in (1, 2, 4)
    else:
        assert info["threads_per_block"] == 128 and info["bricks_per_item"] == 1
    assert info["blocks_per_sm"] >= 1
    assert (info["autotune_trial_ms"] > 0.0) == bool(autotune)
    _check(jobs, its, convs, solo)
    for j in jobs:
        j.close()


def test_batch_run_jobs_stop_at_different_iterations():
    """Jobs with different iteration limits leave the launch one by one; the
    others go on, and every job matches its solo run."""
    slr = _slr()
    kinds = KINDS[:5]
    limits = [12, 40, 25, 3, 31]
    solo = [_solo_one(k, i, m) for i, (k, m) in enumerate(zip(kinds, limits))]
    jobs = [_job(k, i, max_iters=m) for i, (k, m) in enumerate(zip(kinds, limits))]
    its, convs = slr.slr_batch_run([j.ctx for j in jobs], autotune=False)
    assert max(its) <= 40 and min(its) <= 3
    _check(jobs, its, convs, solo)
    for j in jobs:
        j.close()


def test_batch_run_more_than_one_launch_group():
    """More than 64 jobs (and both storage types) run as several launches,
    each job still equal to its solo run."""
    slr = _slr()
    kinds = [(2, 24 + (i % 7), 32 if i % 5 else 64, i % 2) for i in range(70)]
    solo = [_solo_one(k, i, 15) for i, k in enumerate(kinds)]
    jobs = [_job(k, i, max_iters=15) for i, k in enumerate(kinds)]
    its, convs = slr.slr_batch_run([j.ctx for j in jobs], autotune=False)
    _check(jobs, its, convs, solo)
    for j in jobs:
        j.close()


def test_batch_run_then_solo_steps_continue():
    """After a batch the jobs are ordinary contexts again: a further solo
    evolve from the batch's end state equals two solo evolves in a row."""
    slr = _slr()
    k = KINDS[2]
    ref = _job(k, 2, max_iters=10)
    ref.evolve()
    ref.step(3, energy_override=-1.0)
    u_ref = ref.u()
    ref.close()
    j = _job(k, 2, max_iters=10)
    slr.slr_batch_run([j.ctx], autotune=False)
    j.step(3, energy_override=-1.0)
    assert np.array_equal(j.u(), u_ref)
    j.close()


def test_batch_run_rejects_jobs_it_does_not_take():
    """Whole-grid jobs, jobs with the reinitialisation and a job listed twice
    are refused with SLR_E_INVALID before anything runs."""
    slr = _slr()
    ok = _job(KINDS[0], 0)
    full = slr.Reconstruction(dim=2, n=(32, 32, 1), lo=(-1.0, -1.0), hi=(1.0, 1.0), precision=32, interp=0, band=0)
    full.load_cloud(synth.circle_noisy(100, 0.5, 0.01, 1))
    full.build_distance()
    full.init_sphere(0.75)
    for bad in ([ok.ctx, full.ctx], [ok.ctx, ok.ctx]):
        with pytest.raises(slr.SlrError) as e:
            slr.slr_batch_run(bad, autotune=False)
        assert e.value.status == slr.SLR_E_INVALID
    ok.close()
    full.close()
