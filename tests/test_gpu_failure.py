"""Failure detection on the GPU without a fault: the bounded grid barrier of
the cooperative fast-sweeping kernel and the dependency wait of the batched
kernel report a wait that runs out (a barrier that no block completes, a
counter that no work item completes) as SLR_E_TIMEOUT, within the poll
limit, and the device stays usable afterwards."""
import time

import numpy as np
import pytest

import oracle as O
from paper_2410_22205_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_grid_barrier_timeout_is_reported_and_the_device_stays_usable():
    from paper_2410_22205_gb300 import slr

    assert slr.slr_selftest_barrier(0) == slr.SLR_OK
    t0 = time.time()
    assert slr.slr_selftest_barrier(1) == slr.SLR_E_TIMEOUT
    assert time.time() - t0 < 30.0
    assert "ran out" in slr.slr_last_error(None)
    # the same cooperative sweeps still give the oracle's initial data
    n = 48
    rec = slr.Reconstruction(dim=2, n=(n, n, 1), precision=64, interp=0, band=1)
    P = O.params(2, (n, n), (-1.0, -1.0), (1.0, 1.0), band=1, prec=64)
    pts = synth.circle_even_noisy(300, 0.5, 0.002, 1)
    rec.load_cloud(pts)
    rec.build_distance()
    gamma_s = 2.0 * P.h
    rec.init_marking(gamma_s)
    phi, _ = O.init_marking(P, rec.d(), gamma_s)
    assert np.array_equal(rec.u(), np.clip(phi, -P.gamma, P.gamma))
    rec.close()


def test_batch_wait_timeout_is_reported_and_the_device_stays_usable():
    from paper_2410_22205_gb300 import slr

    t0 = time.time()
    assert slr.slr_selftest_barrier(2) == slr.SLR_E_TIMEOUT
    assert time.time() - t0 < 30.0
    assert "batched kernel's wait ran out" in slr.slr_last_error(None)
    # a batch still runs to its stop test afterwards
    n = 40
    rec = slr.Reconstruction(dim=2, n=(n, n, 1), precision=32, interp=0, band=1, max_iters=12)
    rec.load_cloud(synth.circle_even_noisy(300, 0.5, 0.002, 1))
    rec.build_distance()
    rec.init_sphere(0.75)
    its, _ = slr.slr_batch_run([rec.ctx], autotune=False)
    assert its == [12]
    rec.close()
