"""CPU checks of the C ABI: libslr.so loads, exports every entry point that
include/slr.h declares, and validates configurations before touching CUDA."""
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2410_22205_gb300 import slr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "slr.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(slr_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_what_the_binding_wraps():
    assert _declared() == sorted(slr.EXPORTS)


def test_library_exports_every_declared_symbol():
    slr.lib()
    out = subprocess.run(["nm", "-D", "--defined-only", slr.LIB_PATH], capture_output=True, text=True).stdout
    names = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    missing = [s for s in _declared() if s not in names]
    assert not missing, missing


def test_library_is_built_for_sm_103a():
    """One -gencode, for sm_103a, in the build that produced libslr.so."""
    from paper_2410_22205_gb300 import build as B

    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(slr.LIB_PATH)


def test_new_entry_points_check_their_arguments_without_a_device():
    """Argument checks that return before any CUDA call: a batch chunk of a
    null job, the L1 error and the swept distance of a null context, and
    invalid runs-from-coarse-to-fine configurations."""
    L = slr.lib()
    assert L.slr_batch_chunk(None) == 0
    assert L.slr_batch_run(None, 0, 0, None, None, None) == slr.SLR_E_INVALID
    assert L.slr_server_set_policy(None, 1) == slr.SLR_E_INVALID
    assert L.slr_selftest_barrier(3) == slr.SLR_E_INVALID
    assert L.slr_batch_run_info(None, None, None, None, None, None) == slr.SLR_E_INVALID
    out = slr.C.c_double(0.0)
    assert L.slr_l1_error(None, 0, None, None, slr.C.byref(out)) == slr.SLR_E_INVALID
    assert L.slr_build_distance_fsm(None) == slr.SLR_E_INVALID
    pts = np.zeros((4, 2))
    pts[:, 0] = np.arange(4)
    for bad in (dict(runs=0), dict(runs=9), dict(K_s=0.0), dict(sample_frac=0.0), dict(sample_frac=2.0),
                dict(max_nodes=10), dict(max_iters=0), dict(dim=4), dict(distance_fsm=2), dict(exact_sphere=3)):
        kw = dict(dim=2)
        kw.update(bad)
        mc = slr.slr_multirun_default(**kw)
        h = slr.C.c_void_p()
        rep = slr.slr_multirun_report()
        st = L.slr_reconstruct(slr.C.byref(mc), pts.ctypes.data_as(slr._dp), 4, None, None, slr.C.byref(h),
                               slr.C.byref(rep))
        assert st == slr.SLR_E_INVALID, bad


@pytest.mark.parametrize("bad", [
    dict(dim=4),
    dict(dim=2, n=(64, 64, 2)),
    dict(n=(3, 64, 64)),
    dict(n=(64, 64, 64), hi=(1.0, 1.0, 2.0)),
    dict(precision=16),
    dict(interp=2),
    dict(p=0.5),
    dict(energy_R=9),
    dict(gamma=0.01, beta=0.02),
    dict(max_iters=100000),
    dict(stop_k=1024),
    dict(step_kind=3),
    dict(step_kind=1, dim=2, n=(64, 64, 1), lo=(-1.0, -1.0), hi=(1.0, 1.0)),
    dict(step_kind=1, reinit=1),
])
def test_create_rejects_invalid_config(bad):
    cfg = slr.slr_config_default(**bad)
    with pytest.raises(slr.SlrError) as e:
        slr.slr_create(cfg)
    assert e.value.status == slr.SLR_E_INVALID
    assert slr.slr_last_error(None)


def test_create_rejects_grids_of_2_31_nodes_or_more():
    """The node-count limit holds before any device call, including sizes
    whose 64-bit product would wrap around to a small number."""
    big = 2 ** 62 + 1
    for kw in (dict(n=(1300, 1300, 1300)),
               dict(n=(46341, 46341, 4), lo=(0.0, 0.0, 0.0), hi=(46340.0, 46340.0, 3.0)),
               dict(n=(big, 4, 4), lo=(0.0, 0.0, 0.0), hi=(float(big - 1), 3.0, 3.0))):
        cfg = slr.slr_config_default(**kw)
        with pytest.raises(slr.SlrError) as e:
            slr.slr_create(cfg)
        assert e.value.status == slr.SLR_E_INVALID
        assert "2^31" in slr.slr_last_error(None)


def test_noalloc_rejects_grids_of_2_31_nodes_or_more():
    """The allocation-free distance grid checks its sizes before any device
    call (the buffer addresses are never touched), including a wrapping
    product."""
    for n in ((1300, 1300, 1300), (2 ** 62 + 1, 4, 4), (4, 2 ** 62 + 1, 2 ** 62 + 1)):
        with pytest.raises(slr.SlrError) as e:
            slr.slr_distance_grid_noalloc(3, n, (0.0, 0.0, 0.0), 1.0, 32, 256, 10, 512, 768)
        assert e.value.status == slr.SLR_E_INVALID
        assert "2^31" in slr.slr_last_error(None)


def test_default_config_is_the_papers():
    cfg = slr.slr_config_default()
    assert (cfg.p, cfg.delta, cfg.c_sing, cfg.alpha, cfg.energy_R) == (2.0, 1.0, 1e-3, 1.0, 5)
    assert (cfg.stop_tol, cfg.stop_k, cfg.min_iters, cfg.max_iters) == (1e-4, 10, 10, 100)


def test_last_error_without_a_context_is_that_of_the_last_failed_call():
    """slr_last_error(NULL) reports the most recent failed call without a
    context on this thread: a failed allocation-free distance grid followed
    by a failed slr_create reports the create's reason, and the other way
    round. Both fail in their argument checks, before any device call."""
    with pytest.raises(slr.SlrError):
        slr.slr_distance_grid_noalloc(5, (8, 8, 8), (0.0, 0.0, 0.0), 1.0, 32, 256, 10, 512, 768)
    assert "distance_grid_noalloc" in slr.slr_last_error(None)
    with pytest.raises(slr.SlrError):
        slr.slr_create(slr.slr_config_default(dim=4))
    msg = slr.slr_last_error(None)
    assert "dim must be 2 or 3" in msg and "noalloc" not in msg
    with pytest.raises(slr.SlrError):
        slr.slr_distance_grid_noalloc(3, (8, 8, 8), (0.0, 0.0, 0.0), 1.0, 16, 256, 10, 512, 768)
    assert "precision" in slr.slr_last_error(None)


def test_fma_probe_checks_its_arguments_without_a_device():
    L = slr.lib()
    a, b = slr.C.c_double(0.0), slr.C.c_double(0.0)
    assert L.slr_probe_fma(16, 10, slr.C.byref(a), slr.C.byref(b)) == slr.SLR_E_INVALID
    assert L.slr_probe_fma(32, 0, slr.C.byref(a), slr.C.byref(b)) == slr.SLR_E_INVALID
    assert L.slr_probe_fma(32, 10, None, slr.C.byref(b)) == slr.SLR_E_INVALID
