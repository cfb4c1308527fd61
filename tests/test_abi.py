"""CPU checks of the C ABI: libslr.so loads, exports every entry point that
include/slr.h declares, and validates configurations before touching CUDA."""
import os
import re
import subprocess

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
    out = subprocess.run(["cuobjdump", "--list-elf", slr.LIB_PATH], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


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
])
def test_create_rejects_invalid_config(bad):
    cfg = slr.slr_config_default(**bad)
    with pytest.raises(slr.SlrError) as e:
        slr.slr_create(cfg)
    assert e.value.status == slr.SLR_E_INVALID
    assert slr.slr_last_error(None)


def test_default_config_is_the_papers():
    cfg = slr.slr_config_default()
    assert (cfg.p, cfg.delta, cfg.c_sing, cfg.alpha, cfg.energy_R) == (2.0, 1.0, 1e-3, 1.0, 5)
    assert (cfg.stop_tol, cfg.stop_k, cfg.min_iters, cfg.max_iters) == (1e-4, 10, 10, 100)
