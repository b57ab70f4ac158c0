"""The C ABI library loads without a GPU and exports every function include/pff_rve.h declares.

Also checks the host-side argument validation that runs before any device call.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pff_rve.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|long|const char \*)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2508_07424_gb300 import build, capi
    build.build()
    return capi.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("rve_create", "set_microstructure", "step_dissipation", "effective_toughness", "rve_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2508_07424_gb300 import capi
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in capi.EXPORTED, name


def test_create_rejects_bad_sizes_without_touching_the_gpu(lib):
    from paper_2508_07424_gb300 import capi
    from paper_2508_07424_gb300.rve import make_config
    bad = [dict(dim=2, n=(48, 64, 1)), dict(dim=2, n=(64, 64, 2)), dict(dim=3, n=(64, 64, 2)),
           dict(dim=4, n=(64, 64, 1)), dict(dim=2, n=(2048, 64, 1)), dict(dim=3, n=(512, 512, 512)),
           # too small for one warp per x-pass CTA: (nx/4) * min(128/(nx/4), ny*nz/2) < 32
           dict(dim=2, n=(4, 4, 1)), dict(dim=2, n=(8, 8, 1)), dict(dim=2, n=(16, 8, 1)),
           dict(dim=3, n=(8, 4, 1))]
    for b in bad:
        cfg = make_config(b["dim"], b["n"], 2.0)
        h = capi.rve_handle()
        assert lib.rve_create(C.byref(cfg), C.byref(h)) == capi.RVE_EINVAL, b
        assert lib.rve_config_validate(C.byref(cfg)) == capi.RVE_EINVAL, b
    for n, dim in (((64, 64, 1), 2), ((32, 32, 32), 3), ((256, 128, 1), 3)):
        assert lib.rve_config_validate(C.byref(make_config(dim, n, 2.0))) == capi.RVE_OK, n
    # the Newton solver: FP64 only, no split
    for kw in (dict(precision=capi.RVE_FP32R), dict(split=capi.RVE_SPLIT_SPECTRAL), dict(solver_bad=True)):
        cfg = make_config(2, (64, 64, 1), 2.0, solver=capi.RVE_SOLVER_NEWTON,
                          **{k: v for k, v in kw.items() if k != "solver_bad"})
        if "solver_bad" in kw:
            cfg.solver = 7
        h = capi.rve_handle()
        assert lib.rve_create(C.byref(cfg), C.byref(h)) == capi.RVE_EINVAL, kw
    cfg = make_config(2, (64, 64, 1), -1.0)
    h = capi.rve_handle()
    assert lib.rve_create(C.byref(cfg), C.byref(h)) == capi.RVE_EINVAL
    assert lib.rve_create(None, C.byref(h)) == capi.RVE_EINVAL
    assert lib.step_dissipation(None, 1.0, None) == capi.RVE_EINVAL
    assert lib.rve_strerror(capi.RVE_ENOTFRACTURED).decode() == "fracture point not reached"
