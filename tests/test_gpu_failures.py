"""Failure detection, injected on the host (no GPU fault, trap or hang is ever provoked).

* a non-finite damage value is caught by the solver's device scalars (RVE_EBREAKDOWN), the
  committed state is left as it was and a checkpoint restores a clean run;
* an iteration cap that is too small gives RVE_ENOCONV with a message naming the stage, and
  the committed state is untouched;
* calls out of order and bad arguments return their codes without touching the device state.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2508_07424_gb300 import build, capi
    from paper_2508_07424_gb300.rve import Rve
    build.build()
    return capi, Rve


def test_non_finite_damage_is_detected_and_state_is_kept(mods):
    capi, Rve = mods
    w = synth.small_cases()["fibre64x16"]
    g = Rve.from_workload(w)
    g.step(w.dtau)
    blob = g.save()
    s0 = g.scalars()
    phi = g.get(capi.RVE_FIELD_PHI)
    bad = phi.copy()
    bad[0, 3, 5] = np.nan
    g.set(capi.RVE_FIELD_PHI, bad)
    out = capi.rve_step_result()
    rc = capi.lib().step_dissipation(g.h, w.dtau, C.byref(out))
    assert rc == capi.RVE_EBREAKDOWN
    assert "non-finite" in capi.lib().rve_strerror(rc).decode()
    assert g.scalars() == s0
    g.load(blob)
    r = g.step(w.dtau)
    assert r["n"] == s0["n"] + 1 and np.isfinite(r["E"])


def test_iteration_cap_reports_the_stage(mods):
    capi, Rve = mods
    w = synth.small_cases()["poly32"]
    g = Rve.from_workload(w, max_mech_iters=2)
    s0 = g.scalars()
    phi0 = g.get(capi.RVE_FIELD_PHI)
    out = capi.rve_step_result()
    rc = capi.lib().step_dissipation(g.h, w.dtau, C.byref(out))
    assert rc == capi.RVE_ENOCONV
    assert "equilibrium CG" in capi.lib().rve_strerror(rc).decode()
    assert g.scalars() == s0
    assert np.array_equal(g.get(capi.RVE_FIELD_PHI), phi0)


def test_bad_arguments_leave_the_handle_usable(mods):
    capi, Rve = mods
    w = synth.small_cases()["homog32"]
    g = Rve.from_workload(w)
    buf = np.zeros(7)
    assert capi.lib().rve_get_field(g.h, capi.RVE_FIELD_PHI, buf.ctypes.data_as(C.POINTER(C.c_double)), 7) == capi.RVE_EINVAL
    assert capi.lib().rve_get_field(g.h, 42, buf.ctypes.data_as(C.POINTER(C.c_double)), 7) == capi.RVE_EINVAL
    assert capi.lib().rve_load(g.h, b"\\0" * 16, 16) == capi.RVE_EINVAL
    r = g.step(w.dtau)
    assert r["n"] == 1
