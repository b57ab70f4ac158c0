"""Host-side checks of the request server (no GPU): footprint model and argument validation."""
import ctypes as C

import pytest

import synth


@pytest.fixture(scope="module")
def mods():
    from paper_2508_07424_gb300 import build, capi, serve
    build.build()
    return capi, serve


def test_footprint_grows_with_grid_and_precision(mods):
    capi, serve = mods
    small = synth.small_cases()["homog32"]
    big = synth.fibre_composite_512()
    assert serve.Server.footprint(big) > 100 * serve.Server.footprint(small) / 20
    b64 = serve.Server.footprint(big)
    b32 = serve.Server.footprint(synth.replace(big, precision="fp32r"))
    assert b32 < b64


def test_server_rejects_bad_requests(mods):
    capi, serve = mods
    srv = serve.Server(max_inflight=2, hbm_budget_bytes=1 << 30)
    w = synth.small_cases()["homog32"]
    assert srv.submit(1, w, 0) == capi.RVE_EINVAL          # n_inc < 1
    assert srv.submit(2, w, 3, dtau=-1.0) == capi.RVE_EINVAL
    assert srv.stats()["pending"] == 0
    srv.close()
    h = capi.rve_server()
    assert capi.lib().rve_server_create(0, 1, C.byref(h)) == capi.RVE_EINVAL
