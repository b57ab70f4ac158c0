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


def test_newton_solver_footprint_includes_its_vectors(mods):
    capi, serve = mods
    w = synth.fibre_composite_512()
    assert serve.Server.footprint(w, solver=capi.RVE_SOLVER_NEWTON) > serve.Server.footprint(w)


class _FakeClock:
    def __init__(self):
        self.t = 0.0

    def now(self):
        return self.t

    def sleep(self, d):
        self.t += d


class _FakeServer:
    """Accepts requests and completes each one on the next wait, in submission order."""

    def __init__(self, clock, reject=()):
        self.clock, self.reject, self.log, self.pending = clock, set(reject), [], []

    def submit(self, rid, w, n_inc, **kw):
        from paper_2508_07424_gb300 import capi
        if rid in self.reject:
            return capi.RVE_EINVAL
        self.log.append((rid, self.clock.now(), n_inc))
        self.pending.append(rid)
        return capi.RVE_OK

    def wait(self, max_n, timeout):
        done, self.pending = self.pending[:max_n], self.pending[max_n:]
        return [{"id": i, "status": 0} for i in done]


def test_replay_submits_a_poisson_trace_at_its_arrival_times(mods):
    import numpy as np
    capi, serve = mods
    rng = np.random.default_rng(5)
    arrivals = np.cumsum(rng.exponential(0.3, 12))
    reqs = [(float(t), None, 10) for t in arrivals]
    clk = _FakeClock()
    srv = _FakeServer(clk, reject={4})
    out, wall = serve.replay(srv, reqs, time_scale=2.0, clock=clk.now, sleep=clk.sleep)
    assert sorted(out) == list(range(12))
    assert out[4]["status"] == capi.RVE_EINVAL and all(out[i]["status"] == 0 for i in out if i != 4)
    ids = [r for r, _, _ in srv.log]
    assert ids == [i for i in range(12) if i != 4]           # in arrival order
    for rid, t, n_inc in srv.log:                             # never before its scaled arrival time
        assert t >= 2.0 * arrivals[rid] - 1e-12 and n_inc == 10
    assert wall >= 2.0 * arrivals[-1] - 1e-12
