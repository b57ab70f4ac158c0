"""Serving helper over the library's request server (rve_server_*): marshalling and trace replay.

The scheduling itself (admission by HBM footprint, worker threads, one stream per request) is
native code in csrc/pff_serve.cu; this module submits requests at their arrival times and
collects the results.
"""
import ctypes as C
import dataclasses
import math
import threading
import time

from . import capi
from .rve import make_micro, workload_config


class Server:
    def __init__(self, max_inflight=8, hbm_budget_bytes=64 << 30, batching=False):
        self.h = capi.rve_server()
        capi.check(capi.lib().rve_server_create(max_inflight, hbm_budget_bytes, C.byref(self.h)), "rve_server_create")
        capi.check(capi.lib().rve_server_set_batching(self.h, int(batching)), "rve_server_set_batching")
        self._keep = []

    @staticmethod
    def footprint(w, **kw):
        cfg = workload_config(w, **kw)
        return capi.lib().rve_footprint_bytes(C.byref(cfg))

    def submit(self, rid, w, n_inc, dtau=None, **kw):
        cfg = workload_config(w, **kw)
        mi, keep = make_micro(w.micro)
        rc = capi.lib().rve_server_submit(self.h, rid, C.byref(cfg), C.byref(mi), n_inc, dtau or w.dtau)
        return rc

    def wait(self, max_n=64, timeout=1.0):
        buf = (capi.rve_request_result * max_n)()
        n = C.c_int()
        capi.check(capi.lib().rve_server_wait(self.h, buf, max_n, timeout, C.byref(n)), "rve_server_wait")
        return [{k: getattr(buf[i], k) for k, _ in buf[i]._fields_} for i in range(n.value)]

    def stats(self):
        p, b, q = C.c_int(), C.c_size_t(), C.c_long()
        capi.check(capi.lib().rve_server_stats(self.h, C.byref(p), C.byref(b), C.byref(q)), "rve_server_stats")
        return {"peak_inflight": p.value, "peak_bytes": b.value, "pending": q.value}

    def close(self):
        if self.h:
            capi.lib().rve_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def percentile(xs, q):
    xs = sorted(xs)
    if not xs:
        return math.nan
    k = (len(xs) - 1) * q
    lo, hi = int(math.floor(k)), int(math.ceil(k))
    return xs[lo] + (xs[hi] - xs[lo]) * (k - lo)


def replay(server, requests, time_scale=1.0, clock=time.perf_counter, sleep=time.sleep, **kw):
    """requests: list of (arrival_s, workload, n_inc). Submits each at its (scaled) arrival time,
    collects every result. Returns (results by id, wall seconds). ``clock`` and ``sleep`` are the
    time source (replaceable for tests)."""
    t0 = clock()
    out = {}
    done = threading.Event()

    def feeder():
        for i, (ta, w, n_inc) in enumerate(requests):
            delay = t0 + ta * time_scale - clock()
            if delay > 0:
                sleep(delay)
            rc = server.submit(i, w, n_inc, **kw)
            if rc != capi.RVE_OK:
                out[i] = {"id": i, "status": rc}
        done.set()

    th = threading.Thread(target=feeder, daemon=True)
    th.start()
    while len(out) < len(requests):
        for r in server.wait(64, 0.5):
            out[r["id"]] = r
    th.join()
    return out, clock() - t0


def crack_position_sampling(server, w, positions, n_inc=None, timeout_s=600.0, **kw):
    """Toughness of one RVE sampled over initial-crack positions (Sec. 3: the crack position can
    bias the crack path, so the estimate is the minimum over positions).

    positions: (row, x0) pairs for the crack of ``w.micro.crack`` (same kind, length, phi_M). Each
    position is one request of the native server, so the solves run concurrently on the GPU.
    Returns (minimum toughness over the positions that reached the fracture point, per-position
    results in the order given). A position whose run fails or does not fracture within n_inc
    increments keeps its status and fractured flag and is left out of the minimum."""
    for i, (row, x0) in enumerate(positions):
        cr = dataclasses.replace(w.micro.crack, row=int(row), x0=int(x0))
        wi = dataclasses.replace(w, micro=dataclasses.replace(w.micro, crack=cr))
        capi.check(server.submit(i, wi, n_inc or w.n_inc, **kw), "rve_server_submit")
    out = {}
    t_end = time.perf_counter() + timeout_s
    while len(out) < len(positions):
        if time.perf_counter() > t_end:
            raise TimeoutError("crack_position_sampling: results missing after %.0f s" % timeout_s)
        for r in server.wait(64, 0.5):
            out[r["id"]] = r
    res = [dict(out[i], row=int(positions[i][0]), x0=int(positions[i][1])) for i in range(len(positions))]
    ok = [r["toughness"] for r in res if r["status"] == capi.RVE_OK and r["fractured"]]
    return (min(ok) if ok else math.nan), res
