"""Run an RVE to its fracture point and log every increment as one JSON line.

Host-side driver over the library's calls (``Rve.step``, ``Rve.toughness``,
``Rve.toughness_functional``); all computation stays in the CUDA library. One line per committed
increment holds the step result of ``step_dissipation`` (E, Sigma, D, E_mec, T, Gamma, tau,
instantaneous G, iteration counts, staggered error, flags) and the wall time since the start;
the last line summarises the run (fractured, toughness from the load curve and from the
functional).
"""
import json
import math
import time


def _clean(v):
    if isinstance(v, float) and not math.isfinite(v):
        return None
    return v


def run_to_fracture(rve, dtau, max_increments, log=None, clock=time.perf_counter):
    """Step ``rve`` with constant dissipation increments ``dtau`` until the fracture point or
    ``max_increments``. ``log`` is a path or a writable text stream (or None). Returns the
    summary dict."""
    own = isinstance(log, str)
    out = open(log, "w") if own else log
    t0 = clock()
    last = None
    try:
        for _ in range(max_increments):
            r = rve.step(dtau)
            last = r
            if out is not None:
                rec = {k: _clean(v) for k, v in r.items()}
                rec["wall_s"] = clock() - t0
                out.write(json.dumps(rec) + "\n")
            if r["fractured"]:
                break
        summary = {"summary": True, "increments": last["n"] if last else 0,
                   "fractured": bool(last and last["fractured"]), "wall_s": clock() - t0,
                   "toughness": None, "toughness_functional": None}
        if summary["fractured"]:
            summary["toughness"] = _clean(rve.toughness())
            summary["toughness_functional"] = _clean(rve.toughness_functional())
        if out is not None:
            out.write(json.dumps(summary) + "\n")
        return summary
    finally:
        if own:
            out.close()
