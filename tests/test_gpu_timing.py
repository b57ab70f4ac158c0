"""Per-kernel timing classes (measurement support of this implementation; the paper has no
counterpart). The single-kernel classes must be subsets of their templates, every class must be
a subset of all launches, and timing must not change any result bit."""
import math

import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case,precision", [("poly32", "fp64"), ("poly3d", "fp32r")])
def test_timing_classes_are_consistent_and_do_not_change_results(case, precision):
    from paper_2508_07424_gb300 import build
    from paper_2508_07424_gb300.rve import Rve
    build.build()
    w = synth.small_cases()[case]
    w.precision = precision
    recs = []
    for timed in (False, True):
        g = Rve.from_workload(w)
        g.step(w.dtau)
        if timed:
            g.timing(True)
        r = g.step(w.dtau)
        if timed:
            k = g.timing_kinds()
            g.timing(False)
        recs.append(r)
        g.close()
    a, b = recs
    for key in a:
        x, y = a[key], b[key]
        assert x == y or (isinstance(x, float) and math.isnan(x) and math.isnan(y)), key
    ms = {n: v[0] for n, v in k.items()}
    cnt = {n: v[1] for n, v in k.items()}
    # single kernels inside their templates
    assert 0 < cnt["projection_pass"] <= cnt["k_axis"] and ms["projection_pass"] <= ms["k_axis"]
    assert 0 < cnt["cg_x_fwd"] <= cnt["k_x_fwd"] and ms["cg_x_fwd"] <= ms["k_x_fwd"]
    assert 0 < cnt["cg_x_inv"] <= cnt["k_x_inv"] and ms["cg_x_inv"] <= ms["k_x_inv"]
    # one forward and one inverse x pass per CG iteration, one projection pass each as well
    assert cnt["cg_x_fwd"] == cnt["cg_x_inv"] <= cnt["projection_pass"]
    # the template classes (and the FP64 residual passes of the FP32 path) partition all launches
    parts = ("k_axis", "k_x_fwd", "k_x_inv", "k_x_mid", "k_pointwise", "fp64_residual")
    assert sum(cnt[n] for n in parts) == cnt["all"]
    assert abs(sum(ms[n] for n in parts) - ms["all"]) <= 1e-6 * ms["all"] + 1e-3
    if precision == "fp64":
        assert cnt["fp64_residual"] == 0
    else:
        assert cnt["fp64_residual"] > 0
    # FFT flops and algorithmic bytes are recorded per launch
    assert k["projection_pass"][2] > 0 and k["projection_pass"][3] > 0
    assert k["cg_x_fwd"][2] > 0 and k["cg_x_fwd"][3] > 0
