"""Lockstep batching of several RVEs of one grid (rve_step_batch; the batching pattern of this
library, not from the paper). Each RVE of a batch runs its own control and performs exactly the
solver iterations it performs alone, with the same kernels and reduction order, so its increments
and fields must be bit-identical to stepping it alone; and the batched RVEs still match the FP64
oracle (checked through the alone run, which the parity tests compare with the oracle)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cap():
    from paper_2508_07424_gb300 import build, capi
    build.build()
    return capi


def _poly2d(seed, precision):
    crack = synth.Crack(synth.CRACK_CTE, row=16, x0=0, length=6, phi_M=0.8)
    m = synth.voronoi((32, 32), 9, seed, beta=2.0, sigma_Gc=0.2, crack=crack)
    w = synth.Workload(m, ell=2.0, n_inc=8, precision=precision)
    w.dtau = 1.5 * w.A_g / 24
    return w


def _poly3d(seed, precision):
    crack = synth.Crack(synth.CRACK_CTE, row=8, x0=0, length=4, phi_M=0.8)
    m = synth.voronoi((16, 16, 8), 6, seed, orientation="so3", sigma_Gc=0.3, crack=crack)
    w = synth.Workload(m, ell=2.0, n_inc=6, precision=precision)
    w.dtau = 1.5 * float(np.mean(m.Gc)) * w.A_g / 24
    return w


@pytest.mark.parametrize("kind,precision", [("2d", "fp64"), ("2d", "fp32r"), ("3d", "fp32r"), ("3d", "fp64")])
def test_batched_increments_are_bit_identical_to_alone(cap, kind, precision):
    from paper_2508_07424_gb300.rve import Rve, step_batch
    make = _poly2d if kind == "2d" else _poly3d
    ws = [make(s, precision) for s in (11, 12, 13)]
    alone = [Rve.from_workload(w) for w in ws]
    batch = [Rve.from_workload(w) for w in ws]
    for inc in range(2):
        ra = [g.step(w.dtau) for g, w in zip(alone, ws)]
        rb = step_batch(batch, [w.dtau for w in ws])
        for i, (a, b) in enumerate(zip(ra, rb)):
            assert a["mech_iters"] > 0 and a["dmg_iters"] > 0
            for k in a:
                same = (a[k] == b[k]) or (a[k] != a[k] and b[k] != b[k])
                assert same, (inc, i, k, a[k], b[k])
    for ga, gb in zip(alone, batch):
        for f in (cap.RVE_FIELD_PHI, cap.RVE_FIELD_H, cap.RVE_FIELD_EPS):
            assert np.array_equal(ga.get(f), gb.get(f))


def test_batch_refuses_mixed_grids(cap):
    from paper_2508_07424_gb300.rve import Rve
    import ctypes as C
    a = Rve.from_workload(_poly2d(11, "fp64"))
    b = Rve.from_workload(_poly3d(12, "fp64"))
    hs = (cap.rve_handle * 2)(a.h, b.h)
    dt = (C.c_double * 2)(0.1, 0.1)
    assert cap.lib().rve_step_batch(hs, 2, dt, None) == cap.RVE_EINVAL
    hs = (cap.rve_handle * 2)(a.h, a.h)
    assert cap.lib().rve_step_batch(hs, 2, dt, None) == cap.RVE_EINVAL
