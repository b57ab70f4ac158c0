"""Column-tile autotuner of the y / z FFT passes (a tuning aid of this implementation; the paper
has no counterpart). Every kx column is transformed by the same code whatever the tile width, so
the width must not change any result, bit for bit; the tuner's choice must persist in its cache."""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cap():
    from paper_2508_07424_gb300 import build, capi
    build.build()
    return capi


def _poly2d():
    crack = synth.Crack(synth.CRACK_CTE, row=32, x0=0, length=8, phi_M=0.8)
    m = synth.voronoi((64, 64), 9, 21, beta=2.0, crack=crack)
    w = synth.Workload(m, ell=2.0, n_inc=10)
    w.dtau = 1.5 * w.A_g / 24
    return w


@pytest.mark.parametrize("case", ["poly2d", "poly3d"])
def test_tile_width_does_not_change_results(cap, monkeypatch, case):
    from paper_2508_07424_gb300.rve import Rve
    if case == "poly2d":
        w, widths = _poly2d(), [(2, 2), (16, 2)]
    else:
        w, widths = synth.small_cases()["poly3d"], [(8, 16), (16, 16)]
    out = []
    for y, z in widths:
        monkeypatch.setenv("PFF_TILE_CW", f"{y},{z}")
        g = Rve.from_workload(w)
        assert g.tiles() == (y, z if w.micro.dim == 3 else 0)
        rs = [g.step(w.dtau) for _ in range(2)]
        out.append((rs, g.get(cap.RVE_FIELD_PHI), g.get(cap.RVE_FIELD_EPS), g.get(cap.RVE_FIELD_H)))
        g.close()
    a, b = out
    assert a[0] == b[0]
    for x, y in zip(a[1:], b[1:]):
        assert np.array_equal(x, y)


_PROBE = """
import sys
sys.path.insert(0, {root!r})
import synth
from paper_2508_07424_gb300.rve import Rve
crack = synth.Crack(synth.CRACK_CTE, row=16, x0=0, length=8, phi_M=0.8)
w = synth.Workload(synth.homogeneous((128, 32), crack=crack), ell=2.0)
g = Rve.from_workload(w)
print(*g.tiles())
"""


def test_tuned_widths_persist_in_the_cache(cap, tmp_path):
    cache = tmp_path / "tiles.txt"
    env = dict(os.environ, PFF_TILE_CACHE=str(cache))
    env.pop("PFF_TILE_CW", None)
    env.pop("PFF_TILE_TUNE", None)
    probe = _PROBE.format(root=ROOT)
    y, z = map(int, subprocess.run([sys.executable, "-c", probe], env=env, check=True, capture_output=True,
                                   text=True).stdout.split())
    assert z == 0 and y in (1, 2, 4, 8, 16)    # every width up to 16 fits the shared memory here
    lines = cache.read_text().split("\n")
    key, cy, cz = lines[0].split()
    assert "|d2|128x32x1|fp64" in key and int(cy) == y
    # a later process takes the cached width (the last line for a key wins) instead of measuring
    other = [v for v in (1, 2, 4, 8, 16) if v != y][0]
    with open(cache, "a") as f:
        f.write(f"{key} {other} {cz}\n")
    y2, _ = map(int, subprocess.run([sys.executable, "-c", probe], env=env, check=True, capture_output=True,
                                    text=True).stdout.split())
    assert y2 == other
