"""The seeded workload configurations (synth/configs.json) build with their stated shapes."""
import numpy as np
import pytest

import synth

EXPECT = {
    "c0_homogeneous_plate_64": ((64, 64, 1), 2, 1),
    "c1_fibre_composite_512": ((512, 512, 1), 2, 0),
    "c2_polycrystal_1024": ((1024, 1024, 1), 2, 0),
    "plate_polycrystal_256": ((256, 128, 1), 3, 0),
}


@pytest.mark.parametrize("name", sorted(EXPECT))
def test_single_configurations(name):
    w = synth.load_config(name)
    n, dim, split = EXPECT[name]
    assert w.micro.n == n and w.micro.dim == dim and w.split == split
    assert w.dtau > 0 and w.micro.crack.kind == synth.CRACK_CTE


def test_config_names_cover_the_five_benchmark_configurations():
    names = synth.config_names()
    for prefix in ("c0_", "c1_", "c2_", "c3_", "c4_"):
        assert any(n.startswith(prefix) for n in names)


def test_serving_mix_is_seeded_and_mixed():
    a = synth.load_config("c4_serving_mix")
    b = synth.load_config("c4_serving_mix")
    assert len(a) == 24
    assert all(np.array_equal(x.micro.grain_id, y.micro.grain_id) for x, y in zip(a, b))
    dims = {w.micro.dim for w in a}
    assert dims == {2, 3} and all(w.precision == "fp32r" for w in a)
