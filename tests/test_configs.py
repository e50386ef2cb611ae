"""The named workload presets (host side only: descriptions and states)."""
import numpy as np
import pytest

from paper_2105_01722_gb300 import configs, gdg


def _dof(pb):
    n1 = pb.N + 1
    return int(np.prod([pb.n_elem[k] for k in range(pb.dim)])) * n1 ** pb.dim


def test_every_preset_builds_consistent_descriptions():
    small = {"standing_wave_1d": {}, "const_2d_64": {"n": 4}, "mapped_2d_128": {"n": 4},
             "batched_48": {"count": 4, "nmin": 2, "nmax": 5}, "learned_128": {"n": 4}}
    for name, kw in small.items():
        c = configs.preset(name, **kw)
        assert c["name"] == name and len(c["problems"]) == len(c["states"]) == len(c["dt"]) >= 1
        for pb, (U, V), dt in zip(c["problems"], c["states"], c["dt"]):
            assert U.size == V.size == _dof(pb) and dt > 0
            assert np.all(np.isfinite(U)) and np.all(np.isfinite(V))


def test_paper_sizes_and_exact_solutions():
    c = configs.preset("standing_wave_1d")
    pb = c["problems"][0]
    assert (pb.dim, pb.n_elem[0], pb.N, pb.p) == (1, 16, 8, 3)
    assert c["steps"] == 256 and abs(c["dt"][0] * c["steps"] - 1.0) < 1e-15    # CFL 0.5, h = 1/128
    U, V = c["states"][0]
    Ue, Ve = c["exact"](0.0)
    assert np.array_equal(U, Ue) and np.array_equal(V, Ve)
    c = configs.preset("const_2d_64")
    assert _dof(c["problems"][0]) == 331776 and c["problems"][0].p == 5
    c = configs.preset("mapped_2d_128", p=3)
    pb = c["problems"][0]
    assert pb.coef == gdg.COEF_NODAL and _dof(pb) == 128 * 128 * 81 and pb.pcg_rtol == 1e-10
    assert abs(c["dt"][0] * c["steps"] - 0.25) < 1e-12
    with pytest.raises(KeyError):
        configs.preset("no_such_workload")
