"""Checkpoint file round trip (host only): state, time, step and the problem
description, including the nodal geometry and c^2 arrays of a mapped
variable-coefficient problem, come back unchanged."""
import numpy as np

from paper_2105_01722_gb300 import checkpoint, gdg, inputs


def test_round_trip(tmp_path):
    X, Y = inputs.mapped_nodes((3, 2), 8, 0.05)
    C2 = inputs.c2_sine(X, Y)
    kw = dict(dim=2, n=(3, 2), N=8, p=5, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
              bc=(gdg.BC_PERIODIC, gdg.BC_DIRICHLET), flux=gdg.FLUX_ALTERNATING, pcg_rtol=1e-11,
              solver=gdg.SOLVE_INVERSE)
    u = inputs.random_state(X.size, 1)
    v = inputs.random_state(X.size, 2)
    checkpoint.save(tmp_path / "c.npz", u, v, 0.125, 40, kw)
    u2, v2, t, step, kw2 = checkpoint.load(tmp_path / "c.npz")
    assert np.array_equal(u, u2) and np.array_equal(v, v2) and t == 0.125 and step == 40
    assert set(kw2) == set(kw)
    for k, a in kw.items():
        if isinstance(a, np.ndarray):
            assert np.array_equal(kw2[k], a)
        else:
            assert kw2[k] == a, k
    pb = checkpoint.make_problem(kw2)
    assert pb.flux == gdg.FLUX_ALTERNATING and pb.solver == gdg.SOLVE_INVERSE and pb.n_elem[0] == 3
