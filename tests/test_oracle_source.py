"""Pins of the oracle's forcing (the f of u_tt = div(c^2 grad u) + f, added as
int phi_a f to r_v) for a point source f = s(t) delta(x - x_s), independent
of the CUDA path.

* Energy rate: with a conservative flux (central or alternating) the
  semi-discrete energy E = 1/2 sum_e (V^T M_J V + U^T S U) changes only by the
  work of the source, dE/dt = sum_e V_e . F_e, where F is the load vector.
* The load phi_a(x_s) of a point at reference (r, s): it sums to 1 (the GD
  basis reproduces constants), its first moments are (r, s) (it reproduces
  linears), and it is the unit vector when x_s is a node (the basis is
  interpolatory).
"""
import numpy as np
import pytest

from oracle import dg_var as dv, gd_basis as gb
from paper_2105_01722_gb300 import inputs


def _load(p, N, r, s):
    pr, _ = gb.eval_basis(p, N, r)
    ps, _ = gb.eval_basis(p, N, s)
    return np.outer(ps, pr).ravel()


@pytest.mark.parametrize("flux", ["central", "alternating"])
@pytest.mark.parametrize("periodic", [(False, False), (True, False)])
def test_energy_rate_is_the_source_power(flux, periodic):
    n, N, p = (3, 2), 5, 3
    X, Y = inputs.mapped_nodes(n, N, 0.05)
    vp = dv.VarProblem(n=n, N=N, p=p, X=X, Y=Y, C2=inputs.c2_sine(X, Y), flux=flux, periodic=periodic)
    ops = dv.assemble(vp)
    ne, na = n[0] * n[1], (N + 1) ** 2
    rng = np.random.default_rng(3)
    U = rng.standard_normal((ne, na))
    V = rng.standard_normal((ne, na))
    F = np.zeros((ne, na))
    F[4] = 1.7 * _load(p, N, 0.3, 0.8)
    ru, rv = dv.residuals(vp, ops, U, V, forcing=F)
    Ut, Vt = dv.solve_direct(ops, V, ru, rv)
    rate = np.einsum("ea,eab,eb->", V, ops.M, Vt) + np.einsum("ea,eab,eb->", U, ops.S, Ut)
    power = float(np.sum(V * F))
    scale = np.abs(np.einsum("ea,eab,eb->", V, ops.M, Vt)) + abs(power)
    assert abs(rate - power) < 1e-10 * scale
    # the source does change the rate: without it the rate vanishes
    ru0, rv0 = dv.residuals(vp, ops, U, V)
    Ut0, Vt0 = dv.solve_direct(ops, V, ru0, rv0)
    rate0 = np.einsum("ea,eab,eb->", V, ops.M, Vt0) + np.einsum("ea,eab,eb->", U, ops.S, Ut0)
    assert abs(rate0) < 1e-10 * scale and abs(power) > 1e-3


@pytest.mark.parametrize("p,N", [(3, 8), (5, 8), (5, 6), (7, 9)])
def test_point_load_weights(p, N):
    rng = np.random.default_rng(p * 10 + N)
    nodes = np.arange(N + 1) / N
    for _ in range(5):
        r, s = rng.uniform(0.0, 1.0, 2)
        w = _load(p, N, r, s)
        assert abs(w.sum() - 1.0) < 1e-13
        # linears: sum_a phi_a(r, s) (r_a, s_a) = (r, s)
        ri = np.tile(nodes, N + 1)
        si = np.repeat(nodes, N + 1)
        assert abs(w @ ri - r) < 1e-13 and abs(w @ si - s) < 1e-13
    for (i, j) in [(0, 0), (N, N), (2, N - 1)]:
        w = _load(p, N, nodes[i], nodes[j])
        e = np.zeros((N + 1) ** 2)
        e[j * (N + 1) + i] = 1.0
        assert np.abs(w - e).max() < 1e-13
