"""The oracle's classic RK4 (Section 6 integrates every test with it) pinned
to what the method of Runge and Kutta fixes, without retyping its tableau:

* on a linear system y' = A y one step is the degree-4 Taylor polynomial of
  exp(dt A) applied to y (the stability function 1 + z + z^2/2 + z^3/6 +
  z^4/24 of every four-stage fourth-order method); a wrong weight or stage
  coefficient changes a power of dt;
* for y' = g(t) the step is Simpson's rule, exact for cubics in t (pins the
  stage times t, t + dt/2, t + dt/2, t + dt);
* on the DG semi-discretisation at fixed h the error against a run with a
  far smaller step falls 16 times per halving of dt (temporal order 4)."""
import numpy as np
import pytest

from oracle import dg_const as dc, timeint as ti


def _taylor4(M):
    out, term = np.eye(M.shape[0]), np.eye(M.shape[0])
    for k in range(1, 5):
        term = term @ M / k
        out = out + term
    return out


@pytest.mark.parametrize("dt", [0.3, 0.05, 1.7])
def test_linear_step_is_taylor_polynomial(dt):
    rng = np.random.default_rng(7)
    n = 3
    A = rng.standard_normal((2 * n, 2 * n))
    y = rng.standard_normal(2 * n)
    f = lambda t, U, V: tuple(np.split(A @ np.concatenate([U, V]), 2))
    U, V = ti.rk4_step(f, y[:n], y[n:], 0.0, dt)
    want = _taylor4(dt * A) @ y
    assert np.allclose(np.concatenate([U, V]), want, rtol=0, atol=1e-13 * max(1.0, np.abs(want).max()))


def test_quadrature_of_cubics_in_time():
    # y' = g(t), g cubic: RK4 is Simpson's rule on each step, exact
    g = lambda t: 1.0 - 2.0 * t + 3.0 * t ** 2 + 4.0 * t ** 3
    G = lambda t: t - t ** 2 + t ** 3 + t ** 4
    f = lambda t, U, V: (np.array([g(t)]), np.array([0.0]))
    t0, dt, steps = 0.25, 0.125, 6
    U, V = ti.integrate(f, np.array([0.0]), np.array([0.0]), t0, dt, steps)
    assert abs(U[0] - (G(t0 + steps * dt) - G(t0))) < 1e-14
    # a quartic is not integrated exactly: the stage times matter
    f4 = lambda t, U, V: (np.array([5.0 * t ** 4]), np.array([0.0]))
    U4, _ = ti.integrate(f4, np.array([0.0]), np.array([0.0]), 0.0, 0.5, 2)
    assert abs(U4[0] - 1.0) > 1e-4


def test_temporal_order_four_on_the_semidiscretisation():
    prob = dc.Problem(dim=1, n=(4,), N=6, p=3, flux="upwind")
    ops = dc.operators(prob)
    (X,) = dc.node_coordinates(prob)
    U0, V0 = np.sin(2 * np.pi * X), np.zeros_like(X)
    f = lambda t, U, V: dc.time_derivative(prob, U, V, ops)
    T = 0.25
    ref = ti.integrate(f, U0, V0, 0.0, T / 640, 640)
    errs = []
    for steps in (20, 40, 80):     # dt = 0.3 h, 0.15 h, 0.075 h (stable for upwind p = 3)
        U, V = ti.integrate(f, U0, V0, 0.0, T / steps, steps)
        errs.append(np.sqrt(np.sum((U - ref[0]) ** 2 + (V - ref[1]) ** 2)))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 13.0) & (ratios < 19.0)), (errs, ratios)
