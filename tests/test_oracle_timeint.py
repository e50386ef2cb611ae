"""The oracle's classic RK4 (Section 6 integrates every test with it) pinned
to what the method of Runge and Kutta fixes, without retyping its tableau:

* on a linear system y' = A y one step is the degree-4 Taylor polynomial of
  exp(dt A) applied to y (the stability function 1 + z + z^2/2 + z^3/6 +
  z^4/24 of every four-stage fourth-order method); a wrong weight or stage
  coefficient changes a power of dt;
* for y' = g(t) the step is Simpson's rule, exact for cubics in t (pins the
  stage times t, t + dt/2, t + dt/2, t + dt);
* on the DG semi-discretisation at fixed h the error against a run with a
  far smaller step falls 16 times per halving of dt (temporal order 4).

and its two error norms of Section 6 (L2 and energy) pinned to closed-form
integrals (a zero discrete state against sin(pi x) on a shifted box, and
sin(pi x) sin(pi y)) and to zero for polynomials the GD basis reproduces."""
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


# ---- the error norms of Section 6 (timeint.errors) ----

def test_error_norms_of_a_zero_state_are_the_exact_norms_1d():
    """U = V = 0 on [a, b]: the L2 error is ||u|| and the energy-norm error
    (||u_x||^2 + ||v||^2)^1/2, both known in closed form for u = sin(pi x),
    v = c (Gauss quadrature with p + 3 points per cell, exact to rounding
    for these smooth integrands at this resolution)."""
    a, b, c = -1.0, 0.5, 0.7
    prob = dc.Problem(dim=1, n=(3,), N=6, p=3, lo=(a,), hi=(b,))
    Z = np.zeros((3, 7))
    exact = lambda t, x: (np.sin(np.pi * x), [np.pi * np.cos(np.pi * x)], np.full_like(x, c))
    l2, en = ti.errors(prob, Z, Z, exact, 0.0)
    s = (np.sin(2 * np.pi * b) - np.sin(2 * np.pi * a)) / (4 * np.pi)
    assert abs(l2 - np.sqrt((b - a) / 2 - s)) < 1e-12
    assert abs(en - np.sqrt(np.pi ** 2 * ((b - a) / 2 + s) + c * c * (b - a))) < 1e-12


def test_error_norms_of_a_zero_state_are_the_exact_norms_2d():
    """u = sin(pi x) sin(pi y) on the unit square: ||u|| = 1/2 and
    ||grad u|| = pi / sqrt2."""
    prob = dc.Problem(dim=2, n=(3, 2), N=5, p=3)
    Z = np.zeros((6, 36))
    exact = lambda t, X, Y: (np.sin(np.pi * X) * np.sin(np.pi * Y),
                             [np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y),
                              np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)], np.zeros_like(X))
    l2, en = ti.errors(prob, Z, Z, exact, 0.0)
    assert abs(l2 - 0.5) < 1e-12 and abs(en - np.pi / np.sqrt(2.0)) < 1e-12


@pytest.mark.parametrize("p", [3, 5])
def test_polynomials_the_basis_reproduces_have_zero_error(p):
    """Nodal values of a polynomial of degree <= p: the GD basis reproduces
    it, so both error norms vanish; the polynomials are not symmetric in x
    and y, so a transposed evaluation does not vanish."""
    prob = dc.Problem(dim=1, n=(4,), N=7, p=p, lo=(0.2,), hi=(1.4,))
    (X,) = dc.node_coordinates(prob)
    P = lambda x: x ** p - 0.3 * x ** 2 + 1.0
    dP = lambda x: p * x ** (p - 1) - 0.6 * x
    exact = lambda t, x: (P(x), [dP(x)], 2.0 * P(x))
    l2, en = ti.errors(prob, P(X), 2.0 * P(X), exact, 0.0)
    assert l2 < 1e-12 and en < 1e-11, (l2, en)
    prob2 = dc.Problem(dim=2, n=(2, 3), N=p + 1, p=p, lo=(0.0, -0.5), hi=(1.0, 1.0))
    X, Y = dc.node_coordinates(prob2)
    Q = lambda x, y: x ** p * y + 2.0 * y ** 2 - x
    exact2 = lambda t, x, y: (Q(x, y), [p * x ** (p - 1) * y - 1.0, x ** p + 4.0 * y], np.zeros_like(x))
    U = Q(X, Y).reshape(6, -1)
    l2, en = ti.errors(prob2, U, np.zeros_like(U), exact2, 0.0)
    assert l2 < 1e-12 and en < 1e-11, (l2, en)
    # the same nodal values read with x and y exchanged are not the polynomial
    Ut = Q(Y, X).reshape(6, -1)
    assert ti.errors(prob2, Ut, np.zeros_like(U), exact2, 0.0)[0] > 1e-2
