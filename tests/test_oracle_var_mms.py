"""Pins of the oracle's variable-coefficient volume term and of its IC(0)
preconditioner (Section 7.1).

The energy identities and the constant-c^2 reductions in test_oracle_var.py
cannot see where a spatially varying c^2 enters the stiffness integral.
Manufactured solutions can: f = u_tt - div(c^2 grad u) is computed here
from the exact u, c^2 and grad c^2 (not from the oracle), loaded as
int phi f |J|, and the discrete solution must converge at the optimal rate
p+1.  Evaluating c^2 anywhere but at the right quadrature points leaves an
O(1) consistency error and the rate collapses.

* Table 5's problem: c^2 = 1 + x^2 + y^2, u = sin(8 sqrt2 pi t)
  sin(8 pi x) sin(8 pi y), p = 3, 2 x 2 elements, N+1 = 11 and 21, T = 0.2.
  The paper imposes periodic conditions, under which this c^2 jumps across
  the periodic seam and c^2 du/dn is discontinuous there; u vanishes on the
  boundary of the unit square, so Dirichlet u = 0 is used instead.  The
  printed L2 errors are then a soft bound (same magnitude), the rate a hard
  one.
* The sine-mapped unit square with c^2 = 1 + 0.5 sin 2pi x cos 2pi y and
  u = sin(2 sqrt2 pi t) sin(2 pi x) sin(2 pi y).

IC(0) is pinned against the exact Cholesky factor where the factor has no
fill outside the pattern (a banded matrix; a Kronecker product of banded
matrices, which is every Cartesian element mass matrix), against a 4 x 4
factor worked by hand with one dropped fill entry, and against Table 5's
iteration counts (v_t: 1 iteration at every resolution; u_t: below 6).
"""
import os

import numpy as np
import pytest

from oracle import dg_var as dv, gd_basis, timeint as ti
from paper_2105_01722_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table5():
    rows = []
    for line in open(os.path.join(GOLDEN, "table5_pcg.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return np.array(rows)


def _manufactured(k, c2, grad_c2):
    """u = sin(w t) sin(k pi x) sin(k pi y), w = sqrt2 k pi, for
    u_tt = div(c^2 grad u) + f: returns (u(t, x, y), v(t, x, y), f(t, x, y))."""
    K = k * np.pi
    w = np.sqrt(2.0) * K

    def u(t, x, y):
        return np.sin(w * t) * np.sin(K * x) * np.sin(K * y)

    def v(t, x, y):
        return w * np.cos(w * t) * np.sin(K * x) * np.sin(K * y)

    def f(t, x, y):
        s = np.sin(w * t)
        uu = s * np.sin(K * x) * np.sin(K * y)
        ux = s * K * np.cos(K * x) * np.sin(K * y)
        uy = s * K * np.sin(K * x) * np.cos(K * y)
        gx, gy = grad_c2(x, y)
        # u_tt = -w^2 u; div(c^2 grad u) = c^2 lap u + grad c^2 . grad u, lap u = -2 K^2 u
        return -w * w * uu + 2.0 * K * K * c2(x, y) * uu - gx * ux - gy * uy

    return u, v, f


def _solve_mms(vp, u, v, f, T, cfl):
    """RK4 with the forcing evaluated at each stage's time; element systems
    solved with their exact inverses (formed once; the oracle's dense route)."""
    ops = dv.assemble(vp)
    ne = vp.n[0] * vp.n[1]
    Ainv = np.array([np.linalg.inv(dv.spd_u_matrix(ops, e)) for e in range(ne)])
    Minv = np.array([np.linalg.inv(ops.M[e]) for e in range(ne)])

    def rhs(t, U, V):
        F = dv.distributed_load(vp, lambda x, y: f(t, x, y))
        ru, rv = dv.residuals(vp, ops, U, V, forcing=F)
        return V + np.einsum("eab,eb->ea", Ainv, ru), np.einsum("eab,eb->ea", Minv, rv)

    U = u(0.0, vp.X, vp.Y).reshape(ne, -1)       # nodal interpolation of the data
    V = v(0.0, vp.X, vp.Y).reshape(ne, -1)
    h = 1.0 / (vp.n[0] * vp.N)
    steps = int(np.ceil(T / (cfl * h)))
    U, V = ti.integrate(rhs, U, V, 0.0, T / steps, steps)
    return dv.l2_error(vp, U, lambda x, y: u(T, x, y))


def _table5_problem(N):
    X, Y = inputs.cartesian_nodes((2, 2), N)
    c2 = lambda x, y: 1.0 + x * x + y * y
    return dv.VarProblem(n=(2, 2), N=N, p=3, X=X, Y=Y, C2=c2(X, Y)), c2


def test_table5_manufactured_solution():
    """Section 7.1, Table 5 (Dirichlet instead of periodic, see above).
    CFL 0.05 instead of 0.075/(2 pi): the errors agree to three digits and
    the run is 4x shorter."""
    gold = _table5()
    errs = []
    for N in (10, 20):
        vp, c2 = _table5_problem(N)
        u, v, f = _manufactured(8, c2, lambda x, y: (2.0 * x, 2.0 * y))
        errs.append(_solve_mms(vp, u, v, f, T=0.2, cfl=0.05))
    rate = np.log2(errs[0] / errs[1])
    assert rate > 3.7, (errs, rate)                       # optimal p+1 = 4 (Table 5: 4.31)
    for e, g in zip(errs, gold[:2, 1]):                   # same magnitude as the printed errors
        assert g / 2.0 < e < 2.0 * g, (errs, gold[:2, 1])


def test_mapped_manufactured_solution():
    """Sine-mapped mesh, c^2 = 1 + 0.5 sin 2pi x cos 2pi y (physical x, y):
    L2 rate about p+1 = 4 from 2x2 to 4x4 elements of 6x6 cells."""
    c2 = lambda x, y: 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    gc2 = lambda x, y: (np.pi * np.cos(2 * np.pi * x) * np.cos(2 * np.pi * y),
                        -np.pi * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y))
    u, v, f = _manufactured(2, c2, gc2)
    errs = []
    for n in (2, 4):
        X, Y = inputs.mapped_nodes((n, n), 6, 0.05)
        vp = dv.VarProblem(n=(n, n), N=6, p=3, X=X, Y=Y, C2=c2(X, Y))
        errs.append(_solve_mms(vp, u, v, f, T=0.1, cfl=0.05))
    rate = np.log2(errs[0] / errs[1])
    assert rate > 3.6 and errs[1] < 2e-4, (errs, rate)


def test_distributed_load_moments():
    """int phi_a f |J| summed over a reproduces int f over the (mapped)
    domain: f = 1 gives the area (1 up to the geometry's interpolation
    error), f = x gives int x = 1/2, and both are exact on a Cartesian mesh."""
    for amp, tol in ((0.0, 1e-14), (0.05, 1e-6)):
        X, Y = inputs.mapped_nodes((3, 2), 6, amp)
        vp = dv.VarProblem(n=(3, 2), N=6, p=3, X=X, Y=Y, C2=np.ones_like(X))
        assert abs(dv.distributed_load(vp, lambda x, y: 1.0 + 0.0 * x).sum() - 1.0) < tol
        assert abs(dv.distributed_load(vp, lambda x, y: x).sum() - 0.5) < tol


def _read_ic0_golden():
    A, L, cur = [], [], None
    for line in open(os.path.join(GOLDEN, "ic0_4x4.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line in ("A", "L"):
            cur = A if line == "A" else L
            continue
        cur.append([float(x) for x in line.split()])
    return np.array(A), np.array(L)


def test_ic0_hand_worked_dropped_fill():
    A, L = _read_ic0_golden()
    got = dv.ic0(A)
    assert np.abs(got - L).max() < 1e-15
    exact = np.linalg.cholesky(A)
    assert abs(exact[2, 1]) > 0.1 and got[2, 1] == 0.0       # the dropped fill


def test_ic0_exact_without_fill():
    """Banded SPD (the 1-D GD mass and shifted stiffness matrices, half
    bandwidth p) and the Kronecker product of two of them (a Cartesian
    element mass matrix): the Cholesky factor lies inside the pattern, so
    IC(0) is exact."""
    Mh, Sh = gd_basis.mass_stiffness(5, 12)
    for A in (Mh, Sh + Mh, np.kron(Mh, Mh), np.kron(Mh, Sh + Mh)):
        Lx = np.linalg.cholesky(A)
        assert np.abs(dv.ic0(A) - Lx).max() < 1e-13 * np.abs(Lx).max()
    # a random banded SPD matrix
    rng = np.random.default_rng(11)
    n, bw = 30, 4
    B = np.triu(np.tril(rng.standard_normal((n, n)), bw), -bw)
    A = B @ B.T + n * np.eye(n)           # half bandwidth 2 bw
    Lx = np.linalg.cholesky(A)
    assert np.abs(dv.ic0(A) - Lx).max() < 1e-13 * np.abs(Lx).max()


@pytest.mark.parametrize("N", [10, 20])
def test_ic0_pcg_iterations_table5(N):
    """Table 5 iteration counts with IC(0) at the printed tolerances (rtol
    1e-3 / 16^k): the v_t system (M, a Kronecker product on the Cartesian
    elements) needs exactly 1 iteration, as printed; the u_t system a few,
    growing with N and below 6 (printed averages 1.58, 2.13)."""
    gold = _table5()
    vp, c2 = _table5_problem(N)
    ops = dv.assemble(vp)
    u, v, _ = _manufactured(8, c2, lambda x, y: (2.0 * x, 2.0 * y))
    U = u(0.05, vp.X, vp.Y).reshape(4, -1)
    V = v(0.05, vp.X, vp.Y).reshape(4, -1)
    ru, rv = dv.residuals(vp, ops, U, V)
    rtol = gold[{10: 0, 20: 1}[N], 2]
    Ut, Vt, iu, iv = dv.solve_pcg(vp, ops, V, ru, rv, precond="ic0", rtol=rtol, maxit=50)
    assert np.all(iv == 1), iv
    assert 1 <= iu.mean() < 6, iu
    Ud, Vd = dv.solve_direct(ops, V, ru, rv)
    assert np.linalg.norm(Vt - Vd) <= 2 * rtol * np.linalg.norm(Vd)
    if N == 20:
        vp10, _ = _table5_problem(10)
        ops10 = dv.assemble(vp10)
        U = u(0.05, vp10.X, vp10.Y).reshape(4, -1)
        V = v(0.05, vp10.X, vp10.Y).reshape(4, -1)
        ru, rv = dv.residuals(vp10, ops10, U, V)
        _, _, iu10, _ = dv.solve_pcg(vp10, ops10, V, ru, rv, precond="ic0", rtol=gold[0, 2], maxit=50)
        assert iu.mean() > iu10.mean()


@pytest.mark.parametrize("amp", [0.0, 0.05])
def test_l2_error_norm_on_mapped_elements(amp):
    """dg_var.l2_error, the error measure of the mapped tests: with a zero
    discrete state it is ||sin(pi x) sin(pi y)|| = 1/2 over the unit square.
    The interpolated sine map still maps the reference square onto the unit
    square (its boundary nodes lie on the boundary, and so does their
    interpolant), so the change of variables is exact and only quadrature
    rounding remains; a wrong Jacobian determinant or mapped point breaks
    it.  On the Cartesian mesh a polynomial of degree <= p (not symmetric in
    x and y) has zero error."""
    for n, N, p in ((2, 6, 3), (3, 8, 5)):
        X, Y = inputs.mapped_nodes((n, n), N, amp)
        vp = dv.VarProblem(n=(n, n), N=N, p=p, X=X, Y=Y, C2=np.ones_like(X))
        Z = np.zeros((n * n, (N + 1) ** 2))
        l2 = dv.l2_error(vp, Z, lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y))
        assert abs(l2 - 0.5) < 1e-14, (n, N, p, l2)
        if amp == 0.0:
            P = lambda x, y: x ** p * y - 0.5 * y ** 2 + x
            assert dv.l2_error(vp, P(X, Y).reshape(n * n, -1), P) < 1e-14
            assert dv.l2_error(vp, P(Y, X).reshape(n * n, -1), P) > 1e-2
