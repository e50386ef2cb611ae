"""Pins of the oracle's variable-coefficient / mapped-element path
(Section 7.1): reduction to the Cartesian constant-coefficient oracle,
energy identities by brute force, exact kernels and constraints, PCG
against the dense solve, and convergence on a mapped mesh."""
import numpy as np
import pytest

from oracle import dg_const as dc, dg_var as dv, timeint as ti
from paper_2105_01722_gb300 import inputs


def _var_problem(n, N, p, flux="upwind", amp=0.05, c2="sine", periodic=(False, False), xi=0.0):
    X, Y = inputs.mapped_nodes(n, N, amp)
    if c2 == "sine":
        C2 = inputs.c2_sine(X, Y)
    elif c2 == "one":
        C2 = np.ones_like(X)
    else:
        C2 = inputs.smooth_random_c2(X, Y, seed=5)
    return dv.VarProblem(n=n, N=N, p=p, X=X, Y=Y, C2=C2, flux=flux, periodic=periodic, xi=xi)


def _dense(vp, ops):
    ne = vp.n[0] * vp.n[1]
    nd = ne * vp.n1 ** 2
    L = np.zeros((2 * nd, 2 * nd))
    for c in range(2 * nd):
        z = np.zeros(2 * nd)
        z[c] = 1.0
        Ut, Vt = dv.time_derivative(vp, ops, z[:nd].reshape(ne, -1), z[nd:].reshape(ne, -1))
        L[:nd, c] = Ut.ravel()
        L[nd:, c] = Vt.ravel()
    from scipy.linalg import block_diag
    E = block_diag(block_diag(*ops.S), block_diag(*ops.M))
    return L, E


@pytest.mark.parametrize("flux", ["central", "upwind", "alternating"])
@pytest.mark.parametrize("periodic", [(False, False), (True, False), (False, True)])
def test_reduces_to_cartesian_constant(flux, periodic):
    """Affine (Cartesian) geometry and constant c^2: the quadrature route
    reproduces the Kronecker route (exact quadrature with p+1 points)."""
    prob = dc.Problem(dim=2, n=(3, 2), N=5, p=3, lo=(0.2, -0.1), hi=(1.7, 0.7),
                      periodic=periodic, flux=flux, c2=2.3)
    X, Y = dc.node_coordinates(prob)
    vp = dv.VarProblem(n=prob.n, N=prob.N, p=prob.p, X=X, Y=Y, C2=np.full_like(X, 2.3),
                       periodic=periodic, flux=flux)
    ops = dv.assemble(vp)
    opc = dc.operators(prob)
    assert np.abs(ops.M - opc.M).max() < 1e-14 * np.abs(opc.M).max() * 10
    assert np.abs(ops.S - 2.3 * opc.S).max() < 1e-13 * np.abs(opc.S).max()
    rng = np.random.default_rng(1)
    U = rng.standard_normal((6, 36))
    V = rng.standard_normal((6, 36))
    ru, rv = dc.residuals(prob, U, V, opc)
    ru2, rv2 = dv.residuals(vp, ops, U, V)
    assert np.abs(2.3 * ru - ru2).max() < 1e-13 * np.abs(ru2).max()
    assert np.abs(rv - rv2).max() < 1e-13 * np.abs(rv).max()
    Ut, Vt = dc.time_derivative(prob, U, V, opc)
    Ut2, Vt2 = dv.time_derivative(vp, ops, U, V)
    assert np.abs(Ut - Ut2).max() < 1e-12 * np.abs(Ut).max()
    assert np.abs(Vt - Vt2).max() < 1e-12 * np.abs(Vt).max()


@pytest.mark.parametrize("c2", ["sine", "random"])
def test_central_conserves_energy_mapped(c2):
    vp = _var_problem((2, 2), 3, 3, flux="central", amp=0.05, c2=c2)
    ops = dv.assemble(vp)
    L, E = _dense(vp, ops)
    A = E @ L + L.T @ E
    assert np.abs(A).max() < 1e-10 * np.abs(E @ L).max()


@pytest.mark.parametrize("periodic", [(False, False), (True, False)])
def test_alternating_conserves_energy_mapped(periodic):
    vp = _var_problem((2, 2), 3, 3, flux="alternating", amp=0.05, c2="sine", periodic=periodic)
    ops = dv.assemble(vp)
    L, E = _dense(vp, ops)
    A = E @ L + L.T @ E
    assert np.abs(A).max() < 1e-10 * np.abs(E @ L).max()


@pytest.mark.parametrize("periodic", [(False, False), (True, True)])
def test_upwind_dissipates_mapped(periodic):
    vp = _var_problem((2, 2), 3, 3, flux="upwind", amp=0.05, periodic=periodic)
    ops = dv.assemble(vp)
    L, E = _dense(vp, ops)
    A = -(E @ L + L.T @ E)
    lam = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert lam.min() > -1e-9 * np.abs(lam).max()
    assert lam.max() > 1e-3


def test_matrices_and_constraints_mapped():
    vp = _var_problem((3, 3), 4, 3)
    ops = dv.assemble(vp)
    one = np.ones(25)
    for e in range(9):
        M, S = ops.M[e], ops.S[e]
        assert np.abs(M - M.T).max() < 1e-15
        assert np.abs(S - S.T).max() < 1e-13 * np.abs(S).max()
        assert np.linalg.eigvalsh(M).min() > 0
        assert np.abs(S @ one).max() < 1e-12 * np.abs(S).max()
    # the mapped unit square keeps area 1 (interpolated geometry: ~h^(p+1))
    area = sum(one @ ops.M[e] @ one for e in range(9))
    assert abs(area - 1.0) < 1e-5
    rng = np.random.default_rng(2)
    U = rng.standard_normal((9, 25))
    V = rng.standard_normal((9, 25))
    ru, rv = dv.residuals(vp, ops, U, V)
    assert np.abs(ru.sum(axis=1)).max() < 1e-11 * np.abs(ru).max()
    Ut, Vt = dv.time_derivative(vp, ops, U, V)
    w = np.einsum("eab,b->ea", ops.M, one)
    assert np.abs(np.einsum("ea,ea->e", w, Ut - V)).max() < 1e-12 * np.abs(Ut).max()


@pytest.mark.parametrize("precond", ["fdm", "ic0", "none"])
def test_pcg_matches_direct(precond):
    vp = _var_problem((2, 2), 8, 5)
    ops = dv.assemble(vp)
    rng = np.random.default_rng(4)
    U = rng.standard_normal((4, 81))
    V = rng.standard_normal((4, 81))
    ru, rv = dv.residuals(vp, ops, U, V)
    Ut, Vt = dv.solve_direct(ops, V, ru, rv)
    Ut2, Vt2, iu, iv = dv.solve_pcg(vp, ops, V, ru, rv, precond=precond, rtol=1e-13, maxit=500)
    assert np.abs(Ut - Ut2).max() < 1e-9 * np.abs(Ut).max()
    assert np.abs(Vt - Vt2).max() < 1e-9 * np.abs(Vt).max()
    if precond == "fdm":
        assert iu.max() < 40 and iv.max() < 25


def test_fdm_preconditioner_exact_on_affine():
    """On an affine element with constant c^2 the frozen-coefficient
    diagonalisation is the exact inverse: PCG ends after one iteration."""
    prob = dc.Problem(dim=2, n=(2, 2), N=8, p=5, c2=1.3)
    X, Y = dc.node_coordinates(prob)
    vp = dv.VarProblem(n=(2, 2), N=8, p=5, X=X, Y=Y, C2=np.full_like(X, 1.3))
    ops = dv.assemble(vp)
    rng = np.random.default_rng(9)
    U = rng.standard_normal((4, 81))
    V = rng.standard_normal((4, 81))
    ru, rv = dv.residuals(vp, ops, U, V)
    _, _, iu, iv = dv.solve_pcg(vp, ops, V, ru, rv, precond="fdm", rtol=1e-10)
    assert iu.max() == 1 and iv.max() == 1


def test_convergence_on_mapped_mesh():
    """c^2 = 1 on the sine-mapped unit square: the exact mode
    cos(sqrt2 pi t) sin(pi x) sin(pi y) (physical x, y) is still a solution;
    the L2 error falls at about the optimal rate."""
    errs = []
    for n in (2, 4):
        vp = _var_problem((n, n), 4, 3, c2="one", amp=0.05)
        ops = dv.assemble(vp)
        U0, V0 = inputs.standing_mode_2d(vp.X, vp.Y)
        ne = n * n
        U, V = U0.reshape(ne, -1), V0.reshape(ne, -1)
        h = 1.0 / (4 * n)
        T = 0.1
        steps = int(np.ceil(T / (0.1 * h)))
        f = lambda t, U, V: dv.time_derivative(vp, ops, U, V)
        U, V = ti.integrate(f, U, V, 0.0, T / steps, steps)
        # nodal error at the mapped nodes (exact there by interpolation)
        ue, _ = inputs.standing_mode_2d(vp.X, vp.Y, T)
        errs.append(np.sqrt(np.mean((U.reshape(ue.shape) - ue) ** 2)))
    rate = np.log2(errs[0] / errs[1])
    assert rate > 3.3, (errs, rate)


@pytest.mark.parametrize("p,rate,floor", [(3, 3.5, 3e-7), (5, 5.0, 2e-8)])
def test_energy_of_interpolants_converges_to_the_continuous_energy(p, rate, floor):
    """dg_var.energy of the nodal interpolants of u = sin(pi x) sin(pi y) and
    v = sin(2 pi x) y (1 - y) on the sine-mapped square with c^2 = 1 + 0.5
    sin 2pi x cos 2pi y approaches E = 1/2 int (v^2 + c^2 |grad u|^2), here
    computed by a 60 x 60 Gauss-Legendre rule in physical coordinates (the
    interpolated map covers the unit square exactly).  Measured relative gaps
    on 2 x 2, 4 x 4, 8 x 8 elements of 6 x 6 cells: p = 3 4.4e-5, 2.7e-6,
    1.6e-7; p = 5 8.5e-5, 3.8e-7, 7.5e-9."""
    g, w = np.polynomial.legendre.leggauss(60)
    x, wx = 0.5 * (g + 1.0), 0.5 * w
    Xq, Yq = np.meshgrid(x, x, indexing="ij")
    W = np.outer(wx, wx)
    c2 = lambda X, Y: 1.0 + 0.5 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
    u = lambda X, Y: np.sin(np.pi * X) * np.sin(np.pi * Y)
    grad2 = lambda X, Y: (np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)) ** 2 + \
        (np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)) ** 2
    v = lambda X, Y: np.sin(2 * np.pi * X) * Y * (1.0 - Y)
    Ec = 0.5 * np.sum(W * (v(Xq, Yq) ** 2 + c2(Xq, Yq) * grad2(Xq, Yq)))
    gaps = []
    for n in (2, 4, 8):
        X, Y = inputs.mapped_nodes((n, n), 6, 0.05)
        vp = dv.VarProblem(n=(n, n), N=6, p=p, X=X, Y=Y, C2=c2(X, Y))
        gaps.append(abs(dv.energy(dv.assemble(vp), u(X, Y), v(X, Y)) - Ec) / Ec)
    rates = np.log2(np.array(gaps[:-1]) / np.array(gaps[1:]))
    assert rates.min() > rate and gaps[-1] < floor, (gaps, rates)


def _face_rate_cartesian(vp, U, V, Hx, Hy):
    """Independent restatement, on a Cartesian mesh with variable c^2, of the
    energy rate of the upwind flux (Section 2.2.1 with the coefficient under
    the face integrals):
        dE/dt = - sum_interior int c^2 (tau [v]^2 + beta [d_n u]^2) dS
                - sum_Dirichlet int 2 c^2 tau v^2 dS,
    xi = c at the face point (or the problem's fixed xi), beta = xi / 2,
    tau = 1 / (2 xi); traces from the 1-D face data, c^2 traced from the
    face nodes, the face rule p + 1 Gauss points per GD cell."""
    from oracle import gd_basis as gb
    p, N, n1 = vp.p, vp.N, vp.n1
    r, w, cell = gb.quadrature_points(p, N, p + 1)
    B, _ = gb.basis_at_points(p, N, r, cell)
    _, _, dL, dR = gb.face_data(p, N)
    nx, ny = vp.n
    U = U.reshape(ny, nx, n1, n1)
    V = V.reshape(ny, nx, n1, n1)
    C2 = vp.C2.reshape(ny, nx, n1, n1)

    def pen(c2, jv, jd, length):
        xi = np.full_like(c2, vp.xi) if vp.xi > 0 else np.sqrt(c2)
        return length * np.sum(w * c2 * (jv ** 2 / (2 * xi) + 0.5 * xi * jd ** 2))

    rate = 0.0
    for ey in range(ny):
        for ex in range(nx):
            # x faces (j along the face, i = N on the + face, 0 on the - face)
            if ex + 1 < nx or vp.periodic[0]:
                f = (ex + 1) % nx
                jv = B @ (V[ey, ex][:, -1] - V[ey, f][:, 0])
                jd = B @ (U[ey, ex] @ dR - U[ey, f] @ dL) / Hx
                rate -= pen(B @ C2[ey, ex][:, -1], jv, jd, Hy)
            else:
                rate -= 2 * pen(B @ C2[ey, ex][:, -1], B @ V[ey, ex][:, -1], 0.0, Hy)
            if ex == 0 and not vp.periodic[0]:
                rate -= 2 * pen(B @ C2[ey, 0][:, 0], B @ V[ey, 0][:, 0], 0.0, Hy)
            # y faces (i along the face)
            if ey + 1 < ny or vp.periodic[1]:
                f = (ey + 1) % ny
                jv = B @ (V[ey, ex][-1, :] - V[f, ex][0, :])
                jd = B @ (dR @ U[ey, ex] - dL @ U[f, ex]) / Hy
                rate -= pen(B @ C2[ey, ex][-1, :], jv, jd, Hx)
            else:
                rate -= 2 * pen(B @ C2[ey, ex][-1, :], B @ V[ey, ex][-1, :], 0.0, Hx)
            if ey == 0 and not vp.periodic[1]:
                rate -= 2 * pen(B @ C2[0, ex][0, :], B @ V[0, ex][0, :], 0.0, Hx)
    return rate


@pytest.mark.parametrize("periodic", [(False, False), (True, False), (False, True)])
@pytest.mark.parametrize("xi", [0.0, 0.8])
def test_upwind_energy_rate_identity_variable_c2(periodic, xi):
    """dE/dt of the variable-coefficient oracle equals minus the flux
    penalties on the face jumps, with c^2 varying along every face and xi
    the local c (xi = 0) or fixed.  The energy identities above only bound
    the sign; this fixes where c^2 and xi enter the dissipative terms."""
    n, N, p = (3, 2), 5, 3
    lo, hi = (0.1, -0.3), (1.1, 0.7)     # unit periods: c^2 (period 1) is continuous across a periodic seam
    from oracle import dg_const as dcx
    prob = dcx.Problem(dim=2, n=n, N=N, p=p, lo=lo, hi=hi)
    X, Y = dcx.node_coordinates(prob)
    C2 = inputs.smooth_random_c2(X, Y, seed=11)
    vp = dv.VarProblem(n=n, N=N, p=p, X=X, Y=Y, C2=C2, flux="upwind", periodic=periodic, xi=xi)
    ops = dv.assemble(vp)
    rng = np.random.default_rng(3)
    ne = n[0] * n[1]
    U = rng.standard_normal((ne, (N + 1) ** 2))
    V = rng.standard_normal((ne, (N + 1) ** 2))
    Ut, Vt = dv.time_derivative(vp, ops, U, V)
    dEdt = np.einsum("ea,eab,eb->", V, ops.M, Vt) + np.einsum("ea,eab,eb->", U, ops.S, Ut)
    expect = _face_rate_cartesian(vp, U, V, (hi[0] - lo[0]) / n[0], (hi[1] - lo[1]) / n[1])
    assert expect < 0.0
    assert abs(dEdt - expect) < 1e-10 * abs(expect), (dEdt, expect)
