"""Pins of the oracle's constant-coefficient energy-DG semi-discretisation
(Sections 2.2, 3; Eqs. DG1, DG2, DG1_extra) by brute force on tiny meshes,
energy identities derived from the variational statement, and convergence
on exact solutions (Section 6)."""
import numpy as np
import pytest

from oracle import dg_const as dc, gd_basis as gb, timeint as ti

TINY = [
    dict(dim=1, n=(3,), N=4, p=3, periodic=(False,)),
    dict(dim=1, n=(2,), N=5, p=5, periodic=(True,)),
    dict(dim=1, n=(4,), N=3, p=1, periodic=(False,)),
    dict(dim=2, n=(2, 2), N=3, p=3, periodic=(False, False)),
    dict(dim=2, n=(2, 1), N=4, p=3, periodic=(True, False), lo=(0.0, 0.0), hi=(1.0, 0.7)),
    dict(dim=2, n=(1, 2), N=5, p=5, periodic=(False, True)),
]


def _prob(case, flux, c2=1.7, xi=0.0):
    kw = dict(case)
    return dc.Problem(flux=flux, c2=c2, xi=xi, **kw)


@pytest.mark.parametrize("case", TINY)
def test_central_flux_conserves_energy(case):
    """beta = tau = 0: the semi-discrete energy is conserved exactly, i.e.
    E L + L^T E = 0 for the dense global operator L (Section 2.2.1)."""
    prob = _prob(case, "central")
    L = dc.dense_operator(prob)
    E = dc.energy_matrix(prob)
    A = E @ L + L.T @ E
    assert np.abs(A).max() < 1e-11 * np.abs(E @ L).max()
    ev = np.linalg.eigvals(L)
    assert np.abs(ev.real).max() < 1e-8 * np.abs(ev).max()


@pytest.mark.parametrize("case", TINY)
def test_alternating_flux_conserves_energy(case):
    """Alternating flux (alpha = 1, sides by a fixed orientation, Dirichlet
    closure v* = 0, q* = d_in): conservative like the central flux, E L +
    L^T E = 0 and an imaginary spectrum, yet a different operator."""
    prob = _prob(case, "alternating")
    L = dc.dense_operator(prob)
    E = dc.energy_matrix(prob)
    A = E @ L + L.T @ E
    assert np.abs(A).max() < 1e-11 * np.abs(E @ L).max()
    ev = np.linalg.eigvals(L)
    assert np.abs(ev.real).max() < 1e-8 * np.abs(ev).max()
    Lc = dc.dense_operator(_prob(case, "central"))
    assert np.abs(L - Lc).max() > 1e-3 * np.abs(Lc).max()


@pytest.mark.parametrize("case", TINY)
def test_upwind_flux_dissipates(case):
    prob = _prob(case, "upwind")
    L = dc.dense_operator(prob)
    E = dc.energy_matrix(prob)
    A = -(E @ L + L.T @ E)
    lam = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert lam.min() > -1e-10 * np.abs(lam).max()
    assert lam.max() > 1e-3                      # it does dissipate
    ev = np.linalg.eigvals(L)
    assert ev.real.max() < 1e-8 * np.abs(ev).max()


def _face_jumps(prob, U, V):
    """Independent restatement of the energy rate for the upwind flux:
    dE/dt = -sum_interior c^2 int (tau [v]^2 + beta [d_n u]^2)
            -sum_Dirichlet 2 c^2 tau int v^2
    computed from nodal traces with the 1-D face data."""
    beta, tau = prob.beta_tau()
    c2 = prob.c2
    p, N, n1 = prob.p, prob.N, prob.n1
    _, _, dL, dR = gb.face_data(p, N)
    Mh, _ = gb.mass_stiffness(p, N)
    rate = 0.0
    if prob.dim == 1:
        H = prob.H(0)
        U = U.reshape(-1, n1)
        V = V.reshape(-1, n1)
        ne = U.shape[0]
        for e in range(ne):
            # the + face of e
            if e + 1 < ne or prob.periodic[0]:
                f = (e + 1) % ne
                jv = V[e, -1] - V[f, 0]
                jd = U[e] @ dR / H - U[f] @ dL / H   # n1.grad u1 + n2.grad u2
                rate -= c2 * (tau * jv ** 2 + beta * jd ** 2)
            else:
                rate -= 2 * c2 * tau * V[e, -1] ** 2
            if e == 0 and not prob.periodic[0]:
                rate -= 2 * c2 * tau * V[0, 0] ** 2
        return rate
    nx, ny = prob.n
    Hx, Hy = prob.H(0), prob.H(1)
    U = U.reshape(ny, nx, n1, n1)
    V = V.reshape(ny, nx, n1, n1)
    Mx, My = Hx * Mh, Hy * Mh
    for ey in range(ny):
        for ex in range(nx):
            # + x face
            if ex + 1 < nx or prob.periodic[0]:
                fx = (ex + 1) % nx
                jv = V[ey, ex, :, -1] - V[ey, fx, :, 0]
                jd = U[ey, ex] @ dR / Hx - U[ey, fx] @ dL / Hx
                rate -= c2 * (tau * jv @ My @ jv + beta * jd @ My @ jd)
            else:
                v = V[ey, ex, :, -1]
                rate -= 2 * c2 * tau * v @ My @ v
            if ex == 0 and not prob.periodic[0]:
                v = V[ey, ex, :, 0]
                rate -= 2 * c2 * tau * v @ My @ v
            # + y face
            if ey + 1 < ny or prob.periodic[1]:
                fy = (ey + 1) % ny
                jv = V[ey, ex, -1, :] - V[fy, ex, 0, :]
                jd = dR @ U[ey, ex] / Hy - dL @ U[fy, ex] / Hy
                rate -= c2 * (tau * jv @ Mx @ jv + beta * jd @ Mx @ jd)
            else:
                v = V[ey, ex, -1, :]
                rate -= 2 * c2 * tau * v @ Mx @ v
            if ey == 0 and not prob.periodic[1]:
                v = V[ey, ex, 0, :]
                rate -= 2 * c2 * tau * v @ Mx @ v
    return rate


@pytest.mark.parametrize("case", TINY)
@pytest.mark.parametrize("xi", [0.0, 0.6])
def test_upwind_energy_rate_identity(case, xi):
    """dE/dt equals minus the flux penalties on the face jumps exactly.
    A wrong sign or factor in the beta / tau terms (the dissipative B and C
    terms of Eqs. DG_matrix1/2) fails this identity."""
    prob = _prob(case, "upwind", xi=xi)
    rng = np.random.default_rng(7)
    ndof = int(np.prod(prob.n)) * prob.n1 ** prob.dim
    U = rng.standard_normal(ndof)
    V = rng.standard_normal(ndof)
    ops = dc.operators(prob)
    Ut, Vt = dc.time_derivative(prob, U, V, ops)
    ne = int(np.prod(prob.n))
    U2, V2, Ut2, Vt2 = (a.reshape(ne, -1) for a in (U, V, Ut, Vt))
    dEdt = (np.einsum("ea,ab,eb->", V2, ops.M, Vt2)
            + prob.c2 * np.einsum("ea,ab,eb->", U2, ops.S, Ut2))
    expect = _face_jumps(prob, U, V)
    assert abs(dEdt - expect) < 1e-10 * (abs(expect) + np.abs(U).max() ** 2)
    assert expect < 0.0


@pytest.mark.parametrize("case", TINY)
def test_mean_constraint(case):
    """Eq. DG1_extra: w^T (dU/dt - V) = 0 element by element (w = M 1)."""
    prob = _prob(case, "upwind")
    rng = np.random.default_rng(3)
    ne = int(np.prod(prob.n))
    na = prob.n1 ** prob.dim
    U = rng.standard_normal((ne, na))
    V = rng.standard_normal((ne, na))
    ops = dc.operators(prob)
    Ut, Vt = dc.time_derivative(prob, U, V, ops)
    w = ops.M @ np.ones(na)
    assert np.abs((Ut - V) @ w).max() < 1e-12 * np.abs(Ut).max()
    # and the S equation holds: S (dU/dt - V) = r_u
    r_u, r_v = dc.residuals(prob, U, V, ops)
    assert np.abs((Ut - V) @ ops.S.T - r_u).max() < 1e-10 * np.abs(r_u).max()
    assert np.abs(Vt @ ops.M.T - r_v).max() < 1e-11 * np.abs(r_v).max()
    assert np.abs(r_u.sum(axis=1)).max() < 1e-11 * np.abs(r_u).max()


@pytest.mark.parametrize("case", TINY)
def test_diagonalised_solve_matches_dense(case):
    """Section 3.2: M^-1 = Psi Psi^T and the constrained S solve is
    Psi Lambda^+ Psi^T (zero on the constant mode), with Psi the Kronecker
    product of the 1-D modified bases."""
    prob = _prob(case, "upwind")
    rng = np.random.default_rng(11)
    ne = int(np.prod(prob.n))
    na = prob.n1 ** prob.dim
    U = rng.standard_normal((ne, na))
    V = rng.standard_normal((ne, na))
    ops = dc.operators(prob)
    r_u, r_v = dc.residuals(prob, U, V, ops)
    Ut, Vt = dc.solve(ops, V, r_u, r_v)
    Psis, lams = [], []
    for k in range(prob.dim):
        P, lam = gb.simultaneous_diagonalisation(ops.M1[k], ops.S1[k])
        Psis.append(P)
        lams.append(lam)
    if prob.dim == 1:
        Psi, lam = Psis[0], lams[0]
    else:
        Psi = np.kron(Psis[1], Psis[0])
        lam = (lams[1][:, None] + lams[0][None, :]).ravel()
    inv = np.zeros_like(lam)
    inv[1:] = 1.0 / lam[1:]
    y = (r_u @ Psi) * inv @ Psi.T
    z = (r_v @ Psi) @ Psi.T
    assert np.abs(V + y - Ut).max() < 1e-11 * np.abs(Ut).max()
    assert np.abs(z - Vt).max() < 1e-11 * np.abs(Vt).max()


def _standing_wave_1d(t, x):
    w = 2 * np.pi
    return (np.cos(w * t) * np.sin(w * x), [w * np.cos(w * t) * np.cos(w * x)],
            -w * np.sin(w * t) * np.sin(w * x))


def _run_1d(n, p, N, flux, T, cfl):
    prob = dc.Problem(dim=1, n=(n,), N=N, p=p, flux=flux)
    ops = dc.operators(prob)
    (X,) = dc.node_coordinates(prob)
    U, V = np.sin(2 * np.pi * X), np.zeros_like(X)
    h = prob.H(0) / N
    steps = int(np.ceil(T / (cfl * h)))
    dt = T / steps
    f = lambda t, U, V: dc.time_derivative(prob, U, V, ops)
    U, V = ti.integrate(f, U, V, 0.0, dt, steps)
    return ti.errors(prob, U, V, _standing_wave_1d, T), h


@pytest.mark.parametrize("flux", ["central", "upwind", "alternating"])
@pytest.mark.parametrize("p", [3, 5])
def test_convergence_1d_dirichlet(flux, p):
    """Exact standing wave cos(2 pi t) sin(2 pi x), Dirichlet: the L2 error
    falls at about the optimal rate p+1 (Section 6) as elements are added."""
    errs = [_run_1d(n, p, 8, flux, 0.25, 0.05)[0][0] for n in (2, 4, 8)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > p + 0.5, (errs, rates)


def _travelling_wave_1d(t, x):
    w = 2 * np.pi
    return (np.sin(w * (x - t)), [w * np.cos(w * (x - t))], -w * np.cos(w * (x - t)))


@pytest.mark.parametrize("p", [3, 5])
def test_convergence_1d_periodic_alternating(p):
    """Section 6's periodic test for the alternating flux (Tables 1, 2 report
    L2 rates of about p+1 for p >= 3): travelling wave sin 2pi(x - t) on a
    periodic mesh, elements added at N = 8."""
    errs = []
    for n in (2, 4, 8):
        prob = dc.Problem(dim=1, n=(n,), N=8, p=p, flux="alternating", periodic=(True,))
        ops = dc.operators(prob)
        (X,) = dc.node_coordinates(prob)
        U, V = np.sin(2 * np.pi * X), -2 * np.pi * np.cos(2 * np.pi * X)
        h = prob.H(0) / 8
        T = 0.25
        steps = int(np.ceil(T / (0.05 * h)))
        f = lambda t, U, V: dc.time_derivative(prob, U, V, ops)
        U, V = ti.integrate(f, U, V, 0.0, T / steps, steps)
        errs.append(ti.errors(prob, U, V, _travelling_wave_1d, T)[0])
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > p + 0.3, (errs, rates)


def test_config0_energy_and_error():
    """16 elements x 8 cells, p = 3, to T = 1 at dt = h/2: E_h(0) is close
    to pi^2 (the exact energy of sin(2 pi x)); central RK4 energy drift is
    tiny, upwind energy is non-increasing step by step."""
    for flux in ("central", "upwind"):
        prob = dc.Problem(dim=1, n=(16,), N=8, p=3, flux=flux)
        ops = dc.operators(prob)
        (X,) = dc.node_coordinates(prob)
        U, V = np.sin(2 * np.pi * X), np.zeros_like(X)
        E0 = dc.energy(prob, U, V, ops)
        assert abs(E0 - np.pi ** 2) < 1e-6
        dt = 1.0 / 256
        Es = []
        f = lambda t, U, V: dc.time_derivative(prob, U, V, ops)
        U, V = ti.integrate(f, U, V, 0.0, dt, 256,
                            callback=lambda s, t, U, V: Es.append(dc.energy(prob, U, V, ops)))
        l2, en = ti.errors(prob, U, V, _standing_wave_1d, 1.0)
        assert l2 < 1e-6 and en < 1e-4
        if flux == "central":
            assert abs(Es[-1] - E0) < 1e-7 * E0
        else:
            assert np.all(np.diff([E0] + Es) <= 1e-14 * E0)


def test_2d_initial_energy():
    """sin(pi x) sin(pi y): E(0) = pi^2/4 (config of the 2-D constant case)."""
    prob = dc.Problem(dim=2, n=(4, 4), N=8, p=5)
    X, Y = dc.node_coordinates(prob)
    U = np.sin(np.pi * X) * np.sin(np.pi * Y)
    E0 = dc.energy(prob, U.reshape(16, -1), np.zeros((16, 81)))
    assert abs(E0 - np.pi ** 2 / 4) < 1e-7


def _mode_2d(t, X, Y):
    w = np.sqrt(2) * np.pi
    s = np.sin(np.pi * X) * np.sin(np.pi * Y)
    return (np.cos(w * t) * s,
            [np.cos(w * t) * np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y),
             np.cos(w * t) * np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)],
            -w * np.sin(w * t) * s)


def test_convergence_2d_dirichlet():
    """2-D mode cos(sqrt2 pi t) sin(pi x) sin(pi y): L2 rate about p+1."""
    errs = []
    for n in (1, 2, 4):
        prob = dc.Problem(dim=2, n=(n, n), N=4, p=3)
        ops = dc.operators(prob)
        X, Y = dc.node_coordinates(prob)
        ne = n * n
        U = (np.sin(np.pi * X) * np.sin(np.pi * Y)).reshape(ne, -1)
        V = np.zeros_like(U)
        h = 1.0 / (n * 4)
        steps = int(np.ceil(0.2 / (0.05 * h)))
        f = lambda t, U, V: dc.time_derivative(prob, U, V, ops)
        U, V = ti.integrate(f, U, V, 0.0, 0.2 / steps, steps)
        errs.append(ti.errors(prob, U, V, _mode_2d, 0.2)[0])
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 3.5, (errs, rates)


def test_spectral_radius_grows_linearly_in_p():
    """Section 5: the spectral radius of the semi-discretisation grows about
    linearly with p (not quadratically), n = 1, N + 1 = 31, periodic."""
    rho = []
    ps = [1, 3, 5, 7, 9]
    for p in ps:
        prob = dc.Problem(dim=1, n=(1,), N=30, p=p, flux="upwind", periodic=(True,))
        rho.append(np.abs(np.linalg.eigvals(dc.dense_operator(prob))).max())
    rho = np.array(rho)
    growth = rho[1:] / rho[:-1]
    assert np.all(growth > 1.0)
    ratio = rho / np.array(ps)
    # linear in p: rho/p stays within a modest band; quadratic would give ~9x
    assert ratio[1:].max() / ratio[1:].min() < 2.0
