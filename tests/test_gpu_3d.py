"""GPU parity of the 3-D constant-coefficient path (dim = 3; the
tensor-product construction of Sections 2.1.2 and 3 for d = 3) with the
FP64 oracle through the C ABI: gdg_rhs, gdg_mass_solve, gdg_step after every
step and through the captured graph, gdg_energy, edge cases (a single
self-periodic element, mixed boundary conditions, every flux, p = 3, 5, 7),
and a 32 x 32 x 32 mesh checked on sampled elements against 3 x 3 x 3
oracle patches."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dg_const as dc, gd_basis as gb, timeint as ti
from paper_2105_01722_gb300 import gdg, inputs

TOL = 1e-12
FLUX = {"upwind": gdg.FLUX_UPWIND, "central": gdg.FLUX_CENTRAL, "alternating": gdg.FLUX_ALTERNATING}

CASES = [
    dict(n=(2, 2, 2), N=4, p=3, periodic=(False, False, False), flux="upwind"),
    dict(n=(3, 2, 2), N=5, p=5, periodic=(True, False, False), flux="central", c2=2.2),
    dict(n=(2, 3, 1), N=8, p=5, periodic=(True, False, True), flux="alternating", c2=1.7),
    dict(n=(1, 1, 1), N=3, p=3, periodic=(True, True, True), flux="upwind"),
    dict(n=(2, 1, 3), N=9, p=7, periodic=(False, True, False), flux="upwind", xi=0.6,
         lo=(0.0, -1.0, 0.5), hi=(1.5, 0.0, 1.4)),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gdg.lib()


def _ids(c):
    return "n%s-N%d-p%d-%s-per%s" % ("x".join(map(str, c["n"])), c["N"], c["p"], c["flux"],
                                      "".join("1" if q else "0" for q in c["periodic"]))


def _oracle(c):
    return dc.Problem(dim=3, n=c["n"], N=c["N"], p=c["p"], lo=c.get("lo", (0.0, 0.0, 0.0)),
                      hi=c.get("hi", (1.0, 1.0, 1.0)), periodic=c["periodic"], flux=c["flux"],
                      xi=c.get("xi", 0.0), c2=c.get("c2", 1.0))


def _gpu(c):
    bc = tuple(gdg.BC_PERIODIC if q else gdg.BC_DIRICHLET for q in c["periodic"])
    return gdg.make_problem(3, c["n"], c["N"], c["p"], lo=c.get("lo", (0.0, 0.0, 0.0)),
                            hi=c.get("hi", (1.0, 1.0, 1.0)), bc=bc, flux=FLUX[c["flux"]],
                            xi=c.get("xi", 0.0), c2=c.get("c2", 1.0))


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")


def _rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _state(c, seed):
    ne = int(np.prod(c["n"]))
    na = (c["N"] + 1) ** 3
    return inputs.random_state((ne, na), seed), inputs.random_state((ne, na), seed + 1)


def _route_floor(prob, U, V):
    """Rounding floor of the oracle itself on this input: the gap between its
    dense (row-replaced LU) and diagonalised solves of the u_t system;
    parity is required to max(1e-12, 3 x that gap)."""
    ops = dc.operators(prob)
    ru, rv = dc.residuals(prob, U, V, ops)
    Ut, _ = dc.solve(ops, V, ru, rv)
    Ps = [gb.simultaneous_diagonalisation(ops.M1[k], ops.S1[k]) for k in range(3)]
    Psi = np.kron(Ps[2][0], np.kron(Ps[1][0], Ps[0][0]))
    lam = (Ps[2][1][:, None, None] + Ps[1][1][None, :, None] + Ps[0][1][None, None, :]).ravel()
    inv = np.zeros_like(lam)
    inv[1:] = 1.0 / lam[1:]
    y = (ru @ Psi) * inv @ Psi.T
    return max(TOL, 3.0 * _rel(V + y, Ut))


@pytest.mark.parametrize("c", CASES, ids=_ids)
def test_rhs_parity_3d(c):
    prob = _oracle(c)
    U, V = _state(c, 60)
    Ut, Vt = dc.time_derivative(prob, U, V)
    ctx = gdg.Context(_gpu(c))
    assert ctx.n == U.size
    u, v = _dev(U), _dev(V)
    du, dv = torch.empty_like(u), torch.empty_like(v)
    ctx.rhs(u, v, du, dv)
    tol = _route_floor(prob, U, V)
    assert _rel(du.cpu().numpy(), Ut) < tol
    assert _rel(dv.cpu().numpy(), Vt) < tol
    ctx.close()


@pytest.mark.parametrize("c", CASES[:3], ids=_ids)
def test_mass_solve_parity_3d(c):
    prob = _oracle(c)
    ops = dc.operators(prob)
    U, V = _state(c, 70)
    ru, rv = dc.residuals(prob, U, V, ops)
    Ut, Vt = dc.solve(ops, np.zeros_like(V), ru, rv)
    ctx = gdg.Context(_gpu(c))
    x = torch.empty(U.size, dtype=torch.float64, device="cuda")
    ctx.mass_solve(gdg.OP_M, _dev(rv), x)
    assert _rel(x.cpu().numpy(), Vt) < 1e-12
    ctx.mass_solve(gdg.OP_S, _dev(ru), x)
    assert _rel(x.cpu().numpy(), Ut) < _route_floor(prob, U, V)
    ctx.close()


@pytest.mark.parametrize("c", CASES, ids=_ids)
def test_step_parity_every_step_3d(c):
    prob = _oracle(c)
    ops = dc.operators(prob)
    U, V = _state(c, 80)
    ctx = gdg.Context(_gpu(c))
    u, v = _dev(U), _dev(V)
    h = min(prob.H(k) for k in range(3)) / prob.N
    dt = 0.08 * h / np.sqrt(c.get("c2", 1.0))
    f = lambda t, U, V: dc.time_derivative(prob, U, V, ops)
    tol = _route_floor(prob, U, V)
    for s in range(3):
        ctx.step(u, v, s * dt, dt, 1)
        U, V = ti.rk4_step(f, U, V, s * dt, dt)
        a = np.concatenate([u.cpu().numpy(), v.cpu().numpy()])
        assert _rel(a, np.concatenate([U.ravel(), V.ravel()])) < tol, s
    ctx.close()


def test_graph_path_and_energy_3d():
    """nsteps >= 16 runs through the captured graph: same as the oracle after
    19 steps; gdg_energy matches the oracle's energy, and with the central
    flux the fully discrete energy does not grow (RK4 only damps)."""
    c = CASES[1]
    prob = _oracle(c)
    ops = dc.operators(prob)
    U, V = _state(c, 90)
    ctx = gdg.Context(_gpu(c))
    u, v = _dev(U), _dev(V)
    E0 = ctx.energy(u, v)
    assert abs(E0 - dc.energy(prob, U, V, ops)) < 1e-12 * E0
    h = min(prob.H(k) for k in range(3)) / prob.N
    dt = 0.05 * h / np.sqrt(c["c2"])
    steps = 19
    floor = _route_floor(prob, U, V)
    ctx.step(u, v, 0.0, dt, steps)
    f = lambda t, U, V: dc.time_derivative(prob, U, V, ops)
    U, V = ti.integrate(f, U, V, 0.0, dt, steps)
    a = np.concatenate([u.cpu().numpy(), v.cpu().numpy()])
    # one step of either side is within the rounding floor of the exact step
    # and the step map is non-expansive here, so the gap grows at most
    # linearly: steps x floor
    gap = _rel(a, np.concatenate([U.ravel(), V.ravel()]))
    assert gap < steps * floor
    E1 = ctx.energy(u, v)
    # a quadratic form of two states a relative gap g apart differs by at
    # most 2 g relative, plus the rounding of the energy sum itself
    assert abs(E1 - dc.energy(prob, U, V, ops)) < (2 * steps * floor + TOL) * E1
    assert E1 <= E0 * (1 + 1e-12) and E1 > 0.99 * E0
    ctx.close()


def _patch_rhs(U, V, n, N, p, ez, ey, ex):
    """Oracle time derivative of element (ez, ey, ex) of the unit-cube mesh
    from the 3 x 3 x 3 patch around it (its value depends on its own data
    and its neighbours' traces; patch sides on the domain boundary keep the
    Dirichlet condition)."""
    lo_i = [max(i - 1, 0) for i in (ex, ey, ez)]
    hi_i = [min(i + 1, n - 1) for i in (ex, ey, ez)]
    m = tuple(h - l + 1 for l, h in zip(lo_i, hi_i))
    H = 1.0 / n
    prob = dc.Problem(dim=3, n=m, N=N, p=p, lo=tuple(l * H for l in lo_i), hi=tuple((h + 1) * H for h in hi_i),
                      periodic=(False, False, False), flux="upwind")
    sl = (slice(lo_i[2], hi_i[2] + 1), slice(lo_i[1], hi_i[1] + 1), slice(lo_i[0], hi_i[0] + 1))
    ne = m[0] * m[1] * m[2]
    Us, Vs = U[sl].reshape(ne, -1), V[sl].reshape(ne, -1)
    Ut, Vt = dc.time_derivative(prob, Us, Vs)
    c = ((ez - lo_i[2]) * m[1] + (ey - lo_i[1])) * m[0] + (ex - lo_i[0])
    return Ut[c], Vt[c], _route_floor(prob, Us, Vs)


def test_full_size_32cubed_p5_sampled():
    """32^3 elements of 8^3 cells, p = 5 (23.9 M DOF per field), upwind,
    Dirichlet: gdg_rhs on sampled elements against 3 x 3 x 3 oracle patches;
    then RK4 steps of the standing wave with non-increasing energy."""
    n, N, p = 32, 8, 5
    c = dict(n=(n, n, n), N=N, p=p, periodic=(False, False, False), flux="upwind")
    prob = _oracle(c)
    X, Y, Z = dc.node_coordinates(prob)
    U = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z) + 0.01 * inputs.random_state(X.shape, 5)
    V = 0.01 * inputs.random_state(X.shape, 6)
    ctx = gdg.Context(_gpu(c))
    u, v = _dev(U), _dev(V)
    du, dv = torch.empty_like(u), torch.empty_like(v)
    ctx.rhs(u, v, du, dv)
    du = du.cpu().numpy().reshape(U.shape[:3] + (-1,))
    dvv = dv.cpu().numpy().reshape(U.shape[:3] + (-1,))
    for ez, ey, ex in [(0, 0, 0), (31, 31, 31), (15, 16, 17), (0, 31, 9), (20, 0, 31)]:
        Ut, Vt, floor = _patch_rhs(U, V, n, N, p, ez, ey, ex)
        a = np.concatenate([du[ez, ey, ex], dvv[ez, ey, ex]])
        assert _rel(a, np.concatenate([Ut, Vt])) < floor, (ez, ey, ex)
    U0 = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    u, v = _dev(U0), torch.zeros(U0.size, dtype=torch.float64, device="cuda")
    E = [ctx.energy(u, v)]
    dt = 0.1 / (n * N)
    for _ in range(3):
        ctx.step(u, v, 0.0, dt, 8)
        E.append(ctx.energy(u, v))
    assert all(b <= a * (1 + 1e-13) for a, b in zip(E, E[1:])) and E[-1] > 0.99 * E[0]
    ctx.close()
