"""GPU parity of the point source, the forcing f of u_tt = div(c^2 grad u) + f
with f = a sin(w t) delta(x - x_s), on a mapped mesh with variable c^2.

The oracle's RK4 gets the forcing array of its residuals: the load
int phi_a f = phi_a(x_s) a sin(w t) on the element holding x_s (Section 7.1's
right-hand side; the delta function makes the Jacobian drop out), with
phi_a(x_s) = phi_j(s) phi_i(r) from the oracle's own GD basis and the stage
times t, t + dt/2, t + dt/2, t + dt of the classic RK4 step.  The library
advances the state with gdg_step from t0 over 9 steps (a captured graph of 8
steps and one more), once with element inverses and once with converged
element PCG; both are compared with the oracle's direct element solves.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dg_var as dv, gd_basis as gb, timeint as ti
from paper_2105_01722_gb300 import gdg, inputs

EPS = np.finfo(np.float64).eps


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gdg.lib()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")


def _rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _load(vp, e, r, s):
    """phi_a(x_s) on element e, a = j n1 + i (x fastest)."""
    pr, _ = gb.eval_basis(vp.p, vp.N, r)
    ps, _ = gb.eval_basis(vp.p, vp.N, s)
    return np.outer(ps, pr).ravel()


@pytest.mark.parametrize("solver", ["inverse", "pcg"])
@pytest.mark.parametrize("flux,periodic", [("upwind", (False, False)), ("central", (True, False)),
                                           ("alternating", (False, True))])
def test_point_source_steps_match_oracle(solver, flux, periodic):
    n, N, p = (4, 3), 8, 5
    ne = n[0] * n[1]
    X, Y = inputs.mapped_nodes(n, N, 0.05)
    C2 = inputs.c2_sine(X, Y)
    vp = dv.VarProblem(n=n, N=N, p=p, X=X, Y=Y, C2=C2, periodic=periodic, flux=flux)
    ops = dv.assemble(vp)
    e, r, s, amp, omega = 5, 0.37, 0.61, 3.0, 25.0
    w = _load(vp, e, r, s)

    def forcing(t):
        out = np.zeros((ne, (N + 1) ** 2))
        out[e] = amp * np.sin(omega * t) * w
        return out

    K = 6   # PCG form: exactly K iterations per element solve on both sides

    def f(t, U, V):
        ru, rv = dv.residuals(vp, ops, U, V, forcing=forcing(t))
        if solver == "inverse":
            return dv.solve_direct(ops, V, ru, rv)
        return dv.solve_pcg(vp, ops, V, ru, rv, precond="fdm", rtol=0.0, maxit=K)[:2]

    bc = tuple(gdg.BC_PERIODIC if q else gdg.BC_DIRICHLET for q in periodic)
    fl = {"upwind": gdg.FLUX_UPWIND, "central": gdg.FLUX_CENTRAL, "alternating": gdg.FLUX_ALTERNATING}[flux]
    pb = gdg.make_problem(2, n, N, p, bc=bc, flux=fl, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                          solver=gdg.SOLVE_INVERSE if solver == "inverse" else gdg.SOLVE_PCG,
                          pcg_rtol=0.0, pcg_maxit=K)
    ctx = gdg.Context(pb)
    ctx.set_point_source(e, r, s, amp, omega)
    U = 0.1 * inputs.random_state((ne, (N + 1) ** 2), 71)
    V = 0.1 * inputs.random_state((ne, (N + 1) ** 2), 72)
    t0, dt, steps = 0.3, 0.05 / (max(n) * N), 9
    u, v = _dev(U), _dev(V)
    ctx.step(u, v, t0, dt, steps)
    Uo, Vo = U, V
    for k in range(steps):
        Uo, Vo = ti.rk4_step(f, Uo, Vo, t0 + k * dt, dt)
    # element inverses: an explicit inverse applied to a vector has relative
    # error up to about kappa eps per solve, against the oracle's direct solve
    # (50 kappa eps covers the fold's extra products); fixed-iteration PCG on
    # both sides differs by up to sqrt(n) kappa eps, n = (N+1)^2 terms per
    # element product (rounding order only).  Over `steps` steps the per-step
    # gaps add up at most linearly.
    kappa = max(max(np.linalg.cond(dv.spd_u_matrix(ops, q)), np.linalg.cond(ops.M[q])) for q in range(ne))
    per_step = max(1e-12, (50.0 if solver == "inverse" else np.sqrt((N + 1) ** 2)) * kappa * EPS)
    tol = steps * per_step
    got = np.concatenate([u.cpu().numpy(), v.cpu().numpy()])
    ref = np.concatenate([Uo.ravel(), Vo.ravel()])
    assert _rel(got, ref) < tol
    # the source acts: without it the oracle's state differs by far more than tol
    Un, Vn = U, V
    def g(t, U_, V_):
        ru, rv = dv.residuals(vp, ops, U_, V_)
        if solver == "inverse":
            return dv.solve_direct(ops, V_, ru, rv)
        return dv.solve_pcg(vp, ops, V_, ru, rv, precond="fdm", rtol=0.0, maxit=K)[:2]

    for k in range(steps):
        Un, Vn = ti.rk4_step(g, Un, Vn, t0 + k * dt, dt)
    assert _rel(np.concatenate([Un.ravel(), Vn.ravel()]), ref) > 1e3 * tol
    # amplitude 0 removes it: the context then steps without forcing
    ctx.set_point_source(e, r, s, 0.0, omega)
    u, v = _dev(U), _dev(V)
    ctx.step(u, v, t0, dt, steps)
    got0 = np.concatenate([u.cpu().numpy(), v.cpu().numpy()])
    assert _rel(got0, np.concatenate([Un.ravel(), Vn.ravel()])) < tol
    ctx.close()


def test_rhs_evaluates_the_source_at_its_time():
    """gdg_rhs(t) adds the load a sin(w t) phi(x_s) at its own t: the
    derivative at two times differs by exactly the source term, which the
    oracle forms from its residuals and dense solves."""
    n, N, p = (3, 3), 8, 5
    ne = n[0] * n[1]
    X, Y = inputs.mapped_nodes(n, N, 0.05)
    C2 = inputs.c2_sine(X, Y)
    vp = dv.VarProblem(n=n, N=N, p=p, X=X, Y=Y, C2=C2)
    ops = dv.assemble(vp)
    e, r, s_, amp, omega = 4, 0.3, 0.55, 2.0, 7.0
    w = _load(vp, e, r, s_)
    U = 0.1 * inputs.random_state((ne, (N + 1) ** 2), 81)
    V = 0.1 * inputs.random_state((ne, (N + 1) ** 2), 82)
    pb = gdg.make_problem(2, n, N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                          solver=gdg.SOLVE_INVERSE)
    ctx = gdg.Context(pb)
    ctx.set_point_source(e, r, s_, amp, omega)
    kappa = max(max(np.linalg.cond(dv.spd_u_matrix(ops, q)), np.linalg.cond(ops.M[q])) for q in range(ne))
    tol = max(1e-12, 50.0 * kappa * EPS)
    for t in (0.0, 0.37, 1.9):
        F = np.zeros((ne, (N + 1) ** 2))
        F[e] = amp * np.sin(omega * t) * w
        ru, rv = dv.residuals(vp, ops, U, V, forcing=F)
        Ut, Vt = dv.solve_direct(ops, V, ru, rv)
        u, v = _dev(U), _dev(V)
        du, dv_ = torch.empty_like(u), torch.empty_like(v)
        ctx.rhs(u, v, du, dv_, t=t)
        got = np.concatenate([du.cpu().numpy(), dv_.cpu().numpy()])
        assert _rel(got, np.concatenate([Ut.ravel(), Vt.ravel()])) < tol, t
    ctx.close()


def test_point_source_arguments():
    X, Y = inputs.mapped_nodes((2, 2), 8, 0.05)
    C2 = inputs.c2_sine(X, Y)
    ctx = gdg.Context(gdg.make_problem(2, (2, 2), 8, 5, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2))
    for args in ((4, 0.5, 0.5, 1.0, 1.0), (-1, 0.5, 0.5, 1.0, 1.0), (0, 1.5, 0.5, 1.0, 1.0),
                 (0, 0.5, -0.1, 1.0, 1.0), (0, 0.5, 0.5, float("nan"), 1.0)):
        with pytest.raises(gdg.GdgError) as err:
            ctx.set_point_source(*args)
        assert err.value.status == gdg.EINVAL
    ctx.close()
    const = gdg.Context(gdg.make_problem(2, (2, 2), 8, 5))
    with pytest.raises(gdg.GdgError):
        const.set_point_source(0, 0.5, 0.5, 1.0, 1.0)
    const.close()
