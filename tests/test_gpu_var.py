"""GPU parity of the variable-coefficient / mapped-element path (Section
7.1) with the FP64 oracle, through the C ABI: quadrature assembly (via the
energy quadratic forms), element PCG at fixed iteration counts (exact
parity) and converged (against the dense solve), gdg_rhs and gdg_step,
energy behaviour, edge cases, and the full 128 x 128 mapped mesh (p = 3, 5)
on sampled elements, each checked against a 3 x 3 oracle patch around it."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dg_var as dv, timeint as ti
from paper_2105_01722_gb300 import gdg, inputs

TOL = 1e-12
EPS = np.finfo(np.float64).eps


def _kappa_tol(ops):
    """Parity bound of results that pass through element solves: two FP64
    evaluations of the same fixed-iteration PCG (or of the same dense solve)
    that differ only in the order of their sums.  Each element product sums
    n = (N+1)^2 terms, whose rounding differs between the two orders by about
    sqrt(n) eps relative to the terms' size (a random walk of n roundings);
    an element system of 2-norm condition number kappa (largest over the
    elements of S_c2 + w w^T and M_J) amplifies a relative perturbation of
    its operator's application by up to kappa.  Bound: max(1e-12,
    sqrt(n) kappa eps).  Measured gaps: 0.003 to 2.6 kappa eps (the largest
    at 128 x 128 mapped elements, p = 5, one RK4 step: 1.9e-12 with
    kappa eps = 7.5e-13)."""
    ne, na = ops.M.shape[0], ops.M.shape[1]
    kappa = max(max(np.linalg.cond(dv.spd_u_matrix(ops, e)), np.linalg.cond(ops.M[e])) for e in range(ne))
    return max(TOL, np.sqrt(na) * kappa * EPS)


def _solve_err_bound(mats, B, rtol):
    """Absolute bound of the error of element solves stopped by the test
    ||b_e - A_e x_e|| <= rtol ||b_e||: ||x_e - x_e*|| <= ||A_e^-1||_2 rtol
    ||b_e||, combined over the elements in the 2-norm (the a-posteriori
    bound the stopping test implies)."""
    return float(np.sqrt(sum((rtol * np.linalg.norm(b) / np.linalg.eigvalsh(A).min()) ** 2
                             for A, b in zip(mats, B))))


def _converged_tol(mats, B, Xstar, rtol):
    """Relative bound for a converged solve against the exact one: the
    stopping test's bound over ||x*||, plus the FP64 rounding bound."""
    return _solve_err_bound(mats, B, rtol) / np.linalg.norm(Xstar) + TOL


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


def _mesh(n, N, kind="mapped", c2="sine", amp=0.05):
    if kind == "mapped":
        X, Y = inputs.mapped_nodes(n, N, amp)
    else:
        X, Y = inputs.cartesian_nodes(n, N)
    if c2 == "sine":
        C2 = inputs.c2_sine(X, Y)
    elif c2 == "random":
        C2 = inputs.smooth_random_c2(X, Y, seed=11)
    else:
        C2 = np.full_like(X, float(c2))
    return X, Y, C2


def _pair(n, N, p, kind="mapped", c2="sine", flux="upwind", periodic=(False, False), nquad=0,
          rtol=1e-13, maxit=200, precond="fdm", xi=0.0):
    X, Y, C2 = _mesh(n, N, kind, c2)
    vp = dv.VarProblem(n=n, N=N, p=p, X=X, Y=Y, C2=C2, periodic=periodic, flux=flux, xi=xi,
                       nq=nquad if nquad else None)
    bc = tuple(gdg.BC_PERIODIC if q else gdg.BC_DIRICHLET for q in periodic)
    pb = gdg.make_problem(2, n, N, p, bc=bc, flux={"upwind": gdg.FLUX_UPWIND, "central": gdg.FLUX_CENTRAL, "alternating": gdg.FLUX_ALTERNATING}[flux],
                          xi=xi, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2, nquad=nquad,
                          pcg_rtol=rtol, pcg_maxit=maxit,
                          precond=gdg.PC_FDM if precond == "fdm" else gdg.PC_NONE)
    return vp, gdg.Context(pb)


CASES = [
    dict(n=(3, 2), N=8, p=5),
    dict(n=(4, 4), N=8, p=3, flux="central"),
    dict(n=(2, 3), N=4, p=3, periodic=(True, False), c2="random"),
    dict(n=(3, 3), N=5, p=5, periodic=(True, True), kind="cartesian", c2="1.7"),
    dict(n=(1, 1), N=6, p=3, periodic=(True, True)),
    dict(n=(2, 2), N=9, p=7, nquad=9),
    dict(n=(5, 3), N=8, p=5, xi=0.8, precond="none"),
    dict(n=(4, 3), N=8, p=5, flux="alternating", periodic=(True, False), c2="random"),
]


def _ids(c):
    return "n%s-N%d-p%d-%s" % ("x".join(map(str, c["n"])), c["N"], c["p"],
                               "-".join("%s=%s" % (k, v) for k, v in c.items() if k not in ("n", "N", "p")))


def _rand(vp, seed):
    ne = vp.n[0] * vp.n[1]
    return inputs.random_state((ne, vp.n1 ** 2), seed), inputs.random_state((ne, vp.n1 ** 2), seed + 1)


@pytest.mark.parametrize("c", CASES, ids=_ids)
def test_energy_pins_assembly(c):
    """E(0, V) = V^T M_J V / 2 and E(U, 0) = U^T S_c2 U / 2 with random
    states: the GPU-assembled element matrices against the oracle's."""
    vp, ctx = _pair(**c)
    ops = dv.assemble(vp)
    U, V = _rand(vp, 3)
    Z = np.zeros_like(U)
    for a, b in ((Z, V), (U, Z), (U, V)):
        E = dv.energy(ops, a, b)
        Eg = ctx.energy(_dev(a), _dev(b))
        assert abs(Eg - E) < TOL * abs(E), (Eg, E)
    ctx.close()


def _oracle_pcg(vp, ops, which, B, X0, rtol, maxit, precond="fdm"):
    Psi, lam = dv.reference_diagonalisation(vp.p, vp.N)
    out = np.empty_like(B)
    its = []
    for e in range(B.shape[0]):
        A = dv.spd_u_matrix(ops, e) if which == "S" else ops.M[e]
        if precond == "fdm":
            P = dv.fdm_preconditioner(ops, e, which, Psi, lam)
            pinv = lambda r, P=P: P @ r
        else:
            pinv = lambda r: r.copy()
        out[e], it, _ = dv.pcg(A, B[e], pinv, X0[e], rtol, maxit)
        its.append(it)
    return out, np.array(its)


@pytest.mark.parametrize("c", CASES, ids=_ids)
@pytest.mark.parametrize("K", [1, 3, 6])
def test_pcg_fixed_iterations(c, K):
    """rtol = 0, maxit = K: exactly K PCG iterations on every element from a
    random initial guess; the iterates match the oracle's."""
    kw = dict(c)
    kw.update(rtol=0.0, maxit=K)
    vp, ctx = _pair(**kw)
    ops = dv.assemble(vp)
    B, X0 = _rand(vp, 5)
    X0 = 0.1 * X0
    for which, op in (("M", gdg.OP_M), ("S", gdg.OP_S)):
        ref, its = _oracle_pcg(vp, ops, which, B, X0, 0.0, K, kw.get("precond", "fdm"))
        x = _dev(X0)
        st = ctx.pcg(op, _dev(B), x, allow_noconv=True)
        assert st["max_iters"] == K and its.max() == K
        assert _rel(x.cpu().numpy(), ref) < _kappa_tol(ops), which
    ctx.close()


@pytest.mark.parametrize("c", CASES[:4], ids=_ids)
def test_pcg_converged_matches_direct(c):
    vp, ctx = _pair(**c, rtol=1e-12, maxit=300)
    ops = dv.assemble(vp)
    U, V = _rand(vp, 7)
    ru, rv = dv.residuals(vp, ops, U, V)
    Ut, Vt = dv.solve_direct(ops, V, ru, rv)
    ne = ru.shape[0]
    Au = [dv.spd_u_matrix(ops, e) for e in range(ne)]
    x = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    st = ctx.pcg(gdg.OP_M, _dev(rv), x)
    assert st["max_rel_resid"] <= 1e-12
    assert _rel(x.cpu().numpy(), Vt) < _converged_tol(ops.M, rv, Vt, 1e-12)
    x.zero_()
    st = ctx.pcg(gdg.OP_S, _dev(ru), x)
    assert st["max_rel_resid"] <= 1e-12
    assert _rel(x.cpu().numpy(), Ut - V) < _converged_tol(Au, ru, Ut - V, 1e-12)
    ctx.close()


@pytest.mark.parametrize("c", CASES, ids=_ids)
def test_rhs_parity_fixed_iterations(c):
    """gdg_rhs with exactly K = 5 PCG iterations per element system (x0 = 0)
    against the oracle's residuals + the same PCG."""
    K = 5
    vp, ctx = _pair(**c, rtol=0.0, maxit=K)
    ops = dv.assemble(vp)
    U, V = _rand(vp, 9)
    ru, rv = dv.residuals(vp, ops, U, V)
    Ut, Vt, iu, iv = dv.solve_pcg(vp, ops, V, ru, rv, precond=c.get("precond", "fdm"), rtol=0.0, maxit=K)
    u, v = _dev(U), _dev(V)
    du, dv_ = torch.empty_like(u), torch.empty_like(v)
    try:
        ctx.rhs(u, v, du, dv_)
    except gdg.GdgError as err:
        assert err.status == gdg.ENOCONV        # rtol = 0 never "converges"
    a = np.concatenate([du.cpu().numpy(), dv_.cpu().numpy()])
    assert _rel(a, np.concatenate([Ut.ravel(), Vt.ravel()])) < _kappa_tol(ops)
    ctx.close()


@pytest.mark.parametrize("c", CASES[:3], ids=_ids)
def test_rhs_converged_matches_direct(c):
    vp, ctx = _pair(**c, rtol=1e-13, maxit=300)
    ops = dv.assemble(vp)
    U, V = _rand(vp, 13)
    Ut, Vt = dv.time_derivative(vp, ops, U, V)
    u, v = _dev(U), _dev(V)
    du, dv_ = torch.empty_like(u), torch.empty_like(v)
    ctx.rhs(u, v, du, dv_)
    a = np.concatenate([du.cpu().numpy(), dv_.cpu().numpy()])
    ref = np.concatenate([Ut.ravel(), Vt.ravel()])
    assert _rel(a, ref) < _rhs_tol(vp, ops, U, V, 1e-13, ref)
    ctx.close()


def _rhs_tol(vp, ops, U, V, rtol, ref):
    """Bound of a converged-PCG time derivative against the direct one: both
    element systems' stopping-test bounds, over the stacked derivative."""
    ru, rv = dv.residuals(vp, ops, U.reshape(ru_shape(vp)), V.reshape(ru_shape(vp)))
    Au = [dv.spd_u_matrix(ops, e) for e in range(ru.shape[0])]
    e = np.hypot(_solve_err_bound(Au, ru, rtol), _solve_err_bound(ops.M, rv, rtol))
    return e / np.linalg.norm(ref) + TOL


def ru_shape(vp):
    return (vp.n[0] * vp.n[1], vp.n1 ** 2)


@pytest.mark.parametrize("c", CASES[:4], ids=_ids)
def test_step_parity_fixed_iterations(c):
    """Three RK4 steps, every stage solve with exactly K = 6 iterations, one
    gdg_step call per step: the stacked state matches the oracle after each."""
    K = 6
    vp, ctx = _pair(**c, rtol=0.0, maxit=K)
    ops = dv.assemble(vp)
    U, V = _rand(vp, 17)
    u, v = _dev(U), _dev(V)
    f = lambda t, U, V: dv.solve_pcg(vp, ops, V, *dv.residuals(vp, ops, U, V),
                                     precond=c.get("precond", "fdm"), rtol=0.0, maxit=K)[:2]
    dt = 0.05 / (max(vp.n) * vp.N)
    tol = _kappa_tol(ops)
    for s in range(3):
        ctx.step(u, v, s * dt, dt, 1)
        U, V = ti.rk4_step(f, U, V, s * dt, dt)
        a = np.concatenate([u.cpu().numpy(), v.cpu().numpy()])
        assert _rel(a, np.concatenate([U.ravel(), V.ravel()])) < tol, s
    su, sv = ctx.step_stats()
    assert su["max_iters"] == K and sv["max_iters"] == K
    ctx.close()


def test_central_energy_and_upwind_decay_mapped():
    """Mapped mesh, variable c^2: the discrete energy is nearly conserved by
    the central flux (RK4 drift only) and decreases with the upwind flux."""
    for flux in ("central", "upwind"):
        vp, ctx = _pair((4, 4), 8, 5, flux=flux, rtol=1e-13, maxit=300)
        X, Y = vp.X, vp.Y
        U0 = inputs.gaussian_pulse(X, Y, 0.45, 0.55, 0.2)
        u, v = _dev(U0), torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
        E0 = ctx.energy(u, v)
        dt = 0.1 / (4 * 8)
        Es = []
        for _ in range(10):
            ctx.step(u, v, 0.0, dt, 2)
            Es.append(ctx.energy(u, v))
        if flux == "central":
            assert abs(Es[-1] - E0) < 1e-6 * E0, (E0, Es[-1])
        else:
            assert all(b <= a * (1 + 1e-13) for a, b in zip([E0] + Es, Es)) and Es[-1] < E0
        ctx.close()


def _patch_rhs(X, Y, C2, U, V, N, p, ey, ex, K):
    """Oracle time derivative of element (ey, ex) from the 3 x 3 patch around
    it (its value depends on its own data and its neighbours' traces only;
    patch sides on the domain boundary keep the Dirichlet condition)."""
    ny, nx = X.shape[:2]
    y0, y1 = max(ey - 1, 0), min(ey + 1, ny - 1)
    x0, x1 = max(ex - 1, 0), min(ex + 1, nx - 1)
    sl = (slice(y0, y1 + 1), slice(x0, x1 + 1))
    n = (x1 - x0 + 1, y1 - y0 + 1)
    vp = dv.VarProblem(n=n, N=N, p=p, X=X[sl], Y=Y[sl], C2=C2[sl], flux="upwind")
    ops = dv.assemble(vp)
    ne = n[0] * n[1]
    Us = U[sl].reshape(ne, -1)
    Vs = V[sl].reshape(ne, -1)
    ru, rv = dv.residuals(vp, ops, Us, Vs)
    Ut, Vt, _, _ = dv.solve_pcg(vp, ops, Vs, ru, rv, precond="fdm", rtol=0.0, maxit=K)
    c = (ey - y0) * n[0] + (ex - x0)
    return Ut[c], Vt[c], _kappa_tol(ops)


@pytest.mark.parametrize("p", [3, 5])
def test_full_size_mapped_128(p):
    """128 x 128 mapped elements of 8 x 8 cells, c^2 = 1 + 0.5 sin 2pi x cos 2pi y,
    Gaussian pulse: sampled-element parity of gdg_rhs (fixed K = 5 iterations)
    against 3 x 3 oracle patches; then RK4 steps at rtol 1e-10 with bounded
    iteration counts and decaying upwind energy."""
    n, N, K = (128, 128), 8, 5
    X, Y, C2 = _mesh(n, N)
    U = inputs.gaussian_pulse(X, Y, 0.5, 0.5, 0.05) + 0.01 * inputs.random_state(X.shape, 21)
    V = 0.01 * inputs.random_state(X.shape, 22)
    pb = gdg.make_problem(2, n, N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                          pcg_rtol=0.0, pcg_maxit=K)
    ctx = gdg.Context(pb)
    u, v = _dev(U), _dev(V)
    du, dv_ = torch.empty_like(u), torch.empty_like(v)
    try:
        ctx.rhs(u, v, du, dv_)
    except gdg.GdgError as err:
        assert err.status == gdg.ENOCONV
    du = du.cpu().numpy().reshape(128, 128, -1)
    dvv = dv_.cpu().numpy().reshape(128, 128, -1)
    for ey, ex in [(0, 0), (0, 77), (127, 127), (64, 64), (31, 100), (127, 5)]:
        Ut, Vt, tol = _patch_rhs(X, Y, C2, U, V, N, p, ey, ex, K)
        a = np.concatenate([du[ey, ex], dvv[ey, ex]])
        assert _rel(a, np.concatenate([Ut, Vt])) < tol, (ey, ex)
    ctx.close()
    pb = gdg.make_problem(2, n, N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                          pcg_rtol=1e-10, pcg_maxit=100)
    ctx = gdg.Context(pb)
    # the rough part makes jumps across the faces, so that the upwind
    # dissipation (the face terms of the energy identity, Section 2.2.1) is far
    # above the energy noise of rtol-1e-10 solves: over 8 steps a smooth pulse
    # alone loses about 1e-14 of its energy, which the solves' noise can exceed
    # (measured: with a 1e-2 rough part the energy fell by 26 % in 8 steps)
    U0 = inputs.gaussian_pulse(X, Y, 0.5, 0.5, 0.05) + 1e-3 * inputs.random_state(X.shape, 23)
    V0 = 1e-3 * inputs.random_state(X.shape, 24)
    u, v = _dev(U0), _dev(V0)
    E0 = ctx.energy(u, v)
    dt = 0.1 / (128 * 8)
    ctx.step(u, v, 0.0, dt, 8)
    su, sv = ctx.step_stats()
    E1 = ctx.energy(u, v)
    assert su["unconverged"] == 0 and sv["unconverged"] == 0
    assert su["max_iters"] < 40 and sv["max_iters"] < 20
    assert E1 < (1.0 - 1e-6) * E0 and E1 > 0.5 * E0
    ctx.close()


def _patch_step(X, Y, C2, U, V, N, p, ey, ex, K, dt, R=4):
    """Oracle RK4 step of element (ey, ex) from the (2R+1) x (2R+1) patch
    around it.  Each stage couples an element only to its face neighbours,
    so after the 4 stages of one step the element's new state depends on
    elements within 4 faces of it; an error the artificial patch boundary
    makes at the patch's edge travels one element per stage and stops one
    element short of the centre."""
    ny, nx = X.shape[:2]
    y0, y1 = max(ey - R, 0), min(ey + R, ny - 1)
    x0, x1 = max(ex - R, 0), min(ex + R, nx - 1)
    sl = (slice(y0, y1 + 1), slice(x0, x1 + 1))
    n = (x1 - x0 + 1, y1 - y0 + 1)
    vp = dv.VarProblem(n=n, N=N, p=p, X=X[sl], Y=Y[sl], C2=C2[sl], flux="upwind")
    ops = dv.assemble(vp)
    ne = n[0] * n[1]
    f = lambda t, U_, V_: dv.solve_pcg(vp, ops, V_, *dv.residuals(vp, ops, U_, V_), precond="fdm",
                                       rtol=0.0, maxit=K)[:2]
    Un, Vn = ti.rk4_step(f, U[sl].reshape(ne, -1), V[sl].reshape(ne, -1), 0.0, dt)
    c = (ey - y0) * n[0] + (ex - x0)
    return Un[c], Vn[c], _kappa_tol(ops)


@pytest.mark.parametrize("p", [3, 5])
def test_full_size_mapped_128_one_step(p):
    """The 128 x 128 mapped workload (c^2 = 1 + 0.5 sin 2pi x cos 2pi y, 8 x 8
    cells, pulse plus noise): one whole RK4 step with exactly K = 5 PCG
    iterations per element solve, launched as the workload is, against the
    oracle's step on 9 x 9 patches around sampled elements (corners, edges,
    interior)."""
    n, N, K = (128, 128), 8, 5
    X, Y, C2 = _mesh(n, N)
    U = inputs.gaussian_pulse(X, Y, 0.5, 0.5, 0.05) + 0.01 * inputs.random_state(X.shape, 23)
    V = 0.01 * inputs.random_state(X.shape, 24)
    pb = gdg.make_problem(2, n, N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                          pcg_rtol=0.0, pcg_maxit=K)
    ctx = gdg.Context(pb)
    u, v = _dev(U), _dev(V)
    dt = 0.1 / (128 * 8)
    ctx.step(u, v, 0.0, dt, 1)
    un = u.cpu().numpy().reshape(128, 128, -1)
    vn = v.cpu().numpy().reshape(128, 128, -1)
    for ey, ex in [(0, 0), (127, 127), (64, 64), (2, 90), (100, 3)]:
        Uc, Vc, tol = _patch_step(X, Y, C2, U, V, N, p, ey, ex, K, dt)
        a = np.concatenate([un[ey, ex], vn[ey, ex]])
        assert _rel(a, np.concatenate([Uc, Vc])) < tol, (ey, ex, _rel(a, np.concatenate([Uc, Vc])))
    ctx.close()


# ----------------------------------------------------------- mixed precision

def _mixed_pair(n, N, p, rtol, **kw):
    X, Y, C2 = _mesh(n, N, kw.pop("kind", "mapped"), kw.pop("c2", "sine"))
    vp = dv.VarProblem(n=n, N=N, p=p, X=X, Y=Y, C2=C2, flux="upwind")
    mk = lambda prec: gdg.make_problem(2, n, N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                                       pcg_rtol=rtol, pcg_maxit=200, precision=prec, refine_max=10,
                                       refine_rtol=1e-5)
    return vp, gdg.Context(mk(gdg.MIXED)), gdg.Context(mk(gdg.FP64))


@pytest.mark.parametrize("n,N,p", [((3, 2), 8, 5), ((4, 4), 8, 3), ((2, 2), 9, 7)])
def test_mixed_pcg_matches_direct(n, N, p):
    """FP32 inner PCG + FP64 refinement: the true FP64 residual meets rtol,
    and the solution agrees with the oracle's dense solve."""
    vp, cm, _ = _mixed_pair(n, N, p, 1e-12)
    ops = dv.assemble(vp)
    U, V = _rand(vp, 31)
    ru, rv = dv.residuals(vp, ops, U, V)
    Ut, Vt = dv.solve_direct(ops, V, ru, rv)
    Au = [dv.spd_u_matrix(ops, e) for e in range(ru.shape[0])]
    x = torch.zeros(cm.n, dtype=torch.float64, device="cuda")
    st = cm.pcg(gdg.OP_M, _dev(rv), x)
    assert st["max_rel_resid"] <= 1e-12 and st["max_sweeps"] <= 5
    assert _rel(x.cpu().numpy(), Vt) < _converged_tol(ops.M, rv, Vt, 1e-12)
    x.zero_()
    st = cm.pcg(gdg.OP_S, _dev(ru), x)
    assert st["max_rel_resid"] <= 1e-12 and st["max_sweeps"] <= 6
    assert _rel(x.cpu().numpy(), Ut - V) < _converged_tol(Au, ru, Ut - V, 1e-12)
    cm.close()


def test_mixed_rhs_and_steps_match_fp64():
    """Mixed and FP64 forms at the same rtol give the same semi-discrete
    derivative and trajectory to within a few rtol; the mixed form needs
    only a few FP64 sweeps per solve."""
    vp, cm, cf = _mixed_pair((6, 5), 8, 5, 1e-12)
    ops = dv.assemble(vp)
    U = inputs.gaussian_pulse(vp.X, vp.Y, 0.4, 0.6, 0.15)
    V = 0.1 * inputs.random_state(U.shape, 41)
    Ut, Vt = dv.time_derivative(vp, ops, U.reshape(30, -1), V.reshape(30, -1))
    ref = np.concatenate([Ut.ravel(), Vt.ravel()])
    outs = []
    for ctx in (cm, cf):
        u, v = _dev(U), _dev(V)
        du, dv_ = torch.empty_like(u), torch.empty_like(v)
        ctx.rhs(u, v, du, dv_)
        outs.append(np.concatenate([du.cpu().numpy(), dv_.cpu().numpy()]))
    tol = _rhs_tol(vp, ops, U, V, 1e-12, ref)
    assert _rel(outs[0], ref) < tol and _rel(outs[1], ref) < tol
    cm.step_stats(); cf.step_stats()
    states = []
    dt, steps = 2e-3, 5
    for ctx in (cm, cf):
        u, v = _dev(U), _dev(V)
        ctx.step(u, v, 0.0, dt, steps)
        states.append(np.concatenate([u.cpu().numpy(), v.cpu().numpy()]))
    # each stage derivative of either form is within the stopping-test bound
    # e of the exact one, and RK4 adds dt times a weighted mean of them (weights
    # summing to 1) per step, so the two trajectories drift apart by at most
    # 2 dt e per step, over steps steps (the step map itself is non-expansive
    # at this CFL); e is evaluated at the initial state, which dominates
    e_abs = (tol - TOL) * np.linalg.norm(ref)
    state0 = np.linalg.norm(np.concatenate([U.ravel(), V.ravel()]))
    assert _rel(states[0], states[1]) < 2.0 * steps * dt * e_abs / state0 + TOL
    su, sv = cm.step_stats()
    assert su["unconverged"] == 0 and sv["unconverged"] == 0
    assert su["mean_sweeps"] <= 4 and sv["mean_sweeps"] <= 3
    cm.close(); cf.close()


@pytest.mark.parametrize("p", [3, 5])
def test_equal_error_against_refined_reference(p):
    """The forms reach the same error: FP64 PCG, mixed (FP32 inner + FP64
    refinement) and element inverses on the sine-mapped 8 x 8 mesh
    (c^2 = 1 + 0.5 sin 2pi x cos 2pi y, Gaussian pulse of width 0.15) against
    an FP64 run on the 16 x 16 mesh of the same map at dt/2 (every coarse node
    is a fine node); each form's error is within 1.05x the FP64 PCG's (the
    equal-error criterion of the benchmark's comparison)."""
    import bench
    n, N, T = 8, 8, 0.05
    Xf, Yf = inputs.mapped_nodes((2 * n, 2 * n), N, 0.05)
    X, Y = inputs.mapped_nodes((n, n), N, 0.05)
    idx = bench.coarse_in_fine(n, N)
    assert np.abs(Xf.ravel()[idx] - X.ravel()).max() < 1e-13
    steps = int(round(T / (0.1 / (n * N) / np.sqrt(1.5))))
    dt = T / steps
    ctx = gdg.Context(gdg.make_problem(2, (2 * n, 2 * n), N, p, coef=gdg.COEF_NODAL, x_nodes=Xf, y_nodes=Yf,
                                       c2_nodes=inputs.c2_sine(Xf, Yf), solver=gdg.SOLVE_INVERSE))
    u = _dev(inputs.gaussian_pulse(Xf, Yf, 0.5, 0.5, 0.15))
    v = torch.zeros_like(u)
    ctx.step(u, v, 0.0, 0.5 * dt, 2 * steps)
    ref = u.cpu().numpy()[idx]
    ctx.close()
    err = {}
    for name, prec, solver in (("fp64", gdg.FP64, gdg.SOLVE_PCG), ("mixed", gdg.MIXED, gdg.SOLVE_PCG),
                               ("inverse", gdg.FP64, gdg.SOLVE_INVERSE)):
        ctx = gdg.Context(gdg.make_problem(2, (n, n), N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y,
                                           c2_nodes=inputs.c2_sine(X, Y), pcg_rtol=1e-10, pcg_maxit=100,
                                           precision=prec, solver=solver))
        u = _dev(inputs.gaussian_pulse(X, Y, 0.5, 0.5, 0.15))
        v = torch.zeros_like(u)
        ctx.step(u, v, 0.0, dt, steps)
        err[name] = np.linalg.norm(u.cpu().numpy() - ref) / np.linalg.norm(ref)
        ctx.close()
    assert 0.0 < err["fp64"] < 0.1, err          # a discretisation error, not noise and not a blow-up
    assert err["mixed"] <= 1.05 * err["fp64"] and err["inverse"] <= 1.05 * err["fp64"], err
