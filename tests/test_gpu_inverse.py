"""GPU parity of the precomputed-inverse element solves (GDG_SOLVE_INVERSE)
with the FP64 oracle's dense direct solves, through the C ABI: gdg_rhs,
gdg_step over several steps, the full 128 x 128 mapped mesh on sampled
elements (3 x 3 oracle patches), the batched launch, and the PCG trajectory
at rtol 1e-10.

Tolerance: both sides solve the same element systems exactly up to
rounding (the oracle by LU, the library by Cholesky and an explicit
inverse), so each solve's relative error is a small multiple of
kappa * eps; the tests take max(1e-12, 50 kappa_max eps) with kappa_max the
largest 2-norm condition number of the element systems, computed here from
the oracle's matrices."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dg_var as dv, timeint as ti
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


def _mesh(n, N, kind="mapped", c2="sine"):
    X, Y = inputs.mapped_nodes(n, N, 0.05) if kind == "mapped" else inputs.cartesian_nodes(n, N)
    if c2 == "sine":
        C2 = inputs.c2_sine(X, Y)
    elif c2 == "random":
        C2 = inputs.smooth_random_c2(X, Y, seed=11)
    else:
        C2 = np.full_like(X, float(c2))
    return X, Y, C2


def _problem(n, N, p, X, Y, C2, solver=gdg.SOLVE_INVERSE, flux="upwind", periodic=(False, False), **kw):
    bc = tuple(gdg.BC_PERIODIC if q else gdg.BC_DIRICHLET for q in periodic)
    return gdg.make_problem(2, n, N, p, bc=bc, flux={"upwind": gdg.FLUX_UPWIND, "central": gdg.FLUX_CENTRAL, "alternating": gdg.FLUX_ALTERNATING}[flux],
                            coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2, solver=solver, **kw)


def _pair(n, N, p, kind="mapped", c2="sine", flux="upwind", periodic=(False, False)):
    X, Y, C2 = _mesh(n, N, kind, c2)
    vp = dv.VarProblem(n=n, N=N, p=p, X=X, Y=Y, C2=C2, periodic=periodic, flux=flux)
    return vp, gdg.Context(_problem(n, N, p, X, Y, C2, flux=flux, periodic=periodic))


def _kappa(ops):
    ne = ops.M.shape[0]
    return max(max(np.linalg.cond(dv.spd_u_matrix(ops, e)), np.linalg.cond(ops.M[e])) for e in range(ne))


def _tol(ops):
    return max(1e-12, 50.0 * _kappa(ops) * EPS)


CASES = [
    dict(n=(3, 2), N=8, p=5),
    dict(n=(4, 4), N=8, p=3, flux="central"),
    dict(n=(2, 3), N=8, p=5, periodic=(True, False), c2="random"),
    dict(n=(3, 3), N=5, p=5, periodic=(True, True), kind="cartesian", c2="1.7"),
    dict(n=(2, 2), N=9, p=7),
    dict(n=(1, 1), N=6, p=3, periodic=(True, True)),
    dict(n=(3, 4), N=8, p=5, flux="alternating"),
]


def _ids(c):
    return "n%s-N%d-p%d-%s" % ("x".join(map(str, c["n"])), c["N"], c["p"],
                               "-".join("%s=%s" % (k, v) for k, v in c.items() if k not in ("n", "N", "p")))


@pytest.mark.parametrize("c", CASES, ids=_ids)
def test_inverse_rhs_matches_direct(c):
    vp, ctx = _pair(**c)
    ops = dv.assemble(vp)
    ne = vp.n[0] * vp.n[1]
    U = inputs.random_state((ne, vp.n1 ** 2), 31)
    V = inputs.random_state((ne, vp.n1 ** 2), 32)
    Ut, Vt = dv.time_derivative(vp, ops, U, V)
    u, v = _dev(U), _dev(V)
    du, dv_ = torch.empty_like(u), torch.empty_like(v)
    ctx.rhs(u, v, du, dv_)
    a = np.concatenate([du.cpu().numpy(), dv_.cpu().numpy()])
    assert _rel(a, np.concatenate([Ut.ravel(), Vt.ravel()])) < _tol(ops)
    ctx.close()


@pytest.mark.parametrize("c", CASES[:3], ids=_ids)
def test_inverse_steps_match_oracle(c):
    """Three RK4 steps, one gdg_step call per step, against the oracle's RK4
    with dense direct solves, after every step."""
    vp, ctx = _pair(**c)
    ops = dv.assemble(vp)
    tol = _tol(ops)
    ne = vp.n[0] * vp.n[1]
    U = inputs.random_state((ne, vp.n1 ** 2), 41)
    V = inputs.random_state((ne, vp.n1 ** 2), 42)
    u, v = _dev(U), _dev(V)
    f = lambda t, U, V: dv.time_derivative(vp, ops, U, V)
    dt = 0.05 / (max(vp.n) * vp.N)
    for s in range(3):
        ctx.step(u, v, s * dt, dt, 1)
        U, V = ti.rk4_step(f, U, V, s * dt, dt)
        a = np.concatenate([u.cpu().numpy(), v.cpu().numpy()])
        # per-step gaps add up at most linearly (non-expansive step map)
        assert _rel(a, np.concatenate([U.ravel(), V.ravel()])) < (s + 1) * tol, s
    ctx.close()


def _patch_rhs_direct(X, Y, C2, U, V, N, p, ey, ex):
    """Oracle time derivative of element (ey, ex) from the 3 x 3 patch around
    it, with dense direct solves."""
    ny, nx = X.shape[:2]
    y0, y1 = max(ey - 1, 0), min(ey + 1, ny - 1)
    x0, x1 = max(ex - 1, 0), min(ex + 1, nx - 1)
    sl = (slice(y0, y1 + 1), slice(x0, x1 + 1))
    n = (x1 - x0 + 1, y1 - y0 + 1)
    vp = dv.VarProblem(n=n, N=N, p=p, X=X[sl], Y=Y[sl], C2=C2[sl], flux="upwind")
    ops = dv.assemble(vp)
    ne = n[0] * n[1]
    Ut, Vt = dv.time_derivative(vp, ops, U[sl].reshape(ne, -1), V[sl].reshape(ne, -1))
    c = (ey - y0) * n[0] + (ex - x0)
    return Ut[c], Vt[c], _tol(ops), _kappa(ops)


def test_inverse_full_size_mapped_128():
    """128 x 128 mapped elements, p = 5, in the benchmark's launch: gdg_rhs on
    sampled elements against 3 x 3 oracle patches; then the RK4 trajectory
    against the PCG form at rtol 1e-10."""
    n, N, p = (128, 128), 8, 5
    X, Y, C2 = _mesh(n, N)
    U = inputs.gaussian_pulse(X, Y, 0.5, 0.5, 0.05) + 0.01 * inputs.random_state(X.shape, 21)
    V = 0.01 * inputs.random_state(X.shape, 22)
    ctx = gdg.Context(_problem(n, N, p, X, Y, C2))
    u, v = _dev(U), _dev(V)
    du, dv_ = torch.empty_like(u), torch.empty_like(v)
    ctx.rhs(u, v, du, dv_)
    du = du.cpu().numpy().reshape(128, 128, -1)
    dvv = dv_.cpu().numpy().reshape(128, 128, -1)
    kappa = 0.0
    for ey, ex in [(0, 0), (0, 77), (127, 127), (64, 64), (31, 100), (127, 5)]:
        Ut, Vt, tol, k = _patch_rhs_direct(X, Y, C2, U, V, N, p, ey, ex)
        kappa = max(kappa, k)
        a = np.concatenate([du[ey, ex], dvv[ey, ex]])
        assert _rel(a, np.concatenate([Ut, Vt])) < tol, (ey, ex)
    # trajectory: inverse route vs PCG at rtol 1e-10 (same method, PCG residual 1e-10)
    U0 = inputs.gaussian_pulse(X, Y, 0.5, 0.5, 0.05)
    dt = 0.1 / (128 * 8)
    states = []
    for c in (ctx, gdg.Context(_problem(n, N, p, X, Y, C2, solver=gdg.SOLVE_PCG, pcg_rtol=1e-10,
                                        pcg_maxit=100))):
        u, v = _dev(U0), torch.zeros(U0.size, dtype=torch.float64, device="cuda")
        c.step(u, v, 0.0, dt, 8)
        states.append(torch.cat([u, v]).cpu().numpy())
        c.close()
    # PCG's stage derivatives are within kappa rtol (relative) of the exact
    # ones; a step adds dt times a weighted mean of them, and dt |k| <= dt
    # rho(L) |y| <= 2.8 |y| inside RK4's stability interval, so after 8 steps
    # the relative gap is at most 8 x 2.8 x kappa x rtol (kappa from the
    # sampled patches' element systems)
    assert _rel(states[0], states[1]) < 8 * 2.8 * kappa * 1e-10


def test_inverse_batch_equals_individual_steps():
    specs = inputs.batched_problems(count=6, nmin=3, nmax=8)
    built = []
    for sp in specs:
        n, p = sp["n"], sp["p"]
        X, Y = inputs.cartesian_nodes((n, n), 8)
        if sp["variable"]:
            C2 = inputs.smooth_random_c2(X, Y, sp["seed"])
            pb = _problem((n, n), 8, p, X, Y, C2)
            cmax = float(np.sqrt(C2.max()))
        else:
            pb = gdg.make_problem(2, (n, n), 8, p, c2=1.0)
            cmax = 1.0
        built.append((pb, inputs.gaussian_pulse(X, Y, sp["x0"], sp["y0"], 0.05).ravel(), 0.1 / (n * 8) / cmax))
    batch = gdg.Batch([b[0] for b in built])
    us = [_dev(b[1]) for b in built]
    vs = [torch.zeros_like(u) for u in us]
    batch.step(us, vs, [b[2] for b in built], 6)
    for i, (pb, U0, dt) in enumerate(built):
        ctx = gdg.Context(pb)
        u, v = _dev(U0), torch.zeros(U0.size, dtype=torch.float64, device="cuda")
        ctx.step(u, v, 0.0, dt, 6)
        a = torch.cat([us[i], vs[i]]).cpu().numpy()
        b = torch.cat([u, v]).cpu().numpy()
        assert np.abs(a - b).max() <= 1e-15 * np.abs(b).max(), i
        ctx.close()
    batch.close()


def test_inverse_context_still_runs_pcg_and_refuses_the_learned_guess():
    from paper_2105_01722_gb300 import learned
    vp, ctx = _pair((2, 2), 8, 5)
    ops = dv.assemble(vp)
    B = inputs.random_state((4, 81), 51)
    b, x = _dev(B), torch.zeros(4 * 81, dtype=torch.float64, device="cuda")
    ctx.pcg(gdg.OP_M, b, x)
    ref = np.stack([np.linalg.solve(ops.M[e], B[e]) for e in range(4)])
    assert _rel(x.cpu().numpy(), ref) < 1e-7      # rtol 1e-10 x cond(M_J) ~ 3e2
    with pytest.raises(gdg.GdgError):
        ctx.mlp_attach(gdg.Mlp(learned.glorot_params(1)))
    ctx.close()
