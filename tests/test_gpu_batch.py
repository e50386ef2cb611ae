"""Batched persistent launch (gdg_batch_*: one launch per RK stage over every
problem): every problem of a batch ends exactly where its own gdg_step takes
it (the stage bodies are shared), for modal and PCG problems, p = 3, 5, 7,
FP64 and mixed precision, through the graph path and the remainder; the
tuner reports its choice; and every
problem of a mixed batch matches the FP64 oracle's RK4 (FP64 PCG, mixed
precision and element-inverse forms)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2105_01722_gb300 import gdg, inputs

CFL = {3: 0.2, 5: 0.15, 7: 0.12}   # about 0.8 of the largest RK4-stable upwind CFL


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gdg.lib()


def _problem(spec, N=8, precision=gdg.FP64):
    n, p = spec["n"], spec["p"]
    X, Y = inputs.cartesian_nodes((n, n), N)
    if spec["variable"]:
        C2 = inputs.smooth_random_c2(X, Y, spec["seed"])
        pb = gdg.make_problem(2, (n, n), N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                              pcg_rtol=1e-10, pcg_maxit=100, precision=precision, refine_max=10,
                              refine_rtol=1e-5)
        cmax = float(np.sqrt(C2.max()))
    else:
        pb = gdg.make_problem(2, (n, n), N, p, c2=1.0)
        cmax = 1.0
    U = inputs.gaussian_pulse(X, Y, spec["x0"], spec["y0"], 0.05)
    dt = CFL[p] / (n * N) / cmax
    return pb, U.ravel(), dt


def _specs(count, nmin, nmax):
    return inputs.batched_problems(count=count, nmin=nmin, nmax=nmax)


@pytest.mark.parametrize("precision", [gdg.FP64, gdg.MIXED])
def test_batch_equals_individual_steps(precision):
    specs = _specs(8, 4, 12)
    assert {s["p"] for s in specs} >= {3, 5} and any(s["variable"] for s in specs)
    built = [_problem(s, precision=precision) for s in specs]
    batch = gdg.Batch([b[0] for b in built])
    us = [torch.tensor(b[1], device="cuda") for b in built]
    vs = [torch.zeros_like(u) for u in us]
    dts = [b[2] for b in built]
    batch.step(us, vs, dts, 7)       # one graph of 4 steps + 3 direct steps
    tun = batch.tuning()
    assert tun["threads_per_block"] == 96                       # one element block (81 nodes) per CTA
    assert tun["tile_elements"] == 96 // 18                     # half-line modal body: two threads per line
    assert tun["blocks_per_sm"] >= 1 and 0 < tun["registers_per_thread"] <= 255
    for i, (pb, U0, dt) in enumerate(built):
        ctx = gdg.Context(pb)
        u = torch.tensor(U0, device="cuda")
        v = torch.zeros_like(u)
        ctx.step(u, v, 0.0, dt, 7)
        a = torch.cat([us[i], vs[i]]).cpu().numpy()
        b = torch.cat([u, v]).cpu().numpy()
        assert np.abs(a - b).max() <= 1e-15 * np.abs(b).max(), i
        ctx.close()
    for i, s in enumerate(specs):
        if s["variable"]:
            su, sv = batch.stats(i)
            assert su["unconverged"] == 0 and sv["unconverged"] == 0 and su["mean_iters"] > 0
    # a second call with new step sizes reuses the graph and the tuning
    batch.step(us, vs, [0.5 * d for d in dts], 4)
    assert batch.tuning() == tun
    batch.close()


def test_every_launch_shape_gives_the_same_steps():
    """The launch shape (register budget, resident blocks, items per turn)
    only decides which block runs which item: every pinned shape reproduces
    the tuned batch's steps bit for bit."""
    specs = _specs(6, 4, 10)
    built = [_problem(s, precision=gdg.MIXED) for s in specs]
    batch = gdg.Batch([b[0] for b in built])
    dts = [b[2] for b in built]

    def run():
        us = [torch.tensor(b[1], device="cuda") for b in built]
        vs = [torch.zeros_like(u) for u in us]
        batch.step(us, vs, dts, 5)
        return [torch.cat([u, v]).cpu().numpy() for u, v in zip(us, vs)]

    ref = run()
    tun = batch.tuning()
    assert tun["register_budget"] in (0, 1, 2) and tun["items_per_turn"] in (1, 2, 4, 8)
    for budget, r, chunk in ((0, 1, 1), (1, 2, 3), (2, 3, 8), (2, 1, 1000)):
        batch.set_tuning(budget, r, chunk)
        assert batch.tuning()["blocks_per_sm"] == r and batch.tuning()["items_per_turn"] == chunk
        for a, b in zip(run(), ref):
            assert np.array_equal(a, b)
    with pytest.raises(gdg.GdgError):
        batch.set_tuning(0, 64, 1)        # more blocks than fit
    with pytest.raises(gdg.GdgError):
        batch.set_tuning(3, 1, 1)
    batch.set_tuning(0, 0, 1)             # back to the tuner
    for a, b in zip(run(), ref):
        assert np.array_equal(a, b)
    batch.close()


def test_batch_rejects_mixed_cell_counts():
    pbs = [gdg.make_problem(2, (4, 4), 8, 3), gdg.make_problem(2, (4, 4), 9, 3)]
    with pytest.raises(gdg.GdgError):
        gdg.Batch(pbs)


# ---------------------------------------------------------------- oracle parity

EPS = np.finfo(np.float64).eps
TOL = 1e-12
# (variable c^2, p, elements per direction): every degree, both kinds
ORACLE_SPECS = [(False, 3, 4), (True, 3, 3), (False, 5, 3), (True, 5, 4), (True, 7, 3), (False, 7, 3)]


def _rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


def _oracle_rhs(variable, n, p, C2, X, Y, form, K):
    """The oracle's semi-discrete derivative of one batch problem: constant
    c^2 = 1 through the Cartesian oracle (dense solves); variable c^2 through
    the quadrature oracle with exactly K PCG iterations per solve (form
    'fp64') or dense direct solves ('mixed', 'inverse')."""
    from oracle import dg_const as dc, dg_var as dv
    if not variable:
        prob = dc.Problem(dim=2, n=(n, n), N=8, p=p, flux="upwind", c2=1.0)
        ops = dc.operators(prob)
        return (lambda t, U, V: dc.time_derivative(prob, U, V, ops)), None
    vp = dv.VarProblem(n=(n, n), N=8, p=p, X=X, Y=Y, C2=C2, flux="upwind")
    ops = dv.assemble(vp)
    if form == "fp64":
        f = lambda t, U, V: dv.solve_pcg(vp, ops, V, *dv.residuals(vp, ops, U, V), precond="fdm",
                                         rtol=0.0, maxit=K)[:2]
    else:
        f = lambda t, U, V: dv.time_derivative(vp, ops, U, V)
    kappa = max(max(np.linalg.cond(dv.spd_u_matrix(ops, e)), np.linalg.cond(ops.M[e])) for e in range(n * n))
    return f, kappa


@pytest.mark.parametrize("form", ["fp64", "mixed", "inverse"])
def test_batch_matches_oracle(form):
    """A batch of six problems (p = 3, 5, 7; constant and variable c^2), five
    RK4 steps in one gdg_batch_step call (one replay of the 4-step graph and
    one step outside it), each problem against the oracle's RK4.  Bounds per
    step, added over the steps (the step map is non-expansive at these CFLs):
    constant c^2, 1e-12; variable c^2 with K = 6 PCG iterations on both
    sides ('fp64'), max(1e-12, sqrt(81) kappa eps); element inverses against dense
    solves, max(1e-12, 50 kappa eps); FP32 inner PCG refined to the FP64
    residual test rtol = 1e-12 against dense solves ('mixed'), 2.8 kappa rtol
    (each stage derivative within kappa rtol relative, dt |k| <= 2.8 |y| in
    RK4's stability interval)."""
    from oracle import timeint as ti
    K, steps, rtol = 6, 5, 1e-12
    prec = gdg.MIXED if form == "mixed" else gdg.FP64
    solver = gdg.SOLVE_INVERSE if form == "inverse" else gdg.SOLVE_PCG
    pbs, states, dts, oracles = [], [], [], []
    for i, (variable, p, n) in enumerate(ORACLE_SPECS):
        X, Y = inputs.cartesian_nodes((n, n), 8)
        U0 = inputs.gaussian_pulse(X, Y, 0.45, 0.55, 0.2) + 0.01 * inputs.random_state(X.shape, 300 + i)
        V0 = 0.01 * inputs.random_state(X.shape, 400 + i)
        C2 = inputs.smooth_random_c2(X, Y, 77 + i) if variable else None
        if variable:
            pb = gdg.make_problem(2, (n, n), 8, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                                  solver=solver, precision=prec,
                                  pcg_rtol=0.0 if form == "fp64" else rtol,
                                  pcg_maxit=K if form == "fp64" else 300, refine_max=20, refine_rtol=1e-5)
            cmax = float(np.sqrt(C2.max()))
        else:
            pb = gdg.make_problem(2, (n, n), 8, p, c2=1.0)
            cmax = 1.0
        pbs.append(pb)
        states.append((U0, V0))
        dts.append(CFL[p] / (n * 8) / cmax)
        oracles.append(_oracle_rhs(variable, n, p, C2, X, Y, form, K))
    batch = gdg.Batch(pbs)
    us = [torch.tensor(U.ravel(), device="cuda") for U, _ in states]
    vs = [torch.tensor(V.ravel(), device="cuda") for _, V in states]
    batch.step(us, vs, dts, steps)
    for i, ((variable, p, n), (U, V), dt, (f, kappa)) in enumerate(zip(ORACLE_SPECS, states, dts, oracles)):
        ne = n * n
        Uo, Vo = ti.integrate(f, U.reshape(ne, -1), V.reshape(ne, -1), 0.0, dt, steps)
        if not variable:
            per_step = TOL
        elif form == "fp64":
            per_step = max(TOL, 9.0 * kappa * EPS)      # sqrt(n) kappa eps, n = 81 terms per product
        elif form == "inverse":
            per_step = max(TOL, 50.0 * kappa * EPS)
        else:
            per_step = TOL + 2.8 * kappa * rtol
        got = torch.cat([us[i], vs[i]]).cpu().numpy()
        ref = np.concatenate([Uo.ravel(), Vo.ravel()])
        assert _rel(got, ref) < steps * per_step, (form, i, _rel(got, ref), steps * per_step)
    batch.close()


@pytest.mark.parametrize("N", [7, 9])
def test_batch_fluxes_sides_and_cell_counts(N):
    """Batches of N = 7 (64-thread blocks, 4-element modal tiles) and N = 9
    (128-thread blocks, 6-element tiles) whose problems differ in flux
    (central, upwind, alternating), in periodic sides and in rectangular
    element grids, constant and variable c^2 (PCG and element inverses): each
    problem equals its own gdg_step, under the tuner and under every register
    budget (the batch stages each problem's flux and side flags itself)."""
    settings = [
        (gdg.FLUX_CENTRAL, (gdg.BC_PERIODIC, gdg.BC_DIRICHLET), (5, 4), False, gdg.SOLVE_PCG),
        (gdg.FLUX_UPWIND, (gdg.BC_DIRICHLET, gdg.BC_PERIODIC), (3, 6), True, gdg.SOLVE_PCG),
        (gdg.FLUX_ALTERNATING, (gdg.BC_PERIODIC, gdg.BC_PERIODIC), (4, 4), False, gdg.SOLVE_PCG),
        (gdg.FLUX_ALTERNATING, (gdg.BC_DIRICHLET, gdg.BC_DIRICHLET), (4, 3), True, gdg.SOLVE_INVERSE),
        (gdg.FLUX_CENTRAL, (gdg.BC_PERIODIC, gdg.BC_PERIODIC), (6, 5), True, gdg.SOLVE_PCG),
        (gdg.FLUX_UPWIND, (gdg.BC_DIRICHLET, gdg.BC_DIRICHLET), (2, 7), False, gdg.SOLVE_PCG),
    ]
    built = []
    for i, (flux, bc, n, variable, solver) in enumerate(settings):
        p = ((3, 5, 7) if N >= 9 else (3, 5))[i % (3 if N >= 9 else 2)]
        X, Y = inputs.cartesian_nodes(n, N)
        U = np.sin(np.pi * X) * np.cos(np.pi * Y) + 0.1 * inputs.random_state(X.shape, 70 + i)
        if variable:
            C2 = inputs.smooth_random_c2(X, Y, 900 + i)
            pb = gdg.make_problem(2, n, N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2, flux=flux,
                                  bc=bc, pcg_rtol=1e-10, pcg_maxit=100, solver=solver)
            cmax = float(np.sqrt(C2.max()))
        else:
            pb = gdg.make_problem(2, n, N, p, flux=flux, bc=bc, c2=1.3)
            cmax = float(np.sqrt(1.3))
        built.append((pb, U.ravel(), 0.1 / (max(n) * N) / cmax))
    refs = []
    for pb, U0, dt in built:
        ctx = gdg.Context(pb)
        u = torch.tensor(U0, device="cuda")
        v = torch.zeros_like(u)
        ctx.step(u, v, 0.0, dt, 5)
        refs.append(torch.cat([u, v]).cpu().numpy())
        ctx.close()
    batch = gdg.Batch([b[0] for b in built])
    dts = [b[2] for b in built]
    for shape in (None, (0, 1, 1), (1, 2, 2), (2, 3, 1)):
        if shape is not None:
            batch.set_tuning(*shape)
        us = [torch.tensor(b[1], device="cuda") for b in built]
        vs = [torch.zeros_like(u) for u in us]
        batch.step(us, vs, dts, 5)
        if shape is None:
            assert batch.tuning()["tile_elements"] == {7: 64 // 16, 9: 128 // 20}[N]
        for i, ref in enumerate(refs):
            a = torch.cat([us[i], vs[i]]).cpu().numpy()
            assert np.abs(a - ref).max() <= 1e-15 * np.abs(ref).max(), (shape, i)
    batch.close()
