"""Determinism, checkpoint / resume and fault reporting through the C ABI.

* Repeated runs are bitwise equal (a cheap race detector: the kernels use no
  atomics whose order reaches the result, and reductions have a fixed
  order), for every form: modal route (2-D and 3-D), FP64 and mixed PCG,
  element inverses, learned guess, the batched launch.
* A run checkpointed to disk and resumed in a new context continues exactly
  as the uninterrupted run with the same call boundaries.
* Faults are injected on the host and reported as status codes: a NaN in
  the state gives GDG_ENONFINITE from gdg_energy; a one-iteration PCG limit
  gives GDG_ENOCONV with the iterates kept; bad arguments give GDG_EINVAL; a
  wait limit too short for the persistent step's waits between stages
  gives GDG_ETIMEOUT, and the context then steps correctly with a normal
  limit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2105_01722_gb300 import checkpoint, gdg, inputs, learned


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    gdg.lib()


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a).ravel(), dtype=torch.float64, device="cuda")


def _var_kwargs(n=6, p=5, **extra):
    X, Y = inputs.mapped_nodes((n, n), 8, 0.05)
    C2 = inputs.c2_sine(X, Y)
    kw = dict(dim=2, n=(n, n), N=8, p=p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
              pcg_rtol=1e-10, pcg_maxit=100)
    kw.update(extra)
    return kw, X, Y


FORMS = {
    "const2d": lambda: (dict(dim=2, n=(7, 5), N=8, p=5, bc=(gdg.BC_PERIODIC, gdg.BC_DIRICHLET)), 2),
    "const3d": lambda: (dict(dim=3, n=(3, 2, 2), N=6, p=5, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                             bc=(gdg.BC_DIRICHLET, gdg.BC_PERIODIC, gdg.BC_DIRICHLET)), 3),
    "var_fp64": lambda: (_var_kwargs()[0], 2),
    "var_mixed": lambda: (_var_kwargs(precision=gdg.MIXED)[0], 2),
    "var_inverse": lambda: (_var_kwargs(solver=gdg.SOLVE_INVERSE)[0], 2),
}


def _run(kw, nsteps, seed=3, net=None):
    ctx = gdg.Context(gdg.make_problem(**kw))
    if net is not None:
        ctx.mlp_attach(net)
    U = inputs.random_state(ctx.n, seed)
    V = inputs.random_state(ctx.n, seed + 1)
    u, v = _dev(U), _dev(V)
    ctx.step(u, v, 0.0, 2e-4, nsteps)
    out = np.concatenate([u.cpu().numpy(), v.cpu().numpy()])
    ctx.close()
    return out


@pytest.mark.parametrize("form", sorted(FORMS))
def test_repeated_runs_are_bitwise_equal(form):
    kw, _ = FORMS[form]()
    a, b = _run(kw, 19), _run(kw, 19)
    assert np.array_equal(a, b)


def test_learned_guess_is_bitwise_repeatable():
    kw, _, _ = _var_kwargs()
    net = gdg.Mlp(learned.glorot_params(3))
    assert np.array_equal(_run(kw, 6, net=net), _run(kw, 6, net=net))


def test_batched_launch_is_bitwise_repeatable():
    specs = inputs.batched_problems(count=6, nmin=3, nmax=9)
    pbs, U0 = [], []
    for sp in specs:
        n, p = sp["n"], sp["p"]
        X, Y = inputs.cartesian_nodes((n, n), 8)
        if sp["variable"]:
            pbs.append(gdg.make_problem(2, (n, n), 8, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y,
                                        c2_nodes=inputs.smooth_random_c2(X, Y, sp["seed"])))
        else:
            pbs.append(gdg.make_problem(2, (n, n), 8, p, c2=1.0))
        U0.append(inputs.gaussian_pulse(X, Y, sp["x0"], sp["y0"], 0.05).ravel())
    outs = []
    for _ in range(2):
        batch = gdg.Batch(pbs)
        us = [_dev(a) for a in U0]
        vs = [torch.zeros_like(u) for u in us]
        batch.step(us, vs, [1e-3] * len(us), 9)
        outs.append(np.concatenate([torch.cat([u, v]).cpu().numpy() for u, v in zip(us, vs)]))
        batch.close()
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("form", ["const2d", "const3d", "var_fp64"])
def test_checkpoint_resume_matches_uninterrupted(form, tmp_path):
    kw, _ = FORMS[form]()
    dt, n1, n2 = 2e-4, 5, 17
    ctx = gdg.Context(gdg.make_problem(**kw))
    U = inputs.random_state(ctx.n, 9)
    V = inputs.random_state(ctx.n, 10)
    # uninterrupted: the same two calls on one context
    u, v = _dev(U), _dev(V)
    ctx.step(u, v, 0.0, dt, n1)
    ctx.step(u, v, n1 * dt, dt, n2)
    ref = np.concatenate([u.cpu().numpy(), v.cpu().numpy()])
    ctx.close()
    # first leg, checkpoint, resume in a new context from the file alone
    ctx = gdg.Context(gdg.make_problem(**kw))
    u, v = _dev(U), _dev(V)
    ctx.step(u, v, 0.0, dt, n1)
    checkpoint.save(tmp_path / "run.npz", u, v, n1 * dt, n1, kw)
    ctx.close()
    del u, v
    U1, V1, t1, s1, kw1 = checkpoint.load(tmp_path / "run.npz")
    assert s1 == n1 and t1 == n1 * dt
    ctx = gdg.Context(checkpoint.make_problem(kw1))
    u, v = _dev(U1), _dev(V1)
    ctx.step(u, v, t1, dt, n2)
    out = np.concatenate([u.cpu().numpy(), v.cpu().numpy()])
    ctx.close()
    assert np.array_equal(out, ref)


def test_nan_in_state_is_reported_by_energy():
    ctx = gdg.Context(gdg.make_problem(2, (4, 4), 8, 5))
    U = inputs.random_state(ctx.n, 1)
    U[17] = np.nan
    u, v = _dev(U), torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    with pytest.raises(gdg.GdgError) as err:
        ctx.energy(u, v)
    assert err.value.status == gdg.ENONFINITE
    # the context stays usable
    assert np.isfinite(ctx.energy(torch.zeros_like(v), v))
    ctx.close()


def test_one_iteration_limit_reports_noconv():
    kw, _, _ = _var_kwargs(pcg_maxit=1, pcg_rtol=1e-14)
    ctx = gdg.Context(gdg.make_problem(**kw))
    b = _dev(inputs.random_state(ctx.n, 4))
    x = torch.zeros_like(b)
    with pytest.raises(gdg.GdgError) as err:
        ctx.pcg(gdg.OP_S, b, x)
    assert err.value.status == gdg.ENOCONV
    assert torch.isfinite(x).all() and x.abs().sum() > 0    # the iterate is kept
    ctx.close()


def test_wait_limit_reports_timeout():
    """Between stages each block of the persistent step waits for the blocks
    holding its face neighbours; with a 1 ns wait limit the first block that
    has to wait gives up, every block leaves the kernel and gdg_step returns
    GDG_ETIMEOUT.  With the default limit the same context then advances the
    state exactly as the per-stage kernel does."""
    kw = dict(dim=2, n=(12, 10), N=8, p=5, bc=(gdg.BC_DIRICHLET, gdg.BC_PERIODIC))
    ctx = gdg.Context(gdg.make_problem(**kw))
    ctx.set_stage_variant(3)
    U = inputs.random_state(ctx.n, 8)
    V = inputs.random_state(ctx.n, 9)
    u, v = _dev(U), _dev(V)
    ctx.set_wait_limit(1e-9)
    with pytest.raises(gdg.GdgError) as err:
        ctx.step(u, v, 0.0, 2e-4, 64)
    assert err.value.status == gdg.ETIMEOUT
    with pytest.raises(gdg.GdgError):
        ctx.set_wait_limit(0.0)
    ctx.set_wait_limit(1.0)
    u, v = _dev(U), _dev(V)
    ctx.step(u, v, 0.0, 2e-4, 20)
    ref = gdg.Context(gdg.make_problem(**kw))
    ref.set_stage_variant(0)
    ur, vr = _dev(U), _dev(V)
    ref.step(ur, vr, 0.0, 2e-4, 20)
    assert torch.equal(u, ur) and torch.equal(v, vr)
    ref.close()
    ctx.close()
