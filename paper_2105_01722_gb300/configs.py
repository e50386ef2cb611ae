"""Named presets of the five workloads the method is measured on.

Every input is synthetic and seeded (the paper's tests are manufactured
solutions; there is no dataset).  A preset returns a dict with

    name, description
    problems  list of gdg.Problem (host descriptions, ready for gdg.Context
              or gdg.Batch)
    states    list of (U0, V0) numpy arrays, one per problem (nodal, the
              library's element-major layout)
    dt        list of step sizes, one per problem
    steps     RK4 steps to the final time T (of the first problem)
    T         final time
    exact     callable t -> (U, V) of the first problem where the workload
              has an exact solution, else None

and takes keyword overrides of its sizes.  The presets only describe; every
step of the method runs in the library.

    standing_wave_1d   Section 6, Tables 1-2: u_tt = u_xx on [0,1], Dirichlet,
                       u = cos(2 pi t) sin(2 pi x); 16 elements of 8 cells,
                       p = 3; central or upwind flux; RK4 to T = 1 at CFL 0.5
    const_2d_64        Section 6, Tables 3-4: u_tt = Laplace u on [0,1]^2,
                       u = cos(sqrt2 pi t) sin(pi x) sin(pi y); 64 x 64
                       elements of 8 x 8 cells, p = 5; modified-basis route
    mapped_2d_128      Section 7.1: c^2 = 1 + 0.5 sin 2pi x cos 2pi y on the
                       sine-mapped square, 128 x 128 elements, p = 3 or 5,
                       Gaussian pulse of width 0.05, PCG to 1e-10, T = 0.25
    batched_48         48 independent problems, n ~ U{16..128}, p ~ U{3,5,7},
                       alternating constant / smooth random c^2
    learned_128        the learned-guess workload: 128 x 128 Cartesian mesh,
                       smooth random c^2 in [1/2, 2], p = 5, PCG to 1e-10
"""
import numpy as np

from . import gdg, inputs


def standing_wave_1d(n=16, N=8, p=3, flux=gdg.FLUX_CENTRAL, cfl=0.5, T=1.0):
    (X,) = inputs.cartesian_nodes((n,), N)
    h = 1.0 / (n * N)
    steps = int(round(T / (cfl * h)))
    pb = gdg.make_problem(1, (n,), N, p, flux=flux, c2=1.0)
    return dict(name="standing_wave_1d", description="1-D standing wave, %d elements of %d cells, p=%d" % (n, N, p),
                problems=[pb], states=[inputs.standing_wave_1d(X)], dt=[T / steps], steps=steps, T=T,
                exact=lambda t: inputs.standing_wave_1d(X, t))


def const_2d_64(n=64, N=8, p=5, flux=gdg.FLUX_UPWIND, cfl=0.15, T=1.0):
    X, Y = inputs.cartesian_nodes((n, n), N)
    h = 1.0 / (n * N)
    steps = int(round(T / (cfl * h)))
    pb = gdg.make_problem(2, (n, n), N, p, flux=flux, c2=1.0)
    return dict(name="const_2d_64",
                description="2-D constant coefficient, %dx%d elements of %dx%d cells, p=%d" % (n, n, N, N, p),
                problems=[pb], states=[inputs.standing_mode_2d(X, Y)], dt=[T / steps], steps=steps, T=T,
                exact=lambda t: inputs.standing_mode_2d(X, Y, t))


def mapped_2d_128(n=128, N=8, p=5, precision=gdg.FP64, solver=gdg.SOLVE_PCG, T=0.25, amp=0.05):
    X, Y = inputs.mapped_nodes((n, n), N, amp)
    C2 = inputs.c2_sine(X, Y)
    dt0 = 0.1 / (n * N) / np.sqrt(1.5)
    steps = int(round(T / dt0))
    pb = gdg.make_problem(2, (n, n), N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                          pcg_rtol=1e-10, pcg_maxit=100, precision=precision, solver=solver)
    U0 = inputs.gaussian_pulse(X, Y, 0.5, 0.5, 0.05)
    return dict(name="mapped_2d_128",
                description="2-D variable c^2 on the sine-mapped square, %dx%d elements, p=%d" % (n, n, p),
                problems=[pb], states=[(U0, np.zeros_like(U0))], dt=[T / steps], steps=steps, T=T, exact=None)


def batched_48(count=48, nmin=16, nmax=128, N=8, precision=gdg.FP64, solver=gdg.SOLVE_PCG, T=None):
    cfl = {3: 0.2, 5: 0.15, 7: 0.12}
    pbs, states, dts = [], [], []
    for sp in inputs.batched_problems(count, nmin=nmin, nmax=nmax):
        n, p = sp["n"], sp["p"]
        X, Y = inputs.cartesian_nodes((n, n), N)
        if sp["variable"]:
            C2 = inputs.smooth_random_c2(X, Y, sp["seed"])
            pbs.append(gdg.make_problem(2, (n, n), N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                                        pcg_rtol=1e-10, pcg_maxit=100, precision=precision, solver=solver))
            cmax = float(np.sqrt(C2.max()))
        else:
            pbs.append(gdg.make_problem(2, (n, n), N, p, c2=1.0))
            cmax = 1.0
        U0 = inputs.gaussian_pulse(X, Y, sp["x0"], sp["y0"], 0.05)
        states.append((U0, np.zeros_like(U0)))
        dts.append(cfl[p] / (n * N) / cmax)
    steps = 0 if T is None else int(round(T / dts[0]))
    return dict(name="batched_48", description="%d independent problems, n ~ U{%d..%d}" % (count, nmin, nmax),
                problems=pbs, states=states, dt=dts, steps=steps, T=T, exact=None)


def learned_128(n=128, N=8, p=5, seed=31337, precision=gdg.FP64, T=None):
    from . import learned
    pb, X, Y, dt = learned.problem(n, N, p, seed=seed, rtol=1e-10, precision=precision)
    U0 = inputs.gaussian_pulse(X, Y, 0.5, 0.5, 0.05)
    steps = 0 if T is None else int(round(T / dt))
    return dict(name="learned_128", description="%dx%d Cartesian mesh, smooth random c^2, p=%d" % (n, n, p),
                problems=[pb], states=[(U0, np.zeros_like(U0))], dt=[dt], steps=steps, T=T, exact=None)


PRESETS = {f.__name__: f for f in (standing_wave_1d, const_2d_64, mapped_2d_128, batched_48, learned_128)}


def preset(name, **overrides):
    """The preset `name` (a key of PRESETS) with keyword overrides."""
    if name not in PRESETS:
        raise KeyError("unknown preset %r (have %s)" % (name, ", ".join(PRESETS)))
    return PRESETS[name](**overrides)
