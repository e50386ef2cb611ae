"""Small seeded workloads of each kernel family, for profiling and timing.

python -m paper_2105_01722_gb300.cases const [--n 64] [--p 5] [--steps 8] [--variant -1|0|1|2]
python -m paper_2105_01722_gb300.cases const3 [--n 16] [--p 5] [--steps 8]
python -m paper_2105_01722_gb300.cases var   [--n 32] [--p 5] [--steps 2] [--mixed | --inverse]
python -m paper_2105_01722_gb300.cases batch [--problems 12] [--steps 2] [--mixed | --inverse] [--pin B,R,C]
python -m paper_2105_01722_gb300.cases mlp   [--rows 4096] [--steps 4]

Each case builds its inputs with `inputs`, runs a few warm-up calls, then the
timed calls, and prints one JSON line (milliseconds from CUDA events on the
launching stream).  The sizes are chosen so that a profiler capture of one
launch stays small (a few hundred MB on the device at most).
"""
import argparse
import json

import numpy as np

from . import gdg, inputs

CFL = {3: 0.2, 5: 0.15, 7: 0.12}


def _ms(fn):
    import torch
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def case_const(n=64, N=8, p=5, steps=8, warmup=2, variant=-1):
    """2-D constant coefficient standing mode, n x n elements, modal route
    (variant: stage kernel, -1 timed choice, 0 one line per thread, 1 two
    threads per line, 2 one thread per line and field)."""
    import torch
    pb = gdg.make_problem(2, (n, n), N, p, flux=gdg.FLUX_UPWIND, c2=1.0)
    ctx = gdg.Context(pb)
    if variant >= 0:
        ctx.set_stage_variant(variant)
    X, Y = inputs.cartesian_nodes((n, n), N)
    U0, V0 = inputs.standing_mode_2d(X, Y)
    u = torch.tensor(U0.ravel(), device="cuda")
    v = torch.tensor(V0.ravel(), device="cuda")
    dt = CFL[p] / (n * N)
    ctx.step(u, v, 0.0, dt, warmup)
    ms = _ms(lambda: ctx.step(u, v, 0.0, dt, steps))
    chosen = ctx.stage_variant()
    ctx.close()
    dof = n * n * (N + 1) ** 2
    return {"case": "const", "n": n, "N": N, "p": p, "steps": steps, "variant": chosen, "ms": ms,
            "dof_steps_per_s": dof * steps / (ms / 1e3)}


def case_const3(n=16, N=8, p=5, steps=8, warmup=2):
    """3-D constant coefficient standing mode sin(pi x) sin(pi y) sin(pi z),
    n^3 elements, modal route, upwind, Dirichlet."""
    import torch
    pb = gdg.make_problem(3, (n, n, n), N, p, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                          bc=(gdg.BC_DIRICHLET,) * 3, flux=gdg.FLUX_UPWIND, c2=1.0)
    ctx = gdg.Context(pb)
    X, Y, Z = inputs.cartesian_nodes_3d((n, n, n), N)
    u = torch.tensor((np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)).ravel(), device="cuda")
    v = torch.zeros_like(u)
    dt = 0.1 / (n * N)
    ctx.step(u, v, 0.0, dt, warmup)
    ms = _ms(lambda: ctx.step(u, v, 0.0, dt, steps))
    ctx.close()
    dof = n ** 3 * (N + 1) ** 3
    return {"case": "const3", "n": n, "N": N, "p": p, "steps": steps, "ms": ms,
            "dof_steps_per_s": dof * steps / (ms / 1e3)}


def case_var(n=32, N=8, p=5, steps=2, warmup=1, mixed=False, inverse=False):
    """Sine-mapped mesh, c^2 = 1 + 0.5 sin 2pi x cos 2pi y, Gaussian pulse,
    element PCG to rtol 1e-10 (inverse: precomputed element inverses)."""
    import torch
    X, Y = inputs.mapped_nodes((n, n), N, 0.05)
    C2 = inputs.c2_sine(X, Y)
    prec = gdg.MIXED if mixed else gdg.FP64
    pb = gdg.make_problem(2, (n, n), N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                          pcg_rtol=1e-10, pcg_maxit=100, precision=prec,
                          solver=gdg.SOLVE_INVERSE if inverse else gdg.SOLVE_PCG)
    ctx = gdg.Context(pb)
    u = torch.tensor(inputs.gaussian_pulse(X, Y, 0.5, 0.5, 0.05).ravel(), device="cuda")
    v = torch.zeros_like(u)
    dt = 0.1 / (n * N) / np.sqrt(1.5)
    ctx.step(u, v, 0.0, dt, warmup)
    ctx.step_stats()
    ms = _ms(lambda: ctx.step(u, v, 0.0, dt, steps))
    su, sv = ctx.step_stats()
    ctx.close()
    dof = n * n * (N + 1) ** 2
    return {"case": "var", "n": n, "N": N, "p": p, "mixed": mixed, "inverse": inverse, "steps": steps, "ms": ms,
            "dof_steps_per_s": dof * steps / (ms / 1e3), "pcg_u_mean_iters": su["mean_iters"],
            "pcg_v_mean_iters": sv["mean_iters"]}


def case_batch(problems=12, steps=2, warmup=1, mixed=False, sequential=False, pmax=7, inverse=False, pin=None):
    """The seeded mixed batch of `inputs.batched_problems` (sizes, orders,
    constant / variable c^2), advanced by one Batch (sequential: each problem
    by its own gdg_step, one after another on one stream); pmax drops the
    problems of higher order; pin = (register budget, blocks per SM, items
    per turn) fixes the launch shape instead of tuning it."""
    import torch
    specs = [sp for sp in inputs.batched_problems(problems) if sp["p"] <= pmax]
    prec = gdg.MIXED if mixed else gdg.FP64
    solver = gdg.SOLVE_INVERSE if inverse else gdg.SOLVE_PCG
    pbs, us, dts = [], [], []
    for sp in specs:
        n, p = sp["n"], sp["p"]
        X, Y = inputs.cartesian_nodes((n, n), 8)
        if sp["variable"]:
            C2 = inputs.smooth_random_c2(X, Y, sp["seed"])
            pbs.append(gdg.make_problem(2, (n, n), 8, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y,
                                        c2_nodes=C2, pcg_rtol=1e-10, pcg_maxit=100, precision=prec,
                                        solver=solver))
            cmax = float(np.sqrt(C2.max()))
        else:
            pbs.append(gdg.make_problem(2, (n, n), 8, p, c2=1.0))
            cmax = 1.0
        us.append(torch.tensor(inputs.gaussian_pulse(X, Y, sp["x0"], sp["y0"], 0.05).ravel(), device="cuda"))
        dts.append(CFL[p] / (n * 8) / cmax)
    vs = [torch.zeros_like(u) for u in us]
    dof = sum(sp["n"] ** 2 * 81 for sp in specs)
    out = {"case": "batch", "problems": len(specs), "mixed": mixed, "inverse": inverse, "sequential": sequential,
           "steps": steps}
    if sequential:
        ctxs = [gdg.Context(pb) for pb in pbs]
        run = lambda k: [c.step(u, v, 0.0, d, k) for c, u, v, d in zip(ctxs, us, vs, dts)]
        run(warmup)
        ms = _ms(lambda: run(steps))
        for c in ctxs:
            c.close()
    else:
        batch = gdg.Batch(pbs)
        if pin:
            batch.set_tuning(*pin)
        batch.step(us, vs, dts, warmup)
        ms = _ms(lambda: batch.step(us, vs, dts, steps))
        out["tuning"] = batch.tuning()
        batch.close()
    out.update(ms=ms, dof_steps_per_s=dof * steps / (ms / 1e3))
    return out


def case_mlp(rows=4096, steps=4, batch=256, seed=5):
    """Forward over `rows` seeded feature rows and `steps` minibatch
    backward + Adam updates."""
    import torch
    from .learned import glorot_params
    rng = np.random.default_rng(seed)
    X = torch.tensor(rng.standard_normal((rows, gdg.MLP_IN)).astype(np.float32), device="cuda")
    T = torch.tensor(rng.standard_normal((rows, gdg.MLP_OUT)).astype(np.float32), device="cuda")
    Y = torch.empty_like(T)
    net = gdg.Mlp(glorot_params(seed))
    net.forward(X, Y)
    idx = torch.arange(batch, dtype=torch.int32, device="cuda")

    def train():
        for _ in range(steps):
            net.backward(X, T, idx)
            net.adam(1e-3)
    ms_f = _ms(lambda: net.forward(X, Y))
    ms_t = _ms(train)
    return {"case": "mlp", "rows": rows, "forward_ms": ms_f, "train_steps": steps,
            "train_ms_per_step": ms_t / steps}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("case", choices=["const", "const3", "var", "batch", "mlp"])
    ap.add_argument("--n", type=int)
    ap.add_argument("--p", type=int, default=5)
    ap.add_argument("--steps", type=int)
    ap.add_argument("--mixed", action="store_true")
    ap.add_argument("--inverse", action="store_true", help="var: precomputed element inverses")
    ap.add_argument("--problems", type=int, default=12)
    ap.add_argument("--rows", type=int, default=4096)
    ap.add_argument("--sequential", action="store_true")
    ap.add_argument("--pmax", type=int, default=7)
    ap.add_argument("--variant", type=int, default=-1, help="const: stage kernel (-1 timed, 0, 1, 2)")
    ap.add_argument("--pin", help="batch: register budget, blocks per SM, items per turn (e.g. 1,5,1)")
    a = ap.parse_args(argv)
    kw = {"steps": a.steps} if a.steps else {}
    if a.case == "const":
        r = case_const(n=a.n or 64, p=a.p, variant=a.variant, **kw)
    elif a.case == "const3":
        r = case_const3(n=a.n or 16, p=a.p, **kw)
    elif a.case == "var":
        r = case_var(n=a.n or 32, p=a.p, mixed=a.mixed, inverse=a.inverse, **kw)
    elif a.case == "batch":
        pin = tuple(int(x) for x in a.pin.split(",")) if a.pin else None
        r = case_batch(problems=a.problems, mixed=a.mixed, sequential=a.sequential, pmax=a.pmax,
                       inverse=a.inverse, pin=pin, **kw)
    else:
        r = case_mlp(rows=a.rows, **kw)
    print(json.dumps(r))


if __name__ == "__main__":
    main()
