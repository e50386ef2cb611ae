"""Every form of the library on small cases under the index-checking build
(run by tests/test_gpu_checks.py in a child process with GDG_CHECKS=1, so
that the binding loads libgdg_checks.so); prints one JSON line: the check
record after the self-test and after all the forms."""
import json
import os
import sys

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), ".."))

import numpy as np   # noqa: E402
import torch         # noqa: E402

from paper_2105_01722_gb300 import gdg, inputs   # noqa: E402


def _steps(pb, U, V, dt, k=3):
    ctx = gdg.Context(pb)
    u = torch.tensor(np.ascontiguousarray(U).ravel(), device="cuda")
    v = torch.tensor(np.ascontiguousarray(V).ravel(), device="cuda")
    ctx.step(u, v, 0.0, dt, k)
    du, dv = torch.empty_like(u), torch.empty_like(v)
    ctx.rhs(u, v, du, dv)
    torch.cuda.synchronize()
    ctx.close()


def main():
    out = {}
    gdg.check_status(reset=True)
    gdg.check_selftest(5, 3)            # fails: recorded as site 99
    gdg.check_selftest(2, 3)            # passes
    out["selftest"] = gdg.check_status(reset=True)
    # 1-D, both fluxes and a periodic side
    (X,) = inputs.cartesian_nodes((6,), 8)
    for flux in (gdg.FLUX_CENTRAL, gdg.FLUX_UPWIND):
        for bc in ((gdg.BC_DIRICHLET,), (gdg.BC_PERIODIC,)):
            U, V = inputs.standing_wave_1d(X)
            _steps(gdg.make_problem(1, (6,), 8, 3, flux=flux, bc=bc), U, V, 1e-3)
    # 2-D modal: every stage kernel, the three fluxes, periodic sides
    for n in ((5, 7), (16, 12)):
        X, Y = inputs.cartesian_nodes(n, 8)
        U = np.sin(np.pi * X) * np.sin(np.pi * Y) + 0.1 * inputs.random_state(X.shape, 3)
        V = 0.1 * inputs.random_state(X.shape, 4)
        for flux in (gdg.FLUX_CENTRAL, gdg.FLUX_UPWIND, gdg.FLUX_ALTERNATING):
            for bc in ((gdg.BC_DIRICHLET, gdg.BC_DIRICHLET), (gdg.BC_PERIODIC, gdg.BC_PERIODIC)):
                pb = gdg.make_problem(2, n, 8, 5, flux=flux, bc=bc, c2=1.2)
                for variant in (0, 1, 2, 3):
                    ctx = gdg.Context(pb)
                    try:
                        ctx.set_stage_variant(variant)
                    except gdg.GdgError:
                        ctx.close()
                        continue
                    u = torch.tensor(U.ravel(), device="cuda")
                    v = torch.tensor(V.ravel(), device="cuda")
                    ctx.step(u, v, 0.0, 1e-3, 3)
                    torch.cuda.synchronize()
                    ctx.close()
    # other cell counts and orders (odd N included)
    for N, p in ((6, 3), (7, 3), (9, 7)):
        X, Y = inputs.cartesian_nodes((5, 4), N)
        U = np.sin(np.pi * X) * np.sin(np.pi * Y)
        _steps(gdg.make_problem(2, (5, 4), N, p, flux=gdg.FLUX_UPWIND), U, 0 * U, 1e-3)
    # 3-D modal
    X, Y, Z = inputs.cartesian_nodes_3d((3, 4, 5), 8)
    U = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    for bc in ((gdg.BC_DIRICHLET,) * 3, (gdg.BC_PERIODIC,) * 3):
        _steps(gdg.make_problem(3, (3, 4, 5), 8, 5, bc=bc, flux=gdg.FLUX_UPWIND), U, 0 * U, 1e-3, 2)
    # variable coefficients on a mapped mesh: FP64 PCG, mixed, element inverses
    n = (6, 5)
    X, Y = inputs.mapped_nodes(n, 8, 0.05)
    C2 = inputs.c2_sine(X, Y)
    U = inputs.gaussian_pulse(X, Y, 0.5, 0.5, 0.2)
    for prec, solver in ((gdg.FP64, gdg.SOLVE_PCG), (gdg.MIXED, gdg.SOLVE_PCG), (gdg.FP64, gdg.SOLVE_INVERSE)):
        for bc in ((gdg.BC_DIRICHLET, gdg.BC_DIRICHLET), (gdg.BC_PERIODIC, gdg.BC_DIRICHLET)):
            pb = gdg.make_problem(2, n, 8, 5, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                                  precision=prec, solver=solver, bc=bc)
            _steps(pb, U, 0 * U, 1e-4)
    # a batch: constant and variable problems, every register budget
    pbs, us, vs, dts = [], [], [], []
    for sp in inputs.batched_problems(6, nmin=3, nmax=9):
        Xb, Yb = inputs.cartesian_nodes((sp["n"], sp["n"]), 8)
        if sp["variable"]:
            pbs.append(gdg.make_problem(2, (sp["n"], sp["n"]), 8, sp["p"], coef=gdg.COEF_NODAL, x_nodes=Xb,
                                        y_nodes=Yb, c2_nodes=inputs.smooth_random_c2(Xb, Yb, sp["seed"])))
        else:
            pbs.append(gdg.make_problem(2, (sp["n"], sp["n"]), 8, sp["p"]))
        us.append(torch.tensor(inputs.gaussian_pulse(Xb, Yb, sp["x0"], sp["y0"], 0.1).ravel(), device="cuda"))
        vs.append(torch.zeros_like(us[-1]))
        dts.append(1e-4)
    batch = gdg.Batch(pbs)
    batch.step(us, vs, dts, 2)
    for budget in (0, 1, 2):
        batch.set_tuning(budget, 1, 3)
        batch.step(us, vs, dts, 1)
    torch.cuda.synchronize()
    batch.close()
    out["forms"] = gdg.check_status(reset=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
