"""Batched persistent launch (gdg_batch_*): every problem of a batch ends
exactly where its own gdg_step takes it (the stage bodies are shared), for
modal and PCG problems, p = 3, 5, 7, FP64 and mixed precision, through the
graph path and the remainder; the tuner reports its choice."""
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
    assert tun["tile_elements"] in (4, 7, 10, 14, 21, 28)
    assert tun["threads_per_block"] == 9 * tun["tile_elements"]
    assert tun["blocks_per_sm"] in (-1, -2) or tun["blocks_per_sm"] >= 1
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


def test_batch_rejects_mixed_cell_counts():
    pbs = [gdg.make_problem(2, (4, 4), 8, 3), gdg.make_problem(2, (4, 4), 9, 3)]
    with pytest.raises(gdg.GdgError):
        gdg.Batch(pbs)
