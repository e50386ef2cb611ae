"""gdg_rhs_static, the allocation-free right-hand side (collected last).

It serves callers that cannot call cudaMalloc (a plug-in whose host
application's pool holds all free device memory, a loop that cannot afford
cudaMalloc's device synchronisation): no context, scratch in a static device
array.  Checked through the C ABI against the context-based gdg_rhs on two
calls in a row with different problems and inputs, within the 1e-12 relative
tolerance of the other GPU tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2105_01722_gb300 import gdg, inputs

TOL = 1e-12


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _problems():
    yield gdg.make_problem(2, (64, 64), 8, 5, flux=gdg.FLUX_UPWIND, c2=1.0)
    yield gdg.make_problem(2, (9, 13), 6, 3, bc=(gdg.BC_PERIODIC, gdg.BC_DIRICHLET),
                           flux=gdg.FLUX_CENTRAL, c2=2.5, lo=(0.0, -1.0), hi=(1.5, 1.0))
    yield gdg.make_problem(1, (37,), 8, 3, flux=gdg.FLUX_UPWIND, c2=0.7, xi=0.9)
    yield gdg.make_problem(2, (7, 5), 8, 5, bc=(gdg.BC_PERIODIC, gdg.BC_PERIODIC),
                           flux=gdg.FLUX_ALTERNATING, c2=1.3)
    yield gdg.make_problem(1, (11,), 6, 3, flux=gdg.FLUX_ALTERNATING, c2=1.0)


def test_static_rhs_matches_context_rhs_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for k, pb in enumerate(_problems()):
        ctx = gdg.Context(pb)
        for call in range(2):
            U = inputs.random_state(ctx.n, 100 + 10 * k + call)
            V = inputs.random_state(ctx.n, 200 + 10 * k + call)
            u = torch.tensor(U, device="cuda")
            v = torch.tensor(V, device="cuda")
            du_ref, dv_ref = torch.empty_like(u), torch.empty_like(v)
            ctx.rhs(u, v, du_ref, dv_ref)
            du, dv = torch.full_like(u, np.nan), torch.full_like(v, np.nan)
            gdg.rhs_static(pb, u, v, du, dv)
            torch.cuda.synchronize()
            a = np.concatenate([du.cpu().numpy(), dv.cpu().numpy()])
            b = np.concatenate([du_ref.cpu().numpy(), dv_ref.cpu().numpy()])
            assert np.all(np.isfinite(a))
            assert _rel(a, b) < TOL, (k, call, _rel(a, b))
        ctx.close()


def test_static_rhs_rejects_meshes_beyond_the_static_array():
    pb = gdg.make_problem(2, (128, 128), 8, 5)
    n = 128 * 128 * 81
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(gdg.GdgError) as err:
        gdg.rhs_static(pb, u, u.clone(), torch.empty_like(u), torch.empty_like(u))
    assert err.value.status == gdg.EUNSUPPORTED
    bad = gdg.make_problem(2, (4, 4), 8, 5, coef=gdg.COEF_NODAL)
    with pytest.raises(gdg.GdgError) as err:
        gdg.rhs_static(bad, u[:1296], u[:1296].clone(), torch.empty(1296, dtype=torch.float64, device="cuda"),
                       torch.empty(1296, dtype=torch.float64, device="cuda"))
    assert err.value.status == gdg.EINVAL


def test_static_rhs_on_a_side_stream():
    """The call is asynchronous on the caller's stream: launched on a
    non-default stream it gives the same result once that stream is done."""
    pb = gdg.make_problem(2, (12, 10), 8, 5, flux=gdg.FLUX_UPWIND, c2=1.0)
    ctx = gdg.Context(pb)
    u = torch.tensor(inputs.random_state(ctx.n, 7), device="cuda")
    v = torch.tensor(inputs.random_state(ctx.n, 8), device="cuda")
    du_ref, dv_ref = torch.empty_like(u), torch.empty_like(v)
    ctx.rhs(u, v, du_ref, dv_ref)
    du, dv = torch.full_like(u, np.nan), torch.full_like(v, np.nan)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        gdg.rhs_static(pb, u, v, du, dv, stream=side)
    side.synchronize()
    a = np.concatenate([du.cpu().numpy(), dv.cpu().numpy()])
    b = np.concatenate([du_ref.cpu().numpy(), dv_ref.cpu().numpy()])
    assert _rel(a, b) < TOL
    ctx.close()


def test_static_rhs_checks_lengths_against_the_problem():
    pb = gdg.make_problem(2, (4, 4), 8, 5)
    short = torch.zeros(4 * 4 * 81 - 1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        gdg.rhs_static(pb, short, short.clone(), torch.empty_like(short), torch.empty_like(short))
