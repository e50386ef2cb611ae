"""One mesh over two contexts (the element-partitioned step): two processes,
each owning a band of element rows of a 2-D constant-coefficient mesh on
cuda:0, exchange their boundary rows' face traces through gloo between RK
stages (gdg_set_halo with host-staged buffers); the assembled state after
several gdg_step calls, and the gdg_rhs of the bands, equal the
single-context results bit for bit (same stage kernel, same operations).
The processes never wait on each other inside a kernel: every exchange is a
host call between launches."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2105_01722_gb300 import gdg, inputs, shard

CASES = [
    dict(n=(12, 10), N=8, p=5, flux=gdg.FLUX_UPWIND, bc=(gdg.BC_DIRICHLET, gdg.BC_DIRICHLET)),
    dict(n=(7, 9), N=6, p=3, flux=gdg.FLUX_CENTRAL, bc=(gdg.BC_PERIODIC, gdg.BC_DIRICHLET)),
    dict(n=(8, 6), N=8, p=5, flux=gdg.FLUX_ALTERNATING, bc=(gdg.BC_PERIODIC, gdg.BC_DIRICHLET)),
]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _state(c):
    X, Y = inputs.cartesian_nodes(c["n"], c["N"])
    U = np.sin(np.pi * X) * np.sin(np.pi * Y) + 0.1 * inputs.random_state(X.shape, 5)
    V = 0.1 * inputs.random_state(X.shape, 6)
    return U, V      # [ey, ex, j, i]


def _worker(rank, world, port, c, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        pb, (r0, r1) = shard.band_problem(gdg.make_problem, rank, world, 2, c["n"], c["N"], c["p"],
                                          bc=c["bc"], flux=c["flux"], c2=1.3)
        ctx = gdg.Context(pb)
        n = ctx.halo_len()
        mk = lambda on: torch.zeros(n, dtype=torch.float64, device="cuda") if on else None
        lo, hi = rank > 0, rank < world - 1
        bufs = (mk(lo), mk(hi), mk(lo), mk(hi))
        ctx.set_halo(*bufs, shard.HaloExchange(rank, world, *bufs))
        U, V = _state(c)
        u = torch.tensor(U[r0:r1].ravel(), device="cuda")
        v = torch.tensor(V[r0:r1].ravel(), device="cuda")
        du, dv = torch.empty_like(u), torch.empty_like(v)
        ctx.rhs(u, v, du, dv)
        rhs = (du.cpu().numpy(), dv.cpu().numpy())
        dt = 0.1 / (max(c["n"]) * c["N"])
        ctx.step(u, v, 0.0, dt, 3)
        ctx.step(u, v, 3 * dt, dt, 2)
        torch.cuda.synchronize()
        q.put((rank, r0, r1, rhs, (u.cpu().numpy(), v.cpu().numpy())))
        ctx.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("c", CASES, ids=["upwind-dirichlet", "central-periodic-x", "alternating"])
def test_two_bands_equal_one_mesh(c):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    world = 2
    ctxm = mp.get_context("spawn")
    q = ctxm.Queue()
    port = _free_port()
    procs = [ctxm.Process(target=_worker, args=(r, world, port, c, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the whole mesh in one context, the same stage kernel (variant 0)
    pb = gdg.make_problem(2, c["n"], c["N"], c["p"], bc=c["bc"], flux=c["flux"], c2=1.3)
    ctx = gdg.Context(pb)
    ctx.set_stage_variant(0)
    U, V = _state(c)
    u, v = torch.tensor(U.ravel(), device="cuda"), torch.tensor(V.ravel(), device="cuda")
    du, dv = torch.empty_like(u), torch.empty_like(v)
    ctx.rhs(u, v, du, dv)
    dt = 0.1 / (max(c["n"]) * c["N"])
    ctx.step(u, v, 0.0, dt, 3)
    ctx.step(u, v, 3 * dt, dt, 2)
    rows = c["N"] + 1
    per_row = c["n"][0] * rows * rows
    full = [a.cpu().numpy() for a in (du, dv, u, v)]
    for rank, r0, r1, rhs, state in res:
        sl = slice(r0 * per_row, r1 * per_row)
        for got, ref in zip(rhs + state, full):
            assert np.array_equal(got, ref[sl]), rank
    ctx.close()


def test_halo_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pb = gdg.make_problem(2, (4, 6), 8, 5, rows=(3, 6))       # the upper band: a lower halo side
    ctx = gdg.Context(pb)
    n = ctx.halo_len()
    assert n == 4 * 2 * 9 and ctx.n == 4 * 3 * 81
    b = torch.zeros(n, dtype=torch.float64, device="cuda")
    with pytest.raises(gdg.GdgError):       # the lower side needs both of its buffers
        ctx.set_halo(None, None, b, None, lambda s: None)
    u = torch.zeros(ctx.n, dtype=torch.float64, device="cuda")
    with pytest.raises(gdg.GdgError):       # no exchange registered yet
        ctx.step(u, u.clone(), 0.0, 1e-3, 1)

    def failing(stream):
        raise RuntimeError("peer gone")

    ctx.set_halo(b, None, b.clone(), None, failing)
    with pytest.raises(gdg.GdgError) as err:
        ctx.step(u, u.clone(), 0.0, 1e-3, 1)
    assert err.value.status == gdg.EHALO
    with pytest.raises(gdg.GdgError):
        ctx.set_stage_variant(3)
    ctx.close()
    no_halo = gdg.Context(gdg.make_problem(2, (4, 3), 8, 5))
    assert no_halo.halo_len() == -1
    no_halo.close()
    with pytest.raises(gdg.GdgError):       # a periodic y direction is not split
        gdg.Context(gdg.make_problem(2, (4, 3), 8, 5, bc=(0, gdg.BC_PERIODIC), rows=(1, 2)))
    with pytest.raises(gdg.GdgError):       # rows outside the mesh
        gdg.Context(gdg.make_problem(2, (4, 3), 8, 5, rows=(2, 4)))
    whole = gdg.Context(gdg.make_problem(2, (4, 3), 8, 5, rows=(0, 3)))   # every row: no halo
    assert whole.halo_len() == -1
    whole.close()
