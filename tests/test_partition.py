"""One mesh over several ranks (host side, CPU): bands of element rows
cover the mesh with the mesh's own element size and the right halo sides,
and the halo exchange routes each rank's lower-side buffer to the rank
below and its upper-side buffer to the rank above, over world_size 2 and 3
gloo groups (host tensors, no GPU)."""
import os
import socket

import pytest

from paper_2105_01722_gb300 import gdg, shard


def test_row_bands_cover_contiguous_balanced():
    for ny in (1, 5, 64, 129):
        for world in range(1, min(ny, 9) + 1):
            b = shard.row_bands(ny, world)
            assert len(b) == world and b[0][0] == 0 and b[-1][1] == ny
            assert all(b[k][1] == b[k + 1][0] for k in range(world - 1))
            sizes = [r1 - r0 for r0, r1 in b]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 1
    with pytest.raises(ValueError):
        shard.row_bands(3, 4)


def test_band_problems_describe_the_whole_mesh():
    """Every band carries the whole mesh's description (so the element
    operators are bit for bit those of the whole mesh) and its own rows."""
    n, lo, hi = (12, 10), (0.0, -1.0), (2.0, 1.5)
    world = 3
    covered = []
    for rank in range(world):
        pb, (r0, r1) = shard.band_problem(gdg.make_problem, rank, world, 2, n, 8, 5, lo=lo, hi=hi)
        assert tuple(pb.n_elem)[:2] == n and tuple(pb.lo)[:2] == lo and tuple(pb.hi)[:2] == hi
        assert (pb.rows[0], pb.rows[1]) == (r0, r1)
        assert pb.bc[1] == gdg.BC_DIRICHLET
        covered += list(range(r0, r1))
    assert covered == list(range(n[1]))
    pb, _ = shard.band_problem(gdg.make_problem, 0, 1, 2, n, 8, 5)
    assert (pb.rows[0], pb.rows[1]) == (0, n[1])
    with pytest.raises(ValueError):
        shard.band_problem(gdg.make_problem, 0, 2, 2, n, 8, 5, bc=(0, gdg.BC_PERIODIC))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 6
        send_lo = torch.full((n,), 10.0 * rank + 1, dtype=torch.float64)
        send_hi = torch.full((n,), 10.0 * rank + 2, dtype=torch.float64)
        recv_lo = torch.full((n,), -1.0, dtype=torch.float64)
        recv_hi = torch.full((n,), -1.0, dtype=torch.float64)
        ex = shard.HaloExchange(rank, world, send_lo if rank > 0 else None, send_hi if rank < world - 1 else None,
                                recv_lo if rank > 0 else None, recv_hi if rank < world - 1 else None, device=False)
        ex()
        q.put((rank, recv_lo.tolist(), recv_hi.tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_halo_exchange_routes_over_gloo(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, lo, hi in res:
        # the lower side receives the rank below's upper buffer, and so on
        assert lo == ([10.0 * (rank - 1) + 2] * 6 if rank > 0 else [-1.0] * 6)
        assert hi == ([10.0 * (rank + 1) + 1] * 6 if rank < world - 1 else [-1.0] * 6)
