"""Placement of independent problems on ranks (one process per GPU).

Independent problems share nothing on the data path, so a multi-GPU run of
a batch gives every rank a subset and needs no collective except the
max-over-ranks time of the benchmark.  `partition` balances an estimate of
each problem's work (greedy longest-first onto the least-loaded rank); it is
deterministic, so every rank computes the same placement without talking.
"""


def work_estimate(spec, N=8):
    """Relative cost of one RK4 step of a problem from `inputs.batched_problems`:
    elements x per-element cost (an element PCG stage costs about 40x a
    modal-route element stage at N = 8)."""
    elements = spec["n"] * spec["n"]
    per_element = 40.0 if spec.get("variable") else 1.0
    return elements * per_element * (N + 1) ** 2 / 81.0


def partition(specs, world, cost=work_estimate):
    """List of `world` lists of problem indices: disjoint, covering, each
    sorted; greedy longest-processing-time-first (ties by index)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(specs)), key=lambda i: (-cost(specs[i]), i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += cost(specs[i])
    return [sorted(x) for x in out]


def max_over_ranks(value):
    """Maximum of a float over the ranks of the default process group (the
    value itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# One mesh over several ranks: bands of element rows and the halo exchange
# between neighbouring bands (the elements couple only through the fluxes of
# shared faces, so a band needs its neighbours' boundary-row face traces
# before every RK stage; the library packs and unpacks them, the exchange
# below moves them between ranks).

def row_bands(ny, world):
    """Contiguous bands [(row0, row1)] of ny element rows over `world` ranks,
    sizes differing by at most one (the larger ones first)."""
    if world < 1 or ny < world:
        raise ValueError("need 1 <= world <= ny")
    base, extra = divmod(ny, world)
    out, r = [], 0
    for k in range(world):
        n = base + (1 if k < extra else 0)
        out.append((r, r + n))
        r += n
    return out


def band_problem(make_problem, rank, world, dim, n, N, p, lo=(0.0, 0.0), hi=(1.0, 1.0),
                 bc=(0, 0), **kw):
    """The problem of rank `rank`'s band of a 2-D constant-coefficient mesh
    of n = (nx, ny) elements on [lo, hi] split by rows: the whole mesh's
    description with `rows` set to the band (so every band builds exactly the
    element operators of the whole mesh), halo sides towards the neighbouring
    bands.  A periodic y direction is not split (the exchange would pair a
    rank with itself or send two buffers to one neighbour)."""
    if dim != 2:
        raise ValueError("bands of rows: 2-D meshes only")
    if world > 1 and bc[1] != 0:
        raise ValueError("a periodic y direction cannot be split into bands")
    r0, r1 = row_bands(n[1], world)[rank]
    pb = make_problem(2, n, N, p, lo=lo, hi=hi, bc=bc, rows=(r0, r1), **kw)
    return pb, (r0, r1)


class HaloExchange:
    """Moves the halo buffers of rank `rank` (lower side to rank - 1, upper
    side to rank + 1) through torch.distributed point-to-point operations of
    the default group.  On NCCL the device buffers go directly (stream
    ordered: the operations wait for the pack kernel and the unpack kernel
    waits for them); on gloo they go through host copies.  Call it with the
    cudaStream_t (as an int) the library passes; `device=False` runs it on
    host tensors only (no GPU), for tests of the routing."""

    def __init__(self, rank, world, send_lo, send_hi, recv_lo, recv_hi, device=True):
        import torch.distributed as dist
        self.rank, self.world = rank, world
        self.bufs = (send_lo, send_hi, recv_lo, recv_hi)
        self.nccl = dist.get_backend() == "nccl"
        self.device = device

    def _ops(self, send_lo, send_hi, recv_lo, recv_hi):
        import torch.distributed as dist
        ops = []
        if self.rank > 0:
            ops.append(dist.P2POp(dist.isend, send_lo, self.rank - 1))
            ops.append(dist.P2POp(dist.irecv, recv_lo, self.rank - 1))
        if self.rank < self.world - 1:
            ops.append(dist.P2POp(dist.isend, send_hi, self.rank + 1))
            ops.append(dist.P2POp(dist.irecv, recv_hi, self.rank + 1))
        return ops

    def _run(self, send_lo, send_hi, recv_lo, recv_hi):
        import torch.distributed as dist
        ops = self._ops(send_lo, send_hi, recv_lo, recv_hi)
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()

    def __call__(self, stream=None):
        import torch
        send_lo, send_hi, recv_lo, recv_hi = self.bufs
        if self.nccl or not self.device:
            if self.device and stream is not None:
                with torch.cuda.stream(torch.cuda.ExternalStream(stream)):
                    self._run(send_lo, send_hi, recv_lo, recv_hi)
            else:
                self._run(send_lo, send_hi, recv_lo, recv_hi)
            return
        # gloo: host copies (the copies wait for the pack kernel on `stream`)
        ctx = torch.cuda.stream(torch.cuda.ExternalStream(stream)) if stream is not None else None
        if ctx is not None:
            ctx.__enter__()
        try:
            host = [None if t is None else t.cpu() for t in (send_lo, send_hi, recv_lo, recv_hi)]
            self._run(*host)
            for dev_t, h in ((recv_lo, host[2]), (recv_hi, host[3])):
                if dev_t is not None:
                    dev_t.copy_(h)
        finally:
            if ctx is not None:
                ctx.__exit__(None, None, None)
