"""Learned initial guess for the element u_t solve (pattern layered on the
element PCG; the paper has no learned component).

Data: (features, target) rows generated by the method itself -- Cartesian
meshes with random smooth c^2 = 2^s in [1/2, 2], Gaussian pulses advanced by
gdg_step, element residuals r_u from gdg_residuals, converged solutions y of
(S_c2 + w w^T) y = r_u from gdg_pcg, rows from gdg_mlp_rows.
Training: minibatch Adam with the library's BF16 forward / backward / update
kernels.  Evaluation: PCG iterations of the u_t solves inside gdg_step with
and without the attached network.  Host code here only orchestrates calls.
"""
import numpy as np

from . import gdg, inputs

CFL = {3: 0.2, 5: 0.15, 7: 0.12}


def glorot_params(seed):
    """Glorot-uniform weights and zero biases in the library's parameter order."""
    rng = np.random.default_rng(seed)
    out = []
    for fan_in, fan_out in ((gdg.MLP_IN, gdg.MLP_HID), (gdg.MLP_HID, gdg.MLP_HID), (gdg.MLP_HID, gdg.MLP_OUT)):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        out.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
        out.append(np.zeros(fan_out))
    return np.concatenate(out).astype(np.float32)


def problem(n, N, p, seed, rtol=1e-10, maxit=200, precision=gdg.FP64):
    """Cartesian n x n mesh on [0,1]^2 with c^2 = 2^s(x,y), s a seeded smooth
    random trigonometric polynomial (c^2 in [1/2, 2])."""
    X, Y = inputs.cartesian_nodes((n, n), N)
    C2 = inputs.smooth_random_c2(X, Y, seed)
    pb = gdg.make_problem(2, (n, n), N, p, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y, c2_nodes=C2,
                          pcg_rtol=rtol, pcg_maxit=maxit, precision=precision)
    dt = CFL[p] / (n * N) / float(np.sqrt(C2.max()))
    return pb, X, Y, dt


def generate(rows, n=16, N=8, p=5, seed0=1000, snapshots=4, substeps=6, device="cuda", per_snapshot=None):
    """About `rows` training rows (features X [M,162], targets T [M,81], FP32);
    per_snapshot: keep a seeded random subset of at most that many elements
    of each snapshot (more c^2 fields for the same number of rows)."""
    import torch
    Xs, Ts = [], []
    total, k = 0, 0
    while total < rows:
        seed = seed0 + k
        k += 1
        pb, X, Y, dt = problem(n, N, p, seed, rtol=1e-12, maxit=400)
        ctx = gdg.Context(pb)
        rng = np.random.default_rng(seed)
        x0, y0 = rng.uniform(0.25, 0.75, size=2)
        width = rng.uniform(0.04, 0.12)
        u = torch.tensor(inputs.gaussian_pulse(X, Y, x0, y0, width).ravel(), device=device)
        v = torch.zeros_like(u)
        ne = ctx.n // 81
        for _ in range(snapshots):
            ctx.step(u, v, 0.0, dt, substeps)
            ru, rv = torch.empty_like(u), torch.empty_like(u)
            ctx.residuals(u, v, ru, rv)
            y = torch.zeros_like(u)
            ctx.pcg(gdg.OP_S, ru, y, allow_noconv=True)
            Xr = torch.empty(ne * gdg.MLP_IN, dtype=torch.float32, device=device)
            Tr = torch.empty(ne * gdg.MLP_OUT, dtype=torch.float32, device=device)
            ctx.mlp_rows(ru, y, Xr, Tr)
            Xr, Tr = Xr.view(ne, -1), Tr.view(ne, -1)
            keep = torch.nonzero(Xr[:, gdg.MLP_OUT:].abs().sum(dim=1) > 0).flatten()   # r_u = 0: no signal
            if per_snapshot is not None and keep.numel() > per_snapshot:
                pick = np.sort(rng.choice(keep.numel(), size=per_snapshot, replace=False))
                keep = keep[torch.tensor(pick, device=keep.device)]
            Xs.append(Xr[keep])
            Ts.append(Tr[keep])
            total += int(keep.numel())
        ctx.close()
    return torch.cat(Xs)[:rows].contiguous(), torch.cat(Ts)[:rows].contiguous()


def train(X, T, epochs=20, batch=256, lr=2e-3, seed=7, net=None, log=None):
    """Adam on the mean-squared error with the library's kernels; returns the
    network and the per-epoch mean training loss."""
    import torch
    net = net or gdg.Mlp(glorot_params(seed), device=X.device)
    rng = np.random.default_rng(seed)
    M = X.shape[0]
    history = []
    for ep in range(epochs):
        perm = torch.tensor(rng.permutation(M).astype(np.int32), device=X.device)
        acc, nb = 0.0, 0
        for b0 in range(0, M - batch + 1, batch):
            loss = net.backward(X, T, perm[b0:b0 + batch])
            net.adam(lr)
            acc += float(loss.item()) if (nb % 16 == 0) else 0.0
            nb += 1
        history.append(acc / max(1, (nb + 15) // 16))
        if log:
            log(ep, history[-1])
    return net, history


def relative_error(net, X, T):
    """Mean over rows of ||net(x) - t|| / ||t|| (FP32 forward)."""
    import torch
    Y = torch.empty_like(T)
    net.forward(X, Y)
    num = torch.linalg.norm(Y - T, dim=1)
    den = torch.linalg.norm(T, dim=1).clamp_min(1e-30)
    return float((num / den).mean())
