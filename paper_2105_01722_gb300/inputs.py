"""Seeded synthetic inputs for the wave-equation workloads.

Holds no arithmetic of the method: only where the nodes sit, what the
caller samples there (initial data, c^2, mapped coordinates) and seeded
random states.  Shared by the tests, the benchmark and the oracle checks.

Nodal layout everywhere: 1-D [e, i]; 2-D [ey, ex, j, i] (i along x),
element e = ey*nx + ex, node (i, j) of an element at
(x0 + i*Hx/N, y0 + j*Hy/N).
"""
import numpy as np

SEED0 = 20210501


def cartesian_nodes_3d(n, N, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    """GD node coordinates (x, y, z), each [ez, ey, ex, k, j, i], of a uniform
    Cartesian 3-D mesh of n = (nx, ny, nz) elements."""
    n1 = N + 1
    r = np.arange(n1) / N
    shape = (n[2], n[1], n[0], n1, n1, n1)
    out = []
    for d, (ax_e, ax_n) in enumerate(((2, 5), (1, 4), (0, 3))):
        H = (hi[d] - lo[d]) / n[d]
        es = [1] * 6
        es[ax_e] = n[d]
        ns = [1] * 6
        ns[ax_n] = n1
        out.append(np.broadcast_to(lo[d] + H * (np.arange(n[d]).reshape(es) + r.reshape(ns)), shape).copy())
    return tuple(out)


def cartesian_nodes(n, N, lo=(0.0, 0.0), hi=(1.0, 1.0)):
    """GD node coordinates of every element of a uniform Cartesian mesh."""
    n1 = N + 1
    r = np.arange(n1) / N
    if len(n) == 1:
        H = (hi[0] - lo[0]) / n[0]
        return (lo[0] + H * (np.arange(n[0])[:, None] + r[None, :]),)
    nx, ny = n
    Hx = (hi[0] - lo[0]) / nx
    Hy = (hi[1] - lo[1]) / ny
    xs = lo[0] + Hx * (np.arange(nx)[:, None] + r[None, :])
    ys = lo[1] + Hy * (np.arange(ny)[:, None] + r[None, :])
    X = np.broadcast_to(xs[None, :, None, :], (ny, nx, n1, n1)).copy()
    Y = np.broadcast_to(ys[:, None, :, None], (ny, nx, n1, n1)).copy()
    return X, Y


def sine_map(XI, ETA, amp=0.05):
    """x = xi + amp sin(2 pi xi) sin(2 pi eta), y = eta (maps the unit
    square onto itself; orientation preserving for amp < 1/(2 pi))."""
    return XI + amp * np.sin(2 * np.pi * XI) * np.sin(2 * np.pi * ETA), ETA.copy()


def mapped_nodes(n, N, amp=0.05):
    XI, ETA = cartesian_nodes(n, N)
    return sine_map(XI, ETA, amp)


def c2_sine(X, Y):
    """c^2 = 1 + 0.5 sin(2 pi x) cos(2 pi y) (physical x, y)."""
    return 1.0 + 0.5 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)


def gaussian_pulse(X, Y, x0=0.5, y0=0.5, width=0.05):
    return np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / width ** 2)


def smooth_random_c2(X, Y, seed, degree=3):
    """c^2 = 2^s(x,y) with s a seeded random trigonometric polynomial of
    degree <= `degree`, scaled so that max |s| = 1 on a fine grid
    (so c^2 lies in [1/2, 2])."""
    rng = np.random.default_rng(seed)
    coef = rng.standard_normal((degree + 1, degree + 1, 4))
    def s_of(x, y):
        s = np.zeros_like(x)
        for a in range(degree + 1):
            for b in range(degree + 1):
                ca, sa = np.cos(2 * np.pi * a * x), np.sin(2 * np.pi * a * x)
                cb, sb = np.cos(2 * np.pi * b * y), np.sin(2 * np.pi * b * y)
                k = coef[a, b]
                s = s + k[0] * ca * cb + k[1] * ca * sb + k[2] * sa * cb + k[3] * sa * sb
        return s
    g = np.linspace(0.0, 1.0, 97)
    GX, GY = np.meshgrid(g, g)
    scale = np.abs(s_of(GX, GY)).max()
    return 2.0 ** (s_of(X, Y) / scale)


def random_state(shape, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal(shape)


def standing_wave_1d(X, t=0.0):
    """u = cos(2 pi t) sin(2 pi x): (u, v) at time t."""
    w = 2 * np.pi
    return np.cos(w * t) * np.sin(w * X), -w * np.sin(w * t) * np.sin(w * X)


def standing_mode_2d(X, Y, t=0.0):
    """u = cos(sqrt2 pi t) sin(pi x) sin(pi y): (u, v) at time t."""
    w = np.sqrt(2.0) * np.pi
    s = np.sin(np.pi * X) * np.sin(np.pi * Y)
    return np.cos(w * t) * s, -w * np.sin(w * t) * s


def batched_problems(count=48, seed0=SEED0, nmin=16, nmax=128):
    """Uneven independent problems: per problem a square element grid with
    n ~ U{nmin..nmax}, p ~ U{3,5,7}, alternating constant / smooth random
    c^2, pulse centre ~ U[0.3, 0.7]^2, width 0.05."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.integers(nmin, nmax + 1))
        p = int(rng.choice([3, 5, 7]))
        x0, y0 = rng.uniform(0.3, 0.7, size=2)
        out.append(dict(n=n, p=p, variable=bool(i % 2), x0=float(x0), y0=float(y0),
                        seed=seed0 + i))
    return out
