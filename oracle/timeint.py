"""Time stepping and error norms (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Classic four-stage fourth-order Runge-Kutta (used for every experiment of
Sections 3.3 and 6), and the two error measures of Section 6: the L2 error
||u - u_h|| and the energy-norm error (||grad(u - u_h)||^2 + ||v - v_h||^2)^1/2,
both by composite Gauss-Legendre quadrature with p+3 points per GD cell.
"""
import numpy as np

from . import gd_basis


def rk4_step(f, U, V, t, dt):
    """One classic RK4 step of d/dt (U, V) = f(t, U, V)."""
    k1 = f(t, U, V)
    k2 = f(t + 0.5 * dt, U + 0.5 * dt * k1[0], V + 0.5 * dt * k1[1])
    k3 = f(t + 0.5 * dt, U + 0.5 * dt * k2[0], V + 0.5 * dt * k2[1])
    k4 = f(t + dt, U + dt * k3[0], V + dt * k3[1])
    Un = U + dt / 6.0 * (k1[0] + 2.0 * k2[0] + 2.0 * k3[0] + k4[0])
    Vn = V + dt / 6.0 * (k1[1] + 2.0 * k2[1] + 2.0 * k3[1] + k4[1])
    return Un, Vn


def integrate(f, U, V, t0, dt, nsteps, callback=None):
    t = t0
    for s in range(nsteps):
        U, V = rk4_step(f, U, V, t, dt)
        t = t0 + (s + 1) * dt
        if callback is not None:
            callback(s + 1, t, U, V)
    return U, V


def errors(prob, U, V, exact, t, nq=None):
    """(L2 error of u, energy-norm error) against exact(t, *coords) which
    returns (u, [du/dx_k ...], v) evaluated at physical points."""
    p, N, n1 = prob.p, prob.N, prob.n1
    nq = p + 3 if nq is None else nq
    r, w, cell = gd_basis.quadrature_points(p, N, nq)
    B, D = gd_basis.basis_at_points(p, N, r, cell)
    if prob.dim == 1:
        H = prob.H(0)
        ne = prob.n[0]
        U = U.reshape(ne, n1)
        V = V.reshape(ne, n1)
        x = prob.lo[0] + H * (np.arange(ne)[:, None] + r[None, :])
        u, (ux,), v = exact(t, x)
        uh = U @ B.T
        uxh = U @ D.T / H
        vh = V @ B.T
        ww = H * w[None, :]
        l2 = np.sqrt(np.sum(ww * (u - uh) ** 2))
        en = np.sqrt(np.sum(ww * ((ux - uxh) ** 2 + (v - vh) ** 2)))
        return l2, en
    if prob.dim == 3:
        nx, ny, nz = prob.n
        Hx, Hy, Hz = prob.H(0), prob.H(1), prob.H(2)
        U = U.reshape(nz, ny, nx, n1, n1, n1)
        V = V.reshape(nz, ny, nx, n1, n1, n1)
        Q = len(r)
        xs = prob.lo[0] + Hx * (np.arange(nx)[:, None] + r[None, :])
        ys = prob.lo[1] + Hy * (np.arange(ny)[:, None] + r[None, :])
        zs = prob.lo[2] + Hz * (np.arange(nz)[:, None] + r[None, :])
        shape = (nz, ny, nx, Q, Q, Q)
        X = np.broadcast_to(xs[None, None, :, None, None, :], shape)
        Y = np.broadcast_to(ys[None, :, None, None, :, None], shape)
        Z = np.broadcast_to(zs[:, None, None, :, None, None], shape)
        u, (ux, uy, uz), v = exact(t, X, Y, Z)
        # point (c along z, b along y, a along x)
        ev = lambda A, Bz, By, Bx: np.einsum("ck,bj,ai,zyxkji->zyxcba", Bz, By, Bx, A)
        uh = ev(U, B, B, B)
        uxh = ev(U, B, B, D) / Hx
        uyh = ev(U, B, D, B) / Hy
        uzh = ev(U, D, B, B) / Hz
        vh = ev(V, B, B, B)
        ww = Hx * Hy * Hz * w[:, None, None] * w[None, :, None] * w[None, None, :]
        l2 = np.sqrt(np.sum(ww * (u - uh) ** 2))
        en = np.sqrt(np.sum(ww * ((ux - uxh) ** 2 + (uy - uyh) ** 2 + (uz - uzh) ** 2 + (v - vh) ** 2)))
        return l2, en
    nx, ny = prob.n
    Hx, Hy = prob.H(0), prob.H(1)
    U = U.reshape(ny, nx, n1, n1)
    V = V.reshape(ny, nx, n1, n1)
    xs = prob.lo[0] + Hx * (np.arange(nx)[:, None] + r[None, :])   # (nx, Q)
    ys = prob.lo[1] + Hy * (np.arange(ny)[:, None] + r[None, :])   # (ny, Q)
    X = np.broadcast_to(xs[None, :, None, :], (ny, nx, len(r), len(r)))
    Y = np.broadcast_to(ys[:, None, :, None], (ny, nx, len(r), len(r)))
    u, (ux, uy), v = exact(t, X, Y)
    # point (b along y, a along x): sum_{j,i} U[j,i] B[b,j] B[a,i]
    uh = np.einsum("bj,yxji,ai->yxba", B, U, B)
    uxh = np.einsum("bj,yxji,ai->yxba", B, U, D) / Hx
    uyh = np.einsum("bj,yxji,ai->yxba", D, U, B) / Hy
    vh = np.einsum("bj,yxji,ai->yxba", B, V, B)
    ww = Hx * Hy * w[:, None] * w[None, :]
    l2 = np.sqrt(np.sum(ww * (u - uh) ** 2))
    en = np.sqrt(np.sum(ww * ((ux - uxh) ** 2 + (uy - uyh) ** 2 + (v - vh) ** 2)))
    return l2, en
