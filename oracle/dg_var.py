"""Energy-DG for variable c^2 and mapped (curvilinear) 2-D elements (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 7 (and 7.1): for a variable speed of sound or a non-Cartesian element
the simultaneous diagonalisation no longer applies; the method keeps the
nodal GD basis and inverts the element matrices of Eqs. DG1 / DG2
iteratively by preconditioned CG.  The weak form is that of Eqs. DG1, DG2,
DG1_extra with the fluxes of Section 2.2.1, now with integrals evaluated by
quadrature on the reference element:

  M_J       = int phi_a phi_b |J|                                (volume)
  S_c2      = int c^2 (J^-T grad_r phi_a) . (J^-T grad_r phi_b) |J|
  r_u       = sum_faces int_face c^2 (n . grad phi_a) (v* - v_in) dS
  r_v       = -S_c2 U + sum_faces int_face c^2 phi_a q* dS
  S_c2 (dU/dt - V) = r_u,  w^T (dU/dt - V) = 0,  w = M_J 1 / |e|
  M_J dV/dt = r_v

Readings made here (the paper leaves them open):
* geometry and c^2 enter as samples at every element's GD nodes and are
  represented in the same GD space (isoparametric): x(r,s) =
  sum X[j,i] phi_i(r) phi_j(s), likewise y and c^2;
* quadrature: nq Gauss-Legendre points per GD cell per direction (default
  p+1, exact for affine elements with constant c^2);
* upwind splitting xi = c at each face point unless a constant xi > 0 is
  given; c^2 on a face is the inside element's trace;
* alternating flux (alpha = 1): sides labelled by a fixed orientation (side
  1 = the element with the smaller reference index across the face), so on
  an element's xm / ym face v* = v_out, q* = d_in and on its xp / yp face
  v* = v_in, q* = -d_out; on a Dirichlet side v* = 0, q* = d_in;
* the constrained u_t system is solved in the equivalent SPD form
  (S_c2 + w w^T) y = r_u (its solution satisfies S_c2 y = r_u, w^T y = 0
  because 1^T r_u = 0); the extra equation of Eq. DG1_extra is weighted by
  1/|e| (|e| = 1^T M_J 1, the element area), w = M_J 1 / |e|: any positive
  weight gives the same y, and this one keeps the rank-one term O(1) so
  rounding in the constant mode is not amplified by 1/|e|^2;
* PCG (element by element) stops when ||r||_2 <= rtol ||b||_2, tested
  before each iteration, or after maxit iterations; rz = 0 ends it;
* the IC(0) preconditioner of Section 7.1 ("of S_c2 and M"): S_c2 is
  singular, so the u_t system's factor is that of S_c2 + w w^T taken on the
  sparsity pattern of S_c2; the v_t system's is that of M_J on its own
  pattern;
* a distributed forcing f enters r_v as int phi_a f |J| (the load Eq. DG2
  omits; the variational statement carries it), by quadrature with p+3
  points per cell.

Layout of nodal arrays: [ey, ex, j, i] with i along the reference r axis.
"""
import functools
from dataclasses import dataclass

import numpy as np
from scipy.linalg import solve_triangular

from . import gd_basis


@dataclass
class VarProblem:
    n: tuple              # (nx, ny) elements
    N: int
    p: int
    X: np.ndarray         # physical x at element nodes, (ny, nx, n1, n1)
    Y: np.ndarray
    C2: np.ndarray        # c^2 at element nodes
    periodic: tuple = (False, False)
    flux: str = "upwind"
    xi: float = 0.0       # <= 0: xi = local c at the face point
    nq: int = None        # Gauss points per cell per direction (None: p+1)

    @property
    def n1(self):
        return self.N + 1

    @property
    def Q(self):
        return self.N * (self.p + 1 if self.nq is None else self.nq)


class VarOps:
    pass


FACES = ("xm", "xp", "ym", "yp")


def _face_geometry(vp, B, D, dphiL, dphiR, Xe, Ye, face):
    """Per face point: trace matrices Tv (value), Tn (n . grad) over the 81
    element nodes, plus surface weight factor |T| (dS = |T| ds)."""
    n1, Q = vp.n1, B.shape[0]
    e_0 = np.zeros(n1); e_0[0] = 1.0
    e_N = np.zeros(n1); e_N[-1] = 1.0
    if face in ("xm", "xp"):
        # face r = 0 or 1, parametrised by s_b
        rv, rd = (e_0, dphiL) if face == "xm" else (e_N, dphiR)
        phi_val = np.einsum("bj,i->bji", B, rv).reshape(Q, n1 * n1)
        phi_r = np.einsum("bj,i->bji", B, rd).reshape(Q, n1 * n1)
        phi_s = np.einsum("bj,i->bji", D, rv).reshape(Q, n1 * n1)
    else:
        # face s = 0 or 1, parametrised by r_a
        sv, sd = (e_0, dphiL) if face == "ym" else (e_N, dphiR)
        phi_val = np.einsum("j,ai->aji", sv, B).reshape(Q, n1 * n1)
        phi_r = np.einsum("j,ai->aji", sv, D).reshape(Q, n1 * n1)
        phi_s = np.einsum("j,ai->aji", sd, B).reshape(Q, n1 * n1)
    xe, ye = Xe.ravel(), Ye.ravel()
    x_r, x_s = phi_r @ xe, phi_s @ xe
    y_r, y_s = phi_r @ ye, phi_s @ ye
    det = x_r * y_s - x_s * y_r
    if face in ("xm", "xp"):
        T = np.hypot(x_s, y_s)
        nx_, ny_ = y_s / T, -x_s / T          # outward at r = 1
    else:
        T = np.hypot(x_r, y_r)
        nx_, ny_ = -y_r / T, x_r / T          # outward at s = 1
    if face in ("xm", "ym"):
        nx_, ny_ = -nx_, -ny_
    # n . (J^-T g) = (J^-1 n) . g,  J = [[x_r, x_s], [y_r, y_s]]
    fr = (y_s * nx_ - x_s * ny_) / det
    fs = (-y_r * nx_ + x_r * ny_) / det
    Tn = fr[:, None] * phi_r + fs[:, None] * phi_s
    return phi_val, Tn, T


def assemble(vp):
    """Element matrices and face data by quadrature (Section 7.1)."""
    p, N, n1 = vp.p, vp.N, vp.n1
    nq = p + 1 if vp.nq is None else vp.nq
    r, w, cell = gd_basis.quadrature_points(p, N, nq)
    B, D = gd_basis.basis_at_points(p, N, r, cell)
    _, _, dphiL, dphiR = gd_basis.face_data(p, N)
    Q = len(r)
    Phi = np.kron(B, B)           # row b*Q + a, column j*n1 + i
    Gr = np.kron(B, D)            # d/dr acts on i
    Gs = np.kron(D, B)            # d/ds acts on j
    W = np.kron(w, w)
    nx, ny = vp.n
    ne = nx * ny
    ops = VarOps()
    ops.M = np.zeros((ne, n1 * n1, n1 * n1))
    ops.S = np.zeros((ne, n1 * n1, n1 * n1))
    ops.w = np.zeros((ne, n1 * n1))
    ops.Tv = {}
    ops.Tn = {f: np.zeros((ne, Q, n1 * n1)) for f in FACES}
    ops.cw = {f: np.zeros((ne, Q)) for f in FACES}     # c^2 * dS weight
    ops.c = {f: np.zeros((ne, Q)) for f in FACES}      # local c
    ops.Gbar = np.zeros((ne, 2))                       # frozen metric (rr, ss)
    ops.Jbar = np.zeros(ne)
    for ey in range(ny):
        for ex in range(nx):
            e = ey * nx + ex
            xe, ye = vp.X[ey, ex].ravel(), vp.Y[ey, ex].ravel()
            ce = vp.C2[ey, ex].ravel()
            x_r, x_s = Gr @ xe, Gs @ xe
            y_r, y_s = Gr @ ye, Gs @ ye
            det = x_r * y_s - x_s * y_r
            if np.any(det <= 0):
                raise ValueError("mapping not orientation preserving")
            c2q = Phi @ ce
            gx = (y_s[:, None] * Gr - y_r[:, None] * Gs) / det[:, None]
            gy = (-x_s[:, None] * Gr + x_r[:, None] * Gs) / det[:, None]
            wd = W * det
            ops.M[e] = Phi.T @ (wd[:, None] * Phi)
            ops.S[e] = gx.T @ ((wd * c2q)[:, None] * gx) + gy.T @ ((wd * c2q)[:, None] * gy)
            # frozen-coefficient data for the diagonalisation preconditioner:
            # G = c^2 |J| J^-1 J^-T, averaged over the element (diagonal part)
            Grr = c2q * (x_s ** 2 + y_s ** 2) / det
            Gss = c2q * (x_r ** 2 + y_r ** 2) / det
            ops.Gbar[e] = [W @ Grr, W @ Gss]
            ops.Jbar[e] = W @ det
            ops.w[e] = ops.M[e] @ np.ones(n1 * n1) / ops.Jbar[e]
            for f in FACES:
                Tv, Tn, T = _face_geometry(vp, B, D, dphiL, dphiR,
                                           vp.X[ey, ex], vp.Y[ey, ex], f)
                ops.Tv[f] = Tv
                ops.Tn[f][e] = Tn
                c2f = Tv @ ce
                ops.cw[f][e] = c2f * T * w
                ops.c[f][e] = np.sqrt(c2f)
    return ops


@functools.lru_cache(maxsize=16)
def quadrature(p, N, nq):
    """Tensor Gauss-Legendre rule on the reference element (nq points per GD
    cell per direction): Phi[q, a] = phi_a at point q, Gr, Gs the r and s
    derivatives, W the weights (index q = b*Q + a, b along s)."""
    r, w, cell = gd_basis.quadrature_points(p, N, nq)
    B, D = gd_basis.basis_at_points(p, N, r, cell)
    return np.kron(B, B), np.kron(B, D), np.kron(D, B), np.kron(w, w)


def _mapped_points(vp, nq):
    """Physical points (x, y) and |J| at every element's quadrature points."""
    Phi, Gr, Gs, W = quadrature(vp.p, vp.N, nq)
    ne = vp.n[0] * vp.n[1]
    Xe, Ye = vp.X.reshape(ne, -1), vp.Y.reshape(ne, -1)
    det = (Xe @ Gr.T) * (Ye @ Gs.T) - (Xe @ Gs.T) * (Ye @ Gr.T)
    return Phi, W, Xe @ Phi.T, Ye @ Phi.T, det


def distributed_load(vp, f, nq=None):
    """int phi_a f |J| over every element (the forcing term of Eq. DG2 for
    u_tt = div(c^2 grad u) + f, Section 7.1), f a callable of the physical
    (x, y) arrays; returns (ne, n1^2), the `forcing` argument of residuals."""
    Phi, W, xq, yq, det = _mapped_points(vp, vp.p + 3 if nq is None else nq)
    return (W * det * f(xq, yq)) @ Phi


def l2_error(vp, U, u_exact, nq=None):
    """||u - u_h||_L2 (Section 6's error measure) on mapped elements by
    quadrature with p+3 points per cell; u_exact a callable of (x, y)."""
    Phi, W, xq, yq, det = _mapped_points(vp, vp.p + 3 if nq is None else nq)
    ne = vp.n[0] * vp.n[1]
    uh = U.reshape(ne, -1) @ Phi.T
    return float(np.sqrt(np.sum(W * det * (u_exact(xq, yq) - uh) ** 2)))


def _neighbour(vp, ey, ex, face):
    """(element index, its face) across `face`, or None on a Dirichlet side."""
    nx, ny = vp.n
    if face == "xp":
        ex2, ey2, f2, k = ex + 1, ey, "xm", 0
    elif face == "xm":
        ex2, ey2, f2, k = ex - 1, ey, "xp", 0
    elif face == "yp":
        ex2, ey2, f2, k = ex, ey + 1, "ym", 1
    else:
        ex2, ey2, f2, k = ex, ey - 1, "yp", 1
    if not (0 <= ex2 < nx and 0 <= ey2 < ny):
        if not vp.periodic[k]:
            return None
        ex2 %= nx
        ey2 %= ny
    return ey2 * nx + ex2, f2


def _beta_tau(vp, c):
    if vp.flux in ("central", "alternating"):
        return 0.0 * c, 0.0 * c
    if vp.flux != "upwind":
        raise ValueError("unknown flux")
    xi = np.full_like(c, vp.xi) if vp.xi > 0 else c
    return 0.5 * xi, 0.5 / xi


def residuals(vp, ops, U, V, forcing=None):
    """(r_u, r_v) per element; U, V of shape (ne, 81).
    forcing: optional array (ne, 81) of int phi_a f |J| added to r_v."""
    nx, ny = vp.n
    ne = nx * ny
    U = U.reshape(ne, -1)
    V = V.reshape(ne, -1)
    r_u = np.zeros_like(U)
    r_v = -np.einsum("eab,eb->ea", ops.S, U)
    if forcing is not None:
        r_v = r_v + forcing
    for ey in range(ny):
        for ex in range(nx):
            e = ey * nx + ex
            for f in FACES:
                v_in = ops.Tv[f] @ V[e]
                d_in = ops.Tn[f][e] @ U[e]
                nb = _neighbour(vp, ey, ex, f)
                if nb is None:
                    v_out, d_out = -v_in, -d_in
                else:
                    e2, f2 = nb
                    v_out = ops.Tv[f2] @ V[e2]
                    d_out = ops.Tn[f2][e2] @ U[e2]
                beta, tau = _beta_tau(vp, ops.c[f][e])
                if vp.flux != "alternating":
                    vstar = 0.5 * (v_in + v_out) - beta * (d_in + d_out)
                    qstar = 0.5 * (d_in - d_out) - tau * (v_in - v_out)
                elif nb is None:                 # Dirichlet side: v* = 0, q* = d_in
                    vstar, qstar = 0.0 * v_in, d_in
                elif f in ("xm", "ym"):          # element on side 2 (right / upper)
                    vstar, qstar = v_out, d_in
                else:                            # element on side 1 (left / lower)
                    vstar, qstar = v_in, -d_out
                cw = ops.cw[f][e]
                r_u[e] += ops.Tn[f][e].T @ (cw * (vstar - v_in))
                r_v[e] += ops.Tv[f].T @ (cw * qstar)
    return r_u, r_v


def spd_u_matrix(ops, e):
    """S_c2 + w w^T of element e (the SPD form of the constrained system)."""
    return ops.S[e] + np.outer(ops.w[e], ops.w[e])


def solve_direct(ops, V, r_u, r_v):
    """Dense direct solves (the truth for PCG)."""
    ne = r_u.shape[0]
    Ut = np.empty_like(r_u)
    Vt = np.empty_like(r_v)
    for e in range(ne):
        Ut[e] = V.reshape(ne, -1)[e] + np.linalg.solve(spd_u_matrix(ops, e), r_u[e])
        Vt[e] = np.linalg.solve(ops.M[e], r_v[e])
    return Ut, Vt


# ---------------------------------------------------------------- PCG ----

def reference_diagonalisation(p, N):
    Mh, Sh = gd_basis.mass_stiffness(p, N)
    Psi, lam = gd_basis.simultaneous_diagonalisation(Mh, Sh)
    return Psi, lam


def fdm_preconditioner(ops, e, which, Psi, lam):
    """Frozen-coefficient diagonalisation preconditioner P^-1 (dense).

    which = "M": P = Jbar * (M_hat (x) M_hat)  ->  P^-1 = Psi2 Psi2^T / Jbar.
    which = "S": P = Grr (M_hat (x) S_hat) + Gss (S_hat (x) M_hat) + wbar wbar^T
                 with wbar = (M_hat (x) M_hat) 1 (the frozen M_J 1 / |e|); in the
                 Psi2 basis it is diagonal: Grr lam_i + Gss lam_j, and 1 on the
                 constant mode.
    Psi2 = Psi (x) Psi (index j*n1 + i), Section 3.2's modified basis."""
    n1 = Psi.shape[0]
    Psi2 = np.kron(Psi, Psi)
    if which == "M":
        d = np.full(n1 * n1, 1.0 / ops.Jbar[e])
    else:
        Grr, Gss = ops.Gbar[e]
        lam2 = (Gss * lam[:, None] + Grr * lam[None, :]).ravel()   # (j, i)
        lam2[0] = 1.0
        d = 1.0 / lam2
    return Psi2 @ (d[:, None] * Psi2.T)


def ic0(A, pattern=None):
    """Zero fill-in incomplete Cholesky A ~ L L^T (textbook IC(0)).

    Section 7.1 preconditions the two element systems with the IC(0)
    factors of S_c2 and M.  IC(0) runs the steps of the right-looking
    Cholesky factorisation but keeps only the entries of L that lie in the
    sparsity pattern (default: the nonzeros of A); every update that would
    create fill outside it is dropped.  Where the exact Cholesky factor has
    no fill outside the pattern (banded matrices, Kronecker products of
    banded matrices) IC(0) is that factor."""
    n = A.shape[0]
    P = (np.tril(A) != 0.0) if pattern is None else np.tril(np.asarray(pattern, dtype=bool))
    L = np.where(P, np.tril(A), 0.0)
    for k in range(n):
        L[k, k] = np.sqrt(L[k, k])
        L[k + 1:, k] = np.where(P[k + 1:, k], L[k + 1:, k] / L[k, k], 0.0)
        col = L[k + 1:, k]
        L[k + 1:, k + 1:] -= np.where(P[k + 1:, k + 1:], np.tril(np.outer(col, col)), 0.0)
    return L


def pcg(A, b, Pinv, x0=None, rtol=1e-10, maxit=200):
    """Preconditioned CG for SPD A; Pinv is a callable z = P^-1 r.
    Returns (x, iterations, final relative residual)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    bnorm = np.linalg.norm(b)
    z = Pinv(r)
    pdir = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        if np.linalg.norm(r) <= rtol * bnorm or rz == 0.0:
            break
        Ap = A @ pdir
        alpha = rz / (pdir @ Ap)
        x = x + alpha * pdir
        r = r - alpha * Ap
        z = Pinv(r)
        rz_new = r @ z
        pdir = z + (rz_new / rz) * pdir
        rz = rz_new
        it += 1
    rel = np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0
    return x, it, rel


def solve_pcg(vp, ops, V, r_u, r_v, precond="fdm", rtol=1e-10, maxit=200,
              x0_u=None, x0_v=None):
    """Element-by-element PCG for dU/dt and dV/dt.
    Returns (dU/dt, dV/dt, iterations_u[ne], iterations_v[ne])."""
    ne = r_u.shape[0]
    V = V.reshape(ne, -1)
    if precond == "fdm":
        Psi, lam = reference_diagonalisation(vp.p, vp.N)
    Ut = np.empty_like(r_u)
    Vt = np.empty_like(r_v)
    it_u = np.zeros(ne, dtype=int)
    it_v = np.zeros(ne, dtype=int)
    for e in range(ne):
        Au = spd_u_matrix(ops, e)
        Am = ops.M[e]
        if precond == "fdm":
            Pu = fdm_preconditioner(ops, e, "S", Psi, lam)
            Pm = fdm_preconditioner(ops, e, "M", Psi, lam)
            pu = lambda r, P=Pu: P @ r
            pm = lambda r, P=Pm: P @ r
        elif precond == "ic0":
            # Section 7.1: IC(0) of S_c2 for the u_t system and of M for the
            # v_t system.  S_c2 is singular (its kernel is the constants), so
            # the factor is taken of the SPD matrix solved, S_c2 + w w^T, on
            # the sparsity pattern of S_c2 (the rank-one term would fill it).
            Lu, Lm = ic0(Au, ops.S[e] != 0.0), ic0(Am, Am != 0.0)
            pu = lambda r, L=Lu: solve_triangular(L.T, solve_triangular(L, r, lower=True), lower=False)
            pm = lambda r, L=Lm: solve_triangular(L.T, solve_triangular(L, r, lower=True), lower=False)
        elif precond == "none":
            pu = pm = lambda r: r.copy()
        else:
            raise ValueError(precond)
        y, it_u[e], _ = pcg(Au, r_u[e], pu, None if x0_u is None else x0_u[e], rtol, maxit)
        Vt[e], it_v[e], _ = pcg(Am, r_v[e], pm, None if x0_v is None else x0_v[e], rtol, maxit)
        Ut[e] = V[e] + y
    return Ut, Vt, it_u, it_v


def energy(ops, U, V):
    ne = ops.M.shape[0]
    U = U.reshape(ne, -1)
    V = V.reshape(ne, -1)
    return 0.5 * (np.einsum("ea,eab,eb->", V, ops.M, V)
                  + np.einsum("ea,eab,eb->", U, ops.S, U))


def time_derivative(vp, ops, U, V, solver="direct", **kw):
    r_u, r_v = residuals(vp, ops, U, V)
    if solver == "direct":
        return solve_direct(ops, V, r_u, r_v)
    Ut, Vt, _, _ = solve_pcg(vp, ops, V, r_u, r_v, **kw)
    return Ut, Vt
