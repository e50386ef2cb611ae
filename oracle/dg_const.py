"""Energy-DG semi-discretisation, constant c^2, Cartesian elements (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Nodal form, written from the element-wise variational statement (Eqs. DG1,
DG2, DG1_extra of Section 2.2) and the fluxes of Section 2.2.1, element by
element.  Where the printed matrix form (Eqs. DG_matrix1/2 of Section 3)
differs in the sign of the dissipative B and C terms, the variational
statement is followed; the energy identities in the tests pin the choice.

Per element, with outward normal n on each face and traces
  v_in, d_in = n . grad u_in          (this element)
  v_out, d_out = n_out . grad u_out   (the neighbour, its own outward normal)
the fluxes of Section 2.2.1 with alpha = 1/2 in normal form are
  v*  = (v_in + v_out)/2 - beta (d_in + d_out)
  q*  = n . (grad u)* = (d_in - d_out)/2 - tau (v_in - v_out)
central: beta = tau = 0; upwind: beta = xi/2, tau = 1/(2 xi).
Alternating flux (Section 2.2.1, alpha = 1, beta = tau = 0): v* = v^1 and
(grad u)* = grad u^2.  With the sides labelled by a fixed orientation (side 1
= the left / lower element of a face), an element's - face has it on side 2
and its + face on side 1:
  - face:  v* = v_out,  q* = d_in;      + face:  v* = v_in,  q* = -d_out,
so both elements of a face use the same v* and (grad u)*.  On a Dirichlet
side the closure is v* = 0, q* = d_in (what the mirror state gives the
central flux), which keeps the scheme conservative.
Then (c^2 constant, divided out of Eq. DG1):
  r_u = sum_faces (n . grad phi)|face (x) M_perp (v* - v_in)
  r_v = -c^2 S U + sum_faces c^2 phi|face (x) M_perp q*
  M dV/dt = r_v
  S (dU/dt - V) = r_u,  w^T (dU/dt - V) = 0,  w = M 1      (Eq. DG1_extra)
M_perp is the 1-D mass matrix along the face (both neighbours share the
transverse GD basis); in 1-D it is the scalar 1.
Homogeneous Dirichlet data u = 0 enters as the mirror state
  v_out = -v_in, d_out = -d_in  (so v* = 0, q* = d_in - 2 tau v_in).

Layout: 1-D U[e, i]; 2-D U[ey, ex, j, i] (i along x), element e = ey*nx+ex;
3-D U[ez, ey, ex, k, j, i], e = (ez*ny + ey)*nx + ex (Sections 2.1.2 and 3:
the tensor-product construction for d = 3, which the paper states but does
not test).  Each face then carries a 2-D trace over its two transverse node
indices and M_perp is the Kronecker product of the two transverse 1-D mass
matrices.
"""
from dataclasses import dataclass, field

import numpy as np

from . import gd_basis


@dataclass
class Problem:
    dim: int
    n: tuple            # elements per direction
    N: int              # GD cells per element per direction
    p: int              # odd GD degree
    lo: tuple = (0.0, 0.0)
    hi: tuple = (1.0, 1.0)
    periodic: tuple = (False, False)
    flux: str = "upwind"   # "central" | "upwind" | "alternating"
    xi: float = 0.0        # upwind splitting; <= 0 means xi = c
    c2: float = 1.0

    @property
    def n1(self):
        return self.N + 1

    def H(self, k):
        return (self.hi[k] - self.lo[k]) / self.n[k]

    def beta_tau(self):
        if self.flux in ("central", "alternating"):
            return 0.0, 0.0
        if self.flux == "upwind":
            xi = self.xi if self.xi > 0 else np.sqrt(self.c2)
            return 0.5 * xi, 0.5 / xi
        raise ValueError("unknown flux " + str(self.flux))


@dataclass
class Operators:
    """Physical 1-D operators per direction plus the element Kronecker forms."""
    M1: list = field(default_factory=list)   # H * M_hat
    S1: list = field(default_factory=list)   # S_hat / H
    aL: list = field(default_factory=list)   # n . grad phi on the - face
    aR: list = field(default_factory=list)   # n . grad phi on the + face
    M: np.ndarray = None
    S: np.ndarray = None


def operators(prob):
    Mh, Sh = gd_basis.mass_stiffness(prob.p, prob.N)
    _, _, dphiL, dphiR = gd_basis.face_data(prob.p, prob.N)
    ops = Operators()
    for k in range(prob.dim):
        H = prob.H(k)
        ops.M1.append(H * Mh)
        ops.S1.append(Sh / H)
        ops.aL.append(-dphiL / H)   # outward normal -x_k
        ops.aR.append(dphiR / H)    # outward normal +x_k
    if prob.dim == 1:
        ops.M, ops.S = ops.M1[0], ops.S1[0]
    elif prob.dim == 3:
        # element index a = (k*n1 + j)*n1 + i: kron(A_z, A_y, A_x)
        Mx, My, Mz = ops.M1
        Sx, Sy, Sz = ops.S1
        ops.M = np.kron(Mz, np.kron(My, Mx))
        ops.S = np.kron(Mz, np.kron(My, Sx)) + np.kron(Mz, np.kron(Sy, Mx)) + np.kron(Sz, np.kron(My, Mx))
    else:
        # element index a = j*n1 + i (i along x): kron(A_y, B_x)
        Mx, My, Sx, Sy = ops.M1[0], ops.M1[1], ops.S1[0], ops.S1[1]
        ops.M = np.kron(My, Mx)
        ops.S = np.kron(My, Sx) + np.kron(Sy, Mx)
    return ops


def _fluxes(v_in, d_in, v_out, d_out, beta, tau, alt=None, bnd=None):
    """(v*, q*) on one face of every element.  alt: None (alpha = 1/2), or
    "minus" / "plus" for the alternating flux on the element's - / + face,
    with bnd marking the faces on a Dirichlet side."""
    if alt is None:
        vstar = 0.5 * (v_in + v_out) - beta * (d_in + d_out)
        qstar = 0.5 * (d_in - d_out) - tau * (v_in - v_out)
        return vstar, qstar
    if alt == "minus":            # this element is side 2 of the face
        vstar, qstar = v_out.copy(), d_in.copy()
    else:                         # side 1
        vstar, qstar = v_in.copy(), -d_out
    if bnd is not None:
        vstar = np.where(bnd, 0.0, vstar)
        qstar = np.where(bnd, d_in, qstar)
    return vstar, qstar


def _boundary_masks(shape, periodic):
    """Masks of the - and + faces on a Dirichlet side (element axis first)."""
    bm = np.zeros(shape, dtype=bool)
    bp = np.zeros(shape, dtype=bool)
    if not periodic:
        bm[0] = True
        bp[-1] = True
    return bm, bp


def _neighbour_traces(vm, dm, vp, dp, periodic):
    """Given per-element traces on the - face (vm, dm) and + face (vp, dp)
    along axis 0 (the element index in the face-normal direction), return the
    outside states seen by each element's - and + faces."""
    if periodic:
        out_p_v, out_p_d = np.roll(vm, -1, axis=0), np.roll(dm, -1, axis=0)
        out_m_v, out_m_d = np.roll(vp, 1, axis=0), np.roll(dp, 1, axis=0)
    else:
        out_p_v, out_p_d = np.empty_like(vp), np.empty_like(dp)
        out_m_v, out_m_d = np.empty_like(vm), np.empty_like(dm)
        out_p_v[:-1], out_p_d[:-1] = vm[1:], dm[1:]
        out_m_v[1:], out_m_d[1:] = vp[:-1], dp[:-1]
        # homogeneous Dirichlet mirror state on the domain boundary
        out_p_v[-1], out_p_d[-1] = -vp[-1], -dp[-1]
        out_m_v[0], out_m_d[0] = -vm[0], -dm[0]
    return out_m_v, out_m_d, out_p_v, out_p_d


def _residuals_3d(prob, U, V, ops, beta, tau, alt):
    """3-D element residuals: the 2-D face terms with 2-D face traces.
    Direction d in (0, 1, 2) = (x, y, z) is node axis (5, 4, 3) and element
    axis (2, 1, 0) of U[ez, ey, ex, k, j, i]."""
    n1, c2 = prob.n1, prob.c2
    nx, ny, nz = prob.n
    U = U.reshape(nz, ny, nx, n1, n1, n1)
    V = V.reshape(nz, ny, nx, n1, n1, n1)
    r_u = np.zeros_like(U)
    r_v = -c2 * (U.reshape(nz * ny * nx, n1 ** 3) @ ops.S.T).reshape(U.shape)
    for d in range(3):
        node_ax, elem_ax = 5 - d, 2 - d
        # transverse directions, in the order of the remaining node axes
        trans = [q for q in (2, 1, 0) if q != d]
        Ud = np.moveaxis(U, node_ax, -1)
        Vd = np.moveaxis(V, node_ax, -1)
        aL, aR = ops.aL[d], ops.aR[d]
        vm, vp = Vd[..., 0], Vd[..., -1]
        dm, dp = Ud @ aL, Ud @ aR
        t = [np.moveaxis(a, elem_ax, 0) for a in (vm, dm, vp, dp)]
        om_v, om_d, op_v, op_d = [np.moveaxis(a, 0, elem_ax) for a in
                                  _neighbour_traces(*t, prob.periodic[d])]
        bm, bp = [np.moveaxis(a, 0, elem_ax) for a in _boundary_masks(t[0].shape, prob.periodic[d])]
        vs_m, qs_m = _fluxes(vm, dm, om_v, om_d, beta, tau, *(("minus", bm) if alt else ()))
        vs_p, qs_p = _fluxes(vp, dp, op_v, op_d, beta, tau, *(("plus", bp) if alt else ()))
        T1, T2 = ops.M1[trans[0]], ops.M1[trans[1]]
        perp = lambda g: np.einsum("...ab,Aa,Bb->...AB", g, T1, T2)
        ru_d = (np.einsum("...ab,n->...abn", perp(vs_m - vm), aL)
                + np.einsum("...ab,n->...abn", perp(vs_p - vp), aR))
        rv_d = np.zeros_like(ru_d)
        rv_d[..., 0] += c2 * perp(qs_m)
        rv_d[..., -1] += c2 * perp(qs_p)
        r_u += np.moveaxis(ru_d, -1, node_ax)
        r_v += np.moveaxis(rv_d, -1, node_ax)
    ne = nx * ny * nz
    return r_u.reshape(ne, n1 ** 3), r_v.reshape(ne, n1 ** 3)


def residuals(prob, U, V, ops=None):
    """(r_u, r_v) of the element equations for nodal states U, V."""
    ops = operators(prob) if ops is None else ops
    beta, tau = prob.beta_tau()
    alt = prob.flux == "alternating"
    c2 = prob.c2
    n1 = prob.n1
    if prob.dim == 3:
        return _residuals_3d(prob, U, V, ops, beta, tau, alt)
    if prob.dim == 1:
        U = U.reshape(prob.n[0], n1)
        V = V.reshape(prob.n[0], n1)
        aL, aR = ops.aL[0], ops.aR[0]
        vm, vp = V[:, 0], V[:, -1]
        dm, dp = U @ aL, U @ aR
        om_v, om_d, op_v, op_d = _neighbour_traces(vm, dm, vp, dp, prob.periodic[0])
        bm, bp = _boundary_masks(vm.shape, prob.periodic[0])
        vs_m, qs_m = _fluxes(vm, dm, om_v, om_d, beta, tau, *(("minus", bm) if alt else ()))
        vs_p, qs_p = _fluxes(vp, dp, op_v, op_d, beta, tau, *(("plus", bp) if alt else ()))
        r_u = np.outer(vs_m - vm, aL) + np.outer(vs_p - vp, aR)
        r_v = -c2 * U @ ops.S.T
        r_v[:, 0] += c2 * qs_m
        r_v[:, -1] += c2 * qs_p
        return r_u, r_v

    nx, ny = prob.n
    U = U.reshape(ny, nx, n1, n1)
    V = V.reshape(ny, nx, n1, n1)
    Mx, My = ops.M1
    r_u = np.zeros_like(U)
    r_v = -c2 * (U.reshape(ny * nx, n1 * n1) @ ops.S.T).reshape(U.shape)

    # x faces: traces are functions of y (index j); neighbours along ex.
    aL, aR = ops.aL[0], ops.aR[0]
    vm, vp = V[..., :, 0], V[..., :, -1]            # (ny, nx, n1_j)
    dm = np.einsum("yxji,i->yxj", U, aL)
    dp = np.einsum("yxji,i->yxj", U, aR)
    t = [np.swapaxes(a, 0, 1) for a in (vm, dm, vp, dp)]   # element axis first
    om_v, om_d, op_v, op_d = [np.swapaxes(a, 0, 1) for a in
                              _neighbour_traces(*t, prob.periodic[0])]
    bm, bp = [np.swapaxes(a, 0, 1) for a in _boundary_masks(t[0].shape, prob.periodic[0])]
    vs_m, qs_m = _fluxes(vm, dm, om_v, om_d, beta, tau, *(("minus", bm) if alt else ()))
    vs_p, qs_p = _fluxes(vp, dp, op_v, op_d, beta, tau, *(("plus", bp) if alt else ()))
    gm = (vs_m - vm) @ My.T            # M_y (v* - v_in), per element
    gp = (vs_p - vp) @ My.T
    r_u += np.einsum("yxj,i->yxji", gm, aL) + np.einsum("yxj,i->yxji", gp, aR)
    r_v[..., :, 0] += c2 * (qs_m @ My.T)
    r_v[..., :, -1] += c2 * (qs_p @ My.T)

    # y faces: traces are functions of x (index i); neighbours along ey.
    aL, aR = ops.aL[1], ops.aR[1]
    vm, vp = V[..., 0, :], V[..., -1, :]            # (ny, nx, n1_i)
    dm = np.einsum("yxji,j->yxi", U, aL)
    dp = np.einsum("yxji,j->yxi", U, aR)
    om_v, om_d, op_v, op_d = _neighbour_traces(vm, dm, vp, dp, prob.periodic[1])
    bm, bp = _boundary_masks(vm.shape, prob.periodic[1])
    vs_m, qs_m = _fluxes(vm, dm, om_v, om_d, beta, tau, *(("minus", bm) if alt else ()))
    vs_p, qs_p = _fluxes(vp, dp, op_v, op_d, beta, tau, *(("plus", bp) if alt else ()))
    gm = (vs_m - vm) @ Mx.T
    gp = (vs_p - vp) @ Mx.T
    r_u += np.einsum("yxi,j->yxji", gm, aL) + np.einsum("yxi,j->yxji", gp, aR)
    r_v[..., 0, :] += c2 * (qs_m @ Mx.T)
    r_v[..., -1, :] += c2 * (qs_p @ Mx.T)
    ne = nx * ny
    return r_u.reshape(ne, n1 * n1), r_v.reshape(ne, n1 * n1)


def constrained_matrix(M, S):
    """S with its first row replaced by w^T = (M 1)^T (Eq. DG1_extra)."""
    A = S.copy()
    A[0, :] = M @ np.ones(M.shape[0])
    return A


def solve(ops, V, r_u, r_v):
    """dU/dt = V + y with S y = r_u, w^T y = 0;  dV/dt = M^-1 r_v.
    Dense direct solves (library LU / Cholesky as primitives)."""
    A = constrained_matrix(ops.M, ops.S)
    b = r_u.copy()
    b[:, 0] = 0.0
    y = np.linalg.solve(A, b.T).T
    L = np.linalg.cholesky(ops.M)
    z = np.linalg.solve(L, r_v.T)
    Vt = np.linalg.solve(L.T, z).T
    return V.reshape(y.shape) + y, Vt


def time_derivative(prob, U, V, ops=None):
    """(dU/dt, dV/dt) of the semi-discretisation at nodal state (U, V)."""
    ops = operators(prob) if ops is None else ops
    r_u, r_v = residuals(prob, U, V, ops)
    return solve(ops, V, r_u, r_v)


def energy(prob, U, V, ops=None):
    """E = 1/2 sum_e (V_e^T M V_e + c^2 U_e^T S U_e)."""
    ops = operators(prob) if ops is None else ops
    ne = int(np.prod(prob.n))
    U = U.reshape(ne, -1)
    V = V.reshape(ne, -1)
    return 0.5 * (np.einsum("ea,ab,eb->", V, ops.M, V)
                  + prob.c2 * np.einsum("ea,ab,eb->", U, ops.S, U))


def node_coordinates(prob):
    """Physical coordinates of every element's GD nodes, in the layout of U.
    1-D: x[e, i];  2-D: (x, y) each [ey, ex, j, i];  3-D: (x, y, z) each
    [ez, ey, ex, k, j, i]."""
    n1 = prob.n1
    r = np.arange(n1) / prob.N
    if prob.dim == 1:
        H = prob.H(0)
        x0 = prob.lo[0] + H * np.arange(prob.n[0])
        return (x0[:, None] + H * r[None, :],)
    if prob.dim == 3:
        nx, ny, nz = prob.n
        shape = (nz, ny, nx, n1, n1, n1)
        out = []
        for d, (ne_d, ax_e, ax_n) in enumerate(((nx, 2, 5), (ny, 1, 4), (nz, 0, 3))):
            H = prob.H(d)
            c0 = prob.lo[d] + H * np.arange(ne_d)
            e_shape = [1] * 6
            e_shape[ax_e] = ne_d
            n_shape = [1] * 6
            n_shape[ax_n] = n1
            out.append(np.broadcast_to(c0.reshape(e_shape) + H * r.reshape(n_shape), shape).copy())
        return tuple(out)
    nx, ny = prob.n
    Hx, Hy = prob.H(0), prob.H(1)
    x0 = prob.lo[0] + Hx * np.arange(nx)
    y0 = prob.lo[1] + Hy * np.arange(ny)
    X = np.broadcast_to(x0[None, :, None, None] + Hx * r[None, None, None, :],
                        (ny, nx, n1, n1))
    Y = np.broadcast_to(y0[:, None, None, None] + Hy * r[None, None, :, None],
                        (ny, nx, n1, n1))
    return X.copy(), Y.copy()


def dense_operator(prob):
    """Global matrix L with d/dt [U; V] = L [U; V] assembled column by column
    from unit vectors (brute force on tiny meshes, used by the tests)."""
    ops = operators(prob)
    ndof = int(np.prod(prob.n)) * prob.n1 ** prob.dim
    L = np.zeros((2 * ndof, 2 * ndof))
    for c in range(2 * ndof):
        z = np.zeros(2 * ndof)
        z[c] = 1.0
        Ut, Vt = time_derivative(prob, z[:ndof], z[ndof:], ops)
        L[:ndof, c] = Ut.ravel()
        L[ndof:, c] = Vt.ravel()
    return L


def energy_matrix(prob):
    """Block diagonal (c^2 S, M) over all elements: E = 1/2 Z^T E Z."""
    ops = operators(prob)
    ne = int(np.prod(prob.n))
    I = np.eye(ne)
    return np.block([[prob.c2 * np.kron(I, ops.S), np.zeros((ne * ops.S.shape[0],) * 2)],
                     [np.zeros((ne * ops.S.shape[0],) * 2), np.kron(I, ops.M)]])
