"""1-D Galerkin-difference basis on the reference element [0, 1] (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 2.1: nodes r_i = i*h, h = 1/N, i = 0..N, odd degree p, q = (p+1)/2.
Eq. GD_basis_lagrange: away from the boundary, on cell [k h, (k+1) h) the
expansion uses the p+1 nodes k-q+1 .. k+q (Eq. GD_basis_nodalformula) and
each basis function is the Lagrange polynomial of its node on that stencil.
Section 2.1.1 (extrapolation basis): ghost values outside [0, 1] are
replaced by degree-p extrapolation from the p+1 nodes nearest the boundary.
The ghost values then lie on the degree-p interpolant of nodes 0..p (resp.
N-p..N), so on a boundary cell the modified expansion equals the Lagrange
interpolant on the clamped stencil s(k) = min(max(k-q+1, 0), N-p).  That is
the construction below; the p = 3 worked example of Section 2.1.1 is a test.

Section 3.1: M_kl = int phi_k phi_l, S_kl = int phi_k' phi_l' (on the
reference element; a physical element of width H has H*M and S/H).  Exact
Gauss-Legendre quadrature with p+1 points per cell (integrand degree 2p).

Section 3.2: S psi = lambda M psi, psi^T M psi = 1 (simultaneous
diagonalisation, the "modified GD basis").
"""
import numpy as np


def check_degree(p, N):
    if p < 1 or p % 2 == 0:
        raise ValueError("GD degree p must be odd and >= 1 (Section 2)")
    if N < p:
        raise ValueError("need N >= p cells per element so the stencil fits")


def stencil_start(k, p, N):
    """First node of the p+1 node stencil used on cell k (clamped at the
    boundary by the extrapolation basis, Section 2.1.1)."""
    q = (p + 1) // 2
    return min(max(k - q + 1, 0), N - p)


def lagrange_on_nodes(nodes, r):
    """Values and derivatives at r of the Lagrange polynomials of `nodes`.

    Returns (L, dL), each of length len(nodes): L[m](r) = prod_{l!=m}
    (r - x_l)/(x_m - x_l) and its derivative by the product rule."""
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    L = np.ones(n)
    dL = np.zeros(n)
    for m in range(n):
        for l in range(n):
            if l == m:
                continue
            denom = nodes[m] - nodes[l]
            # product rule: d/dr [L * f] = dL*f + L*f'
            f = (r - nodes[l]) / denom
            dL[m] = dL[m] * f + L[m] / denom
            L[m] = L[m] * f
    return L, dL


def cell_of(r, N):
    """Cell index containing r in [0,1]; r = 1 belongs to the last cell."""
    k = int(np.floor(r * N))
    return min(max(k, 0), N - 1)


def eval_basis(p, N, r, cell=None):
    """All N+1 basis functions (and derivatives d/dr) at r in [0,1].

    `cell` forces the cell whose polynomial piece is used (needed for the
    one-sided derivative at the element faces and at cell boundaries)."""
    check_degree(p, N)
    h = 1.0 / N
    k = cell_of(r, N) if cell is None else cell
    s = stencil_start(k, p, N)
    nodes = (np.arange(s, s + p + 1)) * h
    L, dL = lagrange_on_nodes(nodes, r)
    phi = np.zeros(N + 1)
    dphi = np.zeros(N + 1)
    phi[s:s + p + 1] = L
    dphi[s:s + p + 1] = dL
    return phi, dphi


def generating_function(p, x):
    """Phi_p(x) for grid spacing h = 1 (Eq. GD_basis_lagrange): on
    [(q-j-1), (q-j)) it is the Lagrange polynomial L_j of the grid
    {-j, ..., p-j} with L_j(0) = 1; even extension, zero for |x| >= q."""
    q = (p + 1) // 2
    ax = abs(x)
    if ax >= q:
        return 0.0
    j = q - 1 - int(np.floor(ax))
    nodes = np.arange(-j, p - j + 1, dtype=np.float64)
    L, _ = lagrange_on_nodes(nodes, ax)
    return float(L[j])  # node 0 sits at index j of the grid -j..p-j


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [0,1] (library primitive)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def quadrature_points(p, N, nq=None):
    """Composite rule: nq Gauss points in each of the N cells of [0,1].
    Returns (r, w, cell) arrays of length N*nq."""
    nq = p + 1 if nq is None else nq
    x, w = gauss_legendre(nq)
    h = 1.0 / N
    r = np.concatenate([(k + x) * h for k in range(N)])
    ww = np.concatenate([w * h for _ in range(N)])
    cell = np.repeat(np.arange(N), nq)
    return r, ww, cell


def basis_at_points(p, N, r, cell):
    """Matrices B[q, i] = phi_i(r_q), D[q, i] = phi_i'(r_q)."""
    B = np.zeros((len(r), N + 1))
    D = np.zeros((len(r), N + 1))
    for a, (rq, kq) in enumerate(zip(r, cell)):
        B[a], D[a] = eval_basis(p, N, rq, cell=int(kq))
    return B, D


def mass_stiffness(p, N):
    """Reference-element M_hat, S_hat (Section 3.1), exact quadrature."""
    r, w, cell = quadrature_points(p, N)
    B, D = basis_at_points(p, N, r, cell)
    M = B.T @ (w[:, None] * B)
    S = D.T @ (w[:, None] * D)
    return M, S


def face_data(p, N):
    """phi(0), phi(1), phi'(0) (from cell 0), phi'(1) (from cell N-1)."""
    phiL, dphiL = eval_basis(p, N, 0.0, cell=0)
    phiR, dphiR = eval_basis(p, N, 1.0, cell=N - 1)
    return phiL, phiR, dphiL, dphiR


def simultaneous_diagonalisation(M, S):
    """Psi, lam with S Psi = M Psi diag(lam), Psi^T M Psi = I (Section 3.2).

    Cholesky M = L L^T, symmetric eigen-solve of L^-1 S L^-T (library
    primitives), ascending order.  The constant mode is set exactly:
    lambda_0 = 0, psi_0 = 1/sqrt(1^T M 1) (the kernel of S is the
    constants; Section 3.2 enforces dU_0/dt = V_0 for it)."""
    n = M.shape[0]
    L = np.linalg.cholesky(M)
    Linv = np.linalg.inv(L)
    A = Linv @ S @ Linv.T
    A = 0.5 * (A + A.T)
    lam, Y = np.linalg.eigh(A)
    Psi = Linv.T @ Y
    one = np.ones(n)
    Psi[:, 0] = one / np.sqrt(one @ M @ one)
    lam[0] = 0.0
    # re-orthogonalise the others against the exact constant mode
    for k in range(1, n):
        Psi[:, k] -= (Psi[:, 0] @ M @ Psi[:, k]) * Psi[:, 0]
        Psi[:, k] /= np.sqrt(Psi[:, k] @ M @ Psi[:, k])
    return Psi, lam
