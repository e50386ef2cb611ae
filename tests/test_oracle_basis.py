"""Pins of the oracle's 1-D GD basis, matrices and diagonalisation against
facts the paper and the mathematics fix (Sections 2.1, 3.1, 3.2)."""
import os

import numpy as np
import pytest

from oracle import gd_basis as gb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CASES = [(1, 1), (1, 4), (3, 3), (3, 4), (3, 8), (5, 5), (5, 8), (7, 8), (7, 11), (5, 13)]


def _points(N, per_cell=7):
    # points strictly inside every cell plus the nodes themselves
    inner = np.concatenate([(k + np.linspace(0.03, 0.97, per_cell)) / N for k in range(N)])
    return np.concatenate([inner, np.arange(N + 1) / N])


def test_p3_worked_example_extrapolation():
    """Section 2.1.1: on the first cell the boundary-modified functions are
    phi_m + c_m phi_{-1} with c = (4, -6, 4, -1) (the ghost extrapolation)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "p3_extrapolation.txt"))
    c = rows[:, 1]
    p, N = 3, 9
    h = 1.0 / N
    Phi = lambda x: gb.generating_function(p, x)
    for r in np.linspace(0.0, h, 13)[:-1]:
        phi, _ = gb.eval_basis(p, N, r)
        ghost = Phi(r / h + 1.0)            # phi_{-1}(r) = Phi((r + h)/h)
        for m in range(4):
            expect = Phi(r / h - m) + c[m] * ghost
            assert abs(phi[m] - expect) < 1e-14
    # the ghost weights are degree-3 extrapolation: exact for cubics
    for k in range(4):
        vals = np.arange(4.0) ** k
        assert abs(c @ vals - (-1.0) ** k) < 1e-13


@pytest.mark.parametrize("p,N", CASES)
def test_interpolatory(p, N):
    """u_i = u(x_i) (Eq. GD_basis_nodalformula): phi_i(x_j) = delta_ij."""
    for j in range(N + 1):
        phi, _ = gb.eval_basis(p, N, j / N)
        e = np.zeros(N + 1)
        e[j] = 1.0
        assert np.abs(phi - e).max() < 1e-13


@pytest.mark.parametrize("p,N", CASES)
def test_polynomial_reproduction(p, N):
    """Degree-p polynomials are reproduced exactly, with derivatives, on
    every cell (interior stencils and extrapolated boundary stencils)."""
    x_nodes = np.arange(N + 1) / N
    for r in _points(N):
        phi, dphi = gb.eval_basis(p, N, r)
        for m in range(p + 1):
            assert abs(phi @ x_nodes ** m - r ** m) < 1e-12
            d_exact = m * r ** (m - 1) if m > 0 else 0.0
            assert abs(dphi @ x_nodes ** m - d_exact) < 1e-9
    # degree p+1 is NOT reproduced on the interior (a dropped or extra
    # stencil node would still pass the test above only by accident)
    if N >= p + 2:
        err = max(abs(gb.eval_basis(p, N, r)[0] @ x_nodes ** (p + 1) - r ** (p + 1))
                  for r in _points(N))
        assert err > 1e-8


@pytest.mark.parametrize("p", [1, 3, 5, 7, 9])
def test_generating_function(p):
    """Phi_p is even with support [-q h, q h]; interior basis functions are
    its translates (Eq. GD_basis_lagrange); p = 1 is the hat function."""
    q = (p + 1) // 2
    xs = np.linspace(-q - 0.5, q + 0.5, 241)
    vals = np.array([gb.generating_function(p, x) for x in xs])
    assert np.allclose(vals, vals[::-1], atol=1e-14)
    assert np.all(vals[np.abs(xs) >= q] == 0.0)
    assert abs(gb.generating_function(p, 0.0) - 1.0) < 1e-15
    if p == 1:
        assert np.allclose(vals, np.maximum(0.0, 1.0 - np.abs(xs)), atol=1e-14)
    N = 4 * q + 4
    h = 1.0 / N
    i = N // 2
    for r in np.linspace((i - q) * h, (i + q) * h, 37)[:-1]:
        phi, _ = gb.eval_basis(p, N, r)
        assert abs(phi[i] - gb.generating_function(p, (r - i * h) / h)) < 1e-13


def test_p1_is_linear_fem():
    """p = 1: textbook linear FEM mass and stiffness matrices."""
    N = 6
    h = 1.0 / N
    M, S = gb.mass_stiffness(1, N)
    Mf = np.diag(np.full(N + 1, 2 * h / 3)) + np.diag(np.full(N, h / 6), 1) + np.diag(np.full(N, h / 6), -1)
    Mf[0, 0] = Mf[-1, -1] = h / 3
    Sf = (np.diag(np.full(N + 1, 2.0)) - np.diag(np.ones(N), 1) - np.diag(np.ones(N), -1)) / h
    Sf[0, 0] = Sf[-1, -1] = 1.0 / h
    assert np.abs(M - Mf).max() < 1e-15
    assert np.abs(S - Sf).max() < 1e-12


@pytest.mark.parametrize("p,N", CASES)
def test_matrix_structure(p, N):
    """Section 3.1: M symmetric positive definite with bandwidth p; S
    symmetric positive semi-definite, bandwidth p, kernel = constants."""
    M, S = gb.mass_stiffness(p, N)
    assert np.abs(M - M.T).max() < 1e-15
    assert np.abs(S - S.T).max() < 1e-11 * np.abs(S).max()
    k, l = np.indices(M.shape)
    assert np.all(M[np.abs(k - l) > p] == 0.0)
    assert np.all(S[np.abs(k - l) > p] == 0.0)
    assert np.linalg.eigvalsh(M).min() > 0.0
    ev = np.linalg.eigvalsh(S)
    assert abs(ev[0]) < 1e-10 * ev[-1]
    assert ev[1] > 1e-3                      # kernel is one-dimensional
    one = np.ones(N + 1)
    assert np.abs(S @ one).max() < 1e-10 * np.abs(S).max()
    assert abs(one @ M @ one - 1.0) < 1e-14  # integral of 1 over [0,1]
    x = np.arange(N + 1) / N
    assert abs(x @ M @ one - 0.5) < 1e-14    # integral of x
    assert abs(x @ S @ x - 1.0) < 1e-11      # integral of (x')^2


@pytest.mark.parametrize("p,N", CASES)
def test_face_data(p, N):
    phiL, phiR, dphiL, dphiR = gb.face_data(p, N)
    assert phiL[0] == 1.0 and np.count_nonzero(phiL) == 1
    assert phiR[-1] == 1.0 and np.count_nonzero(phiR) == 1
    assert np.all(dphiL[p + 1:] == 0.0) and np.all(dphiR[:N - p] == 0.0)
    assert abs(dphiL.sum()) < 1e-10 and abs(dphiR.sum()) < 1e-10
    x = np.arange(N + 1) / N
    assert abs(dphiL @ x - 1.0) < 1e-11 and abs(dphiR @ x - 1.0) < 1e-11
    # one-sided slope = derivative of the cell polynomial (finite difference)
    eps = 1e-6
    fd = (gb.eval_basis(p, N, eps, cell=0)[0] - gb.eval_basis(p, N, 0.0, cell=0)[0]) / eps
    assert np.abs(fd - dphiL).max() < 1e-3 * max(1.0, np.abs(dphiL).max())


@pytest.mark.parametrize("p,N", CASES)
def test_simultaneous_diagonalisation(p, N):
    """Section 3.2: Psi^T M Psi = I, Psi^T S Psi = diag(lambda), exactly one
    zero eigenvalue; eigenvalues agree with a library generalized solver."""
    from scipy.linalg import eigh
    M, S = gb.mass_stiffness(p, N)
    Psi, lam = gb.simultaneous_diagonalisation(M, S)
    assert np.abs(Psi.T @ M @ Psi - np.eye(N + 1)).max() < 1e-12
    assert np.abs(Psi.T @ S @ Psi - np.diag(lam)).max() < 1e-12 * lam.max()
    assert lam[0] == 0.0 and lam[1] > 1.0
    ref = eigh(S, M, eigvals_only=True)
    assert np.abs(ref[1:] - lam[1:]).max() < 1e-9 * lam.max()


def test_low_eigenvalues_are_neumann_laplacian():
    """The discrete Neumann Laplacian's low eigenvalues approach (k pi)^2
    with an error that shrinks as N grows."""
    errs = []
    for N in (8, 16, 32):
        M, S = gb.mass_stiffness(3, N)
        _, lam = gb.simultaneous_diagonalisation(M, S)
        errs.append(abs(lam[2] - (2 * np.pi) ** 2) / (2 * np.pi) ** 2)
        assert abs(lam[1] - np.pi ** 2) / np.pi ** 2 < 1e-3
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] / errs[2] > 8.0            # at least third order


@pytest.mark.parametrize("p,N,nq", [(3, 5, None), (5, 8, 8), (1, 3, 2)])
def test_composite_quadrature_is_exact_cell_by_cell(p, N, nq):
    """quadrature_points: nq Gauss points in every cell (p + 1 by default),
    each point inside the cell it is tagged with, weights summing to 1, and
    exact for any function that is a polynomial of degree <= 2 nq - 1 on each
    cell, kinks at the cell ends included; on degree 2 nq it misses by the
    Gauss remainder."""
    q = p + 1 if nq is None else nq
    r, w, cell = gb.quadrature_points(p, N, nq)
    assert r.shape == w.shape == cell.shape == (N * q,)
    assert np.array_equal(cell, np.floor(r * N).astype(int)) and np.all(w > 0)
    assert abs(w.sum() - 1.0) < 1e-14
    h = 1.0 / N
    d = 2 * q - 1
    left = cell * h
    f = (r - left) ** d * (1.0 + cell)            # a different polynomial on each cell
    exact = sum((1.0 + k) * h ** (d + 1) / (d + 1) for k in range(N))
    assert abs(np.dot(w, f) - exact) < 1e-14 * max(1.0, exact) + 1e-16
    # degree 2 nq: the Gauss remainder, h^(2n+1) (n!)^4 / ((2n+1) ((2n)!)^2) per
    # cell for x^(2n), n = nq (exact minus rule; the rule falls short)
    from math import factorial
    g = (r - left) ** (d + 1)
    rem = N * h ** (d + 2) * factorial(q) ** 4 / ((d + 2) * factorial(d + 1) ** 2)
    assert abs((N * h ** (d + 2) / (d + 2) - np.dot(w, g)) / rem - 1.0) < 1e-6
