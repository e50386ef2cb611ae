"""Pins of the oracle's 3-D constant-coefficient semi-discretisation (the
tensor-product construction of Sections 2.1.2 and 3 for d = 3): brute-force
energy identities on tiny meshes, reduction to the (separately pinned) 2-D
oracle for data that do not depend on one coordinate on a mesh periodic in
it, and convergence on an exact 3-D standing wave."""
import numpy as np
import pytest

from oracle import dg_const as dc, timeint as ti

FLUXES = ["central", "upwind", "alternating"]


def _p3(n, N, p, periodic, flux, c2=1.0, hi=(1.0, 1.0, 1.0)):
    return dc.Problem(dim=3, n=n, N=N, p=p, lo=(0.0, 0.0, 0.0), hi=hi, periodic=periodic, flux=flux, c2=c2)


@pytest.mark.parametrize("flux", FLUXES)
@pytest.mark.parametrize("periodic", [(False, False, False), (True, False, True)])
def test_energy_identities_3d(flux, periodic):
    """Central and alternating: E L + L^T E = 0 (conservative); upwind:
    -(E L + L^T E) positive semidefinite and nonzero (dissipative)."""
    prob = _p3((1, 2, 1), 3, 3, periodic, flux, c2=1.6, hi=(1.0, 0.8, 1.2))
    L = dc.dense_operator(prob)
    E = dc.energy_matrix(prob)
    A = E @ L + L.T @ E
    if flux == "upwind":
        lam = np.linalg.eigvalsh(-0.5 * (A + A.T))
        assert lam.min() > -1e-10 * np.abs(lam).max() and lam.max() > 1e-3
    else:
        assert np.abs(A).max() < 1e-11 * np.abs(E @ L).max()


@pytest.mark.parametrize("flux", FLUXES)
def test_reduces_to_2d_for_z_independent_data(flux):
    p3 = _p3((3, 2, 2), 4, 3, (False, True, True), flux, c2=1.3, hi=(1.0, 0.7, 0.9))
    p2 = dc.Problem(dim=2, n=(3, 2), N=4, p=3, lo=(0.0, 0.0), hi=(1.0, 0.7), periodic=(False, True),
                    flux=flux, c2=1.3)
    rng = np.random.default_rng(0)
    U2 = rng.standard_normal((2, 3, 5, 5))
    V2 = rng.standard_normal((2, 3, 5, 5))
    U3 = np.broadcast_to(U2[None, :, :, None, :, :], (2, 2, 3, 5, 5, 5))
    V3 = np.broadcast_to(V2[None, :, :, None, :, :], (2, 2, 3, 5, 5, 5))
    Ut2, Vt2 = dc.time_derivative(p2, U2.reshape(6, -1), V2.reshape(6, -1))
    Ut3, Vt3 = dc.time_derivative(p3, U3.reshape(12, -1), V3.reshape(12, -1))
    ref_u = np.broadcast_to(Ut2.reshape(2, 3, 5, 5)[None, :, :, None], (2, 2, 3, 5, 5, 5))
    ref_v = np.broadcast_to(Vt2.reshape(2, 3, 5, 5)[None, :, :, None], (2, 2, 3, 5, 5, 5))
    assert np.abs(Ut3.reshape(ref_u.shape) - ref_u).max() < 1e-12 * np.abs(ref_u).max()
    assert np.abs(Vt3.reshape(ref_v.shape) - ref_v).max() < 1e-12 * np.abs(ref_v).max()


@pytest.mark.parametrize("flux", FLUXES)
def test_reduces_to_2d_for_x_independent_data(flux):
    """Data independent of x on an x-periodic mesh: the (y, z) problem, i.e.
    the 2-D oracle with its x, y taken as the 3-D y, z (pins the z faces)."""
    p3 = _p3((2, 3, 2), 4, 3, (True, False, True), flux, c2=0.8, hi=(0.6, 1.0, 0.9))
    p2 = dc.Problem(dim=2, n=(3, 2), N=4, p=3, lo=(0.0, 0.0), hi=(1.0, 0.9), periodic=(False, True),
                    flux=flux, c2=0.8)
    rng = np.random.default_rng(1)
    U2 = rng.standard_normal((2, 3, 5, 5))        # [ez, ey, k, j]
    V2 = rng.standard_normal((2, 3, 5, 5))
    shape = (2, 3, 2, 5, 5, 5)                    # [ez, ey, ex, k, j, i]
    U3 = np.broadcast_to(U2[:, :, None, :, :, None], shape)
    V3 = np.broadcast_to(V2[:, :, None, :, :, None], shape)
    Ut2, Vt2 = dc.time_derivative(p2, U2.reshape(6, -1), V2.reshape(6, -1))
    Ut3, Vt3 = dc.time_derivative(p3, U3.reshape(12, -1), V3.reshape(12, -1))
    ref_u = np.broadcast_to(Ut2.reshape(2, 3, 5, 5)[:, :, None, :, :, None], shape)
    ref_v = np.broadcast_to(Vt2.reshape(2, 3, 5, 5)[:, :, None, :, :, None], shape)
    assert np.abs(Ut3.reshape(shape) - ref_u).max() < 1e-12 * np.abs(ref_u).max()
    assert np.abs(Vt3.reshape(shape) - ref_v).max() < 1e-12 * np.abs(ref_v).max()


def _standing_wave_3d(t, x, y, z):
    w = np.sqrt(3.0) * np.pi
    sx, sy, sz = np.sin(np.pi * x), np.sin(np.pi * y), np.sin(np.pi * z)
    cx, cy, cz = np.cos(np.pi * x), np.cos(np.pi * y), np.cos(np.pi * z)
    u = np.cos(w * t) * sx * sy * sz
    grad = [np.cos(w * t) * np.pi * cx * sy * sz, np.cos(w * t) * np.pi * sx * cy * sz,
            np.cos(w * t) * np.pi * sx * sy * cz]
    return u, grad, -w * np.sin(w * t) * sx * sy * sz


@pytest.mark.parametrize("flux", ["upwind", "central"])
def test_convergence_3d_dirichlet(flux):
    """sin(pi x) sin(pi y) sin(pi z) cos(sqrt3 pi t) on the unit cube with u = 0:
    the L2 error falls at about the optimal rate p + 1 = 4 as elements are added."""
    errs = []
    for n in (1, 2, 4):
        prob = _p3((n, n, n), 4, 3, (False, False, False), flux)
        ops = dc.operators(prob)
        X, Y, Z = dc.node_coordinates(prob)
        U = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
        V = np.zeros_like(U)
        h = 1.0 / (n * 4)
        T = 0.1
        steps = int(np.ceil(T / (0.05 * h)))
        f = lambda t, U, V: dc.time_derivative(prob, U, V, ops)
        U, V = ti.integrate(f, U.reshape(n ** 3, -1), V.reshape(n ** 3, -1), 0.0, T / steps, steps)
        errs.append(ti.errors(prob, U, V, _standing_wave_3d, T)[0])
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > 3.5, (errs, rates)
