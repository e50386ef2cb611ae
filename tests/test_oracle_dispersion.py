"""Dispersion and dissipation of the semi-discretisation (Section 4's
Bloch-wave analysis, restated as tests on the oracle): on a periodic 1-D
mesh of n elements the eigenvalues of the dense semi-discrete operator
contain the physical branch i*2*pi*m (each element sees the Bloch phases
2*pi*j/n).  Pinned: the physical frequencies converge at high order as
elements are added, the conservative fluxes (central, alternating) keep the
physical modes undamped, and the upwind flux damps them by an amount that
vanishes under refinement."""
import numpy as np
import pytest

from oracle import dg_const as dc


def _physical(flux, p, n, modes=(1, 2, 3)):
    prob = dc.Problem(dim=1, n=(n,), N=8, p=p, flux=flux, periodic=(True,))
    ev = np.linalg.eigvals(dc.dense_operator(prob))
    out = []
    for m in modes:
        w = 2 * np.pi * m
        lam = ev[np.argmin(np.abs(ev - 1j * w))]
        out.append((abs(lam.imag - w) / w, lam.real / w))
    return np.array(out)


@pytest.mark.parametrize("flux", ["central", "upwind", "alternating"])
@pytest.mark.parametrize("p", [3, 5])
def test_physical_branch_converges(flux, p):
    e4, e8 = _physical(flux, p, 4), _physical(flux, p, 8)
    # frequency error of the best-resolved mode falls faster than h^(p+1/2)
    rate = np.log2(e4[0, 0] / e8[0, 0])
    assert rate > p + 0.5, rate
    assert e8[0, 0] < (1e-6 if p == 3 else 1e-10)
    # fewer points per wavelength, larger dispersion error
    assert e8[0, 0] < e8[1, 0] < e8[2, 0]


@pytest.mark.parametrize("flux", ["central", "alternating"])
def test_conservative_fluxes_do_not_damp(flux):
    for n in (2, 4):
        e = _physical(flux, 3, n)
        assert np.abs(e[:, 1]).max() < 1e-11


def test_upwind_damps_resolved_modes_less_under_refinement():
    d = [-_physical("upwind", 3, n)[0, 1] for n in (2, 4, 8)]
    assert all(x > 0 for x in d)                      # dissipative
    assert d[0] > d[1] > d[2] and d[2] < 1e-6         # vanishing for resolved modes
