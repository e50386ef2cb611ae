"""The C-ABI library loads, exports every symbol include/gdg.h declares, and
its host-side logic (basis builder, argument validation) behaves; no GPU
compute here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2105_01722_gb300 import gdg
from oracle import gd_basis as gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    if not os.path.exists(gdg.LIB_PATH):
        from paper_2105_01722_gb300 import build
        build.build(verbose=False)
    return gdg.lib()


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            txt = open(os.path.join(inc, f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(gdg_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol():
    L = _lib()
    names = _declared()
    assert {"gdg_create", "gdg_rhs", "gdg_step", "gdg_energy", "gdg_pcg", "gdg_mass_solve"} <= names
    for n in sorted(names):
        assert hasattr(L, n), n
    # and the binding knows all of them
    assert names <= set(gdg.EXPORTS)


@pytest.mark.parametrize("p,N", [(1, 1), (1, 5), (3, 3), (3, 8), (5, 8), (7, 8), (5, 11), (7, 15)])
def test_library_basis_matches_oracle(p, N):
    """The library's own host basis builder (independent code) agrees with
    the oracle's: matrices, face data, eigenvalues, and the modified basis
    up to the sign of each column."""
    _lib()
    b = gdg.basis_1d(p, N)
    M, S = gb.mass_stiffness(p, N)
    phiL, phiR, dphiL, dphiR = gb.face_data(p, N)
    Psi, lam = gb.simultaneous_diagonalisation(M, S)
    assert np.abs(b["M"] - M).max() < 1e-14
    assert np.abs(b["S"] - S).max() < 1e-11 * np.abs(S).max()
    for k, ref in (("phiL", phiL), ("phiR", phiR)):
        assert np.abs(b[k] - ref).max() < 1e-15
    for k, ref in (("dphiL", dphiL), ("dphiR", dphiR)):
        assert np.abs(b[k] - ref).max() < 1e-10 * np.abs(ref).max()
    assert np.abs(b["lam"] - lam).max() < 1e-9 * lam.max()
    P = b["Psi"]
    assert np.abs(P.T @ M @ P - np.eye(N + 1)).max() < 1e-11
    for k in range(N + 1):
        s = np.sign(P[:, k] @ M @ Psi[:, k])
        assert np.abs(P[:, k] - s * Psi[:, k]).max() < 1e-8


def test_basis_argument_errors():
    L = _lib()
    null = ctypes.c_void_p()
    assert L.gdg_basis_1d(2, 8, *([null] * 8)) == gdg.EINVAL
    assert L.gdg_basis_1d(0, 8, *([null] * 8)) == gdg.EINVAL
    assert L.gdg_basis_1d(5, 4, *([null] * 8)) == gdg.EINVAL
    assert L.gdg_basis_1d(3, 16, *([null] * 8)) == gdg.EUNSUPPORTED
    assert L.gdg_basis_1d(3, 8, *([null] * 8)) == gdg.OK


@pytest.mark.parametrize("bad", [
    dict(p=4), dict(p=5, N=3), dict(N=16), dict(n=(0, 4)), dict(c2=-1.0), dict(flux=7),
    dict(bc=(3, 0)), dict(hi=(0.0, 1.0)), dict(coef=gdg.COEF_NODAL),
])
def test_create_rejects_bad_problems(bad):
    """Validation happens before any device work, so it runs without a GPU."""
    L = _lib()
    kw = dict(dim=2, n=(4, 4), N=8, p=5)
    kw.update(bad)
    pb = gdg.make_problem(**kw)
    h = ctypes.c_void_p()
    st = L.gdg_create(ctypes.byref(pb), ctypes.byref(h))
    assert st in (gdg.EINVAL, gdg.EUNSUPPORTED)
    assert not h


def _nodal_kw(**extra):
    import numpy as np
    from paper_2105_01722_gb300 import inputs
    X, Y = inputs.cartesian_nodes((2, 2), 8)
    kw = dict(dim=2, n=(2, 2), N=8, p=5, coef=gdg.COEF_NODAL, x_nodes=X, y_nodes=Y,
              c2_nodes=np.ones_like(X))
    kw.update(extra)
    return kw


@pytest.mark.parametrize("kw, status", [
    (dict(dim=3, n=(2, 2, 2), N=8, p=5, route=gdg.ROUTE_NODAL), "EUNSUPPORTED"),    # nodal route: dim <= 2
    (dict(dim=2, n=(4, 4), N=8, p=5, precision=gdg.MIXED), "EUNSUPPORTED"),      # nothing to refine
    ("inverse_mixed", "EUNSUPPORTED"),
    ("nodal_diag", "EINVAL"),
    ("ic0", "EUNSUPPORTED"),                                                    # oracle only
    ("tf32", "EUNSUPPORTED"),                                                   # refinement would stall
    ("bf16", "EUNSUPPORTED"),
    (dict(dim=3, n=(2, 2, 2), N=10, p=5), "EUNSUPPORTED"),                      # 3-D: N+1 <= 10
    (dict(dim=4, n=(2, 2, 2), N=8, p=5), "EINVAL"),
])
def test_create_rejects_unbuilt_combinations(kw, status):
    """Combinations that are not built are refused, never silently ignored."""
    L = _lib()
    if kw == "inverse_mixed":
        kw = _nodal_kw(solver=gdg.SOLVE_INVERSE, precision=gdg.MIXED)
    elif kw == "nodal_diag":
        kw = _nodal_kw(solver=gdg.SOLVE_DIAG)
    elif kw == "ic0":
        kw = _nodal_kw(precond=gdg.PC_IC0)
    elif kw in ("tf32", "bf16"):
        kw = _nodal_kw(precision=gdg.TF32 if kw == "tf32" else gdg.BF16)
    pb = gdg.make_problem(**kw)
    h = ctypes.c_void_p()
    assert L.gdg_create(ctypes.byref(pb), ctypes.byref(h)) == getattr(gdg, status)
    assert not h


def test_null_arguments():
    L = _lib()
    assert L.gdg_create(None, None) == gdg.EINVAL
    assert L.gdg_rhs(None, None, None, 0.0, None, None, None) == gdg.EINVAL
    assert L.gdg_step(None, None, None, 0.0, 1e-3, 1, None) == gdg.EINVAL
    assert L.gdg_destroy(None) == gdg.EINVAL
    assert L.gdg_state_len(None) == -1
    for s in (0, -1, -2, -3, -4, -5, -6, -7, -8, -99):
        assert isinstance(L.gdg_status_string(s), bytes)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(gdg, "_LIB", None)
    monkeypatch.setattr(gdg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        gdg.lib()


def test_ordinary_build_has_no_index_checks():
    """The index checks exist only in the GDG_CHECKS build: the ordinary
    library answers GDG_EUNSUPPORTED before touching the device."""
    import ctypes
    L = gdg.lib()
    c, si, i, b = ctypes.c_longlong(7), ctypes.c_int(7), ctypes.c_longlong(7), ctypes.c_longlong(7)
    st = L.gdg_check_status(ctypes.byref(c), ctypes.byref(si), ctypes.byref(i), ctypes.byref(b), 0)
    assert st == gdg.EUNSUPPORTED and (c.value, si.value, i.value, b.value) == (0, 0, 0, 0)
    assert L.gdg_check_selftest(5, 3, None) == gdg.EUNSUPPORTED
