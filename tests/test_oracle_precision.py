"""Why the mixed form's inner solves are FP32 and not TF32 or BF16: iterative
refinement of the element systems of Section 7.1 (FP64 residuals, inner
solves with the matrix rounded to the lower precision) converges at a rate
of about kappa x u_low per sweep (u_low the low precision's unit roundoff),
so it needs kappa u_low < 1.  The u_t systems have kappa ~ 1e3 (p = 3) to
1e5 (p = 7): with TF32 (u = 2^-11) or BF16 (u = 2^-8) they need several
times the FP32 sweeps at p = 5, each an FP64 matrix product (the mixed
form's cost), and do not converge at all at p = 7.  The inner solves here
are exact with the rounded matrix, the best a reduced-precision PCG could do.
Oracle matrices on the sine-mapped mesh with c^2 = 1 + 0.5 sin 2pi x cos 2pi y."""
import numpy as np
import pytest

from oracle import dg_var as dv
from paper_2105_01722_gb300 import inputs

MANTISSA = {"fp32": 23, "tf32": 10, "bf16": 7}


def _round(A, bits):
    """Round to nearest with `bits` explicit mantissa bits."""
    m, e = np.frexp(A)
    scale = 2.0 ** (bits + 1)
    return np.ldexp(np.round(m * scale) / scale, e)


def _sweeps_to(A, b, bits, rtol=1e-10, maxsweep=30):
    """FP64 iterative refinement with exact inner solves on the rounded
    matrix: sweeps until ||b - A x|| <= rtol ||b|| (None if it never gets there)."""
    Al = _round(A, bits)
    x = np.zeros_like(b)
    r = b.copy()
    for k in range(1, maxsweep + 1):
        x = x + np.linalg.solve(Al, r)
        r = b - A @ x
        if np.linalg.norm(r) <= rtol * np.linalg.norm(b):
            return k
    return None


@pytest.fixture(scope="module")
def systems():
    out = {}
    rng = np.random.default_rng(1)
    for p in (3, 5, 7):
        X, Y = inputs.mapped_nodes((2, 2), 8, 0.05)
        vp = dv.VarProblem(n=(2, 2), N=8, p=p, X=X, Y=Y, C2=inputs.c2_sine(X, Y))
        ops = dv.assemble(vp)
        out[p] = (dv.spd_u_matrix(ops, 0), rng.standard_normal(81))
    return out


def test_fp32_inner_solves_refine_every_order(systems):
    for p, (A, b) in systems.items():
        assert _sweeps_to(A, b, MANTISSA["fp32"]) <= 3, p


def test_tf32_and_bf16_need_more_sweeps_or_diverge(systems):
    A, b = systems[5]                               # kappa ~ 5e3
    fp32 = _sweeps_to(A, b, MANTISSA["fp32"])
    tf32 = _sweeps_to(A, b, MANTISSA["tf32"])
    bf16 = _sweeps_to(A, b, MANTISSA["bf16"])
    assert tf32 >= 2 * fp32 and bf16 >= 5 * fp32, (fp32, tf32, bf16)
    A, b = systems[7]                               # kappa ~ 1e5 > 1 / u_low
    assert _sweeps_to(A, b, MANTISSA["tf32"]) is None
    assert _sweeps_to(A, b, MANTISSA["bf16"]) is None
    assert _sweeps_to(A, b, MANTISSA["fp32"]) is not None
