"""The seeded synthetic inputs hold what the input recipe states: the
element-major nodal layout (x fastest), the sine map of the unit square onto
itself, the range and smoothness of the random c^2, the batched workload's
distributions, and the closed-form standing waves (which solve the wave
equation and carry v = u_t)."""
import numpy as np
import pytest

from paper_2105_01722_gb300 import inputs


def test_nodal_layout_2d_and_3d():
    nx, ny, N = 3, 2, 4
    X, Y = inputs.cartesian_nodes((nx, ny), N, lo=(0.5, -1.0), hi=(2.0, 1.0))
    assert X.shape == Y.shape == (ny, nx, N + 1, N + 1)
    Hx, Hy = 1.5 / nx, 2.0 / ny
    for ey in range(ny):
        for ex in range(nx):
            for j in range(N + 1):
                for i in range(N + 1):
                    assert abs(X[ey, ex, j, i] - (0.5 + (ex + i / N) * Hx)) < 1e-15
                    assert abs(Y[ey, ex, j, i] - (-1.0 + (ey + j / N) * Hy)) < 1e-15
    n3 = (2, 3, 4)
    X3, Y3, Z3 = inputs.cartesian_nodes_3d(n3, 2)
    assert X3.shape == (4, 3, 2, 3, 3, 3)
    ez, ey, ex, k, j, i = 3, 1, 1, 2, 0, 1
    assert abs(X3[ez, ey, ex, k, j, i] - (ex + i / 2) / 2) < 1e-15
    assert abs(Y3[ez, ey, ex, k, j, i] - (ey + j / 2) / 3) < 1e-15
    assert abs(Z3[ez, ey, ex, k, j, i] - (ez + k / 2) / 4) < 1e-15
    (X1,) = inputs.cartesian_nodes((5,), 3)
    assert X1.shape == (5, 4) and abs(X1[2, 1] - (2 + 1 / 3) / 5) < 1e-15


def test_sine_map_keeps_the_unit_square_and_its_orientation():
    g = np.linspace(0.0, 1.0, 41)
    XI, ETA = np.meshgrid(g, g, indexing="ij")
    X, Y = inputs.sine_map(XI, ETA, 0.05)
    assert np.array_equal(Y, ETA)
    for edge in (X[0, :], X[-1, :]):                     # xi = 0 and xi = 1 stay put
        assert np.abs(edge - edge[0]).max() < 1e-15
    assert np.abs(X[:, 0] - g).max() < 1e-15 and np.abs(X[:, -1] - g).max() < 1e-15
    # dx/dxi = 1 + 0.1 pi cos(2 pi xi) sin(2 pi eta) >= 1 - 0.1 pi > 0
    dxi = np.diff(X, axis=0)
    assert dxi.min() > 0
    assert X.min() >= 0.0 and X.max() <= 1.0


def test_smooth_random_c2_range_and_seeding():
    g = np.linspace(0.0, 1.0, 97)
    GX, GY = np.meshgrid(g, g)
    for seed in (1, 2, 3):
        c2 = inputs.smooth_random_c2(GX, GY, seed)
        # scaled so that max |s| = 1 on this grid: c^2 = 2^s reaches 1/2 or 2
        assert 0.5 - 1e-12 <= c2.min() and c2.max() <= 2.0 + 1e-12
        assert abs(np.log2(c2)).max() == pytest.approx(1.0, abs=1e-12)
    a = inputs.smooth_random_c2(GX, GY, 5)
    assert np.array_equal(a, inputs.smooth_random_c2(GX, GY, 5))
    assert np.abs(a - inputs.smooth_random_c2(GX, GY, 6)).max() > 0.1
    # smooth (a trigonometric polynomial of degree 3 in the exponent): on a
    # grid of spacing 1/96 neighbouring values differ by a few per cent
    assert np.abs(np.diff(np.log2(a), axis=0)).max() < 0.2


def test_batched_workload_distribution():
    probs = inputs.batched_problems()
    assert len(probs) == 48
    assert [q["seed"] for q in probs] == list(range(inputs.SEED0, inputs.SEED0 + 48))
    assert all(16 <= q["n"] <= 128 for q in probs)
    assert {q["p"] for q in probs} <= {3, 5, 7} and len({q["p"] for q in probs}) == 3
    assert [q["variable"] for q in probs] == [bool(i % 2) for i in range(48)]
    assert all(0.3 <= q["x0"] <= 0.7 and 0.3 <= q["y0"] <= 0.7 for q in probs)
    assert probs == inputs.batched_problems()          # deterministic
    dof = sum(q["n"] ** 2 * 81 for q in probs)
    assert 15e6 < dof < 35e6                             # about 24 M DOF in expectation


def test_pulse_and_standing_waves():
    assert inputs.gaussian_pulse(np.array(0.3), np.array(0.6), 0.3, 0.6, 0.05) == 1.0
    r = inputs.gaussian_pulse(np.array(0.35), np.array(0.6), 0.3, 0.6, 0.05)
    assert abs(r - np.exp(-1.0)) < 1e-15
    # u_tt = u_xx (1-D) and u_tt = u_xx + u_yy (2-D) by central differences;
    # v is u_t
    x, y, t, e = 0.31, 0.77, 0.4, 1e-4
    u1 = lambda x, t: inputs.standing_wave_1d(np.array(x), t)[0]
    utt = (u1(x, t + e) - 2 * u1(x, t) + u1(x, t - e)) / e ** 2
    uxx = (u1(x + e, t) - 2 * u1(x, t) + u1(x - e, t)) / e ** 2
    assert abs(utt - uxx) < 1e-5 * max(1.0, abs(uxx))
    ut = (u1(x, t + e) - u1(x, t - e)) / (2 * e)
    assert abs(ut - inputs.standing_wave_1d(np.array(x), t)[1]) < 1e-6
    u2 = lambda x, y, t: inputs.standing_mode_2d(np.array(x), np.array(y), t)[0]
    utt = (u2(x, y, t + e) - 2 * u2(x, y, t) + u2(x, y, t - e)) / e ** 2
    lap = (u2(x + e, y, t) + u2(x - e, y, t) + u2(x, y + e, t) + u2(x, y - e, t) - 4 * u2(x, y, t)) / e ** 2
    assert abs(utt - lap) < 1e-5 * max(1.0, abs(lap))
    ut = (u2(x, y, t + e) - u2(x, y, t - e)) / (2 * e)
    assert abs(ut - inputs.standing_mode_2d(np.array(x), np.array(y), t)[1]) < 1e-6
    # homogeneous Dirichlet data on the unit square
    assert abs(u2(0.0, y, t)) < 1e-15 and abs(u2(x, 1.0, t)) < 1e-15
