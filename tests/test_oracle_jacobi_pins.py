"""Pins of the Jacobi oracle (oracle/jacobi.py) against facts that do not
come from it: a hand-worked sweep, the eigenvalues of the Jacobi iteration
matrix (a sine mode with zero boundary is scaled by
(cos(pi p/(nx-1)) + cos(pi q/(ny-1)))/2 per sweep), discrete-harmonic grids
as fixed points, convergence to the discrete solution, brute force in plain
Python, and the stopping rule."""
import math

import numpy as np
import pytest

from oracle import jacobi


def test_hand_sweep():
    u = np.array([[0.0, 1.0, 0.0, 0.0],
                  [2.0, 5.0, 7.0, 3.0],
                  [0.0, 4.0, 8.0, 0.0],
                  [0.0, 6.0, 1.0, 0.0]])
    v, ch = jacobi.sweep(u)
    # (1,1): (1 + 4 + 2 + 7)/4 = 3.5; (1,2): (0 + 8 + 5 + 3)/4 = 4
    # (2,1): (5 + 6 + 0 + 8)/4 = 4.75; (2,2): (7 + 1 + 4 + 0)/4 = 3
    want = u.copy()
    want[1, 1:3] = [3.5, 4.0]
    want[2, 1:3] = [4.75, 3.0]
    np.testing.assert_array_equal(v, want)
    assert ch == max(abs(3.5 - 5), abs(4 - 7), abs(4.75 - 4), abs(3 - 8))


def test_sweep_brute_force():
    rng = np.random.default_rng(2)
    u = rng.random((7, 9))
    v, ch = jacobi.sweep(u)
    w = [row[:] for row in u.tolist()]
    best = 0.0
    for i in range(1, 6):
        for j in range(1, 8):
            w[i][j] = (u[i - 1][j] + u[i + 1][j] + u[i][j - 1] + u[i][j + 1]) / 4.0
            best = max(best, abs(w[i][j] - u[i][j]))
    np.testing.assert_allclose(v, np.array(w), rtol=0, atol=1e-15)
    assert ch == pytest.approx(best, abs=1e-15)


@pytest.mark.parametrize("p,q", [(1, 1), (2, 3), (5, 1)])
def test_sine_mode_is_an_eigenvector(p, q):
    ny, nx = 33, 41
    y = np.arange(ny)[:, None] / (ny - 1)
    x = np.arange(nx)[None, :] / (nx - 1)
    u = np.sin(math.pi * q * y) * np.sin(math.pi * p * x)
    u[0, :] = u[-1, :] = 0.0
    u[:, 0] = u[:, -1] = 0.0
    lam = (math.cos(math.pi * p / (nx - 1)) + math.cos(math.pi * q / (ny - 1))) / 2.0
    v, _ = jacobi.sweep(u)
    np.testing.assert_allclose(v, lam * u, rtol=0, atol=1e-14)
    w, k, _ = jacobi.solve(u, 0.0, 5)
    assert k == 5
    np.testing.assert_allclose(w, lam ** 5 * u, rtol=0, atol=1e-13)


def test_discrete_harmonic_fixed_point():
    ny, nx = 20, 27
    y = np.arange(ny, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    for u in (x * x - y * y, 3 * x * y + 2 * x - y + 5, np.ones((ny, nx)) * 0.25):
        u = np.broadcast_to(u, (ny, nx)).copy()
        v, ch = jacobi.sweep(u)
        np.testing.assert_allclose(v, u, rtol=0, atol=1e-12)
        assert ch <= 1e-12


def test_converges_to_discrete_solution_and_stops():
    ny, nx = 24, 24
    y = np.arange(ny, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    exact = (x * y) / (nx * ny)
    u0 = exact.copy()
    u0[1:-1, 1:-1] = 0.0
    u, k, ch = jacobi.solve(u0, 1e-10, 100000)
    assert ch <= 1e-10 < jacobi.solve(u0, 0.0, k - 1)[2]   # sweep k - 1 had not converged
    assert np.abs(u - exact).max() < 1e-7
    assert k < 100000
    u2, k2, _ = jacobi.solve(u0, 0.0, 7)      # tol 0: exactly iter_max sweeps
    assert k2 == 7
    w = u0
    for _ in range(7):
        w, _ = jacobi.sweep(w)
    np.testing.assert_array_equal(u2, w)
