"""FP64 oracle of the Jacobi solver of the Laplace equation.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper (Sec. 4) reports a 13.5x speed-up of a sample application that
solves the Laplace equation by the Jacobi method and prints nothing else
about it.  The method, written out:

* u is an ny x nx grid; its first and last rows and columns are fixed
  (Dirichlet) boundary values, the rest is the unknown interior.
* One sweep replaces every interior point by the mean of its four
  neighbours, all read from the previous iterate:
      u'[i, j] = (u[i-1, j] + u[i+1, j] + u[i, j-1] + u[i, j+1]) / 4,
  and keeps the boundary.
* The change of a sweep is max over the interior of |u'[i, j] - u[i, j]|.
* Sweeps repeat while the last change exceeds tol and fewer than iter_max
  sweeps have run; the result is the last iterate, the number of sweeps and
  the last change.

Each step is a numpy array expression over whole slices of the grid (a
library primitive); there is no blocking or reordering beyond the formula.
"""
from __future__ import annotations

import numpy as np


def sweep(u):
    """One Jacobi sweep; returns (new grid, change)."""
    u = np.asarray(u, dtype=np.float64)
    v = u.copy()
    v[1:-1, 1:-1] = (u[:-2, 1:-1] + u[2:, 1:-1] + u[1:-1, :-2] + u[1:-1, 2:]) / 4.0
    change = float(np.abs(v[1:-1, 1:-1] - u[1:-1, 1:-1]).max()) if v.shape[0] > 2 and v.shape[1] > 2 else 0.0
    return v, change


def solve(u0, tol: float, iter_max: int):
    """Sweeps while the change exceeds tol and fewer than iter_max ran:
    returns (grid, sweeps, last change)."""
    u = np.asarray(u0, dtype=np.float64)
    k, change = 0, np.inf
    while change > tol and k < iter_max:
        u, change = sweep(u)
        k += 1
    return u, k, (change if k else 0.0)
