"""Jacobi solver of the Laplace equation on the GPU (net_jacobi_*) against
the FP64 oracle (oracle/jacobi.py).

The kernels sweep in FP32.  One sweep from the same grid differs from the
FP64 sweep by the rounding of three additions and a multiplication (<= 2^-21
of the grid's largest value); k sweeps by at most k times that (a sweep
never amplifies a difference: it averages).  The stopping decision is taken
in FP32 on the device: the GPU's sweep count must sit where its own change
crossed tol, and within a few sweeps of the oracle's."""
import numpy as np
import pytest

from oracle import jacobi
from paper_1811_03882_gb300 import synth

pytestmark = pytest.mark.gpu
ULP = 2.0 ** -21


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1811_03882_gb300 import build
    build.build()


def _solver(ny, nx):
    from paper_1811_03882_gb300 import binding
    return binding.Jacobi(ny, nx)


def _nerr(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-30))


@pytest.mark.parametrize("ny,nx,interior", [(64, 64, "zero"), (37, 53, "random"), (3, 3, "random"),
                                            (3, 130, "random"), (131, 3, "random"), (70, 2050, "zero"),
                                            (257, 515, "random")])
def test_one_sweep_and_ragged_shapes(ny, nx, interior):
    u0 = synth.laplace_grid(21, ny, nx, interior)
    ref, ch = jacobi.sweep(u0.astype(np.float64))
    with _solver(ny, nx) as J:
        out, k, gch = J.solve(u0, 0.0, 1)
    assert k == 1
    assert _nerr(out, ref) <= 4 * ULP
    assert abs(gch - ch) <= 4 * ULP * max(np.abs(ref).max(), 1e-30)
    np.testing.assert_array_equal(out[0], u0[0])           # boundary untouched
    np.testing.assert_array_equal(out[:, -1], u0[:, -1])


def test_many_sweeps_match_oracle():
    ny, nx = 301, 403
    u0 = synth.laplace_grid(22, ny, nx, "random")
    ref, _, ch = jacobi.solve(u0.astype(np.float64), 0.0, 200)
    with _solver(ny, nx) as J:
        out, k, gch = J.solve(u0, 0.0, 200)      # tol 0: exactly iter_max sweeps
        out2, k2, _ = J.solve(u0, 0.0, 200)      # the handle is reusable
    assert k == k2 == 200
    np.testing.assert_array_equal(out, out2)
    assert _nerr(out, ref) <= 200 * 4 * ULP
    assert abs(gch - ch) <= 200 * 4 * ULP * np.abs(ref).max()


def test_stopping_rule_and_degenerate_calls():
    ny, nx = 96, 96
    u0 = synth.laplace_grid(23, ny, nx, "zero")
    tol = 1e-3
    ref, kr, chr_ = jacobi.solve(u0.astype(np.float64), tol, 100000)
    with _solver(ny, nx) as J:
        out, k, gch = J.solve(u0, tol, 100000)
        assert gch <= tol
        assert abs(k - kr) <= 3, (k, kr)
        # the sweep before the stop had not converged, by the GPU's own change
        _, kb, chb = J.solve(u0, 0.0, k - 1)
        assert kb == k - 1 and chb > tol
        assert _nerr(out, jacobi.solve(u0.astype(np.float64), 0.0, k)[0]) <= k * 4 * ULP
        same, k0, c0 = J.solve(u0, tol, 0)        # iter_max 0: the input back
        assert k0 == 0 and c0 == 0.0
        np.testing.assert_array_equal(same, u0)
        _, k1, _ = J.solve(u0, 10.0, 50)          # tol above any change: one sweep
        assert k1 == 1
        _, k7, _ = J.solve(u0, 0.0, 7)            # iter_max not a multiple of the graph chunk
        assert k7 == 7
        from paper_1811_03882_gb300 import binding
        with pytest.raises(binding.NetError) as e:
            J.solve(u0, -1.0, 5)
        assert e.value.status == binding.NET_E_INVAL
    with pytest.raises(binding.NetError) as e:
        _solver(2, 100)                           # no interior
    assert e.value.status == binding.NET_E_INVAL


def test_device_api_full_size():
    """The bench's grid (8192 x 8192, both iterates 268 MB, above L2) through
    the device-buffer entry point, two sweeps, against the oracle."""
    import torch
    ny = nx = 8192
    u0 = synth.laplace_grid(24, ny, nx, "random")
    ref, _, ch = jacobi.solve(u0.astype(np.float64), 0.0, 2)
    d_in = torch.from_numpy(u0).cuda()
    d_out = torch.empty_like(d_in)
    with _solver(ny, nx) as J:
        k, gch = J.solve_device(d_in, 0.0, 2, d_out)
    assert k == 2
    assert _nerr(d_out.cpu().numpy(), ref) <= 8 * ULP


@pytest.mark.parametrize("rows", ["8", "32", "200"])
def test_strip_height_does_not_change_the_result(rows, monkeypatch):
    """Every point's new value depends only on the previous iterate, so the
    strip height (NET_JACOBI_ROWS; 64 rows by default) changes neither the
    grid nor the stopping decision,
    bit for bit.  With 8-row strips the grid has more tiles (513 x 5) than
    a GB300 has resident blocks (16 x 152), so blocks take a second tile."""
    ny, nx = 4099, 2050
    u0 = synth.laplace_grid(25, ny, nx, "random")
    with _solver(ny, nx) as J:
        ref, kr, cr = J.solve(u0, 1e-4, 40)
    monkeypatch.setenv("NET_JACOBI_ROWS", rows)
    with _solver(ny, nx) as J:
        out, k, c = J.solve(u0, 1e-4, 40)
    assert (k, c) == (kr, cr)
    np.testing.assert_array_equal(out, ref)


@pytest.mark.parametrize("ny,nx,interior,tol,iters", [
    (96, 96, "zero", 1e-3, 100000), (96, 96, "zero", 9e-4, 100000), (96, 96, "zero", 8e-4, 100000),
    (37, 53, "random", 0.0, 7), (3, 130, "random", 0.0, 5), (131, 3, "random", 0.0, 4),
    (257, 515, "random", 0.0, 33), (300, 2050, "random", 2e-4, 999), (4099, 2050, "random", 0.0, 3)])
def test_fused_pairs_match_single_sweeps(ny, nx, interior, tol, iters, monkeypatch):
    """Sweeps run in fused pairs (one pass over the grid computes two; a pair
    whose first sweep meets the stopping rule is redone as a single sweep).
    Each value is the single sweep's expression, so the grid, the sweep count
    and the last change equal the one-sweep-a-launch path's
    (NET_JACOBI_FUSE=0) bit for bit, whichever sweep the rule stops at
    (odd and even counts; stops inside and at the end of a graph chunk)."""
    u0 = synth.laplace_grid(26, ny, nx, interior)
    with _solver(ny, nx) as J:
        out, k, ch = J.solve(u0, tol, iters)
    monkeypatch.setenv("NET_JACOBI_FUSE", "0")
    with _solver(ny, nx) as J:
        out1, k1, ch1 = J.solve(u0, tol, iters)
    assert (k, ch) == (k1, ch1)
    np.testing.assert_array_equal(out, out1)
    if tol == 0.0:
        assert k == iters
