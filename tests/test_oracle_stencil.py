"""Pins of the isotropic central stencils: exact on low-order polynomials."""
import numpy as np

from oracle import lbm as olbm


def _interior(a, k=2):
    return a[..., k:-k, k:-k] if a.ndim == 2 or a.shape[0] > 3 else a


def test_gradient_exact_on_linear_and_laplacian_on_quadratic_2d():
    y, x = np.meshgrid(np.arange(20.0), np.arange(24.0), indexing="ij")
    lin = 0.3 * x - 1.7 * y + 2.0
    quad = 0.5 * x * x + 0.25 * y * y - 0.1 * x * y + x
    g, lap = olbm.grad_lap(lin, (True, True))
    s = (slice(2, -2), slice(2, -2))   # away from the periodic seam
    assert np.allclose(g[0][s], 0.3, atol=1e-12) and np.allclose(g[1][s], -1.7, atol=1e-12)
    assert np.allclose(lap[s], 0.0, atol=1e-12)
    g, lap = olbm.grad_lap(quad, (True, True))
    assert np.allclose(lap[s], 1.5, atol=1e-11)
    assert np.allclose(g[0][s], (x - 0.1 * y + 1)[s], atol=1e-11)
    assert np.allclose(g[1][s], (0.5 * y - 0.1 * x)[s], atol=1e-11)


def test_gradient_exact_on_quadratic_3d():
    z, y, x = np.meshgrid(np.arange(9.0), np.arange(8.0), np.arange(10.0), indexing="ij")
    f = x * x - 2 * y * y + 0.5 * z * z + x * z
    g, lap = olbm.grad_lap(f, (True, True, True))
    s = (slice(2, -2),) * 3
    assert np.allclose(lap[s], -1.0, atol=1e-11)
    assert np.allclose(g[0][s], (2 * x + z)[s], atol=1e-11)
    assert np.allclose(g[2][s], (z + x)[s], atol=1e-11)


def test_mirror_ghost_gives_zero_normal_gradient():
    # a field that is even about the half-way wall has zero y-derivative at the first row's ghost
    y, x = np.meshgrid(np.arange(10.0), np.arange(6.0), indexing="ij")
    f = np.cos(0.3 * x) + 0 * y
    g, _ = olbm.grad_lap(f, (True, False))
    assert np.allclose(g[1], 0.0, atol=1e-14)
