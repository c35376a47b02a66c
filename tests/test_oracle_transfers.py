"""Pins for the oracle's grid transfers (Section 3.1 deflation vectors; multigrid FW / bilinear)."""
import numpy as np
import pytest

import model_problems as mp
from oracle.transfers import (bilinear_prolong, deflation_prolong, deflation_restrict, fw_restrict)


@pytest.mark.parametrize("shape", [(9, 9), (17, 33), (33, 17)])
def test_deflation_prolongation_reproduces_bilinear_functions(shape):
    """Z maps samples of a + b x + c y + d x y at coarse nodes (fine coordinates 2I)
    to the same function at every fine node not within 1 of the boundary."""
    ny, nx = shape
    nyc, nxc = (ny + 1) // 2, (nx + 1) // 2
    f = lambda X, Y: 1.5 - 0.25 * X + 0.75 * Y + 0.1 * X * Y + 0j
    Xc, Yc = np.meshgrid(2.0 * np.arange(nxc), 2.0 * np.arange(nyc))
    Xf, Yf = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    t = deflation_prolong(f(Xc, Yc), shape)
    np.testing.assert_allclose(t[1:-1, 1:-1], f(Xf, Yf)[1:-1, 1:-1], rtol=1e-14, atol=1e-13)


def test_deflation_restriction_is_transpose():
    ny, nx = 17, 25
    v = mp.random_complex((ny, nx), seed=1)
    w = mp.random_complex(((ny + 1) // 2, (nx + 1) // 2), seed=2)
    lhs = np.vdot(deflation_restrict(v), w)
    rhs = np.vdot(v, deflation_prolong(w, (ny, nx)))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_deflation_restriction_weights():
    """Z^T of a unit vector at an interior fine node spreads the weights p_a p_b,
    p = [1, 4, 6, 4, 1] / 8, to the coarse nodes whose support contains it."""
    ny = nx = 17
    v = np.zeros((ny, nx), complex)
    v[8, 8] = 1.0                                  # coincides with coarse (4, 4)
    r = deflation_restrict(v)
    assert abs(r[4, 4] - (6 / 8) ** 2) < 1e-15
    assert abs(r[4, 5] - (6 / 8) * (1 / 8)) < 1e-15
    assert abs(r[5, 5] - (1 / 8) ** 2) < 1e-15
    v[:] = 0
    v[9, 9] = 1.0                                  # between coarse 4 and 5 in both directions
    r = deflation_restrict(v)
    assert abs(r[4, 4] - (4 / 8) ** 2) < 1e-15 and abs(r[5, 5] - (4 / 8) ** 2) < 1e-15


def test_bilinear_reproduces_bilinear_functions():
    ny, nx = 17, 33
    f = lambda X, Y: 2.0 + 0.5 * X - Y + 0.3 * X * Y + 0j
    Xc, Yc = np.meshgrid(2.0 * np.arange((nx + 1) // 2), 2.0 * np.arange((ny + 1) // 2))
    Xf, Yf = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    np.testing.assert_allclose(bilinear_prolong(f(Xc, Yc), (ny, nx)), f(Xf, Yf), rtol=1e-14, atol=1e-13)


def test_full_weighting_is_quarter_bilinear_transpose():
    ny, nx = 33, 17
    r = mp.random_complex((ny, nx), seed=3)
    e = mp.random_complex(((ny + 1) // 2, (nx + 1) // 2), seed=4)
    lhs = np.vdot(fw_restrict(r), e)
    rhs = 0.25 * np.vdot(r, bilinear_prolong(e, (ny, nx)))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_full_weighting_preserves_constants_inside():
    r = np.full((17, 17), 3.0 + 1.0j)
    rc = fw_restrict(r)
    np.testing.assert_allclose(rc[1:-1, 1:-1], 3.0 + 1.0j, rtol=1e-15)
    np.testing.assert_allclose(rc[0, 4], 0.75 * (3.0 + 1.0j), rtol=1e-15)   # outside nodes count as zero
