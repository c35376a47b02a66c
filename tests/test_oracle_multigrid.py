"""Pins for the oracle's CSLP multigrid V-cycle."""
import numpy as np
import scipy.sparse.linalg as spla

import model_problems as mp
from helpers import assemble
from oracle.multigrid import CSLPMultigrid
from oracle.operators import apply_helmholtz, apply_level


def _convergence_factor(mg, apply_m, shape, seed, its=8):
    f = mp.random_complex(shape, seed)
    u = np.zeros(shape, complex)
    res = []
    for _ in range(its):
        r = f - apply_m(u)
        res.append(np.linalg.norm(r))
        u = u + mg(r)
    return (res[-1] / res[2]) ** (1.0 / (its - 3))


def test_near_poisson_vcycle_textbook_factor():
    """k small (nearly the Laplacian with Robin-type boundary): V(1,1) with damped
    Jacobi, full weighting and bilinear prolongation contracts each cycle by a
    textbook factor (0.05 - 0.45; measured 0.38)."""
    n, h = 129, 1.0 / 128
    k = np.full((n, n), 0.5)
    mg = CSLPMultigrid(k, 1, h, 1.0 + 0.5j)
    assert len(mg.levels) == 4          # 129, 65, 33, 17
    rho = _convergence_factor(mg, lambda u: apply_helmholtz(u, k, h, 1.0 + 0.5j), (n, n), 1)
    assert 0.05 < rho < 0.45, rho


def test_cslp_vcycle_contracts_at_moderate_kh():
    """CSLP with shift (1, 0.5) at kh = 0.3: the V-cycle iteration still converges."""
    n, h = 129, 1.0 / 128
    k = np.full((n, n), 0.3 / h)
    mg = CSLPMultigrid(k, 1, h, 1.0 + 0.5j)
    rho = _convergence_factor(mg, lambda u: apply_helmholtz(u, k, h, 1.0 + 0.5j), (n, n), 2)
    assert rho < 0.9, rho


def test_level2_vcycle_uses_5x5_operator_and_converges():
    n, h = 65, 1.0 / 128          # level-2 grid of a 129^2 fine grid
    k = np.full((n, n), 0.15 / h)
    mg = CSLPMultigrid(k, 2, h, 1.0 + 0.5j)
    rho = _convergence_factor(mg, lambda u: apply_level(u, k, 2, h, 1.0 + 0.5j), (n, n), 3)
    assert rho < 0.9, rho


def test_single_level_hierarchy_is_exact():
    n, h = 17, 1.0 / 16
    k = mp.random_k(n, n, seed=4, kmin=2, kmax=8)
    mg = CSLPMultigrid(k, 1, h, 1.0 + 0.5j)
    assert len(mg.levels) == 1
    M = assemble(lambda u: apply_helmholtz(u, k, h, 1.0 + 0.5j), (n, n), 1)
    f = mp.random_complex((n, n), seed=5)
    ref = spla.spsolve(M.tocsc(), f.ravel()).reshape(n, n)
    np.testing.assert_allclose(mg(f), ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())
