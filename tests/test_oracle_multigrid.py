"""Pins for the oracle's CSLP multigrid V-cycle."""
import numpy as np
import pytest
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


def _mg_level_errors(level, m, shift, tops):
    """Consistency of multigrid level m of the CSLP V-cycle on deflation level `level`: the
    level's operator divided by the Galerkin factor 4^(level-1), applied to u = exp(alpha x +
    beta y) on its own grid (spacing H_m = 2^m H_level), against -Laplace(u) - shift k^2 u with
    the Sommerfeld data folded in at the boundary as (2/H_m) g.  Returns (boundary, interior)
    maximum errors for each top-grid size."""
    al, be = 1.0 + 2.0j, -0.5 + 1.5j
    out = []
    for Nt in tops:
        Ht = 1.0 / (Nt - 1)
        h = Ht / 2 ** (level - 1)
        xt = np.arange(Nt) * Ht
        Xt, Yt = np.meshgrid(xt, xt)
        kt = 4.0 + 2.0 * Xt + Yt                       # smooth k != 0 on the deflation level
        mg = CSLPMultigrid(kt, level, h, shift, coarsest_side=8)
        lv = mg.levels[m]
        N = lv.shape[0]
        Hm = 1.0 / (N - 1)
        assert abs(Hm - 2 ** m * Ht) < 1e-15
        x = np.arange(N) * Hm
        X, Y = np.meshgrid(x, x)
        k = 4.0 + 2.0 * X + Y
        np.testing.assert_allclose(lv.k, k, rtol=1e-15)  # wavenumber by injection
        u = np.exp(al * X + be * Y)
        f = -(al ** 2 + be ** 2) * u - shift * k * k * u
        g = np.zeros_like(u)
        g[:, 0] += -al * u[:, 0] - 1j * k[:, 0] * u[:, 0]
        g[:, -1] += al * u[:, -1] - 1j * k[:, -1] * u[:, -1]
        g[0, :] += -be * u[0, :] - 1j * k[0, :] * u[0, :]
        g[-1, :] += be * u[-1, :] - 1j * k[-1, :] * u[-1, :]
        r = lv.apply(u) / 4 ** (level - 1) - f - 2.0 / Hm * g
        edge = np.zeros(u.shape, bool)
        edge[:, 0] = edge[:, -1] = edge[0, :] = edge[-1, :] = True
        out.append((np.max(np.abs(r[edge])), np.max(np.abs(r[~edge]))))
    return out


@pytest.mark.parametrize("level,m", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_mg_coarse_levels_consistent_with_sommerfeld(level, m):
    """Multigrid level m >= 1 re-discretises the CSLP with the 5-point stencil at its own
    spacing 2^m H_l, the Sommerfeld ghost at that spacing, and the deflation level's Galerkin
    scale 4^(l-1) (the multigrid reading of Section 3.2).  With k != 0 the ghost term
    2 H_m i k u enters every boundary row, so a ghost at another spacing, a missing scale or a
    wrong wavenumber fails: boundary rows must converge at first order, interior rows at second."""
    shift = 1.0 + 0.5j
    errs = _mg_level_errors(level, m, shift, (65, 129, 257, 513))
    eb = [e[0] for e in errs]
    ei = [e[1] for e in errs]
    rb = [eb[i] / eb[i + 1] for i in range(len(eb) - 1)]
    ri = [ei[i] / ei[i + 1] for i in range(len(ei) - 1)]
    assert all(1.8 < r < 2.2 for r in rb), (eb, rb)
    assert all(3.5 < r < 4.5 for r in ri), (ei, ri)
