"""Pins for the oracle's homogeneous-Dirichlet multilevel path (MP-1a, Section 2.2): the
interior-unknown transfers, the zero-padded level operators, the Dirichlet multigrid and the
recursive deflated solve."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import model_problems as mp
from helpers import assemble
from oracle import transfers as T
from oracle.madp import Hierarchy, MADPConfig
from oracle.multigrid import CSLPMultigrid
from oracle.operators import DIRICHLET, apply_5pt, apply_level_dirichlet, diag_level_dirichlet

# ---- transfers --------------------------------------------------------------------------------


def test_dirichlet_coarse_unknowns_sit_at_odd_fine_unknowns():
    """Coarse unknown I coincides with fine unknown 2I + 1: Z^T puts weight 6/8 there and the
    [1, 4, 6, 4, 1] / 8 row around it; n_coarse = (n_fine - 1) / 2."""
    Zt = T.zt_1d_dirichlet(15).toarray()
    assert Zt.shape == (7, 15)
    for I in range(7):
        assert Zt[I, 2 * I + 1] == 0.75
        for a, w in zip(range(-2, 3), T.P_DEFL):
            j = 2 * I + 1 + a
            if 0 <= j < 15:
                assert Zt[I, j] == w
    assert T.inject_dirichlet(np.arange(15.0)[None, :].repeat(15, 0), 2)[0].tolist() == [1, 3, 5, 7, 9, 11, 13]
    with pytest.raises(ValueError):
        T.coarse_size_dirichlet(14)


def test_dirichlet_restriction_is_transpose():
    v = mp.random_complex((31, 15), seed=1)
    w = mp.random_complex((15, 7), seed=2)
    lhs = np.vdot(T.deflation_restrict_dirichlet(v), w)
    rhs = np.vdot(v, T.deflation_prolong_dirichlet(w, (31, 15)))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_dirichlet_prolongation_reproduces_linear_functions_inside():
    """Z maps samples of a bilinear function (coarse unknown I at fine coordinate 2I + 1) to the
    function itself at every fine unknown whose interpolation stencil stays inside the grid."""
    ny, nx = 31, 15
    cy, cx = T.coarse_size_dirichlet(ny), T.coarse_size_dirichlet(nx)
    f = lambda y, x: 0.3 + 0.7 * x - 0.2 * y + 0.05 * x * y
    Yc, Xc = np.meshgrid(2 * np.arange(cy) + 1.0, 2 * np.arange(cx) + 1.0, indexing="ij")
    Yf, Xf = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    t = T.deflation_prolong_dirichlet(f(Yc, Xc).astype(complex), (ny, nx))
    inside = (slice(2, ny - 2), slice(2, nx - 2))
    np.testing.assert_allclose(t[inside], f(Yf, Xf)[inside], rtol=0, atol=1e-12)


def test_dirichlet_full_weighting_is_quarter_bilinear_transpose():
    fw = sp.kron(T.fw_1d_dirichlet(15), T.fw_1d_dirichlet(31)).toarray()
    bl = sp.kron(T.bilinear_1d_dirichlet(15), T.bilinear_1d_dirichlet(31)).toarray()
    np.testing.assert_allclose(fw, 0.25 * bl.T, rtol=0, atol=1e-15)


# ---- level operators --------------------------------------------------------------------------
def test_dirichlet_level1_is_the_5_point_operator():
    ny, nx, h = 13, 21, 0.05
    k = mp.random_k(ny, nx, seed=3, kmin=2.0, kmax=9.0)
    u = mp.random_complex((ny, nx), seed=4)
    for shift in (1.0, 1.0 + 0.5j):
        ref = apply_5pt(u, k, 1.0 / (h * h), h, shift, 1.0, DIRICHLET)
        np.testing.assert_allclose(apply_level_dirichlet(u, k, 1, h, shift), ref, rtol=1e-13, atol=1e-10)


@pytest.mark.parametrize("level", [2, 3])
def test_dirichlet_interior_rows_are_galerkin(level):
    """With constant k, rows of Z^T A_{l-1} Z whose footprint stays clear of the boundary equal the
    zero-padded level-l operator; rows next to the boundary differ (the Galerkin product would
    also drop the fine boundary value that Z puts outside the grid), which is this reading."""
    nf = 31 if level == 2 else 63
    h = 1.0 / 64
    kc = 11.0
    fine_level = level - 1
    nfl = nf if fine_level == 1 else T.coarse_size_dirichlet(nf)
    kf = np.full((nfl, nfl), kc)
    nc = T.coarse_size_dirichlet(nfl)
    y = mp.random_complex((nc, nc), seed=5 + level)
    Zy = T.deflation_prolong_dirichlet(y, (nfl, nfl))
    gal = T.deflation_restrict_dirichlet(apply_level_dirichlet(Zy, kf, fine_level, h))
    mine = apply_level_dirichlet(y, np.full((nc, nc), kc), level, h)
    m = 2 if level == 2 else 3
    inside = (slice(m, nc - m), slice(m, nc - m))
    np.testing.assert_allclose(mine[inside], gal[inside], rtol=1e-12, atol=1e-9 * np.abs(gal).max())
    assert np.abs(mine[0, :] - gal[0, :]).max() > 1e-6 * np.abs(gal).max()


@pytest.mark.parametrize("level", [1, 2, 3])
def test_dirichlet_level_diagonal_brute_force(level):
    n, h = 9, 0.1
    k = mp.random_k(n, n, seed=6, kmin=1.0, kmax=4.0)
    M = assemble(lambda u: apply_level_dirichlet(u, k, level, h, 1.0 + 0.5j), (n, n), 3)
    np.testing.assert_allclose(M.diagonal().reshape(n, n), diag_level_dirichlet(k, level, h, 1.0 + 0.5j),
                               rtol=1e-13, atol=1e-9)


# ---- multigrid and the recursive solve --------------------------------------------------------
def _factor(mg, apply_m, shape, seed, its=8):
    f = mp.random_complex(shape, seed)
    u = np.zeros(shape, complex)
    res = []
    for _ in range(its):
        r = f - apply_m(u)
        res.append(np.linalg.norm(r))
        u = u + mg(r)
    return (res[-1] / res[2]) ** (1.0 / (its - 3))


def test_dirichlet_poisson_vcycle_textbook_factor():
    """k = 0 on 127^2 interior unknowns: the Dirichlet Laplacian, for which V(1,1) with
    0.8-damped Jacobi, full weighting and bilinear prolongation contracts each cycle by the
    textbook factor: 0.8-damped Jacobi smooths by 0.6 per sweep in 2-D, so two sweeps bound
    the cycle near 0.36 (measured 0.33)."""
    n, h = 127, 1.0 / 128
    k = np.zeros((n, n))
    mg = CSLPMultigrid(k, 1, h, 1.0 + 0.5j, bc=DIRICHLET)
    assert [lv.shape[0] for lv in mg.levels] == [127, 63, 31, 15]
    rho = _factor(mg, lambda u: apply_level_dirichlet(u, k, 1, h, 1.0 + 0.5j), (n, n), 1)
    assert 0.05 < rho < 0.4, rho


def test_dirichlet_single_level_hierarchy_is_exact():
    n, h = 15, 1.0 / 16
    k = mp.random_k(n, n, seed=4, kmin=2, kmax=8)
    mg = CSLPMultigrid(k, 1, h, 1.0 + 0.5j, bc=DIRICHLET)
    assert len(mg.levels) == 1
    M = assemble(lambda u: apply_level_dirichlet(u, k, 1, h, 1.0 + 0.5j), (n, n), 1)
    f = mp.random_complex((n, n), seed=5)
    ref = spla.spsolve(M.tocsc(), f.ravel()).reshape(n, n)
    np.testing.assert_allclose(mg(f), ref, rtol=1e-11, atol=1e-13 * np.abs(ref).max())


def test_dirichlet_adef1_maps_range_of_AZ_to_Z_with_exact_coarse_inverse():
    """P A Z y = Z y when the coarse system E = Z^T A Z is inverted exactly (Section 3.1)."""
    n, h = 31, 1.0 / 32
    k = mp.random_k(n, n, seed=1, kmin=5, kmax=15)
    hier = Hierarchy(k, h, MADPConfig(levels=2, bc="dirichlet"))
    A = assemble(lambda u: apply_level_dirichlet(u, k, 1, h), (n, n), 1)
    Zt = sp.kron(T.zt_1d_dirichlet(n), T.zt_1d_dirichlet(n), format="csr")
    E = (Zt @ A @ Zt.T).toarray()
    nc = T.coarse_size_dirichlet(n)
    hier.coarse_solve = lambda l, b: np.linalg.solve(E, b.ravel()).reshape(nc, nc)
    y = mp.random_complex((nc, nc), seed=2)
    Zy = T.deflation_prolong_dirichlet(y, (n, n))
    x = hier.precond(1, apply_level_dirichlet(Zy, k, 1, h))
    np.testing.assert_allclose(x, Zy, rtol=0, atol=1e-10 * np.abs(Zy).max())


@pytest.mark.parametrize("levels", [1, 2, 3, 4])
def test_mp1a_solution_matches_direct_solve(levels):
    """MP-1a (constant k = 20, 127^2 interior unknowns, centre source) solved by the recursive
    deflated FGMRES reaches the 1e-6 residual of the assembled Dirichlet system and agrees
    with a sparse LU solve accordingly."""
    p = mp.mp1a(128, 20.0, levels=levels)
    u, st = Hierarchy(p.k, p.h, MADPConfig(levels=levels, bc="dirichlet")).solve(p.b[0])
    A = assemble(lambda x: apply_5pt(x, p.k, 1.0 / p.h ** 2, p.h, 1.0, 1.0, DIRICHLET), (p.ny, p.nx), 1).tocsc()
    b = p.b[0]
    rel = np.linalg.norm(b.ravel() - A @ u.ravel()) / np.linalg.norm(b)
    assert rel <= 1e-6 and abs(rel - st.true_relres) <= 1e-9
    ref = spla.spsolve(A, b.ravel()).reshape(p.ny, p.nx)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-4
    if levels >= 2:
        assert st.outer_iterations <= 12        # deflation: 8-9 outer iterations against 19 without
