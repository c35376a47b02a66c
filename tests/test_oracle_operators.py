"""Pins for the oracle's operators (Section 2.1; Eq. for the CSLP; Section 3.3)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import model_problems as mp
from helpers import assemble
from oracle.operators import (DIRICHLET, SOMMERFELD, apply_5pt, apply_helmholtz, apply_level,
                              diag_5pt, diag_level, jacobi, scale_boundary_rows)
from oracle.stencils import stencils_2d
from oracle.transfers import inject, zt_1d


def grid(n, h, x0=0.0):
    x = x0 + np.arange(n) * h
    X, Y = np.meshgrid(x, x)
    return X, Y


@pytest.mark.parametrize("modes", [(1, 1), (2, 3), (7, 4), (15, 15)])
def test_dirichlet_eigenpairs(modes):
    """Constant-k Dirichlet A_h on n x n interior nodes, h = 1/(n+1): sin(i pi x) sin(j pi y)
    is an eigenvector with eigenvalue (4/h^2)(sin^2(i pi h/2) + sin^2(j pi h/2)) - k^2."""
    n, k = 15, 9.0
    h = 1.0 / (n + 1)
    X, Y = grid(n, h, h)
    i, j = modes
    phi = np.sin(i * np.pi * X) * np.sin(j * np.pi * Y) + 0j
    lam = 4 / h ** 2 * (np.sin(i * np.pi * h / 2) ** 2 + np.sin(j * np.pi * h / 2) ** 2) - k ** 2
    v = apply_helmholtz(phi, np.full((n, n), k), h, bc=DIRICHLET)
    assert np.max(np.abs(v - lam * phi)) <= 1e-12 * abs(lam) * np.max(np.abs(phi)) + 1e-10


def _mms_dirichlet_error(n):
    h = 1.0 / (n + 1)
    X, Y = grid(n, h, h)
    k = 3.0 + X * Y
    u_star = np.sin(np.pi * X) * np.sin(2 * np.pi * Y) + 0j
    f = (5 * np.pi ** 2 - k * k) * u_star
    A = assemble(lambda u: apply_helmholtz(u, k, h, bc=DIRICHLET), (n, n), 1)
    u = spla.spsolve(A.tocsc(), f.ravel()).reshape(n, n)
    return np.max(np.abs(u - u_star))


def test_mms_dirichlet_second_order():
    errs = [_mms_dirichlet_error(n) for n in (15, 31, 63)]
    rates = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.6 < r < 4.4 for r in rates), (errs, rates)


def _mms_sommerfeld_error(n):
    """u* = exp(alpha x + beta y) on [0,1]^2 with variable k; Sommerfeld data
    g = du/dn - i k u enters the right-hand side through the ghost equation."""
    h = 1.0 / (n - 1)
    X, Y = grid(n, h)
    al, be = 1.0 + 2.0j, -0.5 + 1.5j
    k = 4.0 + 2.0 * X + Y
    u_star = np.exp(al * X + be * Y)
    f = -(al ** 2 + be ** 2) * u_star - k * k * u_star
    b = f.copy()
    g_left = -al * u_star[:, 0] - 1j * k[:, 0] * u_star[:, 0]
    g_right = al * u_star[:, -1] - 1j * k[:, -1] * u_star[:, -1]
    g_bot = -be * u_star[0, :] - 1j * k[0, :] * u_star[0, :]
    g_top = be * u_star[-1, :] - 1j * k[-1, :] * u_star[-1, :]
    b[:, 0] += 2.0 / h * g_left
    b[:, -1] += 2.0 / h * g_right
    b[0, :] += 2.0 / h * g_bot
    b[-1, :] += 2.0 / h * g_top
    A = assemble(lambda u: apply_helmholtz(u, k, h), (n, n), 1)
    u = spla.spsolve(A.tocsc(), b.ravel()).reshape(n, n)
    return np.max(np.abs(u - u_star))


def test_mms_sommerfeld_second_order():
    """The ghost point u_0 = u_2 + 2 h i k u_1 discretises du/dn - i k u = 0 with
    second-order accuracy: a wrong sign or factor in it breaks the O(h^2) rate."""
    errs = [_mms_sommerfeld_error(n) for n in (17, 33, 65)]
    rates = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.5 < r < 4.5 for r in rates), (errs, rates)


def test_sommerfeld_edge_scaled_matrix_is_symmetric():
    """Halving the boundary rows (quartering corners) of the ghost-eliminated
    Sommerfeld matrix makes it complex symmetric (the matrix Section 2.1 calls
    symmetric): pins the doubled inward neighbour and the corner rows."""
    n, h = 13, 0.1
    k = mp.random_k(n, n + 4, seed=11)
    A = assemble(lambda u: apply_helmholtz(u, k, h), (n, n + 4), 1).toarray()
    s = np.ones((n, n + 4))
    s[:, 0] *= 0.5; s[:, -1] *= 0.5; s[0, :] *= 0.5; s[-1, :] *= 0.5
    S = s.ravel()[:, None] * A
    assert np.max(np.abs(S - S.T)) <= 1e-12 * np.max(np.abs(S))
    assert np.max(np.abs(S.imag)) > 0
    # the oracle's scale_boundary_rows (used by the sym_rows solve) is that scaling
    Sd = assemble(lambda u: scale_boundary_rows(apply_helmholtz(u, k, h)), (n, n + 4), 1).toarray()
    np.testing.assert_allclose(Sd, S, rtol=1e-15, atol=0)


def test_level1_reduces_to_fine_operator():
    ny, nx, h = 11, 14, 0.05
    k = mp.random_k(ny, nx, seed=3)
    u = mp.random_complex((ny, nx), seed=4)
    for shift in (1.0, 1.0 + 0.5j):
        np.testing.assert_allclose(apply_level(u, k, 1, h, shift), apply_helmholtz(u, k, h, shift),
                                   rtol=1e-14, atol=1e-9)


def _galerkin_check(n_fine, level, kval, h):
    """Rows of Z^T A_{level-1} Z at coarse nodes far from the boundary equal the
    level-``level`` stencil (constant k, where Galerkin coarsening is exact)."""
    kf = np.full((n_fine, n_fine), kval)
    Af = assemble(lambda u: apply_level(u, kf, level - 1, h), (n_fine, n_fine), 4)
    Zt = sp.kron(zt_1d(n_fine), zt_1d(n_fine), format="csr")
    E = (Zt @ Af @ Zt.T).tocsr()
    nc = (n_fine + 1) // 2
    kc = inject(kf, 2)
    Ac = assemble(lambda u: apply_level(u, kc, level, h), (nc, nc), 4).tocsr()
    margin = 5
    worst = 0.0
    for J in range(margin, nc - margin):
        for I in range(margin, nc - margin):
            r = J * nc + I
            d = (E[r] - Ac[r]).toarray()
            worst = max(worst, np.max(np.abs(d)) / np.max(np.abs(Ac[r].toarray())))
    return worst


@pytest.mark.parametrize("level", [2, 3])
def test_interior_rows_are_galerkin(level):
    n_fine = 41 if level == 2 else 41
    assert _galerkin_check(n_fine, level, 6.0, 1.0 / 40) < 1e-12


@pytest.mark.parametrize("level", [1, 2, 3, 4])
def test_level_diagonal_brute_force(level):
    ny, nx, h = 15, 12, 0.07
    k = mp.random_k(ny, nx, seed=5 + level)
    for shift in (1.0, 1.0 + 0.5j):
        A = assemble(lambda u: apply_level(u, k, level, h, shift), (ny, nx), 4)
        np.testing.assert_allclose(diag_level(k, level, h, shift).ravel(), A.diagonal(), rtol=1e-13, atol=1e-9)


def test_5pt_diagonal_brute_force():
    ny, nx = 9, 10
    k = mp.random_k(ny, nx, seed=2)
    for bc in (SOMMERFELD, DIRICHLET):
        A = assemble(lambda u: apply_5pt(u, k, 37.0, 0.2, 1.0 + 0.5j, 4.0, bc), (ny, nx), 1)
        np.testing.assert_allclose(diag_5pt(k, 37.0, 0.2, 1.0 + 0.5j, 4.0, bc).ravel(), A.diagonal(),
                                   rtol=1e-13, atol=1e-9)


def test_jacobi_fixed_point():
    """The exact solution of M u = f is a fixed point of the damped Jacobi sweep."""
    n, h = 17, 1.0 / 16
    k = mp.random_k(n, n, seed=9)
    shift = 1.0 + 0.5j
    M = assemble(lambda u: apply_helmholtz(u, k, h, shift), (n, n), 1)
    f = mp.random_complex((n, n), seed=10)
    u = spla.spsolve(M.tocsc(), f.ravel()).reshape(n, n)
    d = diag_5pt(k, 1 / h ** 2, h, shift)
    u2 = jacobi(u, f, lambda x: apply_helmholtz(x, k, h, shift), d, 0.8)
    assert np.max(np.abs(u2 - u)) <= 1e-12 * np.max(np.abs(u))


# ---- coarse-level boundary rows (Section 3.3 "Boundary") -----------------------------------
_AL, _BE = 1.0 + 2.0j, -0.5 + 1.5j


def _smooth_case(N, H, shift):
    """u = exp(alpha x + beta y) on the level grid [0,1]^2 with spacing H, a smooth variable k,
    f = -Laplace(u) - shift k^2 u and the Sommerfeld data g = du/dn - i k u summed over the
    sides each node touches."""
    x = np.arange(N) * H
    X, Y = np.meshgrid(x, x)
    k = 4.0 + 2.0 * X + Y
    u = np.exp(_AL * X + _BE * Y)
    f = -(_AL ** 2 + _BE ** 2) * u - shift * k * k * u
    g = np.zeros_like(u)
    g[:, 0] += -_AL * u[:, 0] - 1j * k[:, 0] * u[:, 0]
    g[:, -1] += _AL * u[:, -1] - 1j * k[:, -1] * u[:, -1]
    g[0, :] += -_BE * u[0, :] - 1j * k[0, :] * u[0, :]
    g[-1, :] += _BE * u[-1, :] - 1j * k[-1, :] * u[-1, :]
    edge = np.zeros(u.shape, bool)
    edge[:, 0] = edge[:, -1] = edge[0, :] = edge[-1, :] = True
    return u, k, f, g, edge


@pytest.mark.parametrize("level", [2, 3, 4])
@pytest.mark.parametrize("shift", [1.0, 1.0 + 0.5j])
def test_level_boundary_rows_consistent(level, shift):
    """Physical-boundary rows of the level-l operator are the second-order 5-point row at the
    level spacing H_l = 2^(l-1) h with the Sommerfeld ghost u_0 = u_2 + 2 H_l i k u_1, scaled by
    the Galerkin factor 4^(l-1) (Section 3.3, "Boundary", read with the ghost equation of
    Section 2.1).  Divided by 4^(l-1) and with the boundary data folded in as (2/H_l) g, the row
    applied to a smooth solution must approach -Laplace(u) - shift k^2 u at the first-order rate
    of a one-sided ghost row: a ghost at the fine spacing h, a wrong scale or a wrong shift in
    front of k^2 leaves an error that does not shrink."""
    errs = []
    for N in (17, 33, 65, 129):
        H = 1.0 / (N - 1)
        h = H / 2 ** (level - 1)
        u, k, f, g, edge = _smooth_case(N, H, shift)
        v = apply_level(u, k, level, h, shift) / 4 ** (level - 1)
        errs.append(np.max(np.abs((v - f - 2.0 / H * g)[edge])))
    rates = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(1.8 < r < 2.2 for r in rates), (errs, rates)
    assert errs[-1] < 0.15, errs


@pytest.mark.parametrize("level", [2, 3, 4])
@pytest.mark.parametrize("side", ["left", "right", "bottom", "top"])
def test_level_ghost_layer_exact_extension(level, side):
    """The first layer outside a level-l grid holds the Sommerfeld ghost value at spacing H_l
    (Section 3.3, "Boundary"; ghost equation of Section 2.1).  For constant k = sin(kappa H_l)/H_l
    the outgoing wave exp(i kappa s) (s the outward coordinate of that side) satisfies the ghost
    relation exactly, so at nodes R - 1 steps inside the side -- whose stencil reaches exactly the
    ghost layer and no farther -- the operator equals the Galerkin stencil applied to the wave
    itself, the wavenumber stencil seeing zero outside the grid (ghost wavenumbers are zero).
    Everything beyond the ghost layer (zero padding) is this implementation's reading of what the
    paper calls an open problem and is not fixed by this check."""
    N, kap, mu = 33, 0.9, 0.4
    H = 1.0 / (N - 1)
    h = H / 2 ** (level - 1)
    shift = 1.0 + 0.5j
    k0 = np.sin(kap * H) / H
    lap, kk = stencils_2d(level, h)
    R = lap.shape[0] // 2

    def U(i, j):
        x, y = i * H, j * H
        return {"left": np.exp(-1j * kap * x + 1j * mu * y), "right": np.exp(1j * kap * x + 1j * mu * y),
                "bottom": np.exp(-1j * kap * y + 1j * mu * x), "top": np.exp(1j * kap * y + 1j * mu * x)}[side]

    J, I = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    u = U(I, J)
    v = apply_level(u, np.full((N, N), k0), level, h, shift)
    near = {"left": R - 1, "right": N - R, "bottom": R - 1, "top": N - R}[side]
    pts = [(near, j) for j in range(R, N - R)] if side in ("left", "right") else [(i, near) for i in range(R, N - R)]
    worst = 0.0
    for i, j in pts:
        e = 0j
        for dy in range(-R, R + 1):
            for dx in range(-R, R + 1):
                e += lap[dy + R, dx + R] * U(i + dx, j + dy)
                if 0 <= i + dx < N and 0 <= j + dy < N:
                    e -= shift * kk[dy + R, dx + R] * k0 * k0 * U(i + dx, j + dy)
        worst = max(worst, abs(v[j, i] - e) / abs(e))
    assert worst < 1e-10, worst
