"""Pins for the oracle's recursive deflated FGMRES (Algorithm 1 with the MADP schedule)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import model_problems as mp
from helpers import assemble
from oracle.madp import Hierarchy, MADPConfig, krylov_cap
from oracle.operators import apply_helmholtz
from oracle.transfers import deflation_prolong, zt_1d


def test_adef1_maps_range_of_AZ_to_Z_with_exact_coarse_inverse():
    """With E = Z^T A Z inverted exactly, lines 5-15 of Algorithm 1 give
    x = M^-1 (v - A Z E^-1 Z^T v) + Z E^-1 Z^T v, so P A Z y = Z y for every y."""
    n, h = 33, 1.0 / 32
    k = mp.random_k(n, n, seed=1, kmin=5, kmax=15)
    hier = Hierarchy(k, h, MADPConfig(levels=2))
    A = assemble(lambda u: apply_helmholtz(u, k, h), (n, n), 1)
    Zt = sp.kron(zt_1d(n), zt_1d(n), format="csr")
    E = (Zt @ A @ Zt.T).toarray()
    nc = (n + 1) // 2
    hier.coarse_solve = lambda l, b: np.linalg.solve(E, b.ravel()).reshape(nc, nc)
    y = mp.random_complex((nc, nc), seed=2)
    Zy = deflation_prolong(y, (n, n))
    x = hier.precond(1, apply_helmholtz(Zy, k, h))
    np.testing.assert_allclose(x, Zy, rtol=0, atol=1e-10 * np.abs(Zy).max())


@pytest.mark.parametrize("levels,shape,kmax,negdef", [
    (1, (33, 33), 12.0, 0),
    (2, (33, 33), 12.0, 0),
    (3, (33, 49), 20.0, 0),
    (3, (33, 49), 20.0, 3),
    (4, (65, 65), 30.0, 4),
])
def test_solution_matches_direct_solve(levels, shape, kmax, negdef):
    """The solver's result satisfies the assembled system to the 1e-6 relative
    residual and agrees with a sparse LU solve accordingly."""
    ny, nx = shape
    h = 1.0 / (nx - 1)
    k = mp.random_k(ny, nx, seed=3, kmin=0.5 * kmax, kmax=kmax)
    b = mp.point_source(nx, ny, nx // 2, ny - 1, h)
    cfg = MADPConfig(levels=levels, negdef_from_level=negdef)
    u, st = Hierarchy(k, h, cfg).solve(b)
    A = assemble(lambda x: apply_helmholtz(x, k, h), (ny, nx), 1).tocsc()
    rel = np.linalg.norm(b.ravel() - A @ u.ravel()) / np.linalg.norm(b)
    assert rel <= 1e-6 and abs(rel - st.true_relres) <= 1e-9
    ref = spla.spsolve(A, b.ravel()).reshape(ny, nx)
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) < 1e-4
    assert 1 <= st.outer_iterations <= 60


def test_krylov_cap():
    assert krylov_cap(6.0, 1025 * 1025) == 192
    assert krylov_cap(6.0, 65 * 65) == 48
    assert krylov_cap(6.0, 129 * 129) == 68


def test_schedule_counts_two_level():
    """Two levels: each outer iteration solves the coarsest level once by CSLP-FGMRES."""
    p = mp.mp1b(32, 10.0)
    cfg = MADPConfig(levels=2)
    u, st = Hierarchy(p.k, p.h, cfg).solve(p.b[0])
    assert st.level_calls[2] == st.outer_iterations
    assert st.true_relres <= 1e-6


def test_deeper_levels_take_one_iteration():
    """Four levels: level 3 (neither level 2 nor the coarsest) runs exactly one
    FGMRES iteration per call; the negative-definite coarsest runs one too."""
    p = mp.random_field(65, 5.0, seed=3, kh_max=0.3, levels=4, negdef_from_level=4)
    cfg = MADPConfig(levels=4, negdef_from_level=4)
    u, st = Hierarchy(p.k, p.h, cfg).solve(p.b[0])
    assert st.level_iterations[3] == st.level_calls[3]
    assert st.level_iterations[4] == st.level_calls[4]
    assert st.level_calls[3] == st.level_iterations[2]
    assert st.true_relres <= 1e-6
