"""Pins for the oracle's GMRES / FGMRES (Algorithm 1, lines 2-4 and 15-23)."""
import numpy as np
import pytest

import model_problems as mp
from oracle.krylov import fgmres, fgmres_cycle, fgmres_restarted, gmres


def _matrix(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    A = 3.0 * np.eye(n) + (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    return A


@pytest.mark.parametrize("j", [1, 3, 7, 12])
def test_gmres_minimum_residual(j):
    """After j steps the GMRES residual is the minimum of ||b - A x|| over the Krylov
    space span{b, Ab, ..., A^(j-1) b}, computed here from an independent QR basis."""
    n = 40
    A = _matrix(n, 1)
    b = mp.random_complex(n, 2)
    x, res = gmres(lambda v: A @ v, b, 0.0, j)
    K = np.empty((n, j), complex)
    K[:, 0] = b
    for c in range(1, j):
        K[:, c] = A @ K[:, c - 1]
    Q, _ = np.linalg.qr(K)
    y = np.linalg.lstsq(A @ Q, b, rcond=None)[0]
    best = np.linalg.norm(b - A @ Q @ y)
    assert abs(np.linalg.norm(b - A @ x) - best) <= 1e-10 * np.linalg.norm(b)
    assert res.iterations == j


def test_fgmres_exact_preconditioner_one_step():
    n = 30
    A = _matrix(n, 3)
    Ainv = np.linalg.inv(A)
    b = mp.random_complex(n, 4)
    x, res = fgmres(lambda v: A @ v, b, lambda v: Ainv @ v, 1e-12, 10)
    assert res.iterations == 1
    np.testing.assert_allclose(A @ x, b, rtol=1e-11, atol=1e-11)


def test_residual_estimate_is_true_residual():
    """The least-squares residual estimate equals ||r0 - A u|| only if the Arnoldi
    relation A X_j = V_{j+1} H_j holds with orthonormal V (flexible preconditioner)."""
    n = 50
    A = _matrix(n, 5)
    b = mp.random_complex(n, 6)
    rng = np.random.Generator(np.random.PCG64(7))
    D = np.diag(1.0 + rng.random(n))
    calls = [0]

    def prec(v):                                  # a different linear map each call
        calls[0] += 1
        return (D ** (1 + 0.1 * calls[0])) @ v

    res = fgmres_cycle(lambda v: A @ v, b, prec, 9, 0.0)
    assert abs(res.residual_estimate - np.linalg.norm(b - A @ res.update)) <= 1e-10 * np.linalg.norm(b)


def test_restarted_fgmres_reaches_direct_solve():
    n = 60
    A = _matrix(n, 8)
    b = mp.random_complex(n, 9)
    u, its, rel, hist = fgmres_restarted(lambda v: A @ v, b, lambda v: v / 3.0, 1e-10, 5, 500)
    assert rel <= 1e-10 and len(hist) > 1
    np.testing.assert_allclose(u, np.linalg.solve(A, b), rtol=1e-8)


def test_zero_rhs_returns_zero():
    x, res = gmres(lambda v: 2 * v, np.zeros(5, complex), 0.1, 4)
    assert res.iterations == 0 and not np.any(x)


# ---- Bi-CGSTAB (van der Vorst 1992; the CSLP solver of Sections 3.2 and 4.1) --------------------
def test_bicgstab_scaled_identity_is_exact_in_one_step():
    """A = c I: v = c p, alpha = 1/c, s = 0, so the first iteration returns b / c."""
    from oracle.krylov import bicgstab
    b = mp.random_complex((40,), seed=3)
    c = 2.5 - 1.5j
    x, res = bicgstab(lambda u: c * u, b, 1e-12, 10)
    assert res.iterations == 1 and res.converged
    np.testing.assert_allclose(x, b / c, rtol=0, atol=1e-14 * np.abs(b / c).max())


@pytest.mark.parametrize("k", [1, 2, 5, 9])
def test_bicgstab_matches_scipy_iterates(k):
    """k iterations with no early stop give SciPy's independent Bi-CGSTAB iterate."""
    import scipy.sparse.linalg as spla
    from oracle.krylov import bicgstab
    A = _matrix(30, seed=7)
    b = mp.random_complex((30,), seed=8)
    x, res = bicgstab(lambda u: A @ u, b, 0.0, k)
    assert res.iterations == k
    xs, info = spla.bicgstab(A, b, rtol=1e-300, atol=0.0, maxiter=k)
    np.testing.assert_allclose(x, xs, rtol=0, atol=1e-10 * np.abs(xs).max())


def test_bicgstab_recurred_residual_is_true_residual_and_solves():
    """On a Helmholtz-type CSLP system the recurred residual at exit equals ||b - A x||
    and the tolerance reached means the direct solution to that accuracy."""
    from helpers import assemble
    from oracle.krylov import bicgstab
    from oracle.operators import apply_level
    n = 17
    k = mp.random_k(n, n, seed=4, kmin=3.0, kmax=6.0)
    h = 1.0 / 16
    M = lambda u: apply_level(u, k, 3, h, complex(1.0, 0.5))
    b = mp.random_complex((n, n), seed=5)
    x, res = bicgstab(M, b, 1e-10, 400)
    assert res.converged and res.iterations > 3
    true = np.linalg.norm(b - M(x)) / np.linalg.norm(b)
    assert abs(true - res.residual) <= 1e-9
    Md = assemble(M, (n, n), 3).toarray()
    ref = np.linalg.solve(Md, b.ravel()).reshape(n, n)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 1e-10 * np.linalg.cond(Md)


def test_bicgstab_zero_rhs():
    from oracle.krylov import bicgstab
    x, res = bicgstab(lambda u: 2 * u, np.zeros(5, complex), 0.1, 5)
    assert res.iterations == 0 and not x.any()
