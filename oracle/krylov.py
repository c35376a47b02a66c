"""Flexible GMRES with modified Gram-Schmidt.  TEST INFRASTRUCTURE ONLY (FP64 oracle).

Follows Algorithm 1 (lines 2-4 and 15-23) with the preconditioning step
(lines 5-14) passed in as a function:

    r0 = b - A u0, beta = ||r0||, v1 = r0 / beta
    for j = 1..m:  x_j = P v_j;  w = A x_j
                   for i = 1..j: h_ij = (w, v_i) = v_i^H w;  w = w - h_ij v_i
                   h_{j+1,j} = ||w||;  v_{j+1} = w / h_{j+1,j}
    u_m = u0 + X_m y_m,  y_m = argmin ||beta e1 - H_m y||

With P the identity this is plain GMRES.  The residual estimate after each
column is min_y ||beta e1 - H_j y|| computed by a dense least-squares solve
(the definition, not an incremental Givens update), and the cycle stops as soon
as it falls to ``tol_abs`` or the Hessenberg subdiagonal vanishes.

Pins (tests/test_oracle_krylov.py): the GMRES residual after j steps equals the
minimum residual over the Krylov space computed from an independent basis;
FGMRES with the exact inverse converges in one step; the Arnoldi relation
A X_j = V_{j+1} H_j holds; restarted FGMRES reaches a direct solve.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class CycleResult:
    update: np.ndarray
    iterations: int
    residual_estimate: float
    converged: bool
    H: np.ndarray = field(repr=False, default=None)


def _lsq(Hbar: np.ndarray, beta: float):
    rhs = np.zeros(Hbar.shape[0], dtype=np.complex128)
    rhs[0] = beta
    y = np.linalg.lstsq(Hbar, rhs, rcond=None)[0]
    return y, float(np.linalg.norm(rhs - Hbar @ y))


def fgmres_cycle(apply_a, r0, precond, m, tol_abs) -> CycleResult:
    """One FGMRES cycle of at most ``m`` iterations on residual ``r0`` (u0 = 0 shift)."""
    beta = float(np.linalg.norm(r0))
    if beta == 0.0:
        return CycleResult(np.zeros_like(r0), 0, 0.0, True)
    V = [r0 / beta]
    X = []
    H = np.zeros((m + 1, m), dtype=np.complex128)
    y, est, j_done, conv = None, beta, 0, False
    for j in range(m):
        x = precond(V[j]) if precond is not None else V[j]
        X.append(x)
        w = apply_a(x)
        for i in range(j + 1):
            H[i, j] = np.vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        j_done = j + 1
        y, est = _lsq(H[:j + 2, :j + 1], beta)
        if est <= tol_abs or abs(H[j + 1, j]) == 0.0:
            conv = est <= tol_abs or abs(H[j + 1, j]) == 0.0
            break
        V.append(w / H[j + 1, j])
    u = np.zeros_like(r0)
    for i in range(j_done):
        u = u + y[i] * X[i]
    return CycleResult(u, j_done, est, conv, H[:j_done + 1, :j_done])


def fgmres(apply_a, b, precond=None, tol=1e-6, maxit=30):
    """Zero-initial-guess FGMRES without restart: stop at relative residual
    estimate ``tol`` or after ``maxit`` iterations.  Returns (u, CycleResult)."""
    res = fgmres_cycle(apply_a, b, precond, maxit, tol * float(np.linalg.norm(b)))
    return res.update, res


def gmres(apply_a, b, tol, maxit):
    """Unpreconditioned GMRES, zero initial guess (CSLP inverse on coarse levels)."""
    return fgmres(apply_a, b, None, tol, maxit)


def fgmres_restarted(apply_a, b, precond, tol, restart, max_iters, u0=None):
    """Restarted FGMRES(restart) to relative residual ``tol`` in the 2-norm.  A cycle
    that stops on its estimate is confirmed with the true residual b - A u; if that
    check fails the method restarts from the current iterate.
    Returns (u, total_iterations, true_relative_residual, history)."""
    bnorm = float(np.linalg.norm(b))
    u = np.zeros_like(b) if u0 is None else u0.copy()
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0, []
    total, history = 0, []
    r = b - apply_a(u) if u0 is not None else b.copy()
    rel = float(np.linalg.norm(r)) / bnorm
    while total < max_iters and rel > tol:
        m = min(restart, max_iters - total)
        cyc = fgmres_cycle(apply_a, r, precond, m, tol * bnorm)
        u = u + cyc.update
        total += cyc.iterations
        r = b - apply_a(u)
        rel = float(np.linalg.norm(r)) / bnorm
        history.append((cyc.iterations, cyc.residual_estimate / bnorm, rel))
        if cyc.iterations == 0:
            break
    return u, total, rel, history
