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

Bi-CGSTAB (van der Vorst, SIAM J. Sci. Stat. Comput. 13(2), 1992), the Krylov
solver the paper's earlier multilevel work used for the CSLP inverse (Section 3.2)
and its own tolerance study used (Section 4.1), is :func:`bicgstab`.

Pins (tests/test_oracle_krylov.py): the GMRES residual after j steps equals the
minimum residual over the Krylov space computed from an independent basis;
FGMRES with the exact inverse converges in one step; the Arnoldi relation
A X_j = V_{j+1} H_j holds; restarted FGMRES reaches a direct solve.  Bi-CGSTAB:
one step on a multiple of the identity is exact, its recurred residual is the
true residual, and it agrees with SciPy's independent implementation.
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


@dataclass
class BicgResult:
    iterations: int
    residual: float          # recurred ||r|| / ||b|| at exit
    converged: bool


def bicgstab(apply_a, b, tol, maxit):
    """Bi-CGSTAB with zero initial guess and shadow residual r_hat = b.

    Each iteration: rho = r_hat^H r; p = r (first) or r + (rho/rho_old)(alpha/omega)(p - omega v);
    v = A p; alpha = rho / (r_hat^H v); s = r - alpha v; t = A s; omega = t^H s / t^H t;
    x += alpha p + omega s; r = s - omega t.  Stops when ||r|| <= tol ||b|| after an iteration,
    after ``maxit`` iterations, or on a vanishing rho, r_hat^H v or t^H t (breakdown; t = 0
    means s = 0, so x + alpha p is then exact).  Returns (x, BicgResult)."""
    bn = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    if bn == 0.0:
        return x, BicgResult(0, 0.0, True)
    r = b.copy()
    rhat = b.copy()
    p = v = None
    rho_old = alpha = omega = 1.0
    its = 0
    for i in range(maxit):
        rho = np.vdot(rhat, r)
        if rho == 0:
            break
        if i == 0:
            p = r.copy()
        else:
            p = r + (rho / rho_old) * (alpha / omega) * (p - omega * v)
        v = apply_a(p)
        rv = np.vdot(rhat, v)
        if rv == 0:
            break
        alpha = rho / rv
        s = r - alpha * v
        t = apply_a(s)
        tt = np.vdot(t, t).real
        its = i + 1
        if tt == 0:
            x = x + alpha * p
            r = s
            break
        omega = np.vdot(t, s) / tt
        x = x + alpha * p + omega * s
        r = s - omega * t
        rho_old = rho
        if float(np.linalg.norm(r)) <= tol * bn:
            break
    rel = float(np.linalg.norm(r)) / bn
    return x, BicgResult(its, rel, rel <= tol)
