"""CSLP approximate inverse by a multigrid V-cycle.  TEST INFRASTRUCTURE ONLY (FP64 oracle).

The paper approximates M_(beta1,beta2)^-1 on the first and second levels by a
multigrid V-cycle (Section 3.2 third remark; Section 4.4, MADP) whose settings
it takes from its earlier matrix-free CSLP work.  The reading used here:

* V(nu1, nu2) cycle, zero initial guess, damped Jacobi with weight omega
  (defaults nu1 = nu2 = 1, omega = 0.8);
* MG level 0 is the deflation level's own CSLP operator M_l (the 5x5 Galerkin
  stencil on level 2) with its exact diagonal;
* MG level m >= 1 re-discretises M with the 5-point stencil at spacing
  2^m H_l, scaled by the same Galerkin factor 4^(l-1) as level l, with the
  wavenumber injected at coincident nodes;
* full-weighting restriction, bilinear prolongation;
* coarsening stops once a side has at most ``coarsest_side`` nodes (or cannot be
  halved); that level is solved exactly by a dense LU factorisation built once.

On a homogeneous Dirichlet grid (interior unknowns, ``bc = "dirichlet"``) the same
cycle runs with the Dirichlet operators, transfers and injection of
``operators`` / ``transfers`` (coarse unknown I at fine unknown 2I + 1).

Pins (tests/test_oracle_multigrid.py): for the Poisson operator (k = 0) the
V(1,1) convergence factor lies in the textbook range (both boundary types); the
exact solution is a fixed point of every Jacobi sweep; a single-level hierarchy
is an exact solve; with k != 0 every coarse multigrid level's operator, divided
by 4^(l-1), is consistent with -Laplace(u) - shift k^2 u (second order inside,
first order on the boundary rows with the Sommerfeld data folded in), which
fixes its spacing, its ghost spacing, its scale and its injected wavenumber.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla

from .operators import (DIRICHLET, SOMMERFELD, apply_5pt, apply_level, apply_level_dirichlet, diag_5pt, diag_level,
                        diag_level_dirichlet, jacobi, level_scale, level_spacing)
from .transfers import (bilinear_prolong, bilinear_prolong_dirichlet, fw_restrict, fw_restrict_dirichlet, inject,
                        inject_dirichlet)


@dataclass
class MGLevel:
    shape: tuple
    k: np.ndarray
    apply: object
    diag: np.ndarray


def _dense_matrix(apply, shape) -> np.ndarray:
    """Assemble an operator column by column from unit vectors."""
    n = shape[0] * shape[1]
    A = np.zeros((n, n), dtype=np.complex128)
    e = np.zeros(shape, dtype=np.complex128)
    for c in range(n):
        e.flat[c] = 1.0
        A[:, c] = apply(e).ravel()
        e.flat[c] = 0.0
    return A


class CSLPMultigrid:
    """V-cycle approximation of M_l^-1 for deflation level ``level``."""

    def __init__(self, k_level, level, h, shift, omega=0.8, nu1=1, nu2=1, coarsest_side=20, bc=SOMMERFELD):
        self.omega, self.nu1, self.nu2 = omega, nu1, nu2
        self.bc = bc
        ks = level_scale(level)
        H = level_spacing(level, h)
        sh = complex(shift)
        k0 = np.asarray(k_level, dtype=np.float64)
        if bc == DIRICHLET:
            top = MGLevel(k0.shape, k0, (lambda u, kk=k0: apply_level_dirichlet(u, kk, level, h, sh)),
                          diag_level_dirichlet(k0, level, h, sh))
            min_side, injector = 3, inject_dirichlet
        else:
            top = MGLevel(k0.shape, k0, (lambda u, kk=k0: apply_level(u, kk, level, h, sh)),
                          diag_level(k0, level, h, sh))
            min_side, injector = 5, inject
        self.levels = [top]
        Hm = H
        while True:
            ny, nx = self.levels[-1].shape
            if min(ny, nx) <= coarsest_side or (ny - 1) % 2 or (nx - 1) % 2 or min(ny, nx) < min_side:
                break
            Hm = 2.0 * Hm
            km = injector(self.levels[-1].k, 2)
            c = ks / (Hm * Hm)
            self.levels.append(MGLevel(km.shape, km,
                                       (lambda u, kk=km, c=c, Hm=Hm: apply_5pt(u, kk, c, Hm, sh, ks, bc)),
                                       diag_5pt(km, c, Hm, sh, ks, bc)))
        last = self.levels[-1]
        self.lu = sla.lu_factor(_dense_matrix(last.apply, last.shape))

    def vcycle(self, f: np.ndarray, m: int = 0) -> np.ndarray:
        lv = self.levels[m]
        if m == len(self.levels) - 1:
            return sla.lu_solve(self.lu, f.ravel()).reshape(f.shape)
        u = np.zeros(lv.shape, dtype=np.complex128)
        for _ in range(self.nu1):
            u = jacobi(u, f, lv.apply, lv.diag, self.omega)
        r = f - lv.apply(u)
        if self.bc == DIRICHLET:
            ec = self.vcycle(fw_restrict_dirichlet(r), m + 1)
            u = u + bilinear_prolong_dirichlet(ec, lv.shape)
        else:
            ec = self.vcycle(fw_restrict(r), m + 1)
            u = u + bilinear_prolong(ec, lv.shape)
        for _ in range(self.nu2):
            u = jacobi(u, f, lv.apply, lv.diag, self.omega)
        return u

    __call__ = vcycle
