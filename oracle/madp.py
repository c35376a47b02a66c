"""Recursive two-level deflated FGMRES with the MADP schedule.  TEST INFRASTRUCTURE ONLY.

Algorithm 1 (TLADP-FGMRES) at level l, FGMRES right-preconditioned by the
A-DEF1 deflation operator of Section 3.1, P = M^-1 (I - A Q) + Q, applied as
Algorithm 1 lines 5-14:

    v_hat = Z^T v_j                                   (line 5)
    v_til ~ E^-1 v_hat     E = A_{l+1}:
        l+1 == ml : CSLP-preconditioned FGMRES on A_ml (line 7)
        otherwise : TLADP-FGMRES(A_{l+1}, v_hat), recursively (line 10)
    t = Z v_til;  s = A_l t;  r_til = v_j - s        (lines 11-13)
    r ~ M_l^-1 r_til                                   (line 14)
    x_j = r + t                                        (line 15)

MADP schedule (Section 4.4; Section 4.1 for the coarsest level):
* level 1: FGMRES(restart) to relative residual ``tol`` (1e-6, Section 4);
* level 2 (when it is not the coarsest): tolerance 0.3, at most 30 iterations
  (``l2_tol = 0`` runs exactly ``l2_maxit`` iterations: MADP-v1's V-cycle,
  Section 4.3.1, is ``l2_tol = 0, l2_maxit = 1``);
* levels 3 .. ml-1: exactly ``cycle_m`` iterations, Algorithm 1's m on the
  coarser levels (1 = V-cycle, 2 = W-cycle, Section 3.2), or, for a level
  listed in ``level_tol``, that relative tolerance within ``l2_maxit``
  iterations (tolerances on the coarser levels, Sections 4.3.3 and 4.5);
* coarsest level ml: one iteration if it is treated as negative definite,
  otherwise tolerance 1e-1, at most floor(6 N_ml^(1/4)) iterations;
* CSLP inverse: multigrid V-cycle on levels 1 and 2; unpreconditioned GMRES to
  tolerance 1e-1, at most floor(6 N_l^(1/4)) iterations, on levels >= 3
  (Section 4.2), with shift beta = (1, 0.5) (Section 4.3); Bi-CGSTAB with the same
  tolerance and cap instead of GMRES with ``cslp_solver = "bicgstab"`` (the solver
  of the earlier multilevel work, Section 3.2).
All inner solves start from a zero initial guess.

Level l has (n_{l-1} + 1) / 2 nodes per side, spacing 2^(l-1) h and the
wavenumber injected at coincident nodes.  With ``bc = "dirichlet"`` (MP-1a,
Section 2.2) the grids hold interior unknowns only: (n_{l-1} - 1) / 2 per side,
the Dirichlet transfers and level operators of ``transfers`` / ``operators``.

Pins (tests/test_oracle_madp.py, tests/test_oracle_dirichlet.py): with the exact
Galerkin coarse inverse the A-DEF1 operator maps A Z y to Z y (both boundary
types); the solver's result solves the assembled system (dense LU) to the
requested residual on small grids; a level solved with as many iterations as
unknowns (or to 1e-12) reproduces the preconditioner built on a dense inverse of
that level; W-cycle and per-level-tolerance runs keep their call and iteration
counts.  Iteration counts against the paper's tables: the three-level k = 100
constant-wavenumber entries of Section 4.3.1 within one iteration; the pattern
the paper draws from the k = 100 rows (five levels need no more outer
iterations than four, three the fewest) holds, with every entry within three.
The exact four- and five-level counts, 2-3 iterations above the paper (setup
details live in other papers), and the wedge tables (synthetic geometry) stay
parity unpinned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from .krylov import bicgstab, fgmres, fgmres_restarted, gmres
from .multigrid import CSLPMultigrid
from .operators import DIRICHLET, SOMMERFELD, apply_level, apply_level_dirichlet, scale_boundary_rows
from .transfers import (coarse_size, coarse_size_dirichlet, deflation_prolong, deflation_prolong_dirichlet,
                        deflation_restrict, deflation_restrict_dirichlet, inject, inject_dirichlet)


@dataclass
class MADPConfig:
    levels: int = 2
    beta1: float = 1.0
    beta2: float = 0.5
    tol: float = 1e-6
    restart: int = 30
    max_outer: int = 300
    l2_tol: float = 0.3
    l2_maxit: int = 30
    cslp_tol: float = 0.1
    c_it: float = 6.0
    coarsest_tol: float = 0.1
    negdef_from_level: int = 0      # first level treated as negative definite; 0 = none
    mg_max_level: int = 2           # CSLP by multigrid on levels <= this, GMRES beyond
    mg_omega: float = 0.8
    mg_nu1: int = 1
    mg_nu2: int = 1
    mg_coarsest_side: int = 20
    cycle_m: int = 1                # iterations on levels 3 .. ml-1 without a tolerance
    level_tol: dict = field(default_factory=dict)   # level (3 .. ml-1) -> relative tolerance
    cslp_solver: str = "gmres"      # Krylov solver of the CSLP inverse beyond mg_max_level: gmres | bicgstab
    bc: str = SOMMERFELD            # "dirichlet": interior unknowns of a zero-boundary grid (MP-1a)
    sym_rows: bool = False          # outer solve on D A_h u = D b (D: 1/2 on edges, 1/4 at corners)


@dataclass
class Stats:
    outer_iterations: int = 0
    true_relres: float = float("nan")
    level_iterations: dict = field(default_factory=dict)    # level -> total deflated-FGMRES iterations
    level_calls: dict = field(default_factory=dict)         # level -> number of solves
    cslp_gmres_iterations: dict = field(default_factory=dict)
    history: list = field(default_factory=list)

    def add(self, d, level, n):
        d[level] = d.get(level, 0) + n


def krylov_cap(c_it: float, n_nodes: int) -> int:
    """Maximum number of Krylov iterations floor(C_it * N_l^(1/4)) (Section 4.2)."""
    return int(math.floor(c_it * n_nodes ** 0.25))


class Hierarchy:
    """Level data for the multilevel method: shapes, injected wavenumbers, CSLP solvers."""

    def __init__(self, k: np.ndarray, h: float, cfg: MADPConfig):
        self.cfg = cfg
        self.h = float(h)
        self.shift = complex(cfg.beta1, cfg.beta2)
        ny, nx = k.shape
        self.dirichlet = cfg.bc == DIRICHLET
        csize = coarse_size_dirichlet if self.dirichlet else coarse_size
        injector = inject_dirichlet if self.dirichlet else inject
        self.shapes = [(ny, nx)]
        for _ in range(cfg.levels - 1):
            ny, nx = csize(ny), csize(nx)
            self.shapes.append((ny, nx))
        self.k = [injector(np.asarray(k, np.float64), 2 ** l) for l in range(cfg.levels)]
        self.mg = {}
        for l in range(1, cfg.levels + 1):
            if l <= cfg.mg_max_level:
                self.mg[l] = CSLPMultigrid(self.k[l - 1], l, self.h, self.shift, cfg.mg_omega,
                                           cfg.mg_nu1, cfg.mg_nu2, cfg.mg_coarsest_side, cfg.bc)
        self.stats = Stats()

    # operators of level l (1-based)
    def A(self, l, u):
        op = apply_level_dirichlet if self.dirichlet else apply_level
        return op(u, self.k[l - 1], l, self.h, 1.0)

    def M(self, l, u):
        op = apply_level_dirichlet if self.dirichlet else apply_level
        return op(u, self.k[l - 1], l, self.h, self.shift)

    def nodes(self, l):
        return self.shapes[l - 1][0] * self.shapes[l - 1][1]

    def cslp_inverse(self, l, r):
        """r ~ M_l^-1 r_til (Algorithm 1, line 14)."""
        if l in self.mg:
            return self.mg[l](r)
        cap = krylov_cap(self.cfg.c_it, self.nodes(l))
        if self.cfg.cslp_solver == "bicgstab":
            x, res = bicgstab(lambda u: self.M(l, u), r, self.cfg.cslp_tol, cap)
        else:
            x, res = gmres(lambda u: self.M(l, u), r, self.cfg.cslp_tol, cap)
        self.stats.add(self.stats.cslp_gmres_iterations, l, res.iterations)
        return x

    def precond(self, l, v):
        """x_j = (M^-1 P + Q) v_j by Algorithm 1 lines 5-14 at level l."""
        ml = self.cfg.levels
        if ml == 1:
            return self.cslp_inverse(1, v)
        if self.dirichlet:
            vhat = deflation_restrict_dirichlet(v)
            vtil = self.coarse_solve(l + 1, vhat)
            t = deflation_prolong_dirichlet(vtil, self.shapes[l - 1])
        else:
            vhat = deflation_restrict(v)
            vtil = self.coarse_solve(l + 1, vhat)
            t = deflation_prolong(vtil, self.shapes[l - 1])
        s = self.A(l, t)
        rtil = v - s
        r = self.cslp_inverse(l, rtil)
        return r + t

    def coarse_solve(self, l, b):
        """v_til ~ A_l^-1 b for l >= 2 with the MADP schedule."""
        cfg = self.cfg
        ml = cfg.levels
        if l == ml:
            negdef = cfg.negdef_from_level > 0 and l >= cfg.negdef_from_level
            if negdef:
                tol, cap = 0.0, 1
            else:
                tol, cap = cfg.coarsest_tol, krylov_cap(cfg.c_it, self.nodes(l))
            u, res = fgmres(lambda x: self.A(l, x), b, lambda v: self.cslp_inverse(l, v), tol, cap)
        else:
            if l == 2:
                tol, cap = cfg.l2_tol, cfg.l2_maxit
            elif cfg.level_tol.get(l, 0.0) > 0:
                tol, cap = cfg.level_tol[l], cfg.l2_maxit
            else:
                tol, cap = 0.0, cfg.cycle_m
            u, res = fgmres(lambda x: self.A(l, x), b, lambda v: self.precond(l, v), tol, cap)
        self.stats.add(self.stats.level_iterations, l, res.iterations)
        self.stats.add(self.stats.level_calls, l, 1)
        return u

    def solve(self, b, u0=None):
        """Outer FGMRES(restart) on A_1 to relative residual tol (Section 4).  With ``sym_rows``
        the outer operator and right-hand side are the row-scaled D A_1 and D b (the symmetric
        form of the Sommerfeld system; the preconditioner is built from A as always)."""
        cfg = self.cfg
        self.stats = Stats()
        if cfg.sym_rows:
            op, rhs = (lambda x: scale_boundary_rows(self.A(1, x))), scale_boundary_rows(b)
        else:
            op, rhs = (lambda x: self.A(1, x)), b
        u, its, rel, hist = fgmres_restarted(op, rhs, lambda v: self.precond(1, v),
                                             cfg.tol, cfg.restart, cfg.max_outer, u0)
        self.stats.outer_iterations = its
        self.stats.true_relres = rel
        self.stats.history = hist
        return u, self.stats


def solve(k, h, b, cfg: MADPConfig):
    """Convenience wrapper: build the hierarchy and solve one right-hand side."""
    hier = Hierarchy(k, h, cfg)
    return hier.solve(b)
