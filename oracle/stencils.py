"""Exact coarse-level stencils (Section 3.3 and Appendix A).  TEST INFRASTRUCTURE ONLY.

The paper builds the level-l Helmholtz and CSLP stencils by Galerkin coarsening
of the Laplace and wavenumber stencils separately, assuming constant k
(Section 3.3), with the higher-order deflation vectors of Section 3.1.  The
prolongation Z is the tensor product of the 1-D weights p = [1, 4, 6, 4, 1] / 8
at stride 2, so Galerkin coarsening acts on each 1-D factor:

    S_{l+1}[d] = sum_{a, e} p[a] * S_l[e] * p[a + e - 2 d]          (1-D)

starting from the fine mass mask M_1 = [1] and the fine second-difference mask
L_1 = [-1, 2, -1].  The 2-D stencils are

    Lap_l = (L_l (x) M_l + M_l (x) L_l) / h^2,      K_l = M_l (x) M_l,

with h the *fine* spacing, and A_l = Lap_l - k^2 K_l, M_l = Lap_l - (beta1 + i beta2) k^2 K_l
(Eq. for A_h and Eq. for the CSLP).  All arithmetic here is exact (Fractions).

Pins: every integer the paper prints for levels 3-6 (Section 3.3, Appendix A)
is reproduced exactly, apart from K_32h entries above 2^53 that the paper
printed after FP64 rounding; the level-2 stencils, which the paper does not
print, are pinned by a sparse Galerkin triple product Z^T A Z built from the
definition of Z (tests/test_oracle_stencils.py).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

# 1-D deflation weights, offsets -2..2 (higher-order deflation vectors, Section 3.1)
P_WEIGHTS = [Fraction(1, 8), Fraction(4, 8), Fraction(6, 8), Fraction(4, 8), Fraction(1, 8)]


def galerkin_1d(s: list[Fraction]) -> list[Fraction]:
    """One Galerkin coarsening Z^T S Z of a symmetric 1-D stencil ``s``
    (odd length, centre in the middle).  Returns the coarse stencil, trimmed to
    its non-zero support but kept symmetric and of odd length."""
    rs = len(s) // 2
    coarse = {}
    for d in range(-(rs + 4), rs + 5):
        acc = Fraction(0)
        for a in range(-2, 3):
            for e in range(-rs, rs + 1):
                m = a + e - 2 * d
                if -2 <= m <= 2:
                    acc += P_WEIGHTS[a + 2] * s[e + rs] * P_WEIGHTS[m + 2]
        coarse[d] = acc
    r = max((abs(d) for d, v in coarse.items() if v != 0), default=0)
    return [coarse[d] for d in range(-r, r + 1)]


def masks_1d(level: int) -> tuple[list[Fraction], list[Fraction]]:
    """Exact 1-D masks (M_l, L_l) for level ``level`` (1 = finest), each of the same
    odd length 2R+1 (the shorter one zero-padded)."""
    if level < 1:
        raise ValueError("level must be >= 1")
    m = [Fraction(1)]
    lap = [Fraction(-1), Fraction(2), Fraction(-1)]
    for _ in range(level - 1):
        m = galerkin_1d(m)
        lap = galerkin_1d(lap)
    n = max(len(m), len(lap))
    pad = lambda v: [Fraction(0)] * ((n - len(v)) // 2) + v + [Fraction(0)] * ((n - len(v)) // 2)
    return pad(m), pad(lap)


def stencils_2d_exact(level: int) -> tuple[list[list[Fraction]], list[list[Fraction]]]:
    """Exact 2-D stencils (Lap_l * h^2, K_l) as nested lists indexed [dy][dx]."""
    m, lap = masks_1d(level)
    n = len(m)
    lap2 = [[lap[a] * m[b] + m[a] * lap[b] for b in range(n)] for a in range(n)]
    k2 = [[m[a] * m[b] for b in range(n)] for a in range(n)]
    return lap2, k2


def stencils_2d(level: int, h: float) -> tuple[np.ndarray, np.ndarray]:
    """FP64 2-D stencils: (Lap_l, K_l) with Lap_l already divided by the fine h^2.
    Each exact value is rounded once to FP64."""
    lap2, k2 = stencils_2d_exact(level)
    lap = np.array([[float(v) for v in row] for row in lap2]) / (h * h)
    kk = np.array([[float(v) for v in row] for row in k2])
    return lap, kk


def radius(level: int) -> int:
    """Stencil radius R of level ``level``: 1 (3x3), 2 (5x5), then 3 (7x7)."""
    return len(masks_1d(level)[0]) // 2
