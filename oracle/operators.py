"""Matrix-free Helmholtz / CSLP operators.  TEST INFRASTRUCTURE ONLY (FP64 oracle).

Arrays are complex128 indexed [j, i] (row = y, x fastest) on a vertex-centred
grid (Section 2.1).  Every operator is applied as the paper defines it: a
stencil sum with ghost points substituted, never an assembled matrix.

* ``apply_5pt``     the 5-point operator c*(4u - u_E - u_W - u_N - u_S) - shift*ks*k^2*u
                    with the Sommerfeld ghost point u_0 = u_2 + 2 H i k_1 u_1
                    (Section 2.1, Eq. for [A_h] and the Sommerfeld ghost equation),
                    or homogeneous Dirichlet (unknowns = interior nodes, outside = 0).
                    shift = 1 gives A_h; shift = beta1 + i beta2 gives the CSLP
                    M_(beta1,beta2) (Section 3.1, Eq. for the CSLP).
* ``apply_level``   the level-l re-discretised operator (Section 3.3): the exact
                    Galerkin 2-D stencil at interior nodes; physical-boundary nodes
                    use the standard second-order 5-point row at spacing H_l (scaled
                    to the level's Galerkin scale 4^(l-1)); near the boundary the
                    first outside layer holds the Sommerfeld ghost value, layers
                    beyond it are zero and ghost wavenumbers are zero
                    (Section 3.3, "Boundary").  The wavenumber stencil K_l acts on
                    k_l^2 * u with k_l the injection of the fine k.
* ``diag_5pt`` / ``diag_level``   the exact diagonal of those operators (the
                    ghost substitution feeds back into the diagonal).
* ``jacobi``        one damped-Jacobi sweep u + omega * D^-1 (f - M u).
* ``scale_boundary_rows``   the symmetric row scaling D (1/2 on boundary edges, 1/4 at corners)
                    of the Sommerfeld system (pins: D A_h is complex symmetric; the scaled
                    system has the same solution).

Pins (tests/test_oracle_operators.py): closed-form Dirichlet eigenpairs, O(h^2)
convergence of manufactured solutions with Dirichlet and Sommerfeld data,
symmetry of the edge-scaled Sommerfeld matrix, a dense direct solve, the
reduction of ``apply_level`` at level 1 to ``apply_5pt``, Galerkin triple
products for the interior rows of levels 2-3, brute-force diagonals, and for
levels 2-4: first-order consistency of the physical-boundary rows with
-Laplace(u) - shift k^2 u plus the folded-in Sommerfeld data (fixes the ghost
spacing H_l and the scale 4^(l-1)), and exactness of the rows whose stencil
reaches the first outside layer on waves that satisfy the ghost relation
exactly (fixes that layer's ghost value and the zero ghost wavenumber).
Not fixed by any pin: the zero padding beyond the first outside layer, which is
this implementation's reading of what the paper calls an open problem.

* ``apply_level_dirichlet`` / ``diag_level_dirichlet``   the level-l operator on a
                    homogeneous Dirichlet grid (MP-1a): the Galerkin stencil at every
                    interior unknown, zero outside.  Pins: level 1 equals the
                    Dirichlet ``apply_5pt``; interior rows equal the Dirichlet Galerkin
                    triple product; rows that reach the boundary differ from it (zero
                    padding is this reading, not the exact product), parity there is
                    pinned to the oracle only.
"""
from __future__ import annotations

import numpy as np

from .stencils import stencils_2d

SOMMERFELD = "sommerfeld"
DIRICHLET = "dirichlet"


def _ghost_padded(u: np.ndarray, k: np.ndarray, H: float, bc: str) -> np.ndarray:
    """u padded by one ghost layer.  Sommerfeld: the ghost beyond a boundary node
    is the inner neighbour plus 2 H i k u_boundary (ghost equation, Section 2.1).
    Dirichlet: zero (homogeneous boundary values outside the interior unknowns).
    The four corner cells of the padding are never used by a 5-point stencil."""
    ny, nx = u.shape
    g = np.zeros((ny + 2, nx + 2), dtype=np.complex128)
    g[1:-1, 1:-1] = u
    if bc == SOMMERFELD:
        g[1:-1, 0] = u[:, 1] + 2j * H * k[:, 0] * u[:, 0]
        g[1:-1, -1] = u[:, -2] + 2j * H * k[:, -1] * u[:, -1]
        g[0, 1:-1] = u[1, :] + 2j * H * k[0, :] * u[0, :]
        g[-1, 1:-1] = u[-2, :] + 2j * H * k[-1, :] * u[-1, :]
    elif bc != DIRICHLET:
        raise ValueError(bc)
    return g


def apply_5pt(u, k, c, H, shift=1.0, ks=1.0, bc=SOMMERFELD):
    """c * (4 u_C - u_E - u_W - u_N - u_S) - shift * ks * k^2 * u_C, ghosts substituted."""
    g = _ghost_padded(u, k, H, bc)
    lap = 4.0 * u - g[1:-1, 2:] - g[1:-1, :-2] - g[2:, 1:-1] - g[:-2, 1:-1]
    return c * lap - shift * ks * (k * k) * u


def apply_helmholtz(u, k, h, shift=1.0, bc=SOMMERFELD):
    """Fine-grid A_h u (shift = 1) or CSLP M u (shift = beta1 + i beta2), spacing h."""
    return apply_5pt(u, k, 1.0 / (h * h), h, shift, 1.0, bc)


def _boundary_count(ny: int, nx: int) -> np.ndarray:
    """Number of physical boundary sides each node touches (0, 1 or 2)."""
    g = np.zeros((ny, nx))
    g[:, 0] += 1
    g[:, -1] += 1
    g[0, :] += 1
    g[-1, :] += 1
    return g


def diag_5pt(k, c, H, shift=1.0, ks=1.0, bc=SOMMERFELD):
    """Diagonal of ``apply_5pt``: c (4 - 2 i H k g) - shift ks k^2, g = boundary sides."""
    ny, nx = k.shape
    d = 4.0 * c - shift * ks * k * k + 0j
    if bc == SOMMERFELD:
        d = d - c * 2j * H * k * _boundary_count(ny, nx)
    return d


def level_spacing(level: int, h: float) -> float:
    """H_l = 2^(l-1) h."""
    return (2 ** (level - 1)) * h


def level_scale(level: int) -> float:
    """Galerkin scale of level l: the wavenumber stencil K_l sums to 4^(l-1)."""
    return float(4 ** (level - 1))


def apply_level(u, k, level, h, shift=1.0):
    """Level-l operator A_l (shift = 1) or M_l (shift = beta1 + i beta2), Sommerfeld.

    Interior nodes: sum over the (2R+1)^2 Galerkin stencil of Lap_l * u_ext minus
    shift * K_l * (k_ext^2 * u_ext), where u_ext is u extended by one ghost layer
    (Sommerfeld ghost value with spacing H_l; corner cells of that layer and all
    farther cells are zero) and k_ext is k inside and zero outside.
    Physical-boundary nodes: 5-point row at spacing H_l times 4^(l-1).
    """
    lap, kk = stencils_2d(level, h)
    R = lap.shape[0] // 2
    H = level_spacing(level, h)
    ks = level_scale(level)
    ny, nx = u.shape
    ue = np.zeros((ny + 2 * R, nx + 2 * R), dtype=np.complex128)
    ue[R:R + ny, R:R + nx] = u
    ue[R:R + ny, R - 1] = u[:, 1] + 2j * H * k[:, 0] * u[:, 0]
    ue[R:R + ny, R + nx] = u[:, -2] + 2j * H * k[:, -1] * u[:, -1]
    ue[R - 1, R:R + nx] = u[1, :] + 2j * H * k[0, :] * u[0, :]
    ue[R + ny, R:R + nx] = u[-2, :] + 2j * H * k[-1, :] * u[-1, :]
    k2e = np.zeros((ny + 2 * R, nx + 2 * R))
    k2e[R:R + ny, R:R + nx] = k * k
    we = k2e * ue
    v = np.zeros((ny, nx), dtype=np.complex128)
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            a = lap[dy + R, dx + R]
            b = kk[dy + R, dx + R]
            if a != 0.0:
                v += a * ue[R + dy:R + dy + ny, R + dx:R + dx + nx]
            if b != 0.0:
                v -= shift * b * we[R + dy:R + dy + ny, R + dx:R + dx + nx]
    vb = apply_5pt(u, k, 1.0 / (h * h), H, shift, ks, SOMMERFELD)
    v[0, :] = vb[0, :]
    v[-1, :] = vb[-1, :]
    v[:, 0] = vb[:, 0]
    v[:, -1] = vb[:, -1]
    return v


def diag_level(k, level, h, shift=1.0):
    """Exact diagonal of ``apply_level``.  At interior nodes it is the stencil centre;
    a node one step inside a boundary also receives the tap that reaches the
    ghost layer two steps away, because that ghost value contains the node itself
    with coefficient 1.  Boundary nodes take the 5-point diagonal."""
    lap, kk = stencils_2d(level, h)
    R = lap.shape[0] // 2
    H = level_spacing(level, h)
    ks = level_scale(level)
    ny, nx = k.shape
    d = lap[R, R] - shift * kk[R, R] * k * k + 0j
    if R >= 2:
        d[:, 1] += lap[R, R - 2]
        d[:, nx - 2] += lap[R, R + 2]
        d[1, :] += lap[R - 2, R]
        d[ny - 2, :] += lap[R + 2, R]
    db = diag_5pt(k, 1.0 / (h * h), H, shift, ks, SOMMERFELD)
    d[0, :] = db[0, :]
    d[-1, :] = db[-1, :]
    d[:, 0] = db[:, 0]
    d[:, -1] = db[:, -1]
    return d


def apply_level_dirichlet(u, k, level, h, shift=1.0):
    """Level-l operator on a homogeneous Dirichlet grid (interior unknowns only): the
    Galerkin stencil of Section 3.3 at every unknown, with zero values outside the grid
    (the boundary values are zero and no boundary rows exist).  Level 1 is the 5-point
    operator of Section 2.1 with Dirichlet data."""
    lap, kk = stencils_2d(level, h)
    R = lap.shape[0] // 2
    ny, nx = u.shape
    ue = np.zeros((ny + 2 * R, nx + 2 * R), dtype=np.complex128)
    ue[R:R + ny, R:R + nx] = u
    we = np.zeros_like(ue)
    we[R:R + ny, R:R + nx] = k * k * u
    v = np.zeros((ny, nx), dtype=np.complex128)
    for dy in range(-R, R + 1):
        for dx in range(-R, R + 1):
            a = lap[dy + R, dx + R]
            b = kk[dy + R, dx + R]
            if a != 0.0:
                v += a * ue[R + dy:R + dy + ny, R + dx:R + dx + nx]
            if b != 0.0:
                v -= shift * b * we[R + dy:R + dy + ny, R + dx:R + dx + nx]
    return v


def diag_level_dirichlet(k, level, h, shift=1.0):
    """Diagonal of ``apply_level_dirichlet``: the stencil centre at every unknown."""
    lap, kk = stencils_2d(level, h)
    R = lap.shape[0] // 2
    return lap[R, R] - shift * kk[R, R] * k * k + 0j


def scale_boundary_rows(v):
    """D v with D = 1/2 on the grid's boundary edges and 1/4 at its corners: the row scaling that
    makes the ghost-eliminated Sommerfeld matrix complex symmetric (Section 2.1 calls the matrix
    symmetric).  Applied to A_h u and to b it leaves the solution of A_h u = b unchanged."""
    d = np.ones(v.shape[-2:])
    d[:, 0] *= 0.5
    d[:, -1] *= 0.5
    d[0, :] *= 0.5
    d[-1, :] *= 0.5
    return d * v


def jacobi(u, f, apply_m, diag, omega):
    """One damped-Jacobi sweep: u + omega * (f - M u) / diag(M)."""
    return u + omega * (f - apply_m(u)) / diag
