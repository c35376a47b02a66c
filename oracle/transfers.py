"""Grid transfers.  TEST INFRASTRUCTURE ONLY (FP64 oracle).

Coarse node I coincides with fine node 2I (vertex-centred coarsening,
n_coarse = (n_fine + 1) / 2).  All operators are tensor products of 1-D sparse
matrices written from their definitions; 2-D application is A_y @ v @ A_x^T.

* Deflation (Section 3.1, higher-order deflation vectors; Algorithm 1 lines 5
  and 11): Z^T has the 1-D rows p = [1, 4, 6, 4, 1] / 8 centred on the
  coincident fine node, (Z^T v)_I = sum_a p_a v_{2I+a}; Z is its exact
  transpose.  Fine nodes outside the grid do not exist, i.e. the weights are
  truncated at the boundary.  These weights are the ones that reproduce every
  coarse stencil the paper prints (Section 3.3, Appendix A).
* Multigrid (the CSLP V-cycle): full weighting FW = (1/16) [1 2 1; 2 4 2; 1 2 1]
  at coincident nodes (outside fine nodes count as zero, no renormalisation)
  and bilinear prolongation (coincident nodes copied, edge midpoints averaged
  from 2 coarse nodes, cell centres from 4).

Homogeneous Dirichlet grids (MP-1a, Section 2.2) hold only the interior nodes: a
grid of n unknowns is the interior of a vertex grid of n + 2 nodes whose boundary
values are zero.  Its transfers are the ones above on that vertex grid, applied to
the zero-extended vector and restricted to interior nodes (``*_dirichlet``):
coarse unknown I coincides with fine unknown 2I + 1, n_coarse = (n_fine - 1) / 2.

Pins (tests/test_oracle_transfers.py): Z reproduces constants and linear
functions in the interior, <Z^T v, w> = <v, Z w>, bilinear interpolation is
exact for bilinear functions, FW equals one quarter of the bilinear transpose,
and Z^T A Z reproduces the printed coarse stencils; the Dirichlet variants
reproduce constants and linear functions away from the boundary and keep the
transpose relations.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

P_DEFL = np.array([1.0, 4.0, 6.0, 4.0, 1.0]) / 8.0


def coarse_size(n_fine: int) -> int:
    if n_fine < 3 or (n_fine - 1) % 2 != 0:
        raise ValueError(f"grid size {n_fine} cannot be coarsened (needs odd n >= 3)")
    return (n_fine + 1) // 2


def zt_1d(n_fine: int) -> sp.csr_matrix:
    """1-D deflation restriction: (Z^T)[I, 2I + a] = p_a, a = -2..2, truncated."""
    nc = coarse_size(n_fine)
    rows, cols, vals = [], [], []
    for I in range(nc):
        for a in range(-2, 3):
            n = 2 * I + a
            if 0 <= n < n_fine:
                rows.append(I)
                cols.append(n)
                vals.append(P_DEFL[a + 2])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nc, n_fine))


def deflation_restrict(v: np.ndarray) -> np.ndarray:
    """v_hat = Z^T v (Algorithm 1, line 5)."""
    ny, nx = v.shape
    return zt_1d(ny) @ v @ zt_1d(nx).T


def deflation_prolong(w: np.ndarray, fine_shape) -> np.ndarray:
    """t = Z w (Algorithm 1, line 11): the transpose of ``deflation_restrict``."""
    ny, nx = fine_shape
    return (zt_1d(ny).T @ w) @ zt_1d(nx)


def fw_1d(n_fine: int) -> sp.csr_matrix:
    """1-D full weighting: row I has [1/4, 1/2, 1/4] at fine nodes 2I-1, 2I, 2I+1."""
    nc = coarse_size(n_fine)
    w = [0.25, 0.5, 0.25]
    rows, cols, vals = [], [], []
    for I in range(nc):
        for a in (-1, 0, 1):
            n = 2 * I + a
            if 0 <= n < n_fine:
                rows.append(I)
                cols.append(n)
                vals.append(w[a + 1])
    return sp.csr_matrix((vals, (rows, cols)), shape=(nc, n_fine))


def bilinear_1d(n_fine: int) -> sp.csr_matrix:
    """1-D linear interpolation: fine 2I <- coarse I; fine 2I+1 <- (I + (I+1)) / 2."""
    nc = coarse_size(n_fine)
    rows, cols, vals = [], [], []
    for n in range(n_fine):
        if n % 2 == 0:
            rows.append(n)
            cols.append(n // 2)
            vals.append(1.0)
        else:
            rows += [n, n]
            cols += [n // 2, n // 2 + 1]
            vals += [0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_fine, nc))


def fw_restrict(r: np.ndarray) -> np.ndarray:
    """Full-weighting restriction of a fine residual."""
    ny, nx = r.shape
    return fw_1d(ny) @ r @ fw_1d(nx).T


def bilinear_prolong(e: np.ndarray, fine_shape) -> np.ndarray:
    """Bilinear prolongation of a coarse correction to the fine grid."""
    ny, nx = fine_shape
    return (bilinear_1d(ny) @ e) @ bilinear_1d(nx).T


def inject(k: np.ndarray, stride: int) -> np.ndarray:
    """Coarse-grid values at coincident nodes (used for the coarse wavenumbers)."""
    return np.ascontiguousarray(k[::stride, ::stride])


# ---- homogeneous Dirichlet grids (interior unknowns only) ---------------------------------
def coarse_size_dirichlet(n_fine: int) -> int:
    if n_fine < 3 or (n_fine - 1) % 2 != 0:
        raise ValueError(f"Dirichlet grid of {n_fine} unknowns cannot be coarsened (needs odd n >= 3)")
    return (n_fine - 1) // 2


def _interior(m: sp.csr_matrix) -> sp.csr_matrix:
    """Drop the first and last row and column (the zero boundary nodes)."""
    return sp.csr_matrix(m[1:-1, :][:, 1:-1])


def zt_1d_dirichlet(n_fine: int) -> sp.csr_matrix:
    """Z^T between interior unknowns: the vertex-grid rows of coarse interior nodes,
    restricted to fine interior columns: (Z^T)[I, 2I + 1 + a] = p_a."""
    coarse_size_dirichlet(n_fine)
    return _interior(zt_1d(n_fine + 2))


def fw_1d_dirichlet(n_fine: int) -> sp.csr_matrix:
    coarse_size_dirichlet(n_fine)
    return _interior(fw_1d(n_fine + 2))


def bilinear_1d_dirichlet(n_fine: int) -> sp.csr_matrix:
    coarse_size_dirichlet(n_fine)
    return _interior(bilinear_1d(n_fine + 2))


def deflation_restrict_dirichlet(v: np.ndarray) -> np.ndarray:
    ny, nx = v.shape
    return zt_1d_dirichlet(ny) @ v @ zt_1d_dirichlet(nx).T


def deflation_prolong_dirichlet(w: np.ndarray, fine_shape) -> np.ndarray:
    ny, nx = fine_shape
    return (zt_1d_dirichlet(ny).T @ w) @ zt_1d_dirichlet(nx)


def fw_restrict_dirichlet(r: np.ndarray) -> np.ndarray:
    ny, nx = r.shape
    return fw_1d_dirichlet(ny) @ r @ fw_1d_dirichlet(nx).T


def bilinear_prolong_dirichlet(e: np.ndarray, fine_shape) -> np.ndarray:
    ny, nx = fine_shape
    return (bilinear_1d_dirichlet(ny) @ e) @ bilinear_1d_dirichlet(nx).T


def inject_dirichlet(k: np.ndarray, stride: int) -> np.ndarray:
    """Values at the fine unknowns that coincide with coarse unknowns: stride (I + 1) - 1."""
    return np.ascontiguousarray(k[stride - 1::stride, stride - 1::stride])
