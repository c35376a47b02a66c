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

Pins (tests/test_oracle_transfers.py): Z reproduces constants and linear
functions in the interior, <Z^T v, w> = <v, Z w>, bilinear interpolation is
exact for bilinear functions, FW equals one quarter of the bilinear transpose,
and Z^T A Z reproduces the printed coarse stencils.
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
