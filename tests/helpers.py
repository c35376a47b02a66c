"""Test-side helpers: brute-force assembly of matrix-free operators by probing."""
import numpy as np
import scipy.sparse as sp


def assemble(apply, shape, reach):
    """Sparse matrix of a linear matrix-free operator whose row n depends only on
    nodes within Chebyshev distance ``reach`` of n.  Probes with P*P colour vectors
    (period P = 2*reach + 1), so each probe response at node n holds exactly one
    matrix entry per colour."""
    ny, nx = shape
    P = 2 * reach + 1
    jj, ii = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    rows, cols, vals = [], [], []
    for cy in range(P):
        for cx in range(P):
            e = ((jj % P == cy) & (ii % P == cx)).astype(np.complex128)
            if not e.any():
                continue
            y = apply(e)
            for dy in range(-reach, reach + 1):
                for dx in range(-reach, reach + 1):
                    mj, mi = jj + dy, ii + dx
                    ok = (mj >= 0) & (mj < ny) & (mi >= 0) & (mi < nx) & (mj % P == cy) & (mi % P == cx)
                    r = (jj * nx + ii)[ok]
                    c = (mj * nx + mi)[ok]
                    v = y[ok]
                    nz = v != 0
                    rows.append(r[nz]); cols.append(c[nz]); vals.append(v[nz])
    n = ny * nx
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def rel_err(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))
