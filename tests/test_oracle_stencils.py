"""Pins for the oracle's exact coarse-stencil generator (Section 3.3, Appendix A)."""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.stencils import masks_1d, radius, stencils_2d_exact
from oracle.transfers import zt_1d

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    den, rows = None, []
    with open(os.path.join(GOLDEN, name + ".txt")) as f:
        for line in f:
            if line.startswith("# denominator:"):
                den = int(line.split(":")[1])
            elif not line.startswith("#") and line.strip():
                rows.append([int(x) for x in line.split()])
    return den, rows


@pytest.mark.parametrize("level", [3, 4, 5, 6])
def test_printed_laplace_stencils_exact(level):
    """Every printed Laplace-stencil integer (Section 3.3 for 4h; Appendix A for
    8h, 16h, 32h) equals the exact Galerkin value."""
    den, printed = load_golden(f"lap_level{level}")
    lap, _ = stencils_2d_exact(level)
    for a in range(7):
        for b in range(7):
            exact = lap[a][b] * den
            assert exact.denominator == 1
            assert int(exact) == printed[a][b], (level, a, b)


@pytest.mark.parametrize("level", [3, 4, 5, 6])
def test_printed_wavenumber_stencils(level):
    """Printed wavenumber-stencil integers equal the exact Galerkin values; entries
    larger than 2^53 may differ by the few FP64 roundings the paper's print carries
    (its K_32h table is visibly asymmetric in those entries): at most 4 ulp."""
    den, printed = load_golden(f"k_level{level}")
    _, kk = stencils_2d_exact(level)
    rounded = 0
    for a in range(7):
        for b in range(7):
            exact = kk[a][b] * den
            assert exact.denominator == 1
            e = int(exact)
            if printed[a][b] != e:
                assert abs(e) > 2 ** 53, (level, a, b)
                ulp = 2.0 ** (np.floor(np.log2(abs(e))) - 52)
                assert abs(printed[a][b] - e) <= 4 * ulp, (level, a, b, printed[a][b], e)
                rounded += 1
    if level < 6:
        assert rounded == 0


def test_level2_masks():
    """Level-2 masks: M_2 = [1, 28, 70, 28, 1] / 64 and L_2 = [-6, -8, 28, -8, -6] / 64."""
    m, lap = masks_1d(2)
    assert [x * 64 for x in m] == [1, 28, 70, 28, 1]
    assert [x * 64 for x in lap] == [-6, -8, 28, -8, -6]


@pytest.mark.parametrize("level", range(1, 7))
def test_mask_invariants(level):
    """Sum M_l = 2^(l-1) (Z^T applied to constants doubles per dimension), the second
    difference annihilates constants and linear functions, both are symmetric,
    and the stencil radius is 1, 2, then 3 from level 3 on (Section 3.3)."""
    m, lap = masks_1d(level)
    assert sum(m) == 2 ** (level - 1)
    assert sum(lap) == 0
    R = len(lap) // 2
    assert sum(lap[d + R] * d for d in range(-R, R + 1)) == 0
    assert m == m[::-1] and lap == lap[::-1]
    assert radius(level) == min(level, 3)


def test_galerkin_by_sparse_triple_product():
    """The recursion equals Z^T S Z with Z assembled from its definition, for the
    mass and second-difference matrices, at interior coarse rows, levels 1 -> 6."""
    n = 257
    M = sp.identity(n, format="csr")
    T = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    for level in range(2, 7):
        Zt = zt_1d(M.shape[0])
        M = (Zt @ M @ Zt.T).tocsr()
        T = (Zt @ T @ Zt.T).tocsr()
        mid = M.shape[0] // 2
        m_ref, l_ref = masks_1d(level)
        R = len(m_ref) // 2
        row_m = M[mid].toarray().ravel()[mid - R:mid + R + 1]
        row_t = T[mid].toarray().ravel()[mid - R:mid + R + 1]
        np.testing.assert_allclose(row_m, [float(x) for x in m_ref], rtol=1e-14, atol=0)
        np.testing.assert_allclose(row_t, [float(x) for x in l_ref], rtol=1e-13, atol=1e-17)
        assert abs(M[mid].sum() - float(sum(m_ref))) < 1e-12


def test_symbol_recursion():
    """Fourier symbols obey S_{l+1}(phi) = 1/2 sum_{t in {phi/2, phi/2+pi}} p(t)^2 S_l(t)
    with p(t) = (1 + cos t)^2 / 2, the symbol of the deflation weights."""
    def sym(s, t):
        R = len(s) // 2
        return sum(float(w) * np.cos((i - R) * t) for i, w in enumerate(s))
    ph = lambda t: (1 + np.cos(t)) ** 2 / 2
    for level in range(1, 6):
        for idx in (0, 1):
            fine = masks_1d(level)[idx]
            coarse = masks_1d(level + 1)[idx]
            for phi in np.linspace(0, np.pi, 17):
                rhs = 0.5 * sum(ph(t) ** 2 * sym(fine, t) for t in (phi / 2, phi / 2 + np.pi))
                assert abs(sym(coarse, phi) - rhs) < 1e-12 * max(1.0, abs(rhs))
