"""GPU parity of the homogeneous-Dirichlet multilevel path (MP-1a, Section 2.2) against the FP64
oracle: interior-unknown transfers, zero-padded level operators, the Dirichlet multigrid, the
CSLP GMRES on a Dirichlet level and whole solves."""
import numpy as np
import pytest

import model_problems as mp
from gpu_common import TOL64, TOL64_COMPOSITE, dev, host, hzlib, rel2, rel_inf, torch
from oracle import operators as O
from oracle import transfers as T
from oracle.madp import Hierarchy, MADPConfig
from oracle.multigrid import CSLPMultigrid

pytestmark = pytest.mark.gpu

SHIFT = 1.0 + 0.5j
NY, NX, H = 63, 127, 1.0 / 128      # levels: 63 x 127, 31 x 63, 15 x 31


@pytest.fixture(scope="module")
def hz():
    return hzlib()


def _k(seed=31):
    return mp.random_k(NY, NX, seed=seed, kmin=5.0, kmax=0.3 / H)


def _kl(k, level):
    return T.inject_dirichlet(k, 2 ** (level - 1)) if level > 1 else k


@pytest.mark.parametrize("level", [1, 2, 3])
@pytest.mark.parametrize("op", ["A", "M"])
def test_dirichlet_level_apply_fp64(hz, level, op):
    k = _k()
    Hh = hz.Helmholtz(dev(k), H, bc="dirichlet", levels=3)
    cy, cx = Hh.level_size(level)
    assert (cy, cx) == {1: (63, 127), 2: (31, 63), 3: (15, 31)}[level]
    u = mp.random_complex((cy, cx), seed=32 + level)
    y = host(Hh.level_apply(level, dev(u), op))
    ref = O.apply_level_dirichlet(u, _kl(k, level), level, H, 1.0 if op == "A" else SHIFT)
    assert rel_inf(y, ref) <= TOL64


@pytest.mark.parametrize("level", [1, 2])
def test_dirichlet_transfers_fp64(hz, level):
    k = _k()
    Hh = hz.Helmholtz(dev(k), H, bc="dirichlet", levels=3)
    cy, cx = Hh.level_size(level)
    ny2, nx2 = Hh.level_size(level + 1)
    assert (ny2, nx2) == (T.coarse_size_dirichlet(cy), T.coarse_size_dirichlet(cx))
    v = mp.random_complex((cy, cx), seed=40 + level)
    assert rel_inf(host(Hh.defl_restrict(level, dev(v))), T.deflation_restrict_dirichlet(v)) <= TOL64
    w = mp.random_complex((ny2, nx2), seed=42 + level)
    assert rel_inf(host(Hh.defl_prolong(level, dev(w))), T.deflation_prolong_dirichlet(w, (cy, cx))) <= TOL64
    t, r = Hh.defl_prolong_residual(level, dev(w), dev(v))
    t_ref = T.deflation_prolong_dirichlet(w, (cy, cx))
    assert rel_inf(host(t), t_ref) <= TOL64
    r_ref = v - O.apply_level_dirichlet(t_ref, _kl(k, level), level, H, 1.0)
    assert rel_inf(host(r), r_ref) <= TOL64_COMPOSITE


@pytest.mark.parametrize("level", [1, 2])
def test_dirichlet_mg_vcycle_fp64(hz, level):
    """Fused V(1,1) (damped Jacobi, full weighting and bilinear prolongation at coarse unknown
    I = fine unknown 2I + 1) against the oracle's Dirichlet multigrid."""
    k = _k(33)
    Hh = hz.Helmholtz(dev(k), H, bc="dirichlet", levels=2)
    cy, cx = Hh.level_size(level)
    f = mp.random_complex((cy, cx), seed=50 + level)
    mg = CSLPMultigrid(_kl(k, level), level, H, SHIFT, bc=O.DIRICHLET)
    assert [Hh.mg_size(level, m) for m in range(len(mg.levels))] == [lv.shape for lv in mg.levels]
    assert rel_inf(host(Hh.mg_vcycle(level, dev(f))), mg(f)) <= TOL64_COMPOSITE


def test_dirichlet_mg_general_path_fp64(hz):
    """nu1 = 2 runs the unfused kernels (residual, full weighting, prolongation and add)."""
    k = _k(34)
    Hh = hz.Helmholtz(dev(k), H, bc="dirichlet", levels=1, mg_nu1=2, mg_nu2=1)
    f = mp.random_complex((NY, NX), seed=55)
    mg = CSLPMultigrid(k, 1, H, SHIFT, nu1=2, nu2=1, bc=O.DIRICHLET)
    assert rel_inf(host(Hh.mg_vcycle(1, dev(f))), mg(f)) <= TOL64_COMPOSITE


@pytest.mark.parametrize("device_gmres", [1, 0])
def test_dirichlet_cslp_gmres_fp64(hz, device_gmres):
    """GMRES CSLP inverse on the Dirichlet level 3 (15 x 31 unknowns, radius-3 operator): the
    persistent kernel (1) and the host-driven steps (0) reproduce the oracle's iterations and x."""
    k = _k(35)
    Hh = hz.Helmholtz(dev(k), H, bc="dirichlet", levels=3, device_gmres=device_gmres)
    b = mp.random_complex((15, 31), seed=60)
    hier = Hierarchy(k, H, MADPConfig(levels=3, bc="dirichlet"))
    x_ref = hier.cslp_inverse(3, b)
    x, its = Hh.cslp_gmres(3, dev(b))
    assert its[0] == hier.stats.cslp_gmres_iterations[3]
    assert rel_inf(host(x), x_ref) <= TOL64_COMPOSITE


@pytest.mark.parametrize("levels,precision", [(1, "fp64"), (2, "fp64"), (3, "fp64"), (4, "fp64"), (3, "mixed"),
                                              (4, "mixed")])
def test_mp1a_solve(hz, levels, precision):
    """MP-1a (constant k = 20 on the unit square, 127^2 interior unknowns, centre source) solved
    on the GPU reaches the 1e-6 residual of the Dirichlet system with the oracle's solution and
    within one outer iteration of it."""
    p = mp.mp1a(128, 20.0, levels=levels)
    ref, rst = Hierarchy(p.k, p.h, MADPConfig(levels=levels, bc="dirichlet")).solve(p.b[0])
    Hh = hz.Helmholtz(dev(p.k), p.h, bc="dirichlet", levels=levels, precision=precision)
    u, st = Hh.solve(dev(p.b[0]), tol=1e-6)
    u = host(u)
    r = p.b[0] - O.apply_helmholtz(u, p.k, p.h, bc=O.DIRICHLET)
    true_rel = np.linalg.norm(r) / np.linalg.norm(p.b[0])
    assert st[0]["status"] == 0 and true_rel <= 1e-6
    assert abs(st[0]["true_relres"] - true_rel) <= 1e-9
    assert rel2(u, ref) <= 1e-5
    assert abs(st[0]["outer_iterations"] - rst.outer_iterations) <= 1
