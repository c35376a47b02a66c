"""Multi-instance batches (per_rhs_k): right-hand side r of a batch solves the problem with its
own wavenumber field r, every sweep one launch over the whole batch.

Each instance of a mixed batch must equal the same problem set up and solved alone (bitwise:
the batched kernels keep each right-hand side's arithmetic separate) and the FP64 oracle's solve
of that problem (solution within 1e-5, outer iterations within one, true residual <= 1e-6 with
the oracle's operator).  The level operators, the residual check and the serving layer take the
per-instance fields as well."""
import ctypes

import numpy as np
import pytest

import model_problems as mp
from gpu_common import TOL64, TOL64_COMPOSITE, dev, host, hzlib, rel2, rel_inf, torch
from oracle.madp import Hierarchy, MADPConfig
from oracle.operators import DIRICHLET, SOMMERFELD, apply_helmholtz

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hz():
    return hzlib()


def _instances(n=129, seeds=(3, 5, 7, 11), kh=(0.3, 0.25, 0.35, 0.2)):
    """Random-velocity problems on one grid with different fields and frequencies; one point
    source each at a different top-row node."""
    ps = [mp.random_field(n, 5.0, seed=s, kh_max=q, levels=3, negdef_from_level=4, nsrc=len(seeds))
          for s, q in zip(seeds, kh)]
    k = np.stack([p.k for p in ps])
    b = np.stack([p.b[r] for r, p in enumerate(ps)])
    return ps, k, b


@pytest.mark.parametrize("device_gmres,precision", [(1, "mixed"), (1, "fp64"), (3, "mixed"), (4, "mixed")])
def test_instance_batch_equals_each_alone(hz, device_gmres, precision):
    """Four instances in one batch equal each problem solved on a handle of its own.  With
    device_gmres 3 (always clusters) and 4 (always the slice grid) both sides run the same
    kernels: bitwise, with the same iteration counts.  With 1 the batch runs the level-3 GMRES
    as one cluster per instance in one launch while a lone right-hand side takes the grid form,
    whose reductions sum in another order: solutions within 1e-5, outer iterations within one."""
    ps, k, b = _instances()
    kw = dict(levels=3, negdef_from_level=4, precision=precision, device_gmres=device_gmres)
    H = hz.Helmholtz(dev(k), ps[0].h, **kw)
    assert H.cfg.per_rhs_k == 1 and H.cfg.max_rhs == 4
    ub, stb = H.solve(dev(b), tol=1e-6)
    ub = host(ub)
    for r, p in enumerate(ps):
        H1 = hz.Helmholtz(dev(p.k), p.h, **kw)
        u1, st1 = H1.solve(dev(b[r]), tol=1e-6)
        assert stb[r]["status"] == 0 and stb[r]["true_relres"] <= 1e-6
        if device_gmres == 1:
            assert rel2(ub[r], host(u1)) <= 1e-5
            assert abs(st1[0]["outer_iterations"] - stb[r]["outer_iterations"]) <= 1
        else:
            assert np.array_equal(host(u1), ub[r]), r
            assert st1[0]["outer_iterations"] == stb[r]["outer_iterations"]
            assert st1[0]["cslp_gmres_iterations"] == stb[r]["cslp_gmres_iterations"]
        H1.close()
    H.close()


def test_instance_batch_matches_oracle(hz):
    """Each instance of a mixed-precision batch against the FP64 oracle's solve of its problem."""
    ps, k, b = _instances(seeds=(3, 5, 7), kh=(0.3, 0.25, 0.35))
    H = hz.Helmholtz(dev(k), ps[0].h, levels=3, negdef_from_level=4, precision="mixed")
    u, st = H.solve(dev(b), tol=1e-6)
    u = host(u)
    for r, p in enumerate(ps):
        ref, rst = Hierarchy(p.k, p.h, MADPConfig(levels=3, negdef_from_level=4)).solve(b[r])
        rel = np.linalg.norm(b[r] - apply_helmholtz(u[r], p.k, p.h)) / np.linalg.norm(b[r])
        assert st[r]["status"] == 0 and rel <= 1e-6
        assert abs(st[r]["true_relres"] - rel) <= 1e-9
        assert rel2(u[r], ref) <= 1e-5
        assert abs(st[r]["outer_iterations"] - rst.outer_iterations) <= 1
    # the statistics differ between instances (different problems, different work)
    assert len({s["outer_iterations"] for s in st}) > 1 or len({tuple(s["cslp_gmres_iterations"]) for s in st}) > 1


@pytest.mark.parametrize("bc", [SOMMERFELD, DIRICHLET])
def test_instance_apply_and_residual(hz, bc):
    """y_r = A_h(k_r) x_r for every right-hand side (FP64, against the oracle's operator), fewer
    right-hand sides than instances take the first fields, and the allocation-free residual uses
    each instance's field."""
    n = 65
    ny, nx = (n, n) if bc == SOMMERFELD else (n - 2, n - 2)
    h = 1.0 / (n - 1)
    k = np.stack([mp.random_k(ny, nx, seed=40 + r, kmin=5.0, kmax=30.0) for r in range(3)])
    x = np.stack([mp.random_complex((ny, nx), seed=50 + r) for r in range(3)])
    H = hz.Helmholtz(dev(k), h, bc="sommerfeld" if bc == SOMMERFELD else "dirichlet", levels=2)
    y = host(H.apply(dev(x)))
    for r in range(3):
        assert rel_inf(y[r], apply_helmholtz(x[r], k[r], h, bc=bc)) <= TOL64
    y2 = host(H.apply(dev(x[:2])))
    assert np.array_equal(y2, y[:2])
    b = np.stack([mp.random_complex((ny, nx), seed=60 + r) for r in range(3)])
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    assert hz.lib().hz_true_residual_noalloc(H._h, dev(b).data_ptr(), dev(x).data_ptr(), 3, out.data_ptr()) == 0
    want = [np.linalg.norm(b[r] - apply_helmholtz(x[r], k[r], h, bc=bc)) / np.linalg.norm(b[r]) for r in range(3)]
    np.testing.assert_allclose(host(out), want, rtol=1e-12)
    # a fourth right-hand side has no field
    x4 = dev(np.stack([x[0]] * 4))
    with pytest.raises(hz.HzError):
        H.apply(x4)
    H.close()


def test_instance_level_operators_and_precond(hz):
    """Coarse-level operators (radius 2 and 3 Galerkin stencils on the injected per-instance
    fields) and the whole preconditioner equal the single-instance handles' results bitwise."""
    ps, k, _ = _instances(seeds=(3, 5), kh=(0.3, 0.2))
    v = np.stack([mp.random_complex((129, 129), seed=70 + r) for r in range(2)])
    H = hz.Helmholtz(dev(k), ps[0].h, levels=3, negdef_from_level=4)
    xb = host(H.precond(dev(v)))
    outs = {}
    for lev in (2, 3):
        ny, nx = H.level_size(lev)
        w = dev(np.stack([mp.random_complex((ny, nx), seed=80 + lev + r) for r in range(2)]))
        outs[lev] = (w, host(H.level_apply(lev, w, "M")))
    for r, p in enumerate(ps):
        H1 = hz.Helmholtz(dev(p.k), p.h, levels=3, negdef_from_level=4)
        assert np.array_equal(host(H1.precond(dev(v[r]))), xb[r])
        for lev, (w, y) in outs.items():
            assert np.array_equal(host(H1.level_apply(lev, w[r].contiguous(), "M")), y[r])
        H1.close()
    ref = Hierarchy(ps[1].k, ps[1].h, MADPConfig(levels=3, negdef_from_level=4)).precond(1, v[1])
    assert rel_inf(xb[1], ref) <= TOL64_COMPOSITE
    H.close()


def test_instance_request_served(hz):
    """A multi-instance request through the server equals the batch solved directly."""
    ps, k, b = _instances(seeds=(3, 5), kh=(0.3, 0.2))
    H = hz.Helmholtz(dev(k), ps[0].h, levels=3, negdef_from_level=4, precision="mixed")
    ud, _ = H.solve(dev(b), tol=1e-6)
    S = hz.Server(8 << 30, max_active=2)
    t = S.submit(k, b, ps[0].h, tol=1e-6, levels=3, negdef_from_level=4, precision="mixed")
    u, st, _ = S.wait(t)
    assert all(s["status"] == 0 for s in st)
    assert np.array_equal(u, host(ud))
    S.close()
    H.close()
