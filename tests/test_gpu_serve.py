"""Serving layer on the GPU: concurrent requests of different sizes, wavenumbers and
precisions give exactly the result each gives alone; admission respects the memory budget;
a request that fails on the host side leaves the others untouched."""
import numpy as np
import pytest

import model_problems as mp
from gpu_common import dev, hzlib, rel2, torch
from oracle.operators import apply_helmholtz

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hz():
    return hzlib()


def _mix():
    """Three problems of different size, wavenumber field and solver configuration."""
    a = mp.named("mp1b_129")
    b = mp.random_field(257, 10.0, seed=5, kh_max=0.3, levels=4)
    c = mp.named("wedge_289x481")
    return [
        (a, dict(levels=a.levels, precision="fp64")),
        (b, dict(levels=b.levels, precision="mixed")),
        (c, dict(levels=c.levels, negdef_from_level=c.negdef_from_level, precision="mixed")),
    ]


def _alone(hz, p, cfg):
    H = hz.Helmholtz(dev(p.k), p.h, **dict(cfg))
    u, st = H.solve_host(p.b[0])
    H.close()
    return u, st[0]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("device_gmres", [1, 2, 3, 0])
@pytest.mark.parametrize("max_rhs", [1, 4])
def test_estimate_bounds_setup_bytes(hz, precision, device_gmres, max_rhs):
    p = mp.random_field(513, 5.0, seed=3, kh_max=0.3, levels=5)
    cfg = dict(levels=5, precision=precision, device_gmres=device_gmres, max_rhs=max_rhs, negdef_from_level=5)
    est = hz.estimate_bytes(513, 513, p.h, **cfg)
    H = hz.Helmholtz(dev(p.k), p.h, **cfg)
    got = H.memory_bytes()
    H.close()
    assert got <= est <= 1.05 * got + (1 << 20)


def test_mix_equals_alone(hz):
    cases = _mix()
    alone = [_alone(hz, p, cfg) for p, cfg in cases]
    srv = hz.Server(budget_bytes=8 << 30, max_active=3)
    tickets = [srv.submit(p.k, p.b[0], p.h, **dict(cfg)) for p, cfg in cases]
    for (p, _), t, (u0, st0) in zip(cases, tickets, alone):
        u, st, ms = srv.wait(t, timeout_s=600)
        assert np.array_equal(u, u0)
        assert st[0]["outer_iterations"] == st0["outer_iterations"]
        assert st[0]["status"] == 0 and ms > 0
        r = p.b[0] - apply_helmholtz(u, p.k, p.h)
        assert np.linalg.norm(r) / np.linalg.norm(p.b[0]) <= 1e-6
    rep = srv.report()
    srv.close()
    assert rep["completed"] == 3 and rep["failed"] == 0 and rep["queued"] == 0
    assert 0 < rep["p50_ms"] <= rep["p99_ms"] and rep["solves_per_s"] > 0


def test_admission_respects_budget(hz):
    """A budget that holds one of the two large footprints at a time runs them one after the
    other (peak <= budget) while the small request is admitted beside them."""
    big = mp.random_field(513, 5.0, seed=7, kh_max=0.3, levels=5)
    small = mp.named("mp1b_129")
    cfg_big = dict(levels=5, precision="mixed", negdef_from_level=5)
    cfg_small = dict(levels=small.levels, precision="fp64")
    n_big, n_small = 513 * 513, 129 * 129
    fb = hz.estimate_bytes(513, 513, big.h, **cfg_big) + n_big * (8 + 32)
    fs = hz.estimate_bytes(129, 129, small.h, **cfg_small) + n_small * (8 + 32)
    budget = fb + fs + fb // 2
    srv = hz.Server(budget_bytes=budget, max_active=3)
    t = [srv.submit(big.k, big.b[0], big.h, **cfg_big), srv.submit(big.k, big.b[0], big.h, **cfg_big),
         srv.submit(small.k, small.b[0], small.h, **cfg_small)]
    outs = [srv.wait(x, timeout_s=600) for x in t]
    rep = srv.report()
    assert rep["completed"] == 3 and rep["peak_bytes"] <= budget
    assert rep["peak_bytes"] >= fb
    assert np.array_equal(outs[0][0], outs[1][0])
    # a footprint above the whole budget is refused at submit
    with pytest.raises(hz.HzError) as e:
        srv.submit(big.k, big.b[0], big.h, levels=5, precision="fp64", max_rhs=8)
    assert e.value.status == hz.HZ_ENOMEM
    srv.close()


def test_host_side_failure_is_isolated(hz):
    """A request whose configuration hz_setup rejects finishes with HZ_EINVAL and its message;
    the requests around it complete with the results they give alone."""
    good = mp.named("mp1b_129")
    u0, _ = _alone(hz, good, dict(levels=2))
    srv = hz.Server(budget_bytes=4 << 30, max_active=2)
    t1 = srv.submit(good.k, good.b[0], good.h, levels=2)
    bad = srv.submit(good.k, good.b[0], good.h, levels=9)       # 129 nodes cannot coarsen 8 times
    t2 = srv.submit(good.k, good.b[0], good.h, levels=2)
    u_bad, _, _ = srv.wait(bad, check=False)
    assert srv.poll(bad)[0] == hz.HZ_EINVAL
    assert "coarsen" in hz.lib().hz_last_error().decode()
    for t in (t1, t2):
        u, st, _ = srv.wait(t)
        assert np.array_equal(u, u0)
    rep = srv.report()
    srv.close()
    assert rep["completed"] == 2 and rep["failed"] == 1


def test_multi_rhs_request(hz):
    p = mp.random_field(129, 10.0, seed=11, kh_max=0.3, levels=2)
    b = mp.random_complex((3, 129, 129), seed=12)
    srv = hz.Server(budget_bytes=2 << 30, max_active=1)
    t = srv.submit(p.k, b, p.h, levels=2, precision="mixed", max_rhs=3)
    u, st, _ = srv.wait(t)
    srv.close()
    H = hz.Helmholtz(dev(p.k), p.h, levels=2, precision="mixed", max_rhs=3)
    ub, _ = H.solve_host(b)
    assert np.array_equal(u, ub)
    assert all(s["status"] == 0 for s in st)
    assert rel2(u[1], ub[1]) == 0


def test_fp64_multi_rhs_deep_hierarchy(hz):
    """Plain FP64, 5 levels on 2049^2, 4 point sources in one batch (the shape of a serving
    request that once broke down): every right-hand side converges to the tolerance."""
    p = mp.random_field(2049, 5.0, seed=1004, kh_max=0.3, levels=5, negdef_from_level=4, nsrc=4)
    H = hz.Helmholtz(dev(p.k), p.h, levels=5, negdef_from_level=4, precision="fp64", max_rhs=4)
    u, st = H.solve(dev(p.b), tol=1e-6)
    H.close()
    assert all(s["status"] == 0 and s["true_relres"] <= 1e-6 for s in st)
    assert bool(np.isfinite(u.cpu().numpy()).all())


def test_dirichlet_request_in_mix(hz):
    """A homogeneous-Dirichlet MP-1a request (interior unknowns, 3 levels) served beside
    Sommerfeld requests: each result equals the same solve alone, and the Dirichlet one solves
    its system to the tolerance (true residual from the oracle's operator)."""
    from oracle.operators import DIRICHLET
    d = mp.mp1a(128, 20.0, levels=3)
    est = hz.estimate_bytes(d.nx, d.ny, d.h, bc=1, levels=3, precision="mixed")
    Hd = hz.Helmholtz(dev(d.k), d.h, bc="dirichlet", levels=3, precision="mixed")
    got = Hd.memory_bytes()
    ud0, sd0 = Hd.solve_host(d.b[0])
    Hd.close()
    assert got <= est <= 1.05 * got + (1 << 20)
    cases = _mix()[:2]
    alone = [_alone(hz, p, cfg) for p, cfg in cases]
    srv = hz.Server(budget_bytes=8 << 30, max_active=3)
    td = srv.submit(d.k, d.b[0], d.h, bc="dirichlet", levels=3, precision="mixed")
    tickets = [srv.submit(p.k, p.b[0], p.h, **dict(cfg)) for p, cfg in cases]
    ud, sd, _ = srv.wait(td, timeout_s=600)
    assert np.array_equal(ud, ud0) and sd[0]["outer_iterations"] == sd0[0]["outer_iterations"]
    r = d.b[0] - apply_helmholtz(ud, d.k, d.h, bc=DIRICHLET)
    assert np.linalg.norm(r) / np.linalg.norm(d.b[0]) <= 1e-6
    for t, (u0, st0) in zip(tickets, alone):
        u, st, _ = srv.wait(t, timeout_s=600)
        assert np.array_equal(u, u0)
    srv.close()


def test_batching_merges_compatible_requests(hz):
    """With batching on, requests of one grid and configuration that are queued together run as
    one multi-instance solve.  A 513^2 request keeps the single worker busy while five 129^2
    requests of the same configuration (different wavenumber fields, 1-3 sources) queue up; they
    merge (the report counts merged solves).  Each merged result matches its solve alone to the
    solve tolerance (solution within 1e-5, outer iterations within one) and reaches 1e-6 with the
    oracle's operator.  A request with another level count is never merged with them."""
    big = mp.random_field(513, 5.0, seed=9, kh_max=0.3, levels=3, negdef_from_level=4, nsrc=4)
    smalls = [mp.random_field(129, 5.0, seed=20 + i, kh_max=0.25 + 0.02 * i, levels=3, negdef_from_level=4,
                              nsrc=1 + i % 3) for i in range(5)]
    other = mp.random_field(129, 5.0, seed=40, kh_max=0.3, levels=2, negdef_from_level=4)
    S = hz.Server(64 << 30, max_active=1, batch_rhs=16)

    def cfg(p):
        return dict(levels=p.levels, negdef_from_level=4, precision="mixed")

    tb = S.submit(big.k, big.b, big.h, **cfg(big))
    ts = [S.submit(p.k, p.b, p.h, **cfg(p)) for p in smalls]
    to = S.submit(other.k, other.b, other.h, **cfg(other))
    _, stb, _ = S.wait(tb)
    assert all(x["status"] == 0 for x in stb)
    outs = [S.wait(t) for t in ts]
    uo, sto, _ = S.wait(to)
    rep = S.report()
    assert rep["merged_solves"] >= 1 and rep["merged_requests"] >= 2, rep
    assert rep["completed"] == 7 and rep["failed"] == 0
    for p, (u, st, _) in zip(smalls, outs):
        H = hz.Helmholtz(dev(p.k), p.h, max_rhs=p.nrhs, **cfg(p))
        ua, sta = H.solve(dev(p.b), tol=1e-6)
        ua = ua.cpu().numpy()
        H.close()
        for r in range(p.nrhs):
            assert st[r]["status"] == 0
            rel = np.linalg.norm(p.b[r] - apply_helmholtz(u[r], p.k, p.h)) / np.linalg.norm(p.b[r])
            assert rel <= 1e-6
            assert rel2(u[r], ua[r]) <= 1e-5
            assert abs(st[r]["outer_iterations"] - sta[r]["outer_iterations"]) <= 1
    H = hz.Helmholtz(dev(other.k), other.h, **cfg(other))
    ua, _ = H.solve(dev(other.b), tol=1e-6)
    assert np.array_equal(uo, ua.cpu().numpy())
    H.close()
    S.close()
