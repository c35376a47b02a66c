"""hz_true_residual_noalloc: the relative residual without any device allocation.

Some callers cannot call cudaMalloc where they check a solution (a plugin whose host
application owns every device allocation, a loop that must not enter the allocator).
The allocation-free entry point keeps its reduction partials in a static device array;
its result must match the true residual that hz_solve reports through its allocated
workspace, call after call.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import model_problems as mp
from gpu_common import TOL64, dev, host, hzlib, torch

pytestmark = pytest.mark.gpu


def _noalloc(hz, H, b, u, nrhs):
    out = torch.full((nrhs,), float("nan"), dtype=torch.float64, device="cuda")
    st = hz.lib().hz_true_residual_noalloc(H._h, b.data_ptr(), u.data_ptr(), nrhs, out.data_ptr())
    assert st == hz.HZ_OK, hz.lib().hz_last_error().decode()
    return host(out)


def test_noalloc_residual_matches_solver_report():
    hz = hzlib()
    p = mp.random_field(129, 5.0, seed=3, kh_max=0.3, levels=3, negdef_from_level=4, nsrc=3)
    H = hz.Helmholtz(dev(p.k), p.h, levels=3, negdef_from_level=4, precision="mixed", max_rhs=3)
    b = dev(p.b)
    u, stats = H.solve(b, tol=1e-6)
    want = np.array([s["true_relres"] for s in stats])
    assert np.all(want <= 1e-6) and np.all(want > 0)
    first = _noalloc(hz, H, b, u, 3)
    second = _noalloc(hz, H, b, u, 3)                      # two calls in a row share the array
    # both values are ||b - A u|| / ||b||; the residual b - A u carries rounding relative to
    # ||b|| (not to the small residual), so they agree to TOL64 in units of ||b||
    for got in (first, second):
        assert np.all(np.abs(got - want) <= TOL64), (got, want)
    # a different input through the same static array, then the first input again
    z = torch.zeros_like(u)
    np.testing.assert_allclose(_noalloc(hz, H, b, z, 3), 1.0, rtol=TOL64)
    assert np.all(np.abs(_noalloc(hz, H, b, u, 3) - want) <= TOL64)


def test_noalloc_rejects_oversized_batch():
    hz = hzlib()
    p = mp.mp1b(16, 5.0)
    H = hz.Helmholtz(dev(p.k), p.h, levels=1)
    b = dev(np.zeros((p.ny, p.nx), complex))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    L = hz.lib()
    assert L.hz_true_residual_noalloc(H._h, b.data_ptr(), b.data_ptr(), 65, out.data_ptr()) == hz.HZ_EINVAL
    assert L.hz_true_residual_noalloc(H._h, b.data_ptr(), b.data_ptr(), 0, out.data_ptr()) == hz.HZ_EINVAL
    assert L.hz_true_residual_noalloc(H._h, None, b.data_ptr(), 1, out.data_ptr()) == hz.HZ_EINVAL
