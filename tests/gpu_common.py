"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle).

Tolerances (normwise, ||gpu - oracle||_inf / ||oracle||_inf unless stated):
* FP64 single operator apply: 1e-12 (the bar the method's FP64 path must meet).
* FP64 composite steps (V-cycle with a dense coarsest inverse, GMRES, the
  preconditioner, which chain up to ~10^2 applies): 1e-10.
* FP32 single apply: 2e-5.  Each output sums at most 4(2R+1) <= 28 rounded terms in
  the separable evaluation, so its error is <= 28 u sum|terms| with u = 2^-24; for random
  inputs sum|terms| / max|y| <= ~10, giving <= 1.7e-5.  The oracle is evaluated on the
  FP32-rounded inputs, so input rounding is not counted.
* FP32 composite (V-cycle, Z + A - v): 2e-4 = 10 stages x 2e-5.
* Converged solutions: 1e-5 relative 2-norm at a 1e-6 residual; outer iterations +-1.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

TOL64 = 1e-12
TOL64_COMPOSITE = 1e-10
TOL32 = 2e-5
TOL32_COMPOSITE = 2e-4


def cuda_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def hzlib():
    cuda_or_skip()
    from paper_2412_04980_gb300 import build
    build.build()
    import paper_2412_04980_gb300 as hz
    hz.lib()
    return hz


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel_inf(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rel2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def round32(a):
    return np.asarray(a, dtype=np.complex64).astype(np.complex128)


def round32r(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)
