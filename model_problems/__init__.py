"""Seeded synthetic inputs for the 2-D heterogeneous Helmholtz model problems.

This module produces *inputs only*: wavenumber fields k(x, y) = 2*pi*f / c(x, y)
(Section 2, the problem statement), point-source right-hand sides and random
test vectors.  It holds none of the solver's arithmetic (no stencil, transfer,
preconditioner or Krylov step), so both the CPU oracle and the CUDA path can
consume it without sharing any of the method's code.

Grids are vertex-centred (Section 2.1): node (i, j), 0-based, sits at
x_i = x0 + i*h, y_j = y0 + j*h.  Arrays are indexed [j, i] (row = y, x fastest).
All random draws use NumPy's PCG64 generator with an explicit seed.

Model problems (the paper's Section 2; geometry that the paper shows only in a
figure is replaced by the synthetic choices stated below):

* ``mp1b``      constant k on the unit square, Sommerfeld boundary, point
                source at the centre (MP-1b).
* ``wedge``     three layers separated by two straight dipping interfaces
                (synthetic stand-in for the Wedge figure): c = 2000 m/s above
                interface 1, 1500 m/s between, 3000 m/s below.
* ``random``    layered background rising 1500 -> 4500 m/s in 8 flat steps plus
                a Gaussian-filtered white-noise field (correlation length
                200 m, sigma 400 m/s), clipped to [1500, 5500] m/s; stands in
                for the Marmousi model, which is not available here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Problem",
    "mp1b",
    "wedge",
    "wedge_square",
    "random_field",
    "random_instances",
    "point_source",
    "random_complex",
    "random_k",
    "named",
]


@dataclass
class Problem:
    """One Helmholtz instance: grid, wavenumber field and right-hand sides."""

    name: str
    nx: int
    ny: int
    h: float
    k: np.ndarray                  # (ny, nx) float64, k = 2*pi*f/c; (nrhs, ny, nx) for a batch of
                                   # instances, right-hand side r with field r
    b: np.ndarray                  # (nrhs, ny, nx) complex128
    levels: int
    negdef_from_level: int         # first level treated as negative definite (0 = none)
    meta: dict = field(default_factory=dict)

    @property
    def nrhs(self) -> int:
        return int(self.b.shape[0])


def point_source(nx: int, ny: int, i: int, j: int, h: float) -> np.ndarray:
    """Discrete unit point source: 1/h^2 at node (i, j), zero elsewhere."""
    b = np.zeros((ny, nx), dtype=np.complex128)
    b[j, i] = 1.0 / (h * h)
    return b


def nearest_node(coord: float, origin: float, h: float, n: int) -> int:
    """Nearest grid index to a coordinate; ties go to the lower index."""
    t = (coord - origin) / h
    lo = math.floor(t)
    idx = lo if (t - lo) <= 0.5 else lo + 1
    return int(min(max(idx, 0), n - 1))


def mp1b(n_interior: int = 128, k: float = 20.0) -> Problem:
    """Constant wavenumber on [0,1]^2 with (n_interior+1)^2 nodes, h = 1/n_interior,
    Sommerfeld boundary, unit point source at (0.5, 0.5); two deflation levels."""
    n = n_interior + 1
    h = 1.0 / n_interior
    kk = np.full((n, n), float(k))
    c = n // 2
    b = point_source(n, n, c, c, h)[None]
    return Problem("mp1b", n, n, h, kk, b, levels=2, negdef_from_level=0,
                   meta={"k": k, "source": (c, c)})


def mp1a(n_interior: int = 128, k: float = 20.0, levels: int = 2) -> Problem:
    """Constant wavenumber on [0,1]^2 with homogeneous Dirichlet boundary (MP-1a): the
    (n_interior-1)^2 interior nodes are the unknowns, h = 1/n_interior, unit point source at
    (0.5, 0.5) (interior index n_interior/2 - 1)."""
    n = n_interior - 1
    h = 1.0 / n_interior
    kk = np.full((n, n), float(k))
    c = n_interior // 2 - 1
    b = point_source(n, n, c, c, h)[None]
    return Problem("mp1a", n, n, h, kk, b, levels=levels, negdef_from_level=0,
                   meta={"k": k, "source": (c, c), "bc": "dirichlet"})


def _wedge_velocity(x: np.ndarray, y: np.ndarray, width: float) -> np.ndarray:
    """Three-layer wedge velocity.  Interface 1 runs from (0, -350) to (600, -150),
    interface 2 from (0, -700) to (600, -550); both are extended linearly beyond
    x = 600 when the domain is wider."""
    y1 = -350.0 + (200.0 / 600.0) * x
    y2 = -700.0 + (150.0 / 600.0) * x
    c = np.where(y >= y1, 2000.0, np.where(y >= y2, 1500.0, 3000.0))
    return c


def wedge(nx: int = 289, ny: int = 481, freq: float = 20.0, levels: int = 4,
          negdef_from_level: int = 5) -> Problem:
    """Wedge problem on [0,600] x [-1000,0] with nx*ny nodes, Sommerfeld boundary,
    source 10 m below the top centre (300, -10)."""
    h = 600.0 / (nx - 1)
    if abs((ny - 1) * h - 1000.0) > 1e-9 * 1000.0:
        raise ValueError("wedge grid must have a uniform spacing on 600 x 1000 m")
    x = np.arange(nx) * h
    y = -1000.0 + np.arange(ny) * h
    X, Y = np.meshgrid(x, y)
    c = _wedge_velocity(X, Y, 600.0)
    k = 2.0 * math.pi * freq / c
    i = nearest_node(300.0, 0.0, h, nx)
    j = nearest_node(-10.0, -1000.0, h, ny)
    b = point_source(nx, ny, i, j, h)[None]
    return Problem("wedge", nx, ny, h, k, b, levels=levels, negdef_from_level=negdef_from_level,
                   meta={"freq": freq, "source": (i, j), "kh_max": float(k.max() * h)})


def wedge_square(n: int = 2049, nrhs: int = 64, kh_max: float = 0.3, levels: int = 6,
                 negdef_from_level: int = 4) -> Problem:
    """Square 1000 x 1000 m version of the wedge (interfaces extended linearly in x),
    n x n nodes, frequency set so that max(k)*h = kh_max, nrhs point sources on the
    top row at nodes round((s + 0.5) * (n - 1) / nrhs)."""
    h = 1000.0 / (n - 1)
    x = np.arange(n) * h
    y = -1000.0 + np.arange(n) * h
    X, Y = np.meshgrid(x, y)
    c = _wedge_velocity(X, Y, 1000.0)
    freq = kh_max * float(c.min()) / (2.0 * math.pi * h)
    k = 2.0 * math.pi * freq / c
    b = np.zeros((nrhs, n, n), dtype=np.complex128)
    for s in range(nrhs):
        i = int(round((s + 0.5) * (n - 1) / nrhs))
        b[s] = point_source(n, n, i, n - 1, h)
    return Problem("wedge_square", n, n, h, k, b, levels=levels,
                   negdef_from_level=negdef_from_level, meta={"freq": freq})


def random_velocity(n: int, h: float, seed: int = 3, corr_len: float = 200.0,
                    sigma: float = 400.0) -> np.ndarray:
    """Layered background plus a Gaussian random field, clipped to [1500, 5500] m/s.

    The background rises linearly from 1500 m/s at the top row to 4500 m/s at the
    bottom in 8 equal flat steps.  The random part is PCG64 white noise filtered in
    Fourier space by exp(-(kappa * corr_len)^2 / 2) and rescaled to std ``sigma``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.standard_normal((n, n))
    kap = 2.0 * math.pi * np.fft.fftfreq(n, d=h)
    KX, KY = np.meshgrid(kap, kap)
    filt = np.exp(-0.5 * (KX * KX + KY * KY) * corr_len * corr_len)
    g = np.real(np.fft.ifft2(np.fft.fft2(noise) * filt))
    g *= sigma / max(float(g.std()), 1e-300)
    depth_frac = (n - 1 - np.arange(n)) / max(n - 1, 1)           # 0 at top row, 1 at bottom
    step = np.minimum(np.floor(depth_frac * 8.0), 7.0)
    c_layer = 1500.0 + step * (3000.0 / 7.0)
    c = c_layer[:, None] + g
    return np.clip(c, 1500.0, 5500.0)


def random_field(n: int = 4097, h: float = 5.0, seed: int = 3, kh_max: float = 0.3,
                 levels: int = 6, negdef_from_level: int = 4, nsrc: int = 1) -> Problem:
    """Seeded random-velocity model on an n x n grid with spacing h; frequency set so
    that max(k)*h = kh_max; ``nsrc`` point sources on the top row (one per RHS),
    the first at the top-centre node."""
    c = random_velocity(n, h, seed)
    freq = kh_max * float(c.min()) / (2.0 * math.pi * h)
    k = 2.0 * math.pi * freq / c
    b = np.zeros((nsrc, n, n), dtype=np.complex128)
    for s in range(nsrc):
        i = (n - 1) // 2 if s == 0 else int(round((s + 0.5) * (n - 1) / nsrc))
        b[s] = point_source(n, n, i, n - 1, h)
    return Problem("random", n, n, h, k, b, levels=levels, negdef_from_level=negdef_from_level,
                   meta={"freq": freq, "seed": seed})


def random_instances(n: int = 1025, count: int = 16, h: float = 5.0, levels: int = 4,
                     negdef_from_level: int = 4, seed0: int = 100) -> Problem:
    """``count`` independent random-velocity problems on one n x n grid (a multi-instance
    batch): instance r draws its velocity model with seed seed0 + r, takes k_max h evenly from
    0.2 to 0.3 and has one point source on the top row, moving from the centre to the right
    with r; k has shape (count, n, n) and b (count, n, n)."""
    ks, bs = [], []
    for r in range(count):
        c = random_velocity(n, h, seed0 + r)
        kh = 0.2 + 0.1 * r / max(count - 1, 1)
        freq = kh * float(c.min()) / (2.0 * math.pi * h)
        ks.append(2.0 * math.pi * freq / c)
        i = (n - 1) // 2 + r * ((n - 1) // 2) // max(count, 1)
        bs.append(point_source(n, n, i, n - 1, h))
    return Problem("random_instances", n, n, h, np.stack(ks), np.stack(bs), levels=levels,
                   negdef_from_level=negdef_from_level, meta={"instances": count, "seed0": seed0})


def random_complex(shape, seed: int) -> np.ndarray:
    """Complex128 array with independent standard-normal real and imaginary parts."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def random_k(ny: int, nx: int, seed: int, kmin: float = 5.0, kmax: float = 40.0) -> np.ndarray:
    """Positive wavenumber field with uniform random entries in [kmin, kmax]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return kmin + (kmax - kmin) * rng.random((ny, nx))


def named(name: str) -> Problem:
    """The workloads used by the tests and the benchmark, by name."""
    if name == "mp1b_129":
        return mp1b(128, 20.0)
    if name == "wedge_289x481":
        return wedge(289, 481, 20.0, levels=4, negdef_from_level=5)
    if name == "random_4097":
        return random_field(4097, 5.0, seed=3, levels=6, negdef_from_level=4)
    if name == "random_1025":
        return random_field(1025, 5.0, seed=3, levels=4, negdef_from_level=4)
    if name == "random_513":
        return random_field(513, 5.0, seed=3, levels=3, negdef_from_level=4)
    if name == "wedge_2049_64rhs":
        return wedge_square(2049, 64)
    if name == "random_1025_16inst":
        return random_instances(1025, 16, levels=4, negdef_from_level=4)
    if name == "mp1a_1023":
        # MP-1a at k h = 0.3125 (Section 4.3.1's resolution): k = 320 on 1023^2 interior unknowns;
        # levels 1023, 511, 255, 127, the fourth negative definite at this k h
        p = mp1a(1024, 320.0, levels=4)
        p.negdef_from_level = 4
        return p
    raise KeyError(name)
