"""GB300 matrix-free multilevel deflation Helmholtz solver: Python binding.

Thin ctypes layer over the C ABI in ``include/hz.h`` (``libhz.so``, built in-tree by
``paper_2412_04980_gb300.build``).  Functions keep the C names (``hz_setup``,
``hz_apply``, ``hz_precond``, ``hz_solve`` ...); :class:`Helmholtz` wraps a handle for
torch CUDA tensors.  Every numerical step runs in the library's CUDA kernels; this module
only marshals pointers, sizes and streams.  There is no CPU fallback: if the library is
missing, importing the symbols raises.

Vectors are complex tensors on the GPU, shaped (nrhs, ny, nx) or (ny, nx), C-contiguous
(x fastest), dtype complex128 or complex64 as each call states.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

__all__ = [
    "HZ_OK", "HZ_EINVAL", "HZ_ENOMEM", "HZ_ENOTCONV", "HZ_EBREAKDOWN", "HZ_ETIMEOUT", "HZ_ECUDA",
    "HZ_ENOTSUP", "HZ_PENDING", "HZ_BC_SOMMERFELD", "HZ_BC_DIRICHLET", "HZ_PREC_FP64", "HZ_PREC_MIXED",
    "HZ_C128", "HZ_C64", "HZ_OP_A", "HZ_OP_M", "HzGrid", "HzConfig", "HzStats", "HzError", "lib",
    "library_path", "Helmholtz", "HzRequest", "HzServerStats", "Server", "estimate_bytes",
]

HZ_OK, HZ_EINVAL, HZ_ENOMEM, HZ_ENOTCONV, HZ_EBREAKDOWN, HZ_ETIMEOUT, HZ_ECUDA, HZ_ENOTSUP, HZ_PENDING = range(9)
HZ_BC_SOMMERFELD, HZ_BC_DIRICHLET = 0, 1
HZ_PREC_FP64, HZ_PREC_MIXED = 0, 1
HZ_C128, HZ_C64 = 0, 1
HZ_OP_A, HZ_OP_M = 0, 1
HZ_MAX_LEVELS = 10
HZ_CSLP_GMRES, HZ_CSLP_BICGSTAB = 0, 1
HZ_SOLVE_INITIAL_GUESS = 1

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "libhz.so")


class HzGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("h", ctypes.c_double), ("bc", ctypes.c_int)]


class HzConfig(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int), ("precision", ctypes.c_int), ("beta1", ctypes.c_double),
        ("beta2", ctypes.c_double), ("restart", ctypes.c_int), ("max_outer", ctypes.c_int),
        ("l2_tol", ctypes.c_double), ("l2_maxit", ctypes.c_int), ("cslp_tol", ctypes.c_double),
        ("c_it", ctypes.c_double), ("coarsest_tol", ctypes.c_double), ("negdef_from_level", ctypes.c_int),
        ("mg_max_level", ctypes.c_int), ("mg_omega", ctypes.c_double), ("mg_nu1", ctypes.c_int),
        ("mg_nu2", ctypes.c_int), ("mg_coarsest_side", ctypes.c_int), ("max_rhs", ctypes.c_int),
        ("timeout_s", ctypes.c_double), ("device_gmres", ctypes.c_int), ("reorth_eta", ctypes.c_double),
        ("graphs", ctypes.c_int), ("autotune", ctypes.c_int), ("cycle_m", ctypes.c_int),
        ("level_tol", ctypes.c_double * HZ_MAX_LEVELS), ("cslp_solver", ctypes.c_int), ("sym_rows", ctypes.c_int),
        ("per_rhs_k", ctypes.c_int),
    ]


class HzStats(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int), ("outer_iterations", ctypes.c_int),
        ("level_iterations", ctypes.c_int * HZ_MAX_LEVELS), ("level_calls", ctypes.c_int * HZ_MAX_LEVELS),
        ("cslp_gmres_iterations", ctypes.c_int * HZ_MAX_LEVELS), ("true_relres", ctypes.c_double),
        ("est_relres", ctypes.c_double), ("ms", ctypes.c_double),
        ("cslp_gmres_reorth", ctypes.c_int * HZ_MAX_LEVELS),
    ]

    def as_dict(self) -> dict:
        return {
            "status": self.status, "outer_iterations": self.outer_iterations,
            "level_iterations": list(self.level_iterations), "level_calls": list(self.level_calls),
            "cslp_gmres_iterations": list(self.cslp_gmres_iterations), "true_relres": self.true_relres,
            "est_relres": self.est_relres, "ms": self.ms,
            "cslp_gmres_reorth": list(self.cslp_gmres_reorth),
        }


class HzRequest(ctypes.Structure):
    _fields_ = [
        ("grid", HzGrid), ("config", HzConfig), ("k_host", ctypes.c_void_p), ("b_host", ctypes.c_void_p),
        ("u_host", ctypes.c_void_p), ("stats_host", ctypes.c_void_p), ("nrhs", ctypes.c_int), ("tol", ctypes.c_double),
    ]


class HzServerStats(ctypes.Structure):
    _fields_ = [
        ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong), ("queued", ctypes.c_longlong),
        ("active", ctypes.c_int), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
        ("solves_per_s", ctypes.c_double), ("peak_bytes", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t),
        ("merged_solves", ctypes.c_longlong), ("merged_requests", ctypes.c_longlong),
    ]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class HzError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


_P, _I, _D, _U = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint
_SIGS = {
    "hz_config_init": (_I, [ctypes.POINTER(HzConfig)]),
    "hz_setup": (_I, [ctypes.POINTER(HzGrid), _P, ctypes.POINTER(HzConfig), _P, ctypes.POINTER(_P)]),
    "hz_destroy": (_I, [_P]),
    "hz_memory_bytes": (_I, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "hz_apply": (_I, [_P, _P, _P, _I]),
    "hz_precond": (_I, [_P, _P, _P, _I]),
    "hz_solve": (_I, [_P, _P, _P, _I, _D, _U, ctypes.POINTER(HzStats)]),
    "hz_solve_host": (_I, [_P, _P, _P, _I, _D, _U, ctypes.POINTER(HzStats)]),
    "hz_level_size": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "hz_level_gmres_form": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "hz_level_apply": (_I, [_P, _I, _I, _I, _P, _P, _I]),
    "hz_level_jacobi": (_I, [_P, _I, _I, _P, _P, _P, _I]),
    "hz_defl_restrict": (_I, [_P, _I, _I, _P, _P, _I]),
    "hz_defl_prolong": (_I, [_P, _I, _I, _P, _P, _I]),
    "hz_defl_prolong_residual": (_I, [_P, _I, _I, _P, _P, _P, _P, _I]),
    "hz_mg_vcycle": (_I, [_P, _I, _I, _P, _P, _I]),
    "hz_mg_size": (_I, [_P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "hz_cslp_gmres": (_I, [_P, _I, _I, _P, _P, _I, ctypes.POINTER(_I)]),
    "hz_cslp_bicgstab": (_I, [_P, _I, _I, _P, _P, _I, ctypes.POINTER(_I)]),
    "hz_strerror": (ctypes.c_char_p, [_I]),
    "hz_last_error": (ctypes.c_char_p, []),
    "hz_profile_enable": (_I, [_P, _I, _I]),
    "hz_profile_read": (_I, [_P, _I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D),
                             ctypes.POINTER(_D)]),
    "hz_kernel_family_name": (ctypes.c_char_p, [_I]),
    "hz_kernel_family_count": (_I, []),
    "hz_launch_count": (_I, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "hz_gmres_device_time": (_I, [_P, _I, _I, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_D),
                                  ctypes.POINTER(_D)]),
    "hz_true_residual_noalloc": (_I, [_P, _P, _P, _I, _P]),
    "hz_estimate_bytes": (_I, [ctypes.POINTER(HzGrid), ctypes.POINTER(HzConfig), ctypes.POINTER(ctypes.c_size_t)]),
    "hz_server_create": (_I, [ctypes.c_size_t, _I, ctypes.POINTER(_P)]),
    "hz_submit": (_I, [_P, ctypes.POINTER(HzRequest), ctypes.POINTER(ctypes.c_uint64)]),
    "hz_poll": (_I, [_P, ctypes.c_uint64, ctypes.POINTER(_D)]),
    "hz_wait": (_I, [_P, ctypes.c_uint64, _D, ctypes.POINTER(_D)]),
    "hz_server_report": (_I, [_P, ctypes.POINTER(HzServerStats)]),
    "hz_server_set_batching": (_I, [_P, _I]),
    "hz_server_destroy": (_I, [_P]),
}

_LIB = None


def lib() -> ctypes.CDLL:
    """Load ``libhz.so`` (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def _check(status: int, where: str):
    if status != HZ_OK:
        L = lib()
        raise HzError(status, where, f"{L.hz_strerror(status).decode()}; {L.hz_last_error().decode()}")


def __getattr__(name):
    # hz_* names resolve to the C functions of the loaded library
    if name.startswith("hz_") and name in _SIGS:
        return getattr(lib(), name)
    raise AttributeError(name)


def config(**kw) -> HzConfig:
    """An HzConfig with the paper's defaults (hz_config_init) updated by keyword fields."""
    c = HzConfig()
    _check(lib().hz_config_init(ctypes.byref(c)), "hz_config_init")
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        if k == "cslp_solver" and isinstance(v, str):
            v = {"gmres": HZ_CSLP_GMRES, "bicgstab": HZ_CSLP_BICGSTAB}[v]
        if k == "level_tol":
            # {level: tolerance} for levels 3 .. levels-1 (entry level-1 of the C array)
            arr = (ctypes.c_double * HZ_MAX_LEVELS)()
            for lev, tol in dict(v).items():
                if not 1 <= int(lev) <= HZ_MAX_LEVELS:
                    raise ValueError(f"level_tol: level {lev} out of range")
                arr[int(lev) - 1] = float(tol)
            v = arr
        setattr(c, k, v)
    return c


def _ptr(t) -> int:
    return t.data_ptr()


@dataclass
class SolveResult:
    stats: list


class Helmholtz:
    """One Helmholtz instance (grid, wavenumber field, configuration) on the current device.

    ``k`` is a real float64 CUDA tensor of shape (ny, nx), or (I, ny, nx) for a multi-instance
    batch: I problems on the same grid, right-hand side r of every call taking field r
    (``per_rhs_k``; ``max_rhs`` becomes I).  Keyword arguments set :class:`HzConfig` fields
    (``levels``, ``precision`` ('fp64' / 'mixed'), ``max_rhs`` ...).
    """

    def __init__(self, k, h: float, bc: str = "sommerfeld", stream=None, **cfg):
        import torch
        if not (k.is_cuda and k.dtype == torch.float64 and k.dim() in (2, 3) and k.is_contiguous()):
            raise ValueError("k must be a contiguous (ny, nx) or (instances, ny, nx) float64 CUDA tensor")
        self.ny, self.nx = int(k.shape[-2]), int(k.shape[-1])
        if k.dim() == 3:
            if cfg.get("max_rhs", k.shape[0]) != k.shape[0]:
                raise ValueError("a multi-instance batch takes max_rhs = number of wavenumber fields")
            cfg["max_rhs"] = int(k.shape[0])
            cfg["per_rhs_k"] = 1
        prec = cfg.pop("precision", "fp64")
        cfg["precision"] = {"fp64": HZ_PREC_FP64, "mixed": HZ_PREC_MIXED}.get(prec, prec)
        self.cfg = config(**cfg)
        self.grid = HzGrid(self.nx, self.ny, float(h), HZ_BC_SOMMERFELD if bc == "sommerfeld" else HZ_BC_DIRICHLET)
        self.stream = stream if stream is not None else torch.cuda.current_stream(k.device)
        self._h = ctypes.c_void_p()
        _check(lib().hz_setup(ctypes.byref(self.grid), _ptr(k), ctypes.byref(self.cfg),
                              ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(self._h)), "hz_setup")
        self.device = k.device

    def close(self):
        if self._h:
            lib().hz_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- helpers ---------------------------------------------------------------------
    @staticmethod
    def _nrhs(t, ny, nx):
        if not t.is_contiguous():
            raise ValueError("vectors must be contiguous")
        if t.dim() == 2:
            n = 1
        elif t.dim() == 3:
            n = int(t.shape[0])
        else:
            raise ValueError("vectors must be (ny, nx) or (nrhs, ny, nx)")
        if tuple(t.shape[-2:]) != (ny, nx):
            raise ValueError(f"vector shape {tuple(t.shape)} does not match grid ({ny}, {nx})")
        return n

    def level_size(self, level: int):
        nx, ny = ctypes.c_int(), ctypes.c_int()
        _check(lib().hz_level_size(self._h, level, ctypes.byref(nx), ctypes.byref(ny)), "hz_level_size")
        return ny.value, nx.value

    def gmres_form(self, level: int) -> dict:
        """hz_level_gmres_form: {'form': 'none'|'slice'|'tile'|'cluster', 'ctas': int, 'cluster': int}."""
        f, c, cl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().hz_level_gmres_form(self._h, level, ctypes.byref(f), ctypes.byref(c), ctypes.byref(cl)),
               "hz_level_gmres_form")
        return {"form": ("none", "slice", "tile", "cluster")[f.value], "ctas": c.value, "cluster": cl.value}

    def mg_size(self, level: int, mg_level: int):
        nx, ny = ctypes.c_int(), ctypes.c_int()
        _check(lib().hz_mg_size(self._h, level, mg_level, ctypes.byref(nx), ctypes.byref(ny)), "hz_mg_size")
        return ny.value, nx.value

    def memory_bytes(self) -> int:
        b = ctypes.c_size_t()
        _check(lib().hz_memory_bytes(self._h, ctypes.byref(b)), "hz_memory_bytes")
        return b.value

    @staticmethod
    def _dt(t):
        import torch
        if t.dtype == torch.complex128:
            return HZ_C128
        if t.dtype == torch.complex64:
            return HZ_C64
        raise ValueError("complex128 or complex64 expected")

    # -- the hot-path calls ------------------------------------------------------------
    def apply(self, x, y=None):
        """y = A_h x (complex128)."""
        import torch
        n = self._nrhs(x, self.ny, self.nx)
        y = torch.empty_like(x) if y is None else y
        _check(lib().hz_apply(self._h, _ptr(x), _ptr(y), n), "hz_apply")
        return y

    def precond(self, v, x=None):
        """x = P v, the A-DEF1 multilevel preconditioner (complex128)."""
        import torch
        n = self._nrhs(v, self.ny, self.nx)
        x = torch.empty_like(v) if x is None else x
        _check(lib().hz_precond(self._h, _ptr(v), _ptr(x), n), "hz_precond")
        return x

    def solve(self, b, u=None, tol: float = 1e-6, initial_guess: bool = False, check: bool = True):
        """Solve A_h u = b (complex128); returns (u, [stats dict per rhs])."""
        import torch
        n = self._nrhs(b, self.ny, self.nx)
        u = torch.empty_like(b) if u is None else u
        stats = (HzStats * n)()
        st = lib().hz_solve(self._h, _ptr(b), _ptr(u), n, float(tol),
                            HZ_SOLVE_INITIAL_GUESS if initial_guess else 0, stats)
        if check and st not in (HZ_OK,):
            _check(st, "hz_solve")
        return u, [s.as_dict() for s in stats]

    def solve_host(self, b_np, tol: float = 1e-6):
        """hz_solve_host on numpy complex128 arrays; returns (u_np, stats)."""
        import numpy as np
        b = np.ascontiguousarray(b_np, dtype=np.complex128)
        n = 1 if b.ndim == 2 else b.shape[0]
        u = np.empty_like(b)
        stats = (HzStats * n)()
        _check(lib().hz_solve_host(self._h, b.ctypes.data, u.ctypes.data, n, float(tol), 0, stats), "hz_solve_host")
        return u, [s.as_dict() for s in stats]

    # -- building blocks -----------------------------------------------------------------
    def level_apply(self, level: int, x, op: str = "A", y=None):
        import torch
        ny, nx = self.level_size(level)
        n = self._nrhs(x, ny, nx)
        y = torch.empty_like(x) if y is None else y
        _check(lib().hz_level_apply(self._h, level, HZ_OP_A if op == "A" else HZ_OP_M, self._dt(x), _ptr(x),
                                    _ptr(y), n), "hz_level_apply")
        return y

    def level_jacobi(self, level: int, u, f, out=None):
        import torch
        ny, nx = self.level_size(level)
        n = self._nrhs(u, ny, nx)
        out = torch.empty_like(u) if out is None else out
        _check(lib().hz_level_jacobi(self._h, level, self._dt(u), _ptr(u), _ptr(f), _ptr(out), n),
               "hz_level_jacobi")
        return out

    def defl_restrict(self, level: int, v):
        import torch
        ny, nx = self.level_size(level)
        n = self._nrhs(v, ny, nx)
        cy, cx = self.level_size(level + 1)
        out = torch.empty((n, cy, cx) if v.dim() == 3 else (cy, cx), dtype=v.dtype, device=v.device)
        _check(lib().hz_defl_restrict(self._h, level, self._dt(v), _ptr(v), _ptr(out), n), "hz_defl_restrict")
        return out

    def defl_prolong(self, level: int, w):
        import torch
        ny, nx = self.level_size(level)
        cy, cx = self.level_size(level + 1)
        n = self._nrhs(w, cy, cx)
        out = torch.empty((n, ny, nx) if w.dim() == 3 else (ny, nx), dtype=w.dtype, device=w.device)
        _check(lib().hz_defl_prolong(self._h, level, self._dt(w), _ptr(w), _ptr(out), n), "hz_defl_prolong")
        return out

    def defl_prolong_residual(self, level: int, vtil, v):
        import torch
        ny, nx = self.level_size(level)
        n = self._nrhs(v, ny, nx)
        t = torch.empty_like(v)
        r = torch.empty_like(v)
        _check(lib().hz_defl_prolong_residual(self._h, level, self._dt(v), _ptr(vtil), _ptr(v), _ptr(t), _ptr(r),
                                              n), "hz_defl_prolong_residual")
        return t, r

    def mg_vcycle(self, level: int, f):
        import torch
        ny, nx = self.level_size(level)
        n = self._nrhs(f, ny, nx)
        u = torch.empty_like(f)
        _check(lib().hz_mg_vcycle(self._h, level, self._dt(f), _ptr(f), _ptr(u), n), "hz_mg_vcycle")
        return u

    def cslp_gmres(self, level: int, b):
        import torch
        ny, nx = self.level_size(level)
        n = self._nrhs(b, ny, nx)
        x = torch.empty_like(b)
        its = (ctypes.c_int * n)()
        _check(lib().hz_cslp_gmres(self._h, level, self._dt(b), _ptr(b), _ptr(x), n, its), "hz_cslp_gmres")
        return x, list(its)

    def cslp_bicgstab(self, level: int, b):
        """CSLP inverse by Bi-CGSTAB on level ``level`` (handle built with cslp_solver="bicgstab")."""
        import torch
        ny, nx = self.level_size(level)
        n = self._nrhs(b, ny, nx)
        x = torch.empty_like(b)
        its = (ctypes.c_int * n)()
        _check(lib().hz_cslp_bicgstab(self._h, level, self._dt(b), _ptr(b), _ptr(x), n, its), "hz_cslp_bicgstab")
        return x, list(its)

    def launch_count(self) -> int:
        n = ctypes.c_longlong()
        _check(lib().hz_launch_count(self._h, ctypes.byref(n)), "hz_launch_count")
        return n.value

    def gmres_device_time(self, level: int = 0, reset: bool = False):
        """hz_gmres_device_time: (launches, ms, algorithmic bytes) of the self-timed persistent
        GMRES launches folded in by the solves since the last reset (level 0: all levels)."""
        n, ms, by = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        _check(lib().hz_gmres_device_time(self._h, level, 1 if reset else 0, ctypes.byref(n), ctypes.byref(ms),
                                          ctypes.byref(by)), "hz_gmres_device_time")
        return n.value, ms.value, by.value

    # -- per-kernel timing ----------------------------------------------------------------
    @staticmethod
    def kernel_families():
        L = lib()
        return [L.hz_kernel_family_name(i).decode() for i in range(L.hz_kernel_family_count())]

    def profile_enable(self, family: int, on: bool = True):
        _check(lib().hz_profile_enable(self._h, family, 1 if on else 0), "hz_profile_enable")

    def profile_read(self, family: int):
        n, ms, by = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double()
        _check(lib().hz_profile_read(self._h, family, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)),
               "hz_profile_read")
        return n.value, ms.value, by.value


def _precision(cfg: dict) -> dict:
    prec = cfg.pop("precision", "fp64")
    cfg["precision"] = {"fp64": HZ_PREC_FP64, "mixed": HZ_PREC_MIXED}.get(prec, prec)
    return cfg


def estimate_bytes(nx: int, ny: int, h: float, bc: int = HZ_BC_SOMMERFELD, **cfg) -> int:
    """hz_estimate_bytes: device bytes hz_setup allocates for this grid and configuration."""
    out = ctypes.c_size_t()
    g = HzGrid(nx, ny, float(h), bc)
    c = config(**_precision(dict(cfg)))
    _check(lib().hz_estimate_bytes(ctypes.byref(g), ctypes.byref(c), ctypes.byref(out)), "hz_estimate_bytes")
    return out.value


class Server:
    """Concurrent solves on the current device (hz_server_*): ``submit`` copies k and b and
    returns a ticket; ``wait`` blocks until the solution is in the numpy array it returns.
    ``batch_rhs`` > 1 merges compatible queued requests into multi-instance solves of up to that
    many right-hand sides (hz_server_set_batching)."""

    def __init__(self, budget_bytes: int, max_active: int = 2, batch_rhs: int = 0):
        self._s = ctypes.c_void_p()
        _check(lib().hz_server_create(int(budget_bytes), int(max_active), ctypes.byref(self._s)), "hz_server_create")
        if batch_rhs:
            _check(lib().hz_server_set_batching(self._s, int(batch_rhs)), "hz_server_set_batching")
        self._live = {}

    def submit(self, k_np, b_np, h: float, tol: float = 1e-6, bc: str = "sommerfeld", **cfg) -> int:
        import numpy as np
        k = np.ascontiguousarray(k_np, dtype=np.float64)
        b = np.ascontiguousarray(b_np, dtype=np.complex128)
        ny, nx = k.shape[-2:]
        nrhs = 1 if b.ndim == 2 else b.shape[0]
        if b.shape[-2:] != (ny, nx):
            raise ValueError("b must have k's grid shape (optionally with a leading rhs axis)")
        cfg = _precision(dict(cfg))
        if k.ndim == 3:  # multi-instance request: right-hand side r takes wavenumber field r
            if nrhs > k.shape[0] or cfg.get("max_rhs", k.shape[0]) != k.shape[0]:
                raise ValueError("a multi-instance request takes max_rhs = fields >= nrhs")
            cfg["max_rhs"] = int(k.shape[0])
            cfg["per_rhs_k"] = 1
        cfg.setdefault("max_rhs", nrhs)
        u = np.empty_like(b)
        stats = (HzStats * nrhs)()
        grid = HzGrid(nx, ny, float(h), HZ_BC_SOMMERFELD if bc == "sommerfeld" else HZ_BC_DIRICHLET)
        req = HzRequest(grid, config(**cfg), k.ctypes.data, b.ctypes.data,
                        u.ctypes.data, ctypes.addressof(stats), nrhs, float(tol))
        t = ctypes.c_uint64()
        _check(lib().hz_submit(self._s, ctypes.byref(req), ctypes.byref(t)), "hz_submit")
        self._live[t.value] = (u, stats)
        return t.value

    def poll(self, ticket: int):
        """None while pending, else (status, latency_ms)."""
        ms = ctypes.c_double()
        st = lib().hz_poll(self._s, ticket, ctypes.byref(ms))
        return None if st == HZ_PENDING else (st, ms.value)

    def wait(self, ticket: int, timeout_s: float = 600.0, check: bool = True):
        """(u, stats, latency_ms) of a finished request; raises HzError on failure if check."""
        ms = ctypes.c_double()
        st = lib().hz_wait(self._s, ticket, float(timeout_s), ctypes.byref(ms))
        if st == HZ_ETIMEOUT and self.poll(ticket) is None:   # still running (not the solve's own timeout)
            _check(st, "hz_wait")
        u, stats = self._live.pop(ticket)
        if check:
            _check(st, "server request")
        return u, [x.as_dict() for x in stats], ms.value

    def report(self) -> dict:
        out = HzServerStats()
        _check(lib().hz_server_report(self._s, ctypes.byref(out)), "hz_server_report")
        return out.as_dict()

    def close(self):
        if self._s:
            lib().hz_server_destroy(self._s)
            self._s = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
