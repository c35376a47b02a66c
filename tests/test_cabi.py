"""Host-side checks of the C ABI (no GPU): the library builds, loads and exports every
function include/hz.h declares; argument validation answers before any device work."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hz.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_]+\*?\s+\*?(hz_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def L():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2412_04980_gb300 import build
    build.build()
    import paper_2412_04980_gb300 as hz
    return hz.lib()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for required in ("hz_setup", "hz_apply", "hz_precond", "hz_solve", "hz_destroy", "hz_strerror"):
        assert required in names
    assert len(names) >= 20


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_config_defaults(L):
    import paper_2412_04980_gb300 as hz
    c = hz.config()
    assert (c.beta1, c.beta2, c.restart, c.l2_tol, c.cslp_tol, c.c_it, c.mg_omega) == (1.0, 0.5, 30, 0.3, 0.1, 6.0, 0.8)
    assert c.mg_max_level == 2 and c.mg_nu1 == 1 and c.mg_nu2 == 1 and c.max_rhs == 1


def test_strerror_names_every_status(L):
    for s in range(9):
        assert L.hz_strerror(s).decode().startswith("HZ_")


def test_setup_rejects_bad_arguments_before_device_work(L):
    import paper_2412_04980_gb300 as hz
    h = ctypes.c_void_p()
    cfg = hz.config(levels=2)
    bad_grid = hz.HzGrid(2, 9, 0.1, 0)
    assert L.hz_setup(ctypes.byref(bad_grid), ctypes.c_void_p(1), ctypes.byref(cfg), None, ctypes.byref(h)) == hz.HZ_EINVAL
    even = hz.HzGrid(10, 9, 0.1, 0)
    assert L.hz_setup(ctypes.byref(even), ctypes.c_void_p(1), ctypes.byref(cfg), None, ctypes.byref(h)) == hz.HZ_EINVAL
    neg_h = hz.HzGrid(9, 9, -1.0, 0)
    assert L.hz_setup(ctypes.byref(neg_h), ctypes.c_void_p(1), ctypes.byref(cfg), None, ctypes.byref(h)) == hz.HZ_EINVAL
    cfg_bad = hz.config(levels=0)
    ok = hz.HzGrid(9, 9, 0.1, 0)
    assert L.hz_setup(ctypes.byref(ok), ctypes.c_void_p(1), ctypes.byref(cfg_bad), None, ctypes.byref(h)) == hz.HZ_EINVAL
    assert L.hz_setup(None, None, None, None, None) == hz.HZ_EINVAL
    assert L.hz_apply(None, None, None, 1) == hz.HZ_EINVAL
    assert "null" in L.hz_last_error().decode()


def test_kernel_families(L):
    n = L.hz_kernel_family_count()
    names = [L.hz_kernel_family_name(i).decode() for i in range(n)]
    assert "mg_down" in names and "level_op" in names


def test_estimate_bytes_host_only(L):
    """hz_estimate_bytes needs no device: it grows with the grid and with max_rhs, and the
    one-rhs basis of the cooperative-grid GMRES (device_gmres = 2) makes multi-rhs estimates
    smaller there than with per-rhs workspace."""
    import paper_2412_04980_gb300 as hz
    e = lambda n, **c: hz.estimate_bytes(n, n, 5.0, **c)
    small, big = e(129, levels=2), e(257, levels=2)
    assert 0 < small < big
    assert e(513, levels=5, max_rhs=1) < e(513, levels=5, max_rhs=4)
    m = dict(levels=5, precision="mixed")
    assert e(513, max_rhs=4, device_gmres=2, **m) < e(513, max_rhs=4, device_gmres=0, **m)
    assert e(513, max_rhs=4, device_gmres=2, **m) < e(513, max_rhs=4, device_gmres=3, **m)
    assert e(513, max_rhs=3, device_gmres=1, **m) == e(513, max_rhs=3, device_gmres=2, **m)
    assert e(513, max_rhs=4, device_gmres=1, **m) == e(513, max_rhs=4, device_gmres=3, **m)
    # FP64 vectors take the cluster form too (per-rhs workspace), like FP32
    assert e(513, levels=5, max_rhs=4, device_gmres=3) > e(513, levels=5, max_rhs=4, device_gmres=2)
    assert e(513, levels=5, max_rhs=4, device_gmres=1) == e(513, levels=5, max_rhs=4, device_gmres=3)
    assert e(513, levels=5, precision="mixed") < e(513, levels=5, precision="fp64")
    # a level with m iterations or a tolerance keeps a larger Krylov basis than a one-iteration level
    assert e(513, levels=5) < e(513, levels=5, cycle_m=2) < e(513, levels=5, cycle_m=3)
    assert e(513, levels=5, cycle_m=2) < e(513, levels=5, level_tol={3: 0.1})
    # Bi-CGSTAB keeps five vectors per Krylov level in place of the persistent GMRES workspace
    assert e(513, levels=5, cslp_solver="bicgstab") != e(513, levels=5)
    assert L.hz_estimate_bytes(None, None, None) == hz.HZ_EINVAL
    # multi-instance batches keep one wavenumber field per right-hand side on every level
    # (FP64 + FP32 copies, 12 bytes per node) and one coarsest multigrid inverse per field
    one, per = e(513, levels=3, max_rhs=4), e(513, levels=3, max_rhs=4, per_rhs_k=1)
    nodes = 513 ** 2 + 257 ** 2 + 129 ** 2
    assert per - one >= 3 * 12 * nodes
    assert e(513, levels=3, max_rhs=1, per_rhs_k=1) == e(513, levels=3, max_rhs=1)


def test_random_instances_inputs():
    """The multi-instance workload generator: one field and one source per instance, fields
    differ between instances (their own seeds), k_max h runs from 0.2 to 0.3."""
    import math

    import model_problems as mp
    p = mp.random_instances(65, count=4, levels=2, negdef_from_level=4)
    assert p.k.shape == (4, 65, 65) and p.b.shape == (4, 65, 65) and p.nrhs == 4
    assert all(not (p.k[0] == p.k[r]).all() for r in range(1, 4))
    khmax = [float(p.k[r].max()) * p.h for r in range(4)]
    assert all(math.isclose(a, b, rel_tol=1e-12) for a, b in zip(khmax, [0.2, 0.2 + 0.1 / 3, 0.2 + 0.2 / 3, 0.3]))
    assert all((p.b[r] != 0).sum() == 1 for r in range(4))


def test_server_rejects_bad_arguments(L):
    import paper_2412_04980_gb300 as hz
    s = ctypes.c_void_p()
    assert L.hz_server_create(0, 1, ctypes.byref(s)) == hz.HZ_EINVAL
    assert L.hz_server_create(1 << 20, 0, ctypes.byref(s)) == hz.HZ_EINVAL
    assert L.hz_server_create(1 << 20, 1, None) == hz.HZ_EINVAL
    t = ctypes.c_uint64()
    assert L.hz_submit(None, None, ctypes.byref(t)) == hz.HZ_EINVAL
    assert L.hz_poll(None, 1, None) == hz.HZ_EINVAL
    assert L.hz_wait(None, 1, 0.0, None) == hz.HZ_EINVAL
    assert L.hz_server_destroy(None) == hz.HZ_OK


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets the C compiler gives the
    header's structs (checked with gcc, no GPU)."""
    import subprocess
    import paper_2412_04980_gb300 as hz
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    structs = {"hz_grid": hz.HzGrid, "hz_config": hz.HzConfig, "hz_stats": hz.HzStats, "hz_request": hz.HzRequest,
               "hz_server_stats": hz.HzServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hz.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines())
    for cname, py in structs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(py, fname).offset, (cname, fname)


def test_diagnostics_reject_null_handles(L):
    import paper_2412_04980_gb300 as hz
    f, c, cl = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert L.hz_level_gmres_form(None, 1, ctypes.byref(f), ctypes.byref(c), ctypes.byref(cl)) == hz.HZ_EINVAL
    n = ctypes.c_longlong()
    assert L.hz_launch_count(None, ctypes.byref(n)) == hz.HZ_EINVAL
    ms, by = ctypes.c_double(), ctypes.c_double()
    assert L.hz_gmres_device_time(None, 0, 0, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)) == hz.HZ_EINVAL


def test_config_validation_of_new_fields(L):
    import paper_2412_04980_gb300 as hz
    h = ctypes.c_void_p()
    g = hz.HzGrid(9, 9, 0.1, 0)
    for bad in (dict(device_gmres=5), dict(device_gmres=-1), dict(autotune=2), dict(reorth_eta=1.5),
                dict(cycle_m=0), dict(l2_tol=1.0), dict(l2_tol=-0.1), dict(cslp_solver=2), dict(sym_rows=2), dict(per_rhs_k=2),
                dict(levels=3, level_tol={2: 0.1}), dict(levels=3, level_tol={3: 0.1}),
                dict(levels=4, level_tol={3: 1.0}), dict(levels=4, level_tol={3: float("nan")})):
        c = hz.config(**bad)
        assert L.hz_setup(ctypes.byref(g), ctypes.c_void_p(1), ctypes.byref(c), None, ctypes.byref(h)) == hz.HZ_EINVAL
        msg = L.hz_last_error().decode()
        assert "coarsened" not in msg, (bad, msg)       # refused for the field itself
    # the symmetric row scaling applies to Sommerfeld boundary rows only
    c = hz.config(sym_rows=1)
    gd = hz.HzGrid(9, 9, 0.1, 1)
    assert L.hz_setup(ctypes.byref(gd), ctypes.c_void_p(1), ctypes.byref(c), None, ctypes.byref(h)) == hz.HZ_EINVAL
    assert "Sommerfeld" in L.hz_last_error().decode()


def test_dirichlet_grid_coarsening_rule(L):
    """Dirichlet grids hold interior unknowns: a side of n coarsens to (n - 1) / 2 and must be odd
    and at least 3; vertex grids need odd sides of at least 5.  Refused before any device work."""
    import paper_2412_04980_gb300 as hz
    h = ctypes.c_void_p()
    for nx, ny, bc, levels in ((8, 15, 1, 2), (15, 15, 1, 5), (3, 15, 0, 2)):
        g = hz.HzGrid(nx, ny, 0.1, bc)
        c = hz.config(levels=levels)
        assert L.hz_setup(ctypes.byref(g), ctypes.c_void_p(1), ctypes.byref(c), None, ctypes.byref(h)) == hz.HZ_EINVAL
        assert "coarsened" in L.hz_last_error().decode()


def test_dirichlet_estimate_follows_interior_sizes():
    """hz_estimate_bytes on a Dirichlet grid uses the (n - 1) / 2 coarse sides: a 127^2 Dirichlet
    grid needs less than the 129^2 vertex grid with the same levels."""
    import paper_2412_04980_gb300 as hz
    L_ = hz.lib()
    g_d, g_s = hz.HzGrid(127, 127, 1 / 128, 1), hz.HzGrid(129, 129, 1 / 128, 0)
    c = hz.config(levels=4)
    bd, bs = ctypes.c_size_t(), ctypes.c_size_t()
    assert L_.hz_estimate_bytes(ctypes.byref(g_d), ctypes.byref(c), ctypes.byref(bd)) == hz.HZ_OK
    assert L_.hz_estimate_bytes(ctypes.byref(g_s), ctypes.byref(c), ctypes.byref(bs)) == hz.HZ_OK
    assert 0 < bd.value < bs.value


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without libhz.so every entry point raises instead of computing."""
    import paper_2412_04980_gb300 as hz
    monkeypatch.setattr(hz, "_LIB", None)
    monkeypatch.setattr(hz, "library_path", lambda: str(tmp_path / "libhz.so"))
    with pytest.raises(RuntimeError, match="missing"):
        hz.lib()
    with pytest.raises(RuntimeError, match="missing"):
        hz.config(levels=2)
    with pytest.raises(RuntimeError, match="missing"):
        hz.estimate_bytes(129, 129, 1 / 128, levels=2)
