"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/*.h declares; argument errors come back as status codes."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gmg_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401  (provides the CUDA runtime the library links against)
    from paper_2604_26441_b300 import build, gmg
    build.build_library()
    return gmg.load_library()


def test_every_declared_symbol_is_exported_and_bound(lib):
    from paper_2604_26441_b300 import gmg
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
        assert n in gmg.exported_symbols(), n


def test_status_strings_and_defaults(lib):
    from paper_2604_26441_b300 import gmg
    assert lib.gmg_status_str(0) == b"ok"
    assert b"invalid" in lib.gmg_status_str(-1)
    o = gmg._Options()
    lib.gmg_default_options(ctypes.byref(o))
    assert o.levels == 4 and o.degree == 2 and o.power_iters_fine == 20 and o.power_iters_coarse == 10
    assert abs(o.cheb_alpha - 1 / 30) < 1e-15 and o.chol_cutoff == 5000
    assert o.fused_coarse_nodes == 0 and o.bsr_tma_nodes == 0 and o.device_loop == 1 and o.ir_factor == 0.0 and o.fine_smoother == 0
    assert o.cycle_index == 1 and o.outer == 0 and o.restart == 32 and o.bsr_kernel == -1


def test_struct_layouts_match_header(tmp_path):
    """The ctypes mirrors of gmg_options / gmg_info / gmg_grid / gmg_bc have the
    sizes and field offsets a C compiler gives the declarations in gmg.h."""
    import shutil
    import subprocess
    from paper_2604_26441_b300 import gmg
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"gmg_options": gmg._Options, "gmg_info": gmg._Info, "gmg_grid": gmg._Grid, "gmg_bc": gmg._BC,
               "gmg_tuning": gmg._Tuning}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gmg.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                              check=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(out[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(out[f"{cname}.{fname}"]) == getattr(cls, fname).offset, f"{cname}.{fname}"


def test_argument_errors_without_device(lib):
    from paper_2604_26441_b300 import gmg
    h = ctypes.c_void_p()
    g = gmg._Grid(4, 2, 2)
    bc = gmg._BC(gmg.BC_CLAMP_XMIN, None)
    assert lib.gmg_setup(None, ctypes.byref(g), None, 3.0, 1.0, 1e-9, 0.3, ctypes.byref(bc), None) == -1
    assert lib.gmg_setup(ctypes.byref(h), ctypes.byref(g), None, 3.0, 1.0, 1e-9, 0.3, ctypes.byref(bc), None) == -1
    bad = gmg._Grid(0, 2, 2)
    assert lib.gmg_setup(ctypes.byref(h), ctypes.byref(bad), ctypes.c_void_p(16), 3.0, 1.0, 1e-9, 0.3,
                         ctypes.byref(bc), None) == -1
    assert b"element counts" in lib.gmg_last_error()
    mask_bc = gmg._BC(gmg.BC_MASK, None)
    assert lib.gmg_setup(ctypes.byref(h), ctypes.byref(g), ctypes.c_void_p(16), 3.0, 1.0, 1e-9, 0.3,
                         ctypes.byref(mask_bc), None) == -1
    assert lib.gmg_solve(None, None, None, 1e-6, 10, None) == -1
    assert lib.gmg_autotune(None, 3, None) == -1
    assert lib.gmg_solve_multi(None, 1, None, None, 1e-6, 10, None) == -1
    assert lib.gmg_apply_multi(None, 1, None, None) == -1
    assert lib.gmg_set_multi_kernel(None, 0) == -1
    assert lib.gmg_num_levels(None) == 0
    lib.gmg_destroy(None)


def test_no_device_is_reported(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    from paper_2604_26441_b300 import gmg
    h = ctypes.c_void_p()
    g = gmg._Grid(4, 2, 2)
    bc = gmg._BC(gmg.BC_CLAMP_XMIN, None)
    rc = lib.gmg_setup(ctypes.byref(h), ctypes.byref(g), ctypes.c_void_p(256), 3.0, 1.0, 1e-9, 0.3, ctypes.byref(bc),
                       None)
    assert rc == -6 and not h.value


def test_warm_start_network_shape_and_argument_errors(lib):
    """The library's network table agrees with the oracle's (both are written
    from the same architecture statement), and bad arguments are refused
    before any device work."""
    from oracle import warmnet
    from paper_2604_26441_b300 import gmg
    assert "gmg_warm_start" in _declared() and "gmg_net_train_step" in _declared()
    assert lib.gmg_net_num_params() == warmnet.n_params()
    shapes = gmg.net_layer_shapes()
    assert [(ci, co, s, int(a)) for _, ci, co, s, a in warmnet.LAYERS] == shapes
    sh = (ctypes.c_int * 4)()
    assert lib.gmg_net_layer_shape(12, sh) == -1
    h = ctypes.c_void_p()
    assert lib.gmg_net_create(None, ctypes.c_void_p(16), None) == -1
    assert lib.gmg_net_create(ctypes.byref(h), None, None) == -1
    assert lib.gmg_net_forward(None, 8, 8, 8, 1, ctypes.c_void_p(16), ctypes.c_void_p(16)) == -1
    assert lib.gmg_net_features(8, 8, 8, None, None, None, None, None) == -1
    assert lib.gmg_net_target(0, 8, 8, ctypes.c_void_p(16), ctypes.c_void_p(16), None) == -1
    assert lib.gmg_warm_start(None, None, None, None, None, None) == -1
    lib.gmg_net_destroy(None)
