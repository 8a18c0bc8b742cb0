"""CPU-side checks of the C ABI: the library builds for sm_103a, loads without
a GPU, exports every function that include/mh3d.h declares, and the ctypes
mirrors of the ABI structs have the C layout.  No compute call is made."""
import ctypes
import glob
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mh3d.h")
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def _declared_functions():
    text = "".join(open(h).read() for h in HEADERS)
    pat = r"^(?:mh3d_status|const char\s*\*|unsigned long long|long long)\s*(mh3d_\w+)\s*\("
    return sorted(set(re.findall(pat, text, re.M)))


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2503_13802_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["mh3d_plan_create", "mh3d_plan_destroy", "mh3d_forward", "mh3d_adjoint", "mh3d_solve",
                     "mh3d_solve_batched", "mh3d_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    for name in _declared_functions():
        assert re.search(r"\bT\s+" + name + r"\b", out), name


def test_binding_covers_every_declared_symbol():
    from paper_2503_13802_gb300 import mh3d, unet

    assert sorted(mh3d.EXPORTS + unet.EXPORTS) == _declared_functions()


@pytest.mark.parametrize("ch", [(2, 3), (8, 16, 32), (16, 32, 64, 128), (2, 3, 4, 5, 6)])
def test_network_layer_tables_match_the_oracle(lib, ch):
    """The library's parameter count (its C layer table, a host function
    callable without a GPU) and the warm start's initialisation table agree
    with the oracle's layer shapes at every depth."""
    from oracle import unet_oracle as U
    from paper_2503_13802_gb300.warmstart import layer_io

    lib.mh3d_unet_param_count_levels.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    lib.mh3d_unet_param_count_levels.restype = ctypes.c_longlong
    arr = (ctypes.c_int * len(ch))(*ch)
    assert lib.mh3d_unet_param_count_levels(len(ch), arr) == U.param_count(*ch)
    io = [(1 if ci is None else ch[ci], 1 if co is None else ch[co]) for ci, co in layer_io(len(ch))]
    assert io == [(ci, co) for _, ci, co in U.layer_shapes(*ch)]
    assert lib.mh3d_unet_param_count_levels(1, arr) == -1


def test_version_without_gpu(lib):
    lib.mh3d_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.mh3d_version()


def test_struct_layouts_match_c(tmp_path):
    """Compile a C program against the header that prints sizeof/offsetof of
    the ABI structs and compare with the ctypes mirrors."""
    from paper_2503_13802_gb300 import mh3d as m

    fields = {
        "mh3d_geometry": ["n", "voxel_mm", "drive_axis", "ds_factor", "ds_offset", "pad", "k_min", "k_max",
                          "gamma_per_mm", "gammaA", "transverse_ratio", "theta", "sensitivity_dev"],
        "mh3d_solve_opts": ["reg_kind", "lambda", "alpha", "shell", "solver", "rel_tol", "max_iter", "fixed_iters",
                            "x0_dev", "normal_mode", "apg_tau", "lambda_relative", "cg_variant", "x0_fallback",
                            "fp32_scalar_div"],
        "mh3d_solve_info": ["iters", "rel_res_recurrence", "rel_res_true", "history", "status", "x0_rejected",
                            "tau"],
        "mh3d_unet_conv_desc": ["nx", "ny", "nz", "cin", "cout", "src_bf16", "skip_bf16", "src_f32", "up"],
    }
    src = ['#include <stdio.h>', '#include <stddef.h>'] + [f'#include "{h}"' for h in HEADERS] + ["int main(void){"]
    for st, fs in fields.items():
        src.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for f in fs:
            src.append(f'printf("{st}.{f} %zu\\n", offsetof({st}, {f}));')
    src.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", str(c), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    from paper_2503_13802_gb300 import unet as u

    py = {"mh3d_geometry": m.mh3d_geometry, "mh3d_solve_opts": m.mh3d_solve_opts, "mh3d_solve_info": m.mh3d_solve_info,
          "mh3d_unet_conv_desc": u.mh3d_unet_conv_desc}
    for st, cls in py.items():
        assert int(got[st]) == ctypes.sizeof(cls), st
        for f in fields[st]:
            pyf = "lambda_" if f == "lambda" else f
            assert int(got[f"{st}.{f}"]) == getattr(cls, pyf).offset, (st, f)
