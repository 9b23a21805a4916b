"""The C-ABI library builds, loads without a GPU, and exports every function
that include/ctd.h declares; the binding keeps the C names."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ctd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ctd_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ctd_create_phantom", "ctd_set_source", "ctd_set_spectrum", "ctd_run", "ctd_get_dose_and_stddev"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1109_3266_gb300 import build, ctd
    build.build()
    L = ctd.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_has_the_c_names():
    from paper_1109_3266_gb300 import ctd
    missing = [n for n in declared_functions() if n not in ("ctd_last_error", "ctd_abi_version") and not hasattr(ctd, n)]
    assert not missing, missing


def test_calls_fail_cleanly_without_a_device():
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1109_3266_gb300 import ctd
    h = ctypes.c_void_p()
    rc = ctd.lib().ctd_create(ctypes.byref(h), None)
    assert rc == 3 and not h.value
    assert ctd.lib().ctd_last_error()
    assert ctd.lib().ctd_abi_version() == 9


def test_kramers_helper_matches_the_input_recipe():
    # a host-only helper: the library's Kramers spectrum equals the input generator's
    from paper_1109_3266_gb300 import ctd, inputs as I
    for kvp, mm, e_min in ((120, 2.5, 1), (80, 0.0, 10), (140, 4.0, 1)):
        lo, hi, w = ctd.ctd_spectrum_kramers(kvp, mm, e_min)
        ref = I.spectrum_kramers(kvp, mm, e_min)
        assert np.array_equal(lo, ref.e_lo) and np.array_equal(hi, ref.e_hi)
        assert np.allclose(w, ref.w, rtol=1e-13, atol=0)
    for bad in ((10, 1.0, 10), (100, -1.0, 1), (100, 1.0, 0)):
        with pytest.raises(ctd.CtdError):
            ctd.ctd_spectrum_kramers(*bad)


C_PROGRAM = r"""
#include <stdio.h>
#include <stddef.h>
#include "ctd.h"

int main(void)
{
    double lo[200], hi[200], w[200];
    int n = 0;
    if (ctd_spectrum_kramers(120, 2.5, 1, lo, hi, w, &n) != CTD_OK) return 1;
    if (ctd_spectrum_kramers(10, 1.0, 10, NULL, NULL, NULL, &n) != CTD_EINVAL) return 2;
    if (ctd_last_error()[0] == '\0') return 3;
    ctd_spectrum_kramers(120, 2.5, 1, lo, hi, w, &n);
    /* the layouts the Python binding mirrors */
    printf("%d %d %.17g %.17g\n", ctd_abi_version(), n, w[0], w[n - 1]);
    printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(ctd_options), sizeof(ctd_material), sizeof(ctd_source),
           sizeof(ctd_physics), sizeof(ctd_run_stats), sizeof(ctd_request), sizeof(ctd_req_status),
           sizeof(ctd_tune_result));
    printf("%zu %zu %zu\n", offsetof(ctd_options, shared_launch), offsetof(ctd_source, z1_cm),
           offsetof(ctd_physics, compton_model));
    {
        /* host physics: water's node-table columns with the independent-atom form factor */
        const ctd_material water = {0.5551, 18.015, 7.42, 1.0, 0.55};
        const int z[2] = {1, 8};
        const double n[2] = {2.0, 1.0};
        double col[3 * 150];
        if (ctd_material_columns(&water, 2, z, n, 1, 150, CTD_COMPTON_WH, col) != CTD_OK) return 4;
        printf("%.17g %.17g\n", col[3 * 59 + 2], col[3 * 149 + 1]);
    }
    return 0;
}
"""


def test_header_is_plain_c_and_layouts_match_the_binding(tmp_path):
    # a C99 program built against the header and linked to the library: the host-only
    # entry points run, and C's struct sizes and offsets are the ones the binding uses
    import ctypes
    import shutil
    import subprocess
    from paper_1109_3266_gb300 import build, ctd
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lib = build.build()
    src = tmp_path / "abi.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "abi"
    r = subprocess.run([cc, "-std=c99", "-pedantic", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), lib, f"-Wl,-rpath,{os.path.dirname(lib)}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    first, sizes, offs, cols = r.stdout.split("\n")[:4]
    abi, n, w0, wl = first.split()
    assert int(abi) == ctd.lib().ctd_abi_version() and int(n) == 119
    lo, hi, w = ctd.ctd_spectrum_kramers(120, 2.5, 1)
    assert float(w0) == w[0] and float(wl) == w[-1]
    want = [ctypes.sizeof(t) for t in (ctd.ctd_options, ctd.ctd_material, ctd.ctd_source, ctd.ctd_physics,
                                       ctd.ctd_run_stats, ctd.ctd_request, ctd.ctd_req_status, ctd.ctd_tune_result)]
    assert [int(x) for x in sizes.split()] == want
    assert [int(x) for x in offs.split()] == [ctd.ctd_options.shared_launch.offset, ctd.ctd_source.z1_cm.offset,
                                              ctd.ctd_physics.compton_model.offset]
    from paper_1109_3266_gb300 import inputs as I
    py = ctd.ctd_material_columns(I.WATER, 1, 150, "wh", ((1, 2.0), (8, 1.0)))
    assert [float(x) for x in cols.split()] == [py[59, 2], py[149, 1]]
