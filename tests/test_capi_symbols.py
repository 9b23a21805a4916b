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
    assert ctd.lib().ctd_abi_version() == 7


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
