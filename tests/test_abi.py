"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and
exports every entry point that include/mbs.h declares."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mbs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mbs_[A-Za-z_0-9]+)\s*\(", src)))


def test_header_declares_the_paper_calls():
    names = _declared()
    for n in ("mbs_build_scattering_matrices", "mbs_apply_operator", "mbs_solve",
              "mbs_evaluate_field", "mbs_rhs", "mbs_create", "mbs_destroy"):
        assert n in names


def test_library_builds_and_exports_every_symbol():
    from paper_2603_19113_gb300 import build as b
    try:
        lib_path = b.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    import ctypes
    lib = ctypes.CDLL(lib_path)
    for n in _declared():
        assert hasattr(lib, n), n
    from paper_2603_19113_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(_declared())


def test_default_options_and_argument_errors_without_gpu():
    """Calls that fail argument validation never touch the device."""
    import ctypes as C

    import paper_2603_19113_gb300 as pkg
    from paper_2603_19113_gb300 import _lib
    try:
        lib = pkg.load_library()
    except ImportError as e:
        pytest.skip(str(e))
    o = _lib.mbs_options()
    lib.mbs_default_options(C.byref(o))
    assert o.precision == 0 and o.restart > 0 and 0 < o.tol < 1e-6
    h = C.c_void_p()
    assert lib.mbs_create(4, 1.0, C.byref(o), C.byref(h)) == 1  # bad dim
    assert lib.mbs_create(2, -1.0, C.byref(o), C.byref(h)) == 1  # bad kappa
    o.restart = 0
    assert lib.mbs_create(2, 1.0, C.byref(o), C.byref(h)) == 1  # bad restart
    lib.mbs_default_options(C.byref(o))
    assert o.fp64_kernel == 2 and o.cuda_graphs == 1 and o.inner_tol == 1e-6
    for field, bad in (("fp64_kernel", 3), ("mac_path", 4), ("inner_tol", 0.0)):
        lib.mbs_default_options(C.byref(o))
        setattr(o, field, bad)
        assert lib.mbs_create(2, 1.0, C.byref(o), C.byref(h)) == 1, field
    assert lib.mbs_serve_create(0, 0, C.byref(h)) == 1
