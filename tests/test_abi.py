"""The C-ABI library loads and exports every entry point include/multipole.h declares;
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "multipole.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2602_02507_gb300 import build as cuda_build
    from paper_2602_02507_gb300 import multipole as mpl
    cuda_build.build()
    return mpl.load_library()


def declared_functions():
    text = open(HEADER).read()
    return re.findall(r"^MP_API\s+[\w\s\*]+?\b(mp_\w+)\s*\(", text, flags=re.M)


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for required in ("mp_mesh_create", "mp_set_density", "mp_solve", "mp_get_phi", "mp_get_moments",
                     "mp_mesh_destroy", "mp_batch_create", "mp_batch_solve", "mp_autotune", "mp_solve_host",
                     "mp_solve_host_async"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    from paper_2602_02507_gb300 import multipole as mpl
    for code, name in mpl.STATUS_NAMES.items():
        assert mpl.status_string(code).startswith(name)
    assert mpl.version() >= 100


def _create(lib, r, th, ph, L=4, G=1.0, prec=0):
    dp = ctypes.POINTER(ctypes.c_double)
    r, th, ph = (np.ascontiguousarray(a, dtype=np.float64) for a in (r, th, ph))
    h = ctypes.c_void_p()
    st = lib.mp_mesh_create(r.ctypes.data_as(dp), r.size - 1, th.ctypes.data_as(dp), th.size - 1,
                            ph.ctypes.data_as(dp), ph.size - 1, L, G, prec, None, ctypes.byref(h))
    return st, h


GOOD = (np.linspace(0, 1, 5), np.linspace(0, np.pi, 5), np.linspace(0, 2 * np.pi, 9))


@pytest.mark.parametrize("case", ["r_decreasing", "r_negative", "theta_beyond_pi", "phi_span", "nan_edge",
                                  "bad_L", "bad_G", "bad_prec"])
def test_argument_errors_are_caught_on_the_host(lib, case):
    r, th, ph = (a.copy() for a in GOOD)
    L, G, prec = 4, 1.0, 0
    if case == "r_decreasing":
        r[2] = r[1]
    elif case == "r_negative":
        r[0] = -0.1
    elif case == "theta_beyond_pi":
        th[-1] = np.pi + 1e-6
    elif case == "phi_span":
        ph[-1] = 2 * np.pi + 1e-6
    elif case == "nan_edge":
        r[3] = np.nan
    elif case == "bad_L":
        L = -1
    elif case == "bad_G":
        G = 0.0
    elif case == "bad_prec":
        prec = 7
    st, h = _create(lib, r, th, ph, L=L, G=G, prec=prec)
    assert st == 1, st  # MP_ERR_INVALID_ARG
    assert h.value is None
    buf = ctypes.create_string_buffer(256)
    lib.mp_last_error_detail(buf, 256)
    assert buf.value


def test_range_error_for_huge_radial_span(lib):
    r = np.geomspace(1e-30, 1e30, 9)
    st, _ = _create(lib, r, GOOD[1], GOOD[2], L=40)
    assert st == 2  # MP_ERR_RANGE


def test_split_precision_degree_limit(lib):
    st, _ = _create(lib, *GOOD, L=128, prec=1)
    assert st == 8  # MP_ERR_UNSUPPORTED


def test_null_handles(lib):
    assert lib.mp_solve(None) == 1
    assert lib.mp_mesh_destroy(None) == 1
    assert lib.mp_set_density(None, None) == 1
