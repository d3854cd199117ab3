"""CPU-side checks of the boundary: the library builds, loads and exports every
entry point include/pvsc.h declares; host-only entry points behave.  No GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pvsc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pvsc_[A-Za-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__
    return __graft_entry__._build_module().build_library()


def test_header_declares_the_core_entry_points():
    names = declared_functions()
    for core in ("pvsc_lattice_create", "pvsc_apply_H", "pvsc_cheb_step", "pvsc_kpm_moments",
                 "pvsc_cheb_propagate"):
        assert core in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"declared in pvsc.h but not exported: {missing}"


def test_binding_imports_and_reports_version(libpath):
    import paper_1708_09689_gb300 as pv
    assert "sm_103a" in pv.version()


def test_propagation_coeffs_host_entry_point(libpath):
    import paper_1708_09689_gb300 as pv
    from scipy.special import jv
    cw = pv.propagation_coeffs(3.055, 1e-14)
    assert len(cw) == 20
    k = np.arange(20)
    ref = 2.0 * ((-1j) ** k) * jv(k, 3.055)
    ref[0] = jv(0, 3.055)
    assert np.max(np.abs(np.array(cw) - ref)) < 1e-15
    # too-small output buffer is an argument error, not a crash
    n = ctypes.c_int()
    buf = (ctypes.c_double * 4)()
    rc = pv.lib().pvsc_propagation_coeffs(3.055, 1e-14, 2, buf, ctypes.byref(n))
    assert rc == pv.PVSC_ERR_ARG and n.value == 20


def test_argument_errors_are_reported_without_a_device(libpath):
    import paper_1708_09689_gb300 as pv
    lib = pv.lib()
    d = pv.LatticeDesc()
    d.model = 7
    h = ctypes.c_void_p()
    assert lib.pvsc_lattice_create(ctypes.byref(d), None, ctypes.byref(h)) == pv.PVSC_ERR_ARG
    assert b"model" in lib.pvsc_last_error()
    d.model = pv.TI
    for i in range(3):
        d.dims[i] = 4
    d.delta1 = 0.5
    assert lib.pvsc_lattice_create(ctypes.byref(d), None, ctypes.byref(h)) == pv.PVSC_ERR_UNSUPPORTED
    assert lib.pvsc_apply_H(None, 1, 0, None, None, None) == pv.PVSC_ERR_ARG
    assert lib.pvsc_work_bytes(None, 0, 1, 0, 0) == 0
