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
    d.delta1 = float("nan")
    assert lib.pvsc_lattice_create(ctypes.byref(d), None, ctypes.byref(h)) == pv.PVSC_ERR_ARG
    d.model, d.dims[2], d.delta1 = pv.GRAPHENE, 1, 0.5  # Delta terms belong to the TI
    assert lib.pvsc_lattice_create(ctypes.byref(d), None, ctypes.byref(h)) == pv.PVSC_ERR_ARG
    assert b"Delta" in lib.pvsc_last_error()
    assert lib.pvsc_apply_H(None, 1, 0, None, None, None) == pv.PVSC_ERR_ARG
    assert lib.pvsc_work_bytes(None, 0, 1, 0, 0) == 0


def test_quantum_dot_descriptor_errors_without_a_device(libpath):
    # PVSC_V_QDOT is checked before any device call: graphene only, 1..16 dots per row,
    # positive finite radius and width, finite heights
    import paper_1708_09689_gb300 as pv
    lib = pv.lib()
    h = ctypes.c_void_p()

    def desc(model=pv.GRAPHENE, count=2, radius=3.0, V0=0.1, width=1.0, dV=0.0):
        d = pv.LatticeDesc()
        d.model = model
        d.dims[0], d.dims[1], d.dims[2] = 8, 8, (4 if model == pv.TI else 1)
        d.t = 1.0
        d.v_source = pv.V_QDOT
        d.qd_count, d.qd_radius, d.qd_V0, d.qd_width, d.qd_dV = count, radius, V0, width, dV
        return d

    for bad, word in [(desc(model=pv.TI), b"graphene"), (desc(count=0), b"qd_count"),
                      (desc(count=17), b"qd_count"), (desc(radius=0.0), b"radius"),
                      (desc(width=-1.0), b"width"), (desc(V0=float("nan")), b"V0"),
                      (desc(dV=float("inf")), b"dV")]:
        assert lib.pvsc_lattice_create(ctypes.byref(bad), None, ctypes.byref(h)) == pv.PVSC_ERR_ARG
        assert word in lib.pvsc_last_error()
    d = desc()
    d.v_source = 6  # past the last potential source
    assert lib.pvsc_lattice_create(ctypes.byref(d), None, ctypes.byref(h)) == pv.PVSC_ERR_ARG
    assert b"v_source" in lib.pvsc_last_error()


@pytest.mark.parametrize("n,seed", [(1, 0), (7, 1), (40, 2), (64, 3)])
def test_host_hermitian_jacobi_matches_numpy(libpath, n, seed):
    # the small dense eigenproblem of ChebFD's Rayleigh-Ritz step, host code only
    lib = ctypes.CDLL(libpath)
    lib.pvsc_debug_eigh.argtypes = [ctypes.c_int] + [ctypes.c_void_p] * 3
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = A + A.conj().T
    if n >= 40:  # Kramers-like degenerate pairs, as in the TI spectrum
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        A = Q @ np.diag(np.repeat(rng.standard_normal(n // 2), 2)) @ Q.conj().T
    Af = np.asfortranarray(A).astype(np.complex128)
    w = np.zeros(n)
    V = np.zeros((n, n), dtype=np.complex128, order="F")
    assert lib.pvsc_debug_eigh(n, Af.ctypes.data, w.ctypes.data, V.ctypes.data) == 0
    scale = np.linalg.norm(A)
    assert np.max(np.abs(w - np.linalg.eigvalsh(A))) < 1e-13 * scale
    assert np.max(np.abs(A @ V - V * w)) < 1e-12 * scale
    assert np.max(np.abs(V.conj().T @ V - np.eye(n))) < 1e-12


@pytest.mark.parametrize("cname,pyname", [("pvsc_lattice_desc", "LatticeDesc"), ("pvsc_tuning", "Tuning"),
                                          ("pvsc_chebfd_params", "ChebFDParams")])
def test_binding_structs_match_the_c_layout(libpath, tmp_path, cname, pyname):
    # the ctypes mirrors of the C structs: same size and the same offset for every field
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mod = pytest.importorskip("paper_1708_09689_gb300")
    py = getattr(mod, pyname)
    fields = [f[0] for f in py._fields_]
    src = tmp_path / "layout.c"
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pvsc.h"', "int main(void) {",
             f'  printf("size %zu\\n", sizeof({cname}));']
    lines += [f'  printf("{f} %zu\\n", offsetof({cname}, {f}));' for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                  text=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(py)
    for f in fields:
        assert int(out[f]) == getattr(py, f).offset, f


@pytest.mark.parametrize("K", list(range(1, 40)) + [202, 4000])
def test_series_accumulator_plan_adds_every_term_once(libpath, K):
    # The series sweeps add their terms to the fp64 accumulator in groups: the
    # groups must tile the terms 0 .. K-1 exactly, in order, with at most three
    # terms per group (a sweep holds only y_in, x and y_new), the last sweep
    # always writing the result, and no sweep before it touching more often
    # than every third sweep.
    lib = ctypes.CDLL(libpath)
    lib.pvsc_debug_series_plan.argtypes = [ctypes.c_int, ctypes.c_void_p]
    terms = np.zeros(K, dtype=np.int32)
    assert lib.pvsc_debug_series_plan(K, terms.ctypes.data) == 0
    if K == 1:
        assert terms.tolist() == [1]
        return
    assert terms[0] == 0 and terms[1] == 2 and terms[K - 1] > 0
    covered = -1
    touches = []
    for j in range(1, K):
        n = int(terms[j])
        if n:
            assert 1 <= n <= 3 and j - n + 1 == covered + 1  # the next terms, ending with term j
            covered = j
            touches.append(j)
    assert covered == K - 1 and int(terms.sum()) == K
    inner = [j for j in touches if 1 < j < K - 1]
    assert all(j % 3 == 1 for j in inner)
    assert len(touches) == 1 + len(inner) + (K - 1 > 1)


def test_series_plan_rejects_bad_arguments(libpath):
    lib = ctypes.CDLL(libpath)
    lib.pvsc_debug_series_plan.argtypes = [ctypes.c_int, ctypes.c_void_p]
    out = np.zeros(4, dtype=np.int32)
    assert lib.pvsc_debug_series_plan(0, out.ctypes.data) != 0
    assert lib.pvsc_debug_series_plan(3, None) != 0
