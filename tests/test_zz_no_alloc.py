"""pvsc_cheb_step_noalloc, the fused Chebyshev step for callers that cannot
allocate device memory, checked through the C ABI against pvsc_cheb_step
(the entry point that takes a caller-allocated work buffer).

Kept in a file of its own that pytest collects last: it exercises the
library's static scratch array, which every call on a device shares, and it
must pass both alone in a fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

pv = pytest.importorskip("paper_1708_09689_gb300")


def _c_doubles(v):
    return (ctypes.c_double * len(v))(*[float(a) for a in v])


def _opt(v):
    return _c_doubles(v) if v is not None else None


def _call_noalloc(lat, x, y, z, alpha, beta, gamma, delta, flags, dots):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return pv.lib().pvsc_cheb_step_noalloc(
        lat.handle, x.shape[1], pv.prec_of(x), ctypes.c_void_p(x.data_ptr()),
        ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(z.data_ptr()) if z is not None else None,
        _c_doubles(alpha), _c_doubles(beta), _opt(gamma), _opt(delta),
        flags, ctypes.c_void_p(dots.data_ptr()) if flags else None, stream)


def _call_with_work(lat, x, y, z, alpha, beta, gamma, delta, flags, dots):
    R, prec = x.shape[1], pv.prec_of(x)
    work = pv.work_buffer(lat.work_bytes(pv.OP_CHEB_STEP, R, prec))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return pv.lib().pvsc_cheb_step(
        lat.handle, R, prec, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
        ctypes.c_void_p(z.data_ptr()) if z is not None else None, _c_doubles(alpha),
        _c_doubles(beta), _opt(gamma), _opt(delta), flags,
        ctypes.c_void_p(dots.data_ptr()) if flags else None, ctypes.c_void_p(work.data_ptr()),
        work.numel(), stream)


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-13), (torch.complex64, 1e-6)])
@pytest.mark.parametrize("flags", [0, 1, 7])
@pytest.mark.parametrize("with_z,with_gamma", [(True, True), (False, True), (True, False)])
def test_noalloc_step_matches_work_buffer_step_on_two_calls(dtype, tol, flags, with_z, with_gamma):
    lat = pv.Lattice.ti((12, 10, 9), (1, 1, 0), t=1.0, m=2.0, disorder=(2.0, 5))
    R = 8
    for call in range(2):  # two calls in a row share (and reuse) the static scratch
        x = torch.from_numpy(W.gaussian_block(lat.D, R, 10 + call)).to("cuda", dtype)
        y0 = torch.from_numpy(W.gaussian_block(lat.D, R, 20 + call)).to("cuda", dtype)
        z0 = torch.from_numpy(W.gaussian_block(lat.D, R, 30 + call)).to("cuda", dtype)
        alpha = [0.2 + 0.01 * r for r in range(R)]
        beta = [0.1 * (r - 3) for r in range(R)]
        gamma = [-1.0] * R if with_gamma else None
        delta = [0.5] * R if with_z else None
        za = z0.clone() if with_z else None
        zb = z0.clone() if with_z else None
        ya, da = y0.clone(), torch.zeros((4, R), dtype=torch.float64, device="cuda")
        yb, db = y0.clone(), torch.zeros((4, R), dtype=torch.float64, device="cuda")
        assert _call_noalloc(lat, x, ya, za, alpha, beta, gamma, delta, flags, da) == pv.PVSC_OK, \
            pv.lib().pvsc_last_error()
        assert _call_with_work(lat, x, yb, zb, alpha, beta, gamma, delta, flags, db) == pv.PVSC_OK, \
            pv.lib().pvsc_last_error()
        torch.cuda.synchronize()
        assert torch.equal(ya, yb)
        if with_z:
            assert torch.equal(za, zb)
        if flags:
            rows = [0] + ([1, 2, 3] if flags & 6 else [])
            scale = db[rows].abs().max().item()
            assert (da[rows] - db[rows]).abs().max().item() <= tol * scale
            assert da[0].min().item() > 0  # <x|x> was really written


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lat = pv.Lattice.ti((8, 8, 8), (1, 1, 1), disorder=(1.0, 1))
    R = 64  # 4 dots x 64 vectors x (SMs x 16) blocks of fp64 partials exceed 2 MiB on GB300
    x = torch.zeros((lat.D, R), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    dots = torch.zeros((4, R), dtype=torch.float64, device="cuda")
    one = [1.0] * R
    rc = _call_noalloc(lat, x, y, None, one, one, one, one, 7, dots)
    assert rc == pv.PVSC_ERR_ARG
    assert b"scratch" in pv.lib().pvsc_last_error()
