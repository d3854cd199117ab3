"""Python binding of libpvsc (matrix-free Chebyshev stencils for Dirac and
topological materials on GB300).

This module only marshals arguments: it turns torch CUDA tensors into device
pointers, the current torch stream into a cudaStream_t and Python numbers into
C values, and calls the C ABI declared in include/pvsc.h.  Every arithmetic
step of the path runs in the library's CUDA kernels.  There is no CPU
fallback: if libpvsc.so has not been built, importing the library raises.

Vectors are torch tensors of shape (D, R) (or (D,) for R = 1) in the layout
of the C ABI, D = orbitals * n_sites: complex128 selects PVSC_C128 and
complex64 PVSC_C64.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import torch

from .build import LIB_PATH

PVSC_OK, PVSC_ERR_ARG, PVSC_ERR_CUDA, PVSC_ERR_OOM, PVSC_ERR_TIMEOUT, PVSC_ERR_UNSUPPORTED = \
    0, -1, -2, -3, -4, -5
TI, GRAPHENE, WSM = 1, 2, 3
C128, C64, Q64 = 0, 1, 2  # Q64: fixed-point vectors, pvsc_kpm_moments on TI only
KERNEL_NONE, KERNEL_JACKSON, KERNEL_LORENTZ = 0, 1, 2  # damping kernels of kpm_density
V_ZERO, V_HOST, V_DEVICE, V_SEED, V_ON_THE_FLY, V_QDOT = 0, 1, 2, 3, 4, 5
DOT_XX, DOT_XY, DOT_YY = 1, 2, 4
OP_APPLY, OP_CHEB_STEP, OP_KPM, OP_SERIES, OP_ADJOINT, OP_KPM_BATCHED = 0, 1, 2, 3, 4, 5
LATTICE_Z_HALO_LO, LATTICE_Z_HALO_HI = 1, 2  # z-slab lattices: halo plane below / above


class PvscError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pvsc error {code}: {msg}")
        self.code = code


class LatticeDesc(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int32),
        ("periodic", ctypes.c_int32 * 3),
        ("dims", ctypes.c_int64 * 3),
        ("t", ctypes.c_double),
        ("m", ctypes.c_double),
        ("delta1", ctypes.c_double),
        ("delta2", ctypes.c_double),
        ("v_source", ctypes.c_int32),
        ("flags", ctypes.c_int32),
        ("V", ctypes.c_void_p),
        ("seed", ctypes.c_uint64),
        ("W", ctypes.c_double),
        ("k0", ctypes.c_double),
        ("qd_count", ctypes.c_int32),
        ("qd_reserved", ctypes.c_int32),
        ("qd_radius", ctypes.c_double),
        ("qd_V0", ctypes.c_double),
        ("qd_width", ctypes.c_double),
        ("qd_dV", ctypes.c_double),
    ]


class Tuning(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("zslab", ctypes.c_int32), ("time_ms", ctypes.c_float), ("vpt", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("kernel", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"threads": self.threads, "blocks_per_sm": self.blocks_per_sm, "zslab": self.zslab,
                "time_ms": self.time_ms, "vpt": self.vpt, "tile_x": self.tile_x,
                "tile_y": self.tile_y, "kernel": self.kernel}


_vp, _i, _sz, _d, _u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_double, ctypes.c_uint64
_dp = ctypes.POINTER(ctypes.c_double)

_SIGNATURES = {
    "pvsc_lattice_create": (_i, [ctypes.POINTER(LatticeDesc), _vp, ctypes.POINTER(_vp)]),
    "pvsc_lattice_destroy": (_i, [_vp]),
    "pvsc_lattice_info": (_i, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]),
    "pvsc_set_potential": (_i, [_vp, _vp, _vp]),
    "pvsc_get_potential": (_i, [_vp, _vp, _vp]),
    "pvsc_spectral_bounds": (_i, [_vp, _d, _dp, _dp, _dp, _dp, _vp, _sz, _vp]),
    "pvsc_random_vectors": (_i, [_vp, _i, _i, _u64, _vp, _vp]),
    "pvsc_apply_H": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
    "pvsc_cheb_step": (_i, [_vp, _i, _i, _vp, _vp, _vp, _dp, _dp, _dp, _dp, _i, _vp, _vp, _sz, _vp]),
    "pvsc_cheb_step_noalloc": (_i, [_vp, _i, _i, _vp, _vp, _vp, _dp, _dp, _dp, _dp, _i, _vp, _vp]),
    "pvsc_kpm_moments": (_i, [_vp, _i, _i, _vp, _u64, _i, _d, _d, _vp, _vp, _sz, _vp]),
    "pvsc_kpm_density": (_i, [_i, _i, _vp, _i, _d, _d, _d, _d, _i, _vp, _vp, _vp]),
    "pvsc_chebfd": (_i, [_vp, _vp, _d, _d, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "pvsc_chebfd_work_bytes": (_sz, [_vp, _i, _i, _i]),
    "pvsc_bloch_vectors": (_i, [_vp, _i, ctypes.POINTER(_d), _i, _vp, _vp]),
    "pvsc_cheb_series": (_i, [_vp, _i, _i, _vp, _vp, _dp, _i, _dp, _d, _d, _vp, _sz, _vp]),
    "pvsc_cheb_filter": (_i, [_vp, _i, _i, _vp, _vp, _dp, _i, _d, _d, _vp, _sz, _vp]),
    "pvsc_propagation_coeffs": (_i, [_d, _d, _i, _dp, ctypes.POINTER(ctypes.c_int)]),
    "pvsc_cheb_propagate": (_i, [_vp, _i, _i, _vp, _d, _i, _d, _d, _d, _vp, _sz, _vp]),
    "pvsc_cheb_adjoint_step": (_i, [_vp, _i, _i, _vp, _vp, _d, _d, _d, _d, _vp, _vp, _sz, _vp]),
    "pvsc_cheb_propagate_checkpointed": (_i, [_vp, _i, _i, _vp, _d, _i, _i, _d, _d, _d, _vp, _vp, _sz, _vp]),
    "pvsc_cheb_propagate_adjoint": (_i, [_vp, _i, _i, _vp, _d, _i, _i, _d, _d, _d, _vp, _vp, _vp, _sz, _vp]),
    "pvsc_propagate_adjoint_work_bytes": (_sz, [_vp, _i, _i, _d, _d]),
    "pvsc_debug_export_pattern": (_i, [_vp, _vp, _vp]),
    "pvsc_debug_fx_arith": (_i, [_i, _vp, ctypes.c_int64, _vp, _vp]),
    "pvsc_debug_series_plan": (_i, [_i, _vp]),
    "pvsc_kpm_sweeps": (_i, [_vp, _i, _i, _i, _i, _vp, _vp, _d, _d, _vp, _i, _vp, _sz, _vp]),
    "pvsc_kpm_moments_batched": (_i, [ctypes.POINTER(_vp), _i, _i, _i, ctypes.POINTER(_u64), _i,
                                      _dp, _dp, _vp, _vp, _sz, _vp]),
    "pvsc_batched_work_bytes": (_sz, [ctypes.POINTER(_vp), _i, _i, _i, _i]),
    "pvsc_work_bytes": (_sz, [_vp, _i, _i, _i, _i]),
    "pvsc_set_wait_limit": (_i, [_u64]),
    "pvsc_debug_inject_stall": (_i, [_i]),
    "pvsc_set_tuning": (_i, [_vp, _i, _i, ctypes.POINTER(Tuning)]),
    "pvsc_get_tuning": (_i, [_vp, _i, _i, ctypes.POINTER(Tuning)]),
    "pvsc_autotune": (_i, [_vp, _i, _i, ctypes.POINTER(Tuning), _vp]),
    "pvsc_autotune_op": (_i, [_vp, _i, _i, _i, ctypes.POINTER(Tuning), _vp]),
    "pvsc_autotune_batched": (_i, [_vp, _i, _i, _i, _vp, _i, _vp, _vp, ctypes.POINTER(Tuning), _vp]),
    "pvsc_debug_neighbours": (_i, [_vp, _vp, _vp]),
    "pvsc_last_error": (ctypes.c_char_p, []),
    "pvsc_version": (ctypes.c_char_p, []),
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (or python -m "
                          "paper_1708_09689_gb300.build) to compile the CUDA library")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def lib():
    return _lib


def _check(rc: int):
    if rc != PVSC_OK:
        raise PvscError(rc, _lib.pvsc_last_error().decode())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _darr(vals):
    vals = [float(v) for v in vals]
    return (ctypes.c_double * len(vals))(*vals)


def prec_of(t: torch.Tensor) -> int:
    if t.dtype == torch.complex128:
        return C128
    if t.dtype == torch.complex64:
        return C64
    raise ValueError(f"vectors must be complex128 or complex64, got {t.dtype}")


def block_R(t: torch.Tensor) -> int:
    return 1 if t.dim() == 1 else int(t.shape[1])


def version() -> str:
    return _lib.pvsc_version().decode()


def work_buffer(nbytes: int, device=None) -> torch.Tensor:
    """Caller-owned device scratch (16-byte aligned by the caching allocator)."""
    return torch.empty(max(int(nbytes), 16), dtype=torch.uint8, device=device or "cuda")


# ---------------------------------------------------------------------------- lattice
class Lattice:
    """A TI (Eq. TB_H_topi) or graphene (Eq. graphene_model) lattice handle.

    V: None (zero), a torch CUDA float64 tensor, or a numpy/CPU float64 array
    (copied into the handle); or disorder=(W, seed) for box disorder from the
    counter hash, stored (on_the_fly=False) or regenerated in every sweep; or, for
    graphene, qdots=(count, radius, V0, width[, dV]) for the gate-defined quantum-dot
    array of Eq. qdotarray regenerated in every sweep.
    """

    def __init__(self, model: int, dims, periodic, t: float = 1.0, m: float = 0.0, V=None,
                 disorder=None, on_the_fly: bool = False, delta1: float = 0.0, delta2: float = 0.0,
                 k0: float = 0.0, qdots=None, z_halo: int = 0, stream=None):
        d = LatticeDesc()
        d.model = model
        d.flags = int(z_halo)  # LATTICE_Z_HALO_LO | LATTICE_Z_HALO_HI for a slab with halo planes
        dims = list(dims) + [1] * (3 - len(dims))
        per = list(periodic) + [0] * (3 - len(periodic))
        for i in range(3):
            d.dims[i] = int(dims[i])
            d.periodic[i] = int(bool(per[i]))
        d.t, d.m, d.delta1, d.delta2 = float(t), float(m), float(delta1), float(delta2)
        d.k0 = float(k0)
        keep = None
        if qdots is not None:
            q = list(qdots) + [0.0] * (5 - len(qdots))
            d.v_source = V_QDOT
            d.qd_count, d.qd_radius, d.qd_V0, d.qd_width, d.qd_dV = (
                int(q[0]), float(q[1]), float(q[2]), float(q[3]), float(q[4]))
        elif disorder is not None:
            W, seed = disorder
            d.v_source = V_ON_THE_FLY if on_the_fly else V_SEED
            d.W, d.seed = float(W), int(seed)
        elif V is None:
            d.v_source = V_ZERO
        elif isinstance(V, torch.Tensor) and V.is_cuda:
            keep = V.to(torch.float64).contiguous()
            d.v_source, d.V = V_DEVICE, keep.data_ptr()
        else:
            import numpy as np
            keep = np.ascontiguousarray(np.asarray(V, dtype=np.float64))
            d.v_source, d.V = V_HOST, keep.ctypes.data
        h = ctypes.c_void_p()
        _check(_lib.pvsc_lattice_create(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
        self._h = h
        self.model = model
        self.dims = tuple(dims)
        self.periodic = tuple(per)
        self.t, self.m = float(t), float(m)
        n = ctypes.c_int64()
        o = ctypes.c_int32()
        _check(_lib.pvsc_lattice_info(self._h, ctypes.byref(n), ctypes.byref(o)))
        self.n_sites, self.orbitals = int(n.value), int(o.value)
        self.D = self.n_sites * self.orbitals

    @classmethod
    def ti(cls, dims, periodic, t=1.0, m=2.0, **kw):
        return cls(TI, dims, periodic, t=t, m=m, **kw)

    @classmethod
    def wsm(cls, dims, periodic, k0=math.pi / 2, **kw):
        """Two-band Weyl semimetal of Eq. TB_H_wsm (Weyl nodes at (+-k0, 0, 0)); Lx even."""
        return cls(WSM, dims, periodic, k0=k0, **kw)

    @classmethod
    def graphene(cls, cells, periodic, t=1.0, **kw):
        return cls(GRAPHENE, list(cells) + [1], list(periodic) + [0], t=t, **kw)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            _lib.pvsc_lattice_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def work_bytes(self, op: int, R: int, prec: int, M: int = 0) -> int:
        return int(_lib.pvsc_work_bytes(self._h, op, R, prec, M))

    def set_potential(self, V: torch.Tensor, stream=None):
        V = V.to(torch.float64).contiguous()
        _check(_lib.pvsc_set_potential(self._h, _ptr(V), _stream(stream)))

    def potential(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.n_sites, dtype=torch.float64, device="cuda")
        _check(_lib.pvsc_get_potential(self._h, _ptr(out), _stream(stream)))
        return out

    def spectral_bounds(self, eps: float = 0.01, stream=None):
        """(emin, emax, a, b): exact Gershgorin interval and the Chebyshev scaling."""
        w = work_buffer(self.work_bytes(OP_APPLY, 1, C128))
        emin, emax, a, b = _d(), _d(), _d(), _d()
        _check(_lib.pvsc_spectral_bounds(self._h, eps, ctypes.byref(emin), ctypes.byref(emax),
                                         ctypes.byref(a), ctypes.byref(b), _ptr(w), w.numel(),
                                         _stream(stream)))
        return emin.value, emax.value, a.value, b.value

    def neighbours(self, stream=None) -> torch.Tensor:
        n = self.n_sites if self.model == TI else self.dims[0] * self.dims[1]
        out = torch.empty((n, 7), dtype=torch.int64, device="cuda")
        _check(_lib.pvsc_debug_neighbours(self._h, _ptr(out), _stream(stream)))
        return out

    def export_pattern(self):
        """(rowptr, col) numpy arrays: the stencil's terms per row (pvsc_debug_export_pattern)."""
        import numpy as np
        rowptr = np.zeros(self.D + 1, dtype=np.int64)
        _check(_lib.pvsc_debug_export_pattern(self._h, rowptr.ctypes.data, None))
        col = np.zeros(int(rowptr[-1]), dtype=np.int32)
        _check(_lib.pvsc_debug_export_pattern(self._h, rowptr.ctypes.data, col.ctypes.data))
        return rowptr, col

    def set_tuning(self, R: int, prec: int, threads: int = 256, blocks_per_sm: int = 0,
                   zslab: int = 0, vpt: int = 0, tile_x: int = 0, tile_y: int = 0,
                   kernel: int = 0):
        t = Tuning(threads, blocks_per_sm, zslab, 0.0, vpt, tile_x, tile_y, kernel)
        _check(_lib.pvsc_set_tuning(self._h, R, prec, ctypes.byref(t)))

    def get_tuning(self, R: int, prec: int) -> dict:
        t = Tuning()
        _check(_lib.pvsc_get_tuning(self._h, R, prec, ctypes.byref(t)))
        return t.as_dict()

    def autotune(self, R: int, prec: int, op: int = OP_KPM, stream=None) -> dict:
        """Time the launch shapes with the sweeps of `op` (OP_KPM, OP_SERIES or
        OP_APPLY) and keep the fastest for (R, prec)."""
        t = Tuning()
        _check(_lib.pvsc_autotune_op(self._h, R, prec, int(op), ctypes.byref(t), _stream(stream)))
        return t.as_dict()


# ---------------------------------------------------------------------------- operations
def random_vectors(lat: Lattice, R: int, prec: int, seed: int, stream=None) -> torch.Tensor:
    """Random-phase block exp(2 pi i u)/sqrt(D) from the counter hash, shape (D, R)."""
    out = torch.empty((lat.D, R), dtype=torch.complex128 if prec == C128 else torch.complex64,
                      device="cuda")
    _check(_lib.pvsc_random_vectors(lat.handle, R, prec, int(seed), _ptr(out), _stream(stream)))
    return out


def apply_H(lat: Lattice, x: torch.Tensor, y: torch.Tensor | None = None, stream=None):
    """y = H x."""
    y = torch.empty_like(x) if y is None else y
    _check(_lib.pvsc_apply_H(lat.handle, block_R(x), prec_of(x), _ptr(x), _ptr(y), _stream(stream)))
    return y


def cheb_step(lat: Lattice, x, y, alpha, beta, gamma=None, z=None, delta=None, dots: int = 0,
              work: torch.Tensor | None = None, stream=None):
    """y <- alpha (H - beta) x + gamma y; z += delta y; returns the dots tensor [4, R] or None."""
    R, prec = block_R(x), prec_of(x)
    d = torch.zeros((4, R), dtype=torch.float64, device=x.device) if dots else None
    if dots and work is None:
        work = work_buffer(lat.work_bytes(OP_CHEB_STEP, R, prec))
    _check(_lib.pvsc_cheb_step(
        lat.handle, R, prec, _ptr(x), _ptr(y), _ptr(z), _darr(alpha), _darr(beta),
        _darr(gamma) if gamma is not None else None, _darr(delta) if delta is not None else None,
        int(dots), _ptr(d), _ptr(work), 0 if work is None else work.numel(), _stream(stream)))
    return d


def cheb_step_noalloc(lat: Lattice, x, y, alpha, beta, gamma=None, z=None, delta=None,
                      dots: int = 0, out_dots: torch.Tensor | None = None, stream=None):
    """cheb_step for callers that cannot allocate: no work buffer, the library's
    static scratch holds the dot partials.  out_dots (float64 [4, R] on the
    device) may be passed in so that this call allocates nothing either."""
    R, prec = block_R(x), prec_of(x)
    if dots and out_dots is None:
        out_dots = torch.zeros((4, R), dtype=torch.float64, device=x.device)
    _check(_lib.pvsc_cheb_step_noalloc(
        lat.handle, R, prec, _ptr(x), _ptr(y), _ptr(z), _darr(alpha), _darr(beta),
        _darr(gamma) if gamma is not None else None, _darr(delta) if delta is not None else None,
        int(dots), _ptr(out_dots) if dots else None, _stream(stream)))
    return out_dots if dots else None


def kpm_moments(lat: Lattice, M: int, a: float, b: float, R: int = 1, prec: int = C128,
                r0: torch.Tensor | None = None, seed: int = 0, work=None, mu=None, stream=None):
    """Per-vector KPM moments mu[r, k] = <r|T_k(H~)|r>, a float64 tensor (R, M)."""
    if r0 is not None:
        if prec == Q64 and r0.dtype != torch.complex128:
            raise PvscError(PVSC_ERR_ARG, "Q64 moments take a complex128 start block")
        R = block_R(r0)
        prec = Q64 if prec == Q64 else prec_of(r0)
    mu = torch.empty((R, M), dtype=torch.float64, device="cuda") if mu is None else mu
    if work is None:
        work = work_buffer(lat.work_bytes(OP_KPM, R, prec, M))
    _check(_lib.pvsc_kpm_moments(lat.handle, R, prec, _ptr(r0), int(seed), int(M), float(a),
                                 float(b), _ptr(mu), _ptr(work), work.numel(), _stream(stream)))
    return mu


def kpm_sweeps(lat: Lattice, k_begin: int, k_end: int, wa, wb, a, b, mu, work=None, stream=None):
    """KPM sweeps k_begin .. k_end-1 on caller-held vectors (pvsc_kpm_sweeps): w_j in wa
    for even j, in wb for odd j; moments into mu (float64 (R, M) on the device)."""
    R, prec = block_R(wa), prec_of(wa)
    if work is None:
        work = work_buffer(lat.work_bytes(OP_CHEB_STEP, R, prec))
    _check(_lib.pvsc_kpm_sweeps(lat.handle, R, prec, int(k_begin), int(k_end), _ptr(wa), _ptr(wb), float(a),
                                float(b), _ptr(mu), int(mu.shape[-1]), _ptr(work), work.numel(), _stream(stream)))
    return mu


def _cplx_arr(coeffs):
    flat = []
    for c in coeffs:
        c = complex(c)
        flat += [c.real, c.imag]
    return _darr(flat)


def cheb_series(lat: Lattice, x, coeffs, a, b, phase=None, y=None, prec: int = C128, work=None,
                stream=None):
    """y = phase sum_k coeffs_k T_k(H~) x (x, y complex128)."""
    R = block_R(x)
    y = torch.empty_like(x) if y is None else y
    K = len(coeffs)
    if work is None:
        work = work_buffer(lat.work_bytes(OP_SERIES, R, prec, K))
    ph = None if phase is None else _darr([complex(phase).real, complex(phase).imag])
    _check(_lib.pvsc_cheb_series(lat.handle, R, prec, _ptr(x), _ptr(y), _cplx_arr(coeffs), K, ph,
                                 float(a), float(b), _ptr(work), work.numel(), _stream(stream)))
    return y


def cheb_filter(lat: Lattice, x, g, a, b, y=None, prec: int = C128, work=None, stream=None):
    """y = sum_k g_k T_k(H~) x with real g (x, y complex128)."""
    R = block_R(x)
    y = torch.empty_like(x) if y is None else y
    if work is None:
        work = work_buffer(lat.work_bytes(OP_SERIES, R, prec, len(g)))
    _check(_lib.pvsc_cheb_filter(lat.handle, R, prec, _ptr(x), _ptr(y), _darr(g), len(g), float(a),
                                 float(b), _ptr(work), work.numel(), _stream(stream)))
    return y


def propagation_coeffs(a_dt: float, trunc: float = 1e-14):
    """Series weights cw_0 = J_0, cw_k = 2 (-i)^k J_k(a dt) of Eq. U_1 (list of complex)."""
    n = ctypes.c_int()
    buf = (ctypes.c_double * 512)()
    _check(_lib.pvsc_propagation_coeffs(float(a_dt), float(trunc), 256, buf, ctypes.byref(n)))
    return [complex(buf[2 * k], buf[2 * k + 1]) for k in range(n.value)]


def cheb_propagate(lat: Lattice, psi, dt, nsteps, a, b, trunc=1e-14, prec: int = C128, work=None,
                   stream=None):
    """psi <- U(dt)^nsteps psi in place (psi complex128)."""
    R = block_R(psi)
    if work is None:
        K = len(propagation_coeffs(a * dt, trunc))
        work = work_buffer(lat.work_bytes(OP_SERIES, R, prec, K))
    _check(_lib.pvsc_cheb_propagate(lat.handle, R, prec, _ptr(psi), float(dt), int(nsteps), float(a),
                                    float(b), float(trunc), _ptr(work), work.numel(), _stream(stream)))
    return psi


def cheb_adjoint_step(lat: Lattice, psi_s, G, dt, a, b, dLdV, trunc=1e-14, work=None, stream=None):
    """G <- dL/dpsi_s and dLdV += the potential gradient of one propagation step."""
    if work is None:
        K = len(propagation_coeffs(a * dt, trunc))
        work = work_buffer(lat.work_bytes(OP_ADJOINT, 1, C128, K))
    _check(_lib.pvsc_cheb_adjoint_step(lat.handle, block_R(psi_s), C128, _ptr(psi_s), _ptr(G), float(dt),
                                       float(a), float(b), float(trunc), _ptr(dLdV), _ptr(work),
                                       work.numel(), _stream(stream)))
    return G


def cheb_propagate_checkpointed(lat: Lattice, psi, dt, nsteps, every, a, b, trunc=1e-14, ckpts=None,
                                work=None, stream=None):
    """psi <- U(dt)^nsteps psi in place (complex128), keeping psi at steps 0, every,
    2 every, ... in ckpts (a complex128 tensor (nseg, D[, R]), allocated if None)."""
    R = block_R(psi)
    nseg = (int(nsteps) + int(every) - 1) // int(every)
    if ckpts is None:
        ckpts = torch.empty((max(nseg, 1),) + tuple(psi.shape), dtype=torch.complex128, device=psi.device)
    if work is None:
        K = len(propagation_coeffs(a * dt, trunc))
        work = work_buffer(lat.work_bytes(OP_SERIES, R, C128, K))
    _check(_lib.pvsc_cheb_propagate_checkpointed(
        lat.handle, R, C128, _ptr(psi), float(dt), int(nsteps), int(every), float(a), float(b), float(trunc),
        _ptr(ckpts), _ptr(work), work.numel(), _stream(stream)))
    return psi, ckpts


def cheb_propagate_adjoint(lat: Lattice, ckpts, G, dt, nsteps, every, a, b, dLdV, trunc=1e-14, work=None,
                           stream=None):
    """G <- dL/dpsi_0 and dLdV += dL/dV of the whole checkpointed propagation
    (G holds dL/dpsi_nsteps on entry)."""
    if work is None:
        nb = int(_lib.pvsc_propagate_adjoint_work_bytes(lat.handle, 1, int(every), float(a * dt), float(trunc)))
        work = work_buffer(nb)
    _check(_lib.pvsc_cheb_propagate_adjoint(
        lat.handle, block_R(G), C128, _ptr(ckpts), float(dt), int(nsteps), int(every), float(a), float(b),
        float(trunc), _ptr(G), _ptr(dLdV), _ptr(work), work.numel(), _stream(stream)))
    return G


def kpm_density(mu: torch.Tensor, E: torch.Tensor, a: float, b: float, kernel: int = KERNEL_JACKSON,
                lam: float = 4.0, scale: float = 1.0, out: torch.Tensor | None = None, stream=None):
    """rho(E) = scale sum_r [g_0 mu_0^r + 2 sum_k g_k mu_k^r T_k(x)] / (pi a sqrt(1 - x^2)), x = (E-b)/a,
    from per-vector moments mu (R, M) (float64, on the device) on energies E (float64)."""
    mu = mu.to(torch.float64).contiguous()
    R, M = mu.shape
    E = E.to(device=mu.device, dtype=torch.float64).contiguous()
    out = torch.empty_like(E) if out is None else out
    _check(_lib.pvsc_kpm_density(R, M, _ptr(mu), int(kernel), float(lam), float(a), float(b),
                                 float(scale), E.numel(), _ptr(E), _ptr(out), _stream(stream)))
    return out


def dos(lat: Lattice, mu: torch.Tensor, E, a, b, kernel: int = KERNEL_JACKSON, lam: float = 4.0):
    """DOS(E) of Eq. DOS from the stochastic-trace moments of R random vectors (integrates to D)."""
    return kpm_density(mu, torch.as_tensor(E, dtype=torch.float64, device="cuda"), a, b, kernel, lam,
                       scale=lat.D / mu.shape[0])


def bloch_vectors(lat: Lattice, ks, prec: int = C128, stream=None) -> torch.Tensor:
    """The states psi(k, nu) of Eq. ak for up to 16 k-points: a (D, O nk) block, vector O q + nu
    (O = orbitals per site: TI 4, Weyl semimetal 2)."""
    ks = [tuple(float(c) for c in k) + (0.0,) * (3 - len(k)) for k in ks]
    nk = len(ks)
    out = torch.empty((lat.D, lat.orbitals * nk), dtype=torch.complex128 if prec == C128 else torch.complex64,
                      device="cuda")
    flat = (ctypes.c_double * (3 * nk))(*[c for k in ks for c in k])
    _check(_lib.pvsc_bloch_vectors(lat.handle, nk, flat, prec, _ptr(out), _stream(stream)))
    return out


def spectral_function(lat: Lattice, ks, M: int, a, b, E, prec: int = C64,
                      kernel: int = KERNEL_JACKSON, lam: float = 4.0, work=None) -> torch.Tensor:
    """A(k, E) of Eq. ak for up to 16 k-points: KPM moments of the O states psi(k, nu) of each
    k-point (one call, R = O nk), summed per k-point; returns (nk, NE) float64."""
    psi = bloch_vectors(lat, ks, prec)
    mu = kpm_moments(lat, M, a, b, r0=psi, work=work)
    E = torch.as_tensor(E, dtype=torch.float64, device="cuda")
    O = lat.orbitals
    return torch.stack([kpm_density(mu[O * q:O * q + O], E, a, b, kernel, lam) for q in range(len(ks))])


class ChebFDParams(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double), ("hi", ctypes.c_double), ("n_search", ctypes.c_int32),
                ("degree", ctypes.c_int32), ("max_iter", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("tol", ctypes.c_double), ("seed", ctypes.c_uint64)]


def chebfd(lat: Lattice, lo: float, hi: float, a: float, b: float, n_search: int = 64,
           degree: int = 500, max_iter: int = 30, tol: float = 1e-10, prec: int = C128,
           seed: int = 1, stream=None):
    """Chebyshev filter diagonalization: the eigenpairs of H in [lo, hi].  Returns
    (theta, resid, X, n_inside, iterations): all n_search Ritz values (ascending, numpy),
    their residual norms, the Ritz vectors (complex128 (D, n_search) on the device)."""
    prm = ChebFDParams(float(lo), float(hi), int(n_search), int(degree), int(max_iter), int(prec),
                       float(tol), int(seed))
    X = torch.empty((lat.D, n_search), dtype=torch.complex128, device="cuda")
    work = work_buffer(_lib.pvsc_chebfd_work_bytes(lat.handle, n_search, prec, degree))
    theta = (ctypes.c_double * n_search)()
    resid = (ctypes.c_double * n_search)()
    n_in, iters = ctypes.c_int(), ctypes.c_int()
    _check(_lib.pvsc_chebfd(lat.handle, ctypes.byref(prm), float(a), float(b), _ptr(X), theta, resid,
                            ctypes.byref(n_in), ctypes.byref(iters), _ptr(work), work.numel(),
                            _stream(stream)))
    return np.array(theta[:]), np.array(resid[:]), X, n_in.value, iters.value


def kpm_moments_batched(lats, M, a, b, R=16, prec=C64, seeds=None, work=None, mu=None, stream=None):
    """Batched KPM over several TI lattices in one persistent launch: mu (n, R, M)."""
    n = len(lats)
    hs = (ctypes.c_void_p * n)(*[l.handle.value for l in lats])
    seeds = list(seeds) if seeds is not None else list(range(n))
    sarr = (ctypes.c_uint64 * n)(*[int(s) for s in seeds])
    mu = torch.empty((n, R, M), dtype=torch.float64, device="cuda") if mu is None else mu
    if work is None:
        work = work_buffer(int(_lib.pvsc_batched_work_bytes(hs, n, R, prec, M)))
    _check(_lib.pvsc_kpm_moments_batched(hs, n, R, prec, sarr, int(M), _darr(a), _darr(b), _ptr(mu),
                                         _ptr(work), work.numel(), _stream(stream)))
    return mu


def autotune_batched(lats, M, a, b, R=16, prec=C64, seeds=None, stream=None) -> dict:
    """Tune the batched KPM's launch shape on the batch itself (pvsc_autotune_batched)."""
    n = len(lats)
    hs = (ctypes.c_void_p * n)(*[l.handle.value for l in lats])
    seeds = list(seeds) if seeds is not None else list(range(n))
    sarr = (ctypes.c_uint64 * n)(*[int(s) for s in seeds])
    t = Tuning()
    _check(_lib.pvsc_autotune_batched(hs, n, R, prec, sarr, int(M), _darr(a), _darr(b), ctypes.byref(t),
                                      _stream(stream)))
    return t.as_dict()


def device_error(clear: bool = True) -> int:
    """The device error word of the staged sweeps (1 if a copy wait ran out since
    the last clear; the sweep's outputs are then invalid).  Synchronises the device."""
    flag = ctypes.c_int(0)
    _check(_lib.pvsc_device_error(ctypes.byref(flag), int(bool(clear))))
    return int(flag.value)


def debug_series_plan(K: int) -> list:
    """Terms each recurrence sweep of a K-term series adds to its accumulator
    (pvsc_debug_series_plan, host only)."""
    out = (ctypes.c_int * max(K, 1))()
    _check(_lib.pvsc_debug_series_plan(K, ctypes.cast(out, ctypes.c_void_p)))
    return list(out)[:K]


def debug_fx_arith(op: int, values, stream=None):
    """The fixed-point sweep arithmetic on given int64 operands (pvsc_debug_fx_arith).
    op 0: values (n, 4) = (c1, x1, c2, x2) -> (n,) rounded updates; op 1: values
    (n, 16) = (x_0..7, y_0..7) -> (4,) exact sums (hi, lo) of x^2 and y x.
    values: a CUDA int64 tensor."""
    v = values.contiguous()
    if v.dtype != torch.int64 or not v.is_cuda:
        raise PvscError(PVSC_ERR_ARG, "values must be a CUDA int64 tensor")
    width = 4 if op == 0 else 16
    if v.dim() != 2 or v.shape[1] != width:
        raise PvscError(PVSC_ERR_ARG, f"values must have shape (n, {width})")
    n = v.shape[0]
    out = torch.zeros((n if op == 0 else 4,), dtype=torch.int64, device=v.device)
    _check(_lib.pvsc_debug_fx_arith(int(op), _ptr(v) if n else None, n, _ptr(out), _stream(stream)))
    return out


def set_wait_limit(spins: int):
    _check(_lib.pvsc_set_wait_limit(int(spins)))


def inject_stall(enable: bool):
    """Fault injection: make the batched kernel's first wait target an unpublished phase."""
    _check(_lib.pvsc_debug_inject_stall(int(bool(enable))))


def batched_work_bytes(lats, R, prec, M) -> int:
    hs = (ctypes.c_void_p * len(lats))(*[l.handle.value for l in lats])
    return int(_lib.pvsc_batched_work_bytes(hs, len(lats), R, prec, M))


def library_path() -> str:
    return LIB_PATH


from .autograd import ChebPropagate, propagate_with_grad  # noqa: E402,F401
