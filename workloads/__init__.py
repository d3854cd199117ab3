"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module produces *inputs* only: lattice sizes, on-site disorder, start
vectors, the gate-defined quantum-dot potential and the Gaussian wave packet.
It holds none of the arithmetic of the method itself (no Hamiltonian
application, no Chebyshev recurrence, no moment or gradient computation), so
both the CPU oracle and the CUDA library can consume what it produces without
sharing any code with one another.

Random numbers come from a counter-based generator so that every value depends
only on (seed, stream, index) and can be regenerated anywhere, in any order:

    mix(z)   = SplitMix64 output finaliser (Steele, Lea & Flood, OOPSLA 2014):
               z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
               z ^= z >> 27; z *= 0x94D049BB133111EB;
               z ^= z >> 31
    h        = mix(mix(seed ^ (stream * 0x9E3779B97F4A7C15)) + idx)   (mod 2^64)
    u        = (h >> 11) * 2^-53                      in [0, 1), exact in fp64

Streams: 0 = on-site disorder (idx = site), 1 = random-phase start vectors
(idx = r * D + i), 2 = complex Gaussian vectors (Box-Muller on idx 2j, 2j+1).

The paper draws its disorder from per-thread xorshift streams (Sec. 3.3); a
counter-based mix replaces them because it needs no sequential state, which is
what a GPU thread that regenerates V_n on the fly needs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_DISORDER = 0
STREAM_PHASE = 1
STREAM_GAUSS = 2

TI_ORBITALS = 4
GRAPHENE_SITES_PER_CELL = 4


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on uint64 arrays (wrap-around arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = z ^ (z >> np.uint64(30))
        z = z * _M1
        z = z ^ (z >> np.uint64(27))
        z = z * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def hash64(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Counter-based 64-bit hash h(seed, stream, idx)."""
    with np.errstate(over="ignore"):
        key = np.uint64(seed) ^ (np.uint64(stream) * GOLDEN_GAMMA)
        k = mix64(np.array([key], dtype=np.uint64))[0]
        return mix64(np.asarray(idx, dtype=np.uint64) + k)


def uniform(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1): the top 53 bits of the hash times 2^-53."""
    h = hash64(seed, stream, idx)
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def disorder_potential(n_sites: int, W: float, seed: int) -> np.ndarray:
    """Box-distributed on-site disorder V_n = W (u_n - 1/2), V_n in [-W/2, W/2).

    The paper draws V_n uniformly from [-gamma/2, gamma/2] (Sec. 4.2, Fig. 10;
    Sec. 4.3).  (u - 1/2) is exact in fp64 and the product is rounded once, so
    any implementation of the same formula yields identical bits.
    """
    u = uniform(seed, STREAM_DISORDER, np.arange(n_sites, dtype=np.uint64))
    return W * (u - 0.5)


def random_phase_block(D: int, R: int, seed: int) -> np.ndarray:
    """R random-phase vectors r_i = exp(2 pi i u) / sqrt(D), shape (D, R).

    Element (i, r) uses idx = r * D + i, so each vector is independent of R.
    With unit-modulus entries scaled by 1/sqrt(D), <r|r> = 1 and mu_0 = 1.
    """
    i = np.arange(D, dtype=np.uint64)[:, None]
    r = np.arange(R, dtype=np.uint64)[None, :]
    u = uniform(seed, STREAM_PHASE, r * np.uint64(D) + i)
    return np.exp(2j * np.pi * u) / math.sqrt(D)


def gaussian_block(D: int, R: int, seed: int) -> np.ndarray:
    """Complex Gaussian vectors (g1 + i g2)/sqrt(2) by Box-Muller, shape (D, R)."""
    i = np.arange(D, dtype=np.uint64)[:, None]
    r = np.arange(R, dtype=np.uint64)[None, :]
    j = r * np.uint64(D) + i
    u1 = uniform(seed, STREAM_GAUSS, np.uint64(2) * j)
    u2 = uniform(seed, STREAM_GAUSS, np.uint64(2) * j + np.uint64(1))
    rad = np.sqrt(-2.0 * np.log1p(-u1))
    return (rad * np.cos(2 * np.pi * u2) + 1j * rad * np.sin(2 * np.pi * u2)) / math.sqrt(2.0)


# ----------------------------------------------------------------------------
# Graphene geometry (4-site rectangular cell of Eq. graphene_model)
# ----------------------------------------------------------------------------
SQRT3 = math.sqrt(3.0)
# In-cell offsets (physical X, physical Y) of the 4 carbon sites, in units of
# the C-C distance.  The cell axis "x" (fastest index) runs along physical Y
# with period sqrt(3); the cell axis "y" runs along physical X with period 3.
# With these offsets every bond of Eq. graphene_model has length exactly 1.
_CELL_OFFSETS = np.array(
    [[0.0, SQRT3 / 2], [0.5, 0.0], [1.5, 0.0], [2.0, SQRT3 / 2]], dtype=np.float64
)


def graphene_positions(Nx: int, Ny: int) -> tuple[np.ndarray, np.ndarray]:
    """Physical (X, Y) of every site, site index = 4 (x + Nx y) + nu."""
    cx = np.arange(Nx, dtype=np.float64)
    cy = np.arange(Ny, dtype=np.float64)
    CX, CY = np.meshgrid(cx, cy, indexing="xy")  # shape (Ny, Nx): c = x + Nx y
    X = 3.0 * CY[..., None] + _CELL_OFFSETS[None, None, :, 0]
    Y = SQRT3 * CX[..., None] + _CELL_OFFSETS[None, None, :, 1]
    return X.reshape(-1), Y.reshape(-1)


def graphene_extent(Nx: int, Ny: int) -> tuple[float, float]:
    return 3.0 * Ny, SQRT3 * Nx


def qdot_potential(Nx: int, Ny: int, ndots: int, R_dot: float, V0: float,
                   w: float, dV: float = 0.0) -> np.ndarray:
    """Gate-defined quantum-dot array potential (Eq. qdotarray), per site.

    V(r) = sum_{l,k} V_k * S(R_dot - |R_{l,k} - r|) with V_k = V0 + dV |k - K/2|
    and a tanh-smoothed step S(s) = (1 + tanh(s / w)) / 2 in place of Theta.
    Dots sit on a square grid of spacing D_dot = 4 R_dot (the paper's 10 nm
    radius : 40 nm spacing), centred in the sample.
    """
    Xe, Ye = graphene_extent(Nx, Ny)
    Xc, Yc = Xe / 2.0, Ye / 2.0
    D_dot = 4.0 * R_dot
    # S is evaluated within R_dot + 20 w of each dot centre and taken as 0 beyond,
    # where it is below exp(-40) V0 (about 4e-18 V0).
    r_cut = R_dot + 20.0 * w
    V = np.zeros((Ny, Nx, 4))
    for l in range(ndots):
        for k in range(ndots):
            Rx = Xc + (l - (ndots - 1) / 2.0) * D_dot
            Ry = Yc + (k - (ndots - 1) / 2.0) * D_dot
            Vk = V0 + dV * abs(k - ndots / 2.0)
            cy0 = max(int(np.floor((Rx - r_cut - 2.0) / 3.0)), 0)
            cy1 = min(int(np.ceil((Rx + r_cut) / 3.0)) + 1, Ny)
            cx0 = max(int(np.floor((Ry - r_cut - SQRT3) / SQRT3)), 0)
            cx1 = min(int(np.ceil((Ry + r_cut) / SQRT3)) + 1, Nx)
            if cy0 >= cy1 or cx0 >= cx1:
                continue
            CY, CX = np.meshgrid(np.arange(cy0, cy1, dtype=np.float64),
                                 np.arange(cx0, cx1, dtype=np.float64), indexing="ij")
            X = 3.0 * CY[..., None] + _CELL_OFFSETS[None, None, :, 0]
            Y = SQRT3 * CX[..., None] + _CELL_OFFSETS[None, None, :, 1]
            d = np.hypot(X - Rx, Y - Ry)
            S = np.where(d < r_cut, 0.5 * (1.0 + np.tanh((R_dot - d) / w)), 0.0)
            V[cy0:cy1, cx0:cx1, :] += Vk * S
    return V.reshape(-1)


def dirac_point() -> tuple[float, float]:
    """A zero of f(k) = sum_delta exp(i k.delta), delta in {(-1,0), (1/2, +-sqrt3/2)}."""
    return 0.0, 4.0 * math.pi / (3.0 * SQRT3)


def gaussian_packet(Nx: int, Ny: int, x0: float, y0: float, sigma: float,
                    q: float) -> np.ndarray:
    """Gaussian wave packet of Eq. qgauwp, shape (4 Nx Ny,), normalised.

    psi(r) = exp(-|r - r0|^2 / (4 sigma^2)) * u_s * exp(i k0.r), with
    k0 = K + (q, 0) near the Dirac point K and the upper-band spinor
    u_A = 1, u_B = -conj(f(k0)) / |f(k0)|, so the packet moves along +X.
    """
    X, Y = graphene_positions(Nx, Ny)
    Kx, Ky = dirac_point()
    kx, ky = Kx + q, Ky
    deltas = [(-1.0, 0.0), (0.5, SQRT3 / 2), (0.5, -SQRT3 / 2)]
    f = sum(np.exp(1j * (kx * dx + ky * dy)) for dx, dy in deltas)
    uB = -np.conj(f) / abs(f)
    nu = np.tile(np.arange(4), Nx * Ny)
    spinor = np.where((nu == 0) | (nu == 2), 1.0 + 0j, uB)
    env = np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (4.0 * sigma ** 2))
    psi = env * spinor * np.exp(1j * (kx * X + ky * Y))
    return psi / np.linalg.norm(psi)


def detector_mask(Nx: int, Ny: int, x_lo: float, width: float, y_c: float,
                  height: float) -> np.ndarray:
    """Boolean per-site mask of the detector rectangle [x_lo, x_lo+width) x [y_c-h/2, y_c+h/2)."""
    X, Y = graphene_positions(Nx, Ny)
    return (X >= x_lo) & (X < x_lo + width) & (Y >= y_c - height / 2) & (Y < y_c + height / 2)


# ----------------------------------------------------------------------------
# Workload definitions (sizes, seeds, tolerances) of the five configurations
# ----------------------------------------------------------------------------
@dataclass
class TIConfig:
    dims: tuple[int, int, int]
    periodic: tuple[int, int, int]
    t: float = 1.0
    m: float = 2.0
    W: float = 1.0
    seed_V: int = 1
    seed_r: int = 3
    R: int = 1
    M: int = 256

    @property
    def n_sites(self) -> int:
        return self.dims[0] * self.dims[1] * self.dims[2]

    @property
    def D(self) -> int:
        return TI_ORBITALS * self.n_sites


@dataclass
class GrapheneConfig:
    cells: tuple[int, int]
    periodic: tuple[int, int] = (0, 0)
    t: float = 1.0
    ndots: int = 8
    R_dot: float = 40.0
    V0: float = 0.1
    w: float = 5.0
    sigma: float = 50.0
    q: float = 0.05
    packet_offset: float = 750.0
    dt: float = 1.0
    nsteps: int = 500
    trunc: float = 1e-14

    @property
    def n_sites(self) -> int:
        return GRAPHENE_SITES_PER_CELL * self.cells[0] * self.cells[1]

    def potential(self) -> np.ndarray:
        return qdot_potential(self.cells[0], self.cells[1], self.ndots, self.R_dot,
                              self.V0, self.w)

    def packet(self) -> np.ndarray:
        Xe, Ye = graphene_extent(*self.cells)
        return gaussian_packet(self.cells[0], self.cells[1], Xe / 2 - self.packet_offset,
                               Ye / 2, self.sigma, self.q)

    def detector(self) -> np.ndarray:
        Xe, Ye = graphene_extent(*self.cells)
        return detector_mask(self.cells[0], self.cells[1], Xe / 2, 100.0, Ye / 2, 100.0)


# 16^3 periodic TI, one H.v and 256 KPM moments with one random-phase vector.
CONFIG_TI_CUBE = TIConfig(dims=(16, 16, 16), periodic=(1, 1, 1), W=1.0, seed_V=1, R=1, M=256)
# TI slab 256x256x64, periodic in x, y and open in z; W in {0,2,4}; R in {1..32}.
CONFIG_TI_SLAB = TIConfig(dims=(256, 256, 64), periodic=(1, 1, 0), W=2.0, seed_V=2, R=8, M=2048)
TI_SLAB_W = (0.0, 2.0, 4.0)
TI_SLAB_R = (1, 4, 8, 16, 32)
# Graphene QD-array propagation: 4096 x 2048 four-site cells (2^25 sites), open.
CONFIG_GRAPHENE_QD = GrapheneConfig(cells=(4096, 2048))
# Adjoint workload: 1024 x 512 four-site cells (2^21 sites), 4x4 dots of radius 30.
CONFIG_GRAPHENE_ADJ = GrapheneConfig(cells=(1024, 512), ndots=4, R_dot=30.0,
                                     packet_offset=250.0, nsteps=200)
ADJ_CHECKPOINT_EVERY = 20
ADJ_FD_SITES = 32
ADJ_FD_SEED = 5
ADJ_FD_H = 1e-6


def batched_lattices(n: int = 64, seed: int = 4,
                     sizes=(24, 32, 48, 64, 96), Wmax: float = 5.0):
    """The batched-KPM workload: n periodic TI cubes of edge L drawn from sizes, W ~ U[0, Wmax).

    Returns a list of (L, W, seed_V) with per-lattice disorder seeds.
    """
    idx = np.arange(n, dtype=np.uint64)
    uL = uniform(seed, 3, idx)
    uW = uniform(seed, 4, idx)
    out = []
    for i in range(n):
        L = sizes[min(int(uL[i] * len(sizes)), len(sizes) - 1)]
        out.append((L, float(Wmax * uW[i]), 1000 + i))
    return out
