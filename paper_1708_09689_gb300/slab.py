"""Domain decomposition of one TI lattice into z-slabs, one per rank.

The paper runs a lattice too large for one socket by splitting it into
domains, one per process, each updating its part of every vector and
exchanging one layer of next-neighbour halo sites with its neighbours before
each stencil sweep (Sec. 3.4).  Here the split is along z, the slowest index
of the site-major layout, so a plane of a vector block is one contiguous
span and a halo exchange is two contiguous sends and two contiguous receives
per sweep.

Rank r owns the planes [z0, z1) of the global Lx x Ly x Lz lattice (sizes
differ by at most one plane) and a local lattice of its nz planes plus one
halo plane on each side that has a neighbouring slab (none at an open end of
the global lattice), created with the library's PVSC_LATTICE_Z_HALO_LO / _HI
flags: the library reads a halo plane as a z-neighbour but updates, writes
and reduces only the slab's own planes.  Before sweep k the rank sends its
first and last own plane of w_k to the slabs below and above (a ring when z
is periodic) and receives theirs into its halo planes.  The
KPM moments are linear in the per-slab dot products (mu_2k = 2 <w_k|w_k> -
mu_0, mu_2k+1 = 2 Re <w_k+1|w_k> - mu_1), so each slab's moments add up to
the global ones: one all-reduce (fp64, sum) of mu[R][M] at the end and no
per-sweep global reduction.  The spectral interval is the min / max of the
slabs' Gershgorin intervals.

The halo exchange goes through a transport: TorchDistTransport (point-to-point
sends and receives of torch.distributed, NCCL between GPUs) by default.  This
module holds no stencil arithmetic: the sweeps are the library's
(pvsc_kpm_sweeps on the slab's lattice) unless a caller passes its own.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch
import torch.distributed as dist


@dataclass(frozen=True)
class SlabPartition:
    """The planes of one rank's slab of a TI lattice split along z."""
    dims: tuple
    periodic: tuple
    world: int
    rank: int

    def __post_init__(self):
        Lz = int(self.dims[2])
        if not (0 <= self.rank < self.world):
            raise ValueError(f"rank {self.rank} outside world of {self.world}")
        if Lz < self.world:
            raise ValueError(f"{Lz} planes cannot be split over {self.world} ranks")

    @property
    def z0(self) -> int:
        return self.rank * int(self.dims[2]) // self.world

    @property
    def z1(self) -> int:
        return (self.rank + 1) * int(self.dims[2]) // self.world

    @property
    def nz(self) -> int:
        return self.z1 - self.z0

    @property
    def below(self):
        """Rank holding the plane below this slab, None at an open end."""
        if self.rank > 0:
            return self.rank - 1
        return self.world - 1 if self.periodic[2] else None

    @property
    def above(self):
        if self.rank < self.world - 1:
            return self.rank + 1
        return 0 if self.periodic[2] else None

    @property
    def lo(self) -> int:
        """1 if the slab has a halo plane below its planes (local plane 0)."""
        return 0 if self.below is None else 1

    @property
    def hi(self) -> int:
        """1 if the slab has a halo plane above its planes (local plane lo + nz)."""
        return 0 if self.above is None else 1

    @property
    def halo_flags(self) -> int:
        """The library's lattice flags: PVSC_LATTICE_Z_HALO_LO (1) | _HI (2)."""
        return self.lo | (self.hi << 1)

    @property
    def local_dims(self) -> tuple:
        """The slab's lattice: its planes plus its halo planes."""
        return (int(self.dims[0]), int(self.dims[1]), self.lo + self.nz + self.hi)

    @property
    def local_periodic(self) -> tuple:
        return (int(self.periodic[0]), int(self.periodic[1]), 0)

    @property
    def plane_sites(self) -> int:
        return int(self.dims[0]) * int(self.dims[1])

    def global_planes(self) -> list:
        """Global plane index of each local plane (halo planes wrapped around a periodic axis)."""
        Lz = int(self.dims[2])
        return [z % Lz for z in range(self.z0 - self.lo, self.z1 + self.hi)]

    def local_rows(self, global_block, orbitals: int = 4):
        """This slab's rows (halo planes included) of a global block of shape
        (D, ...) in the library layout."""
        P = self.plane_sites * orbitals
        return torch.cat([global_block[z * P:(z + 1) * P] for z in self.global_planes()], dim=0)

    def inner_rows(self, local_block, orbitals: int = 4):
        """The rows of the slab's own planes (halo planes dropped)."""
        P = self.plane_sites * orbitals
        return local_block[self.lo * P:(self.lo + self.nz) * P]


class TorchDistTransport:
    """Halo planes and reductions over torch.distributed (NCCL or gloo)."""

    def exchange(self, sends, recvs):
        """sends: [(tensor, peer)], recvs: [(tensor, peer)], matched in posting
        order between every pair of ranks."""
        ops = [dist.P2POp(dist.isend, t, peer) for t, peer in sends]
        ops += [dist.P2POp(dist.irecv, t, peer) for t, peer in recvs]
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()

    def all_reduce(self, t, op: str):
        red = {"sum": dist.ReduceOp.SUM, "min": dist.ReduceOp.MIN, "max": dist.ReduceOp.MAX}[op]
        if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
            dist.all_reduce(t, op=red)
        return t


def halo_exchange(part: SlabPartition, w, transport, orbitals: int = 4):
    """Fill the halo planes of the slab's block w (shape (D_local, ...)) with
    the neighbouring slabs' boundary planes: the plane below the slab into
    local plane 0, the plane above it into the last local plane."""
    P = part.plane_sites * orbitals
    lo, nz = part.lo, part.nz
    first, last = w[lo * P:(lo + 1) * P], w[(lo + nz - 1) * P:(lo + nz) * P]
    lower = w[0:P] if lo else None
    upper = w[(lo + nz) * P:(lo + nz + 1) * P] if part.hi else None
    below, above = part.below, part.above
    if part.world == 1:  # one periodic slab: its own planes wrap around
        if lower is not None:
            lower.copy_(last)
            upper.copy_(first)
        return
    # sends and receives are matched in posting order per pair of ranks: the
    # last plane goes up before the first goes down, and the halo below is
    # received before the halo above (two ranks on a periodic axis are each
    # other's neighbour on both sides)
    sends = [(last, above)] if above is not None else []
    sends += [(first, below)] if below is not None else []
    recvs = [(lower, below)] if below is not None else []
    recvs += [(upper, above)] if above is not None else []
    transport.exchange(sends, recvs)


def spectral_interval(local_emin: float, local_emax: float, transport, device=None):
    """The global Gershgorin interval from the slabs' intervals."""
    lo = torch.tensor([local_emin], dtype=torch.float64, device=device)
    hi = torch.tensor([local_emax], dtype=torch.float64, device=device)
    transport.all_reduce(lo, "min")
    transport.all_reduce(hi, "max")
    return float(lo.item()), float(hi.item())


def kpm_moments(part: SlabPartition, M: int, a: float, b: float, r0, transport=None, sweep=None,
                lat=None, work=None):
    """Global KPM moments mu (R, M) of a z-split lattice, on every rank.

    r0: this slab's start block (D_local, R) (its halo planes are overwritten).
    sweep(k, wa, wb, mu): one KPM sweep of the slab (w_j in wa for even j, in
    wb for odd j); by default the library's pvsc_kpm_sweeps on `lat`, the
    slab's lattice (local_dims, local_periodic, halo_flags)."""
    transport = transport or TorchDistTransport()
    if sweep is None:
        from . import kpm_sweeps  # the library (needs the built extension)

        def sweep(k, wa, wb, mu):
            kpm_sweeps(lat, k, k + 1, wa, wb, a, b, mu, work=work)
    wa = r0.clone().contiguous()
    wb = torch.zeros_like(wa)
    R = 1 if wa.dim() == 1 else wa.shape[1]
    mu = torch.zeros((R, M), dtype=torch.float64, device=wa.device)
    for k in range((M + 1) // 2):
        halo_exchange(part, wa if k % 2 == 0 else wb, transport)
        sweep(k, wa, wb, mu)
    return transport.all_reduce(mu, "sum")
