"""z-slab lattices with halo planes and the per-sweep KPM entry point on the GPU.

One process drives several slabs of one lattice on the one GPU: the slab
driver's halo exchange (paper_1708_09689_gb300/slab.py) moves the boundary
planes between them through an in-process transport, and every slab sweeps
its own lattice (PVSC_LATTICE_Z_HALO_LO / _HI) with pvsc_kpm_sweeps.  Summed
over the slabs, the moments must equal the single-lattice library moments and
the oracle; the slabs' spectral bounds must give the global Gershgorin
interval.  Resumable KPM: sweeps split over two calls equal one call bit for bit.
"""
from collections import defaultdict

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

pv = pytest.importorskip("paper_1708_09689_gb300")
from paper_1708_09689_gb300 import slab as S  # noqa: E402


class _Hub:
    """In-process transport: sends and receives of all slabs of one exchange,
    matched per pair of slabs in posting order (as point-to-point messages are)."""

    def __init__(self):
        self.pending = []

    def view(self, rank):
        hub = self

        class _View:
            def exchange(self, sends, recvs):
                hub.pending.append((rank, sends, recvs))
        return _View()

    def flush(self):
        queues = defaultdict(list)
        for rank, sends, _ in self.pending:
            for t, peer in sends:
                queues[(rank, peer)].append(t)
        for rank, _, recvs in self.pending:
            for t, peer in recvs:
                t.copy_(queues[(peer, rank)].pop(0))
        assert all(not q for q in queues.values())
        self.pending.clear()


@pytest.mark.parametrize("dims,per,world", [((6, 5, 9), (1, 1, 0), 2), ((6, 5, 9), (1, 0, 1), 3),
                                            ((8, 4, 7), (0, 1, 1), 2), ((5, 6, 8), (1, 1, 1), 4)])
@pytest.mark.parametrize("prec,tol", [(pv.C128, 1e-12), (pv.C64, 1e-5)])
def test_slabs_with_halo_exchange_reproduce_the_whole_lattice(dims, per, world, prec, tol):
    n = int(np.prod(dims))
    V = W.disorder_potential(n, 2.0, 6)
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V)
    gmin, gmax = O.gershgorin(H)
    a, b = O.cheb_scale(gmin, gmax)
    R, M = 4, 30
    r = W.random_phase_block(4 * n, R, 8)
    cdt = torch.complex128 if prec == pv.C128 else torch.complex64
    whole = pv.Lattice.ti(dims, per, V=V)
    mu_whole = pv.kpm_moments(whole, M, a, b, r0=torch.from_numpy(r).to("cuda", cdt)).cpu().numpy()
    parts = [S.SlabPartition(dims, per, world, k) for k in range(world)]
    Vt, rt = torch.from_numpy(V), torch.from_numpy(r)
    lats, wa, wb, mus, lo, hi = [], [], [], [], [], []
    for p in parts:
        lat = pv.Lattice.ti(p.local_dims, p.local_periodic, V=p.local_rows(Vt, orbitals=1).numpy(),
                            z_halo=p.halo_flags)
        lats.append(lat)
        wa.append(p.local_rows(rt).to("cuda", cdt).contiguous())
        wb.append(torch.zeros_like(wa[-1]))
        mus.append(torch.zeros((R, M), dtype=torch.float64, device="cuda"))
        emin, emax, _, _ = lat.spectral_bounds()
        lo.append(emin)
        hi.append(emax)
    assert abs(min(lo) - gmin) < 1e-12 and abs(max(hi) - gmax) < 1e-12
    hub = _Hub()
    for k in range((M + 1) // 2):
        for i, p in enumerate(parts):
            S.halo_exchange(p, wa[i] if k % 2 == 0 else wb[i], hub.view(i))
        hub.flush()
        for i in range(world):
            pv.kpm_sweeps(lats[i], k, k + 1, wa[i], wb[i], a, b, mus[i])
    mu = sum(m.cpu().numpy() for m in mus)
    assert np.max(np.abs(mu - mu_whole)) < tol
    ref = O.kpm_moments(H, r, M, a, b).real
    assert np.max(np.abs(mu - ref)) / ref[0, 0] < (1e-12 if prec == pv.C128 else 1e-4)


@pytest.mark.parametrize("prec", [pv.C128, pv.C64])
def test_kpm_sweeps_resume_bit_for_bit(prec):
    dims, per = (10, 8, 6), (1, 1, 0)
    lat = pv.Lattice.ti(dims, per, disorder=(1.5, 3))
    _, _, a, b = lat.spectral_bounds()
    R, M = 2, 41
    cdt = torch.complex128 if prec == pv.C128 else torch.complex64
    r0 = pv.random_vectors(lat, R, prec, 11)
    runs = []
    for cuts in ([0, 21], [0, 7, 21], [0, 1, 2, 13, 21]):
        wa, wb = r0.clone(), torch.zeros_like(r0)
        mu = torch.zeros((R, M), dtype=torch.float64, device="cuda")
        for k0, k1 in zip(cuts[:-1], cuts[1:]):
            pv.kpm_sweeps(lat, k0, k1, wa, wb, a, b, mu)
        runs.append((mu.clone(), wa.clone(), wb.clone()))
    for mu, wa, wb in runs[1:]:
        assert torch.equal(mu, runs[0][0]) and torch.equal(wa, runs[0][1]) and torch.equal(wb, runs[0][2])
    mu_one = pv.kpm_moments(lat, M, a, b, r0=r0.to(cdt))
    assert (runs[0][0] - mu_one).abs().max().item() < (1e-12 if prec == pv.C128 else 1e-6)


def test_halo_lattices_refuse_what_they_do_not_support():
    with pytest.raises(pv.PvscError, match="halo"):
        pv.Lattice.ti((4, 4, 5), (1, 1, 1), z_halo=3)          # periodic z
    with pytest.raises(pv.PvscError, match="halo"):
        pv.Lattice.ti((4, 4, 2), (1, 1, 0), z_halo=3)          # no plane besides the halos
    with pytest.raises(pv.PvscError, match="halo"):
        pv.Lattice.ti((4, 4, 5), (1, 1, 0), disorder=(1.0, 2), z_halo=1)  # a hashed potential
    lat = pv.Lattice.ti((4, 4, 5), (1, 1, 0), z_halo=3)
    r0 = torch.zeros((lat.D, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(pv.PvscError, match="halo"):
        pv.kpm_moments(lat, 8, 8.0, 0.0, r0=r0, prec=pv.Q64)
