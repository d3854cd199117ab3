"""Domain decomposition of one TI lattice into z-slabs (Sec. 3.4), on CPU ranks.

Each gloo rank holds its slab of the lattice as an oracle Hamiltonian (its
planes plus one halo plane on each side, open along z) and runs the slab
driver of paper_1708_09689_gb300/slab.py: a halo exchange of the current
recurrence vector before every KPM sweep, the sweep on the slab (here the
oracle's arithmetic, with dot products over the slab's own planes), and one
sum of the moments at the end.  The result must equal the single-domain
oracle recurrence, for open and periodic z, on 2 and 3 ranks and with uneven
slabs.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _load_slab():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "pvsc_slab", os.path.join(ROOT, "paper_1708_09689_gb300", "slab.py"))
    mod = importlib.util.module_from_spec(spec)
    import sys
    sys.modules["pvsc_slab"] = mod  # dataclasses resolve their module by name
    spec.loader.exec_module(mod)
    return mod


def _global_case(dims, per):
    import oracle as O
    import workloads as W
    n = int(np.prod(dims))
    V = W.disorder_potential(n, 2.0, 9)
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V)
    a, b = O.cheb_scale(*O.gershgorin(H))
    r = W.random_phase_block(4 * n, 2, 4)
    return V, H, a, b, r


def _oracle_slab_sweep(Hl, part, a, b, M):
    """One KPM sweep of a slab with the oracle's arithmetic: the recurrence on
    every local row, the dot products on the slab's own planes only."""
    P = part.plane_sites * 4
    inner = slice(part.lo * P, (part.lo + part.nz) * P)

    def sweep(k, wa, wb, mu):
        x = (wa if k % 2 == 0 else wb).numpy()
        other = wb if k % 2 == 0 else wa
        Ht = (Hl @ x - b * x) / a
        if k == 0:
            y = Ht
            mu[:, 0] = torch.from_numpy(np.sum(np.abs(x[inner]) ** 2, axis=0))
            if M > 1:
                mu[:, 1] = torch.from_numpy(np.sum(np.conj(y[inner]) * x[inner], axis=0).real)
        else:
            y = 2.0 * Ht - other.numpy()
            if 2 * k < M:
                mu[:, 2 * k] = torch.from_numpy(2.0 * np.sum(np.abs(x[inner]) ** 2, axis=0)) - mu[:, 0]
            if 2 * k + 1 < M:
                mu[:, 2 * k + 1] = torch.from_numpy(
                    2.0 * np.sum(np.conj(y[inner]) * x[inner], axis=0).real) - mu[:, 1]
        other.copy_(torch.from_numpy(y))
    return sweep


def _worker(rank, world, port, dims, per, M, out_path):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    S = _load_slab()
    V, H, a, b, r = _global_case(dims, per)
    part = S.SlabPartition(dims, per, world, rank)
    tr = S.TorchDistTransport()
    # the slab's lattice: its planes and the halo planes, open along z
    Vl = part.local_rows(torch.from_numpy(V), orbitals=1).numpy()
    Hl = O.ti_hamiltonian(part.local_dims, part.local_periodic, 1.0, 2.0, Vl)
    # global spectral interval from the slabs' Gershgorin intervals (own rows only)
    P = part.plane_sites * 4
    own = slice(part.lo * P, (part.lo + part.nz) * P)
    rows = Hl[own]
    diag = np.asarray(Hl.diagonal()[own]).real
    rad = np.asarray(abs(rows).sum(axis=1)).ravel() - np.abs(diag)
    emin, emax = S.spectral_interval(float((diag - rad).min()), float((diag + rad).max()), tr)
    r0 = part.local_rows(torch.from_numpy(r))
    mu = S.kpm_moments(part, M, a, b, r0, transport=tr, sweep=_oracle_slab_sweep(Hl, part, a, b, M))
    if rank == 0:
        np.save(out_path, mu.numpy())
        np.save(out_path + ".bounds.npy", np.array([emin, emax]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("dims,per,world", [((4, 3, 7), (1, 1, 0), 2), ((4, 3, 7), (1, 0, 1), 2),
                                            ((3, 4, 8), (1, 1, 1), 3), ((3, 3, 5), (0, 1, 0), 3)])
def test_slab_ranks_reproduce_the_single_domain_oracle(tmp_path, dims, per, world):
    import oracle as O
    M = 40
    out = str(tmp_path / "mu.npy")
    mp.start_processes(_worker, args=(world, _free_port(), dims, per, M, out), nprocs=world, join=True,
                       start_method="spawn")
    mu = np.load(out)
    V, H, a, b, r = _global_case(dims, per)
    ref = O.kpm_moments(H, r, M, a, b).real
    assert np.max(np.abs(mu - ref)) / ref[0, 0] < 1e-14
    emin, emax = np.load(out + ".bounds.npy")
    gmin, gmax = O.gershgorin(H)
    assert abs(emin - gmin) < 1e-13 and abs(emax - gmax) < 1e-13


def test_slab_partition_covers_every_plane_once():
    S = _load_slab()
    for Lz, world in ((7, 2), (8, 3), (5, 5), (64, 4)):
        planes = []
        for rank in range(world):
            p = S.SlabPartition((4, 4, Lz), (1, 1, 0), world, rank)
            planes += list(range(p.z0, p.z1))
            assert p.nz >= 1 and p.local_dims == (4, 4, p.lo + p.nz + p.hi)
            assert p.halo_flags == p.lo + 2 * p.hi
        assert planes == list(range(Lz))
    p = S.SlabPartition((4, 4, 6), (1, 1, 1), 3, 0)
    assert p.below == 2 and p.above == 1 and p.global_planes() == [5, 0, 1, 2]
    p = S.SlabPartition((4, 4, 6), (1, 1, 0), 3, 2)
    assert p.below == 1 and p.above is None and p.global_planes() == [3, 4, 5]
    assert (p.lo, p.hi) == (1, 0)
    with pytest.raises(ValueError):
        S.SlabPartition((4, 4, 2), (1, 1, 0), 3, 0)


def test_single_periodic_slab_wraps_its_own_planes():
    S = _load_slab()
    p = S.SlabPartition((2, 1, 3), (1, 1, 1), 1, 0)
    assert p.global_planes() == [2, 0, 1, 2, 0]
    w = torch.arange(5 * 8, dtype=torch.float64).reshape(40, 1)
    S.halo_exchange(p, w, S.TorchDistTransport())
    assert torch.equal(w[0:8], w[24:32]) and torch.equal(w[32:40], w[8:16])
