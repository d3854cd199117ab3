"""The multi-rank decomposition on CPU with the gloo backend (world size 2).

Each rank computes the oracle KPM moments of its own random vectors; the
gathered result must equal the single-process result exactly (no collective
touches the data path, only the final gather), and the timing reduction must
return the maximum over ranks."""
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


def _load_sharding():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "pvsc_sharding", os.path.join(ROOT, "paper_1708_09689_gb300", "sharding.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _worker(rank, world, port, out_path):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    import workloads as W
    S = _load_sharding()
    dims, per = (5, 4, 3), (1, 1, 0)
    n = 60
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, W.disorder_potential(n, 1.0, 2))
    a, b = O.cheb_scale(*O.gershgorin(H))
    n_units, M = 7, 24
    local = {}
    for u in S.shard(n_units, world, rank):
        r = W.random_phase_block(4 * n, 1, S.vector_seed(3, u))
        local[u] = torch.from_numpy(O.kpm_moments(H, r, M, a, b).real[0])
    mu = S.gather_results(local, n_units)
    tmax = S.max_over_ranks(1.0 + rank)
    units = S.sum_over_ranks(len(local))
    if rank == 0:
        np.save(out_path, mu.numpy())
        with open(out_path + ".txt", "w") as f:
            f.write(f"{tmax} {units}")
    dist.barrier()
    dist.destroy_process_group()


def test_shard_covers_every_unit_once():
    S = _load_sharding()
    for world in (1, 2, 3, 8):
        owned = sorted(u for r in range(world) for u in S.shard(64, world, r))
        assert owned == list(range(64))
    with pytest.raises(ValueError):
        S.shard(4, 2, 2)


def test_two_gloo_ranks_reproduce_single_process_moments(tmp_path):
    import oracle as O
    import workloads as W
    S = _load_sharding()
    out = str(tmp_path / "mu.npy")
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    mu = np.load(out)
    tmax, units = open(out + ".txt").read().split()
    assert float(tmax) == 2.0 and float(units) == 7.0
    dims, per, n = (5, 4, 3), (1, 1, 0), 60
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, W.disorder_potential(n, 1.0, 2))
    a, b = O.cheb_scale(*O.gershgorin(H))
    for u in range(7):
        r = W.random_phase_block(4 * n, 1, S.vector_seed(3, u))
        assert np.array_equal(mu[u], O.kpm_moments(H, r, 24, a, b).real[0])
