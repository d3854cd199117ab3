"""Batched persistent KPM, the autotuner and the bounded device waits."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

pv = pytest.importorskip("paper_1708_09689_gb300")


def _lattices(specs):
    lats, Hs, ab = [], [], []
    for L, Wd, seed in specs:
        dims = (L, L, L) if isinstance(L, int) else L
        n = int(np.prod(dims))
        lat = pv.Lattice.ti(dims, (1, 1, 1), disorder=(Wd, seed))
        H = O.ti_hamiltonian(dims, (1, 1, 1), 1.0, 2.0, W.disorder_potential(n, Wd, seed))
        lats.append(lat)
        Hs.append(H)
        ab.append(O.cheb_scale(*O.gershgorin(H)))
    return lats, Hs, ab


@pytest.mark.parametrize("prec,tol", [(pv.C128, 1e-12), (pv.C64, 1e-4)])
def test_batched_kpm_matches_oracle_on_uneven_lattices(prec, tol):
    specs = [(4, 1.0, 11), ((6, 5, 7), 3.0, 12), (3, 0.0, 13), ((9, 8, 30), 2.0, 14), (5, 4.5, 15)]
    lats, Hs, ab = _lattices(specs)
    R, M = 4, 48
    seeds = [100 + i for i in range(len(lats))]
    mu = pv.kpm_moments_batched(lats, M, [x[0] for x in ab], [x[1] for x in ab], R=R, prec=prec,
                                seeds=seeds).cpu().numpy()
    for i, (H, (a, b)) in enumerate(zip(Hs, ab)):
        r = W.random_phase_block(H.shape[0], R, seeds[i])
        ref = O.kpm_moments(H, r, M, a, b).real
        assert np.max(np.abs(mu[i] - ref)) / ref[0, 0] < tol, i


def test_batched_kpm_equals_single_lattice_kpm_bitwise_for_moments_count():
    lats, Hs, ab = _lattices([(6, 2.0, 21), (8, 1.0, 22)])
    R, M = 2, 20
    mu_b = pv.kpm_moments_batched(lats, M, [x[0] for x in ab], [x[1] for x in ab], R=R,
                                  prec=pv.C128, seeds=[5, 6]).cpu().numpy()
    for i, lat in enumerate(lats):
        mu_s = pv.kpm_moments(lat, M, ab[i][0], ab[i][1], R=R, prec=pv.C128, seed=5 + i).cpu().numpy()
        assert np.max(np.abs(mu_b[i] - mu_s)) < 1e-13


def test_batched_kpm_repeat_is_reproducible_and_replays_graph():
    lats, _, ab = _lattices([(5, 1.0, 31), (7, 2.0, 32), (4, 0.5, 33)])
    args = ([x[0] for x in ab], [x[1] for x in ab])
    work = pv.work_buffer(pv.batched_work_bytes(lats, 8, pv.C64, 32))
    m1 = pv.kpm_moments_batched(lats, 32, *args, R=8, prec=pv.C64, seeds=[1, 2, 3], work=work)
    m2 = pv.kpm_moments_batched(lats, 32, *args, R=8, prec=pv.C64, seeds=[1, 2, 3], work=work)
    assert torch.equal(m1, m2)


def test_batched_wait_timeout_is_reported_and_context_survives():
    lats, Hs, ab = _lattices([(12, 1.0, 41), (10, 1.0, 42)])
    args = ([x[0] for x in ab], [x[1] for x in ab])
    # a wait on a phase that nobody publishes, with a short spin limit
    pv.set_wait_limit(20000)
    pv.inject_stall(True)
    try:
        with pytest.raises(pv.PvscError) as e:
            pv.kpm_moments_batched(lats, 64, *args, R=4, prec=pv.C64, seeds=[1, 2])
        assert e.value.code == pv.PVSC_ERR_TIMEOUT
    finally:
        pv.inject_stall(False)
        pv.set_wait_limit(1 << 26)
    # the context is still usable and the next call is correct
    mu = pv.kpm_moments_batched(lats, 16, *args, R=4, prec=pv.C128, seeds=[1, 2]).cpu().numpy()
    ref = O.kpm_moments(Hs[0], W.random_phase_block(Hs[0].shape[0], 4, 1), 16, *ab[0]).real
    assert np.max(np.abs(mu[0] - ref)) < 1e-12


def test_autotune_picks_a_valid_shape_and_results_do_not_change():
    lat = pv.Lattice.ti((20, 18, 16), (1, 1, 0), disorder=(2.0, 7))
    H = O.ti_hamiltonian((20, 18, 16), (1, 1, 0), 1.0, 2.0, W.disorder_potential(20 * 18 * 16, 2.0, 7))
    a, b = O.cheb_scale(*O.gershgorin(H))
    before = pv.kpm_moments(lat, 40, a, b, R=8, prec=pv.C128, seed=4).cpu().numpy()
    best = lat.autotune(8, pv.C128)
    assert best["threads"] in (64, 128, 256) and best["time_ms"] > 0
    assert lat.get_tuning(8, pv.C128)["threads"] == best["threads"]
    after = pv.kpm_moments(lat, 40, a, b, R=8, prec=pv.C128, seed=4).cpu().numpy()
    assert np.max(np.abs(after - before)) < 1e-13


def test_explicit_tuning_shapes_all_agree():
    lat = pv.Lattice.ti((9, 11, 13), (0, 1, 1), disorder=(1.0, 8))
    x = torch.from_numpy(W.gaussian_block(lat.D, 16, 1)).cuda().to(torch.complex64)
    ref = pv.apply_H(lat, x)
    for th, bps, zs in [(64, 1, 1), (128, 2, 3), (256, 0, 13), (128, 0, 5)]:
        lat.set_tuning(16, pv.C64, th, bps, zs)
        assert torch.equal(pv.apply_H(lat, x), ref)
    with pytest.raises(pv.PvscError):
        lat.set_tuning(16, pv.C64, 100, 0, 0)  # not a multiple of 32
