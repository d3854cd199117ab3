"""Fixed-point (Q64) KPM moments of the TI lattice against the fp64 oracle.

The Q64 path keeps complex128-sized vectors as 64-bit fixed-point integers
(59 fraction bits after an exact power-of-two scaling of each start vector),
adds exactly and rounds each update once at 2^-60, so its moments must agree
with the oracle's fp64 recurrence to the fp64 tolerance.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pv = pytest.importorskip("paper_1708_09689_gb300")
pytestmark = pytest.mark.gpu

TOL = 1e-12  # absolute on moments of unit-norm start vectors (fp64 path tolerance)

CASES = [((7, 5, 6), (1, 0, 1)), ((4, 4, 4), (1, 1, 1)), ((3, 2, 5), (0, 1, 0)),
         ((1, 3, 2), (1, 1, 1)), ((2, 1, 3), (1, 0, 0)), ((9, 8, 11), (1, 1, 0))]


def ti_pair(dims, per, W_=2.0, seed=5):
    n = int(np.prod(dims))
    V = W.disorder_potential(n, W_, seed)
    lat = pv.Lattice.ti(dims, per, disorder=(W_, seed))
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V)
    return lat, H


@pytest.mark.parametrize("dims,per", CASES)
@pytest.mark.parametrize("R", [1, 2, 8])
def test_q64_moments_match_oracle(dims, per, R):
    lat, H = ti_pair(dims, per)
    _, _, a, b = lat.spectral_bounds()
    M = 41
    r = W.random_phase_block(H.shape[0], R, 17)
    mu = pv.kpm_moments(lat, M, a, b, r0=torch.from_numpy(r).cuda(), prec=pv.Q64).cpu().numpy()
    ref = O.kpm_moments(H, r, M, a, b).real
    assert np.max(np.abs(mu - ref)) < TOL


def test_q64_generated_start_block_matches_fp64_path():
    lat, H = ti_pair((10, 9, 8), (1, 1, 0))
    _, _, a, b = lat.spectral_bounds()
    R, M = 4, 64
    mu_q = pv.kpm_moments(lat, M, a, b, R=R, prec=pv.Q64, seed=23).cpu().numpy()
    mu_d = pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C128, seed=23).cpu().numpy()
    assert abs(mu_q[0, 0] - 1.0) < 1e-14
    assert np.max(np.abs(mu_q - mu_d)) < TOL


def test_q64_power_of_two_scaling_is_exact_and_r0_untouched():
    lat, H = ti_pair((6, 7, 5), (1, 0, 1))
    _, _, a, b = lat.spectral_bounds()
    r = W.gaussian_block(H.shape[0], 2, 9) * 0.37  # not unit norm
    rt = torch.from_numpy(r).cuda()
    keep = rt.clone()
    mu1 = pv.kpm_moments(lat, 30, a, b, r0=rt, prec=pv.Q64).cpu().numpy()
    assert torch.equal(rt, keep)
    mu2 = pv.kpm_moments(lat, 30, a, b, r0=rt * 1024.0, prec=pv.Q64).cpu().numpy()
    assert np.array_equal(mu2, mu1 * 1024.0 ** 2)  # same integers, exponent shifted by 10
    ref = O.kpm_moments(O.ti_hamiltonian((6, 7, 5), (1, 0, 1), 1.0, 2.0,
                                         W.disorder_potential(210, 2.0, 5)), r, 30, a, b).real
    norm2 = np.sum(np.abs(r) ** 2, axis=0)[:, None]
    assert np.max(np.abs(mu1 - ref) / norm2) < TOL


def test_q64_bitwise_reproducible_and_zero_vector():
    lat, H = ti_pair((8, 8, 8), (1, 1, 1))
    _, _, a, b = lat.spectral_bounds()
    r = W.random_phase_block(H.shape[0], 2, 3)
    r[:, 1] = 0.0
    rt = torch.from_numpy(r).cuda()
    mu1 = pv.kpm_moments(lat, 20, a, b, r0=rt, prec=pv.Q64).cpu().numpy()
    mu2 = pv.kpm_moments(lat, 20, a, b, r0=rt, prec=pv.Q64).cpu().numpy()
    assert np.array_equal(mu1, mu2)
    assert np.all(mu1[1] == 0.0)


def test_q64_on_the_fly_disorder_equals_stored():
    dims, per = (6, 6, 7), (1, 1, 0)
    lat_s = pv.Lattice.ti(dims, per, disorder=(3.0, 8))
    lat_f = pv.Lattice.ti(dims, per, disorder=(3.0, 8), on_the_fly=True)
    _, _, a, b = lat_s.spectral_bounds()
    mu_s = pv.kpm_moments(lat_s, 24, a, b, R=2, prec=pv.Q64, seed=4).cpu().numpy()
    mu_f = pv.kpm_moments(lat_f, 24, a, b, R=2, prec=pv.Q64, seed=4).cpu().numpy()
    assert np.array_equal(mu_s, mu_f)


def test_q64_rejects_scaling_that_does_not_hold_the_spectrum():
    lat, _ = ti_pair((5, 5, 5), (1, 1, 1))
    emin, emax, a, b = lat.spectral_bounds()
    with pytest.raises(pv.PvscError, match="spectrum"):
        pv.kpm_moments(lat, 8, 0.9 * a, b, R=1, prec=pv.Q64)
    with pytest.raises(pv.PvscError, match="spectrum"):
        pv.kpm_moments(lat, 8, a, b + 0.5, R=1, prec=pv.Q64)


def test_q64_is_kpm_on_ti_only():
    cells = (4, 3)
    latg = pv.Lattice.graphene(cells, (1, 1), V=np.zeros(4 * 12))
    _, _, a, b = latg.spectral_bounds()
    with pytest.raises(pv.PvscError, match="TI lattice only"):
        pv.kpm_moments(latg, 8, a, b, R=1, prec=pv.Q64)
    lat, _ = ti_pair((4, 4, 4), (1, 1, 1))
    assert lat.work_bytes(pv.OP_KPM, 4, pv.Q64, 16) > 0
    for op in (pv.OP_APPLY, pv.OP_CHEB_STEP, pv.OP_SERIES):
        assert lat.work_bytes(op, 4, pv.Q64, 16) == 0  # no other operation takes Q64


def test_q64_prefetch_variants_are_bitwise_identical():
    # The integer arithmetic is exact and the prefetch ring only changes where
    # loads land, so for one launch shape every variant gives the same bits.
    lat, H = ti_pair((9, 7, 12), (1, 0, 1))
    _, _, a, b = lat.spectral_bounds()
    r = torch.from_numpy(W.random_phase_block(H.shape[0], 4, 6)).cuda()
    out = []
    for kernel in (0, 2, 3):
        lat.set_tuning(4, pv.Q64, threads=128, zslab=5, vpt=1, kernel=kernel)
        assert lat.get_tuning(4, pv.Q64)["kernel"] == kernel
        out.append(pv.kpm_moments(lat, 33, a, b, r0=r, prec=pv.Q64).cpu().numpy())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])
    ref = O.kpm_moments(H, r.cpu().numpy(), 33, a, b).real
    assert np.max(np.abs(out[0] - ref)) < TOL
    for bad in (dict(kernel=1), dict(vpt=2), dict(threads=100, kernel=0), dict(tile_x=4, tile_y=4)):
        shape = dict(threads=128, vpt=1, kernel=2)
        shape.update(bad)
        with pytest.raises(pv.PvscError):
            lat.set_tuning(4, pv.Q64, **shape)


def test_q64_scaling_check_follows_a_new_potential():
    # the Gershgorin interval is kept in the handle after the first call; a new
    # potential must renew it, so a scaling that held the old spectrum is refused
    dims, per = (6, 5, 4), (1, 1, 0)
    n = int(np.prod(dims))
    lat = pv.Lattice.ti(dims, per, V=np.zeros(n))
    _, _, a, b = lat.spectral_bounds()
    r0 = torch.from_numpy(W.random_phase_block(4 * n, 2, 3)).cuda()
    pv.kpm_moments(lat, 8, a, b, r0=r0, prec=pv.Q64)
    pv.kpm_moments(lat, 8, a, b, r0=r0, prec=pv.Q64)  # the kept interval
    lat.set_potential(torch.from_numpy(W.disorder_potential(n, 6.0, 1)).cuda())
    with pytest.raises(pv.PvscError) as e:
        pv.kpm_moments(lat, 8, a, b, r0=r0, prec=pv.Q64)
    assert e.value.code == pv.PVSC_ERR_ARG
    _, _, a2, b2 = lat.spectral_bounds()
    mu = pv.kpm_moments(lat, 8, a2, b2, r0=r0, prec=pv.Q64).cpu().numpy()
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, W.disorder_potential(n, 6.0, 1))
    ref = O.kpm_moments(H, r0.cpu().numpy(), 8, a2, b2).real
    assert np.max(np.abs(mu - ref)) < TOL
