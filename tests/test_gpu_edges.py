"""Edge cases across the models and precisions: the smallest moment counts,
the widest blocks, the tiniest lattices and the shortest series."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pv = pytest.importorskip("paper_1708_09689_gb300")
pytestmark = pytest.mark.gpu


def _ti(dims, per, Wd=1.0, seed=2):
    n = int(np.prod(dims))
    return (pv.Lattice.ti(dims, per, disorder=(Wd, seed)),
            O.ti_hamiltonian(dims, per, 1.0, 2.0, W.disorder_potential(n, Wd, seed)))


@pytest.mark.parametrize("M", [1, 2, 3])
@pytest.mark.parametrize("prec,tol", [(pv.C128, 1e-13), (pv.C64, 1e-5), (pv.Q64, 1e-13)])
def test_kpm_with_the_smallest_moment_counts(M, prec, tol):
    lat, H = _ti((5, 4, 6), (1, 0, 1))
    _, _, a, b = lat.spectral_bounds()
    r = W.random_phase_block(H.shape[0], 2, 4)
    r0 = torch.from_numpy(r).cuda()
    if prec == pv.C64:
        r0 = r0.to(torch.complex64)
    mu = pv.kpm_moments(lat, M, a, b, r0=r0, prec=prec).cpu().numpy()
    assert mu.shape == (2, M)
    assert np.max(np.abs(mu - O.kpm_moments(H, r, M, a, b).real)) < tol


@pytest.mark.parametrize("prec,tol", [(pv.C128, 1e-13), (pv.C64, 2e-6)])
def test_widest_block_on_the_weyl_semimetal(prec, tol):
    dims, per = (6, 3, 4), (1, 0, 1)
    n = 72
    lat = pv.Lattice.wsm(dims, per, disorder=(1.0, 5))
    H = O.wsm_hamiltonian(dims, per, W.disorder_potential(n, 1.0, 5))
    x = W.gaussian_block(H.shape[0], 64, 1)
    cdt = torch.complex128 if prec == pv.C128 else torch.complex64
    y = pv.apply_H(lat, torch.from_numpy(x).to("cuda", cdt)).cpu().numpy().astype(np.complex128)
    xr = x.astype(np.complex64).astype(np.complex128) if prec == pv.C64 else x
    assert np.linalg.norm(y - H @ xr) / np.linalg.norm(H @ xr) < tol


def test_widest_block_in_fixed_point():
    lat, H = _ti((4, 5, 3), (1, 1, 0))
    _, _, a, b = lat.spectral_bounds()
    r = W.random_phase_block(H.shape[0], 64, 6)
    mu = pv.kpm_moments(lat, 17, a, b, r0=torch.from_numpy(r).cuda(), prec=pv.Q64).cpu().numpy()
    assert np.max(np.abs(mu - O.kpm_moments(H, r, 17, a, b).real)) < 1e-12


@pytest.mark.parametrize("model", ["ti", "wsm", "graphene"])
def test_tiny_periodic_lattices_through_kpm_and_propagation(model):
    if model == "ti":
        lat, H = _ti((2, 2, 2), (1, 1, 1))
    elif model == "wsm":
        lat = pv.Lattice.wsm((2, 1, 2), (1, 1, 1), disorder=(1.0, 3))
        H = O.wsm_hamiltonian((2, 1, 2), (1, 1, 1), W.disorder_potential(4, 1.0, 3))
    else:
        V = W.disorder_potential(4, 0.5, 3)
        lat = pv.Lattice.graphene((1, 1), (1, 1), V=V)
        H = O.graphene_hamiltonian((1, 1), (1, 1), 1.0, V)
    _, _, a, b = lat.spectral_bounds()
    r = W.random_phase_block(H.shape[0], 1, 2)
    mu = pv.kpm_moments(lat, 12, a, b, r0=torch.from_numpy(r).cuda()).cpu().numpy()
    assert np.max(np.abs(mu - O.kpm_moments(H, r, 12, a, b).real)) < 1e-12
    psi0 = r / np.linalg.norm(r)
    for prec, tol in ((pv.C128, 1e-12), (pv.C64, 1e-5)):
        psi = torch.from_numpy(psi0).cuda()
        pv.cheb_propagate(lat, psi, 0.5, 4, a, b, prec=prec)
        assert np.linalg.norm(psi.cpu().numpy() - O.propagate(H, psi0, 0.5, 4, a, b)) < tol


@pytest.mark.parametrize("dt,K_expected", [(1e-9, 2), (3e-6, 3)])
def test_propagation_with_the_shortest_series(dt, K_expected):
    # tiny time steps truncate the Bessel series to one or two terms
    lat, H = _ti((3, 4, 5), (1, 1, 0))
    _, _, a, b = lat.spectral_bounds()
    assert len(pv.propagation_coeffs(a * dt, 1e-14)) == K_expected
    x = W.gaussian_block(H.shape[0], 2, 3)
    x /= np.linalg.norm(x, axis=0)
    ref = O.propagate(H, x, dt, 3, a, b)
    for prec, tol in ((pv.C128, 1e-13), (pv.C64, 1e-6)):
        psi = torch.from_numpy(x).cuda()
        pv.cheb_propagate(lat, psi, dt, 3, a, b, prec=prec)
        assert np.linalg.norm(psi.cpu().numpy() - ref) / np.linalg.norm(ref) < tol


def test_poisoned_potential_is_detected_on_the_host_without_a_device_fault():
    # failure detection without a GPU fault: a NaN planted in the potential (on
    # the host side of the input) is reported by the spectral bounds as an
    # error, propagates into mu_1 and every later moment while mu_0 = <r|r> stays
    # finite, and into the norm of a propagated state; the context stays usable
    dims, per = (6, 5, 4), (1, 1, 0)
    n = int(np.prod(dims))
    V = W.disorder_potential(n, 1.0, 3)
    lat = pv.Lattice.ti(dims, per, V=V)
    _, _, a, b = lat.spectral_bounds()
    bad = V.copy()
    bad[17] = np.nan
    lat.set_potential(torch.from_numpy(bad).cuda())
    with pytest.raises(pv.PvscError) as e:
        lat.spectral_bounds()
    assert e.value.code == pv.PVSC_ERR_ARG and "non-finite" in str(e.value)
    for prec in (pv.C128, pv.C64):
        mu = pv.kpm_moments(lat, 16, a, b, R=2, prec=prec, seed=4).cpu().numpy()
        assert np.all(np.isfinite(mu[:, 0])) and np.all(np.isnan(mu[:, 1:]))
    psi = torch.from_numpy(W.gaussian_block(4 * n, 1, 2)[:, 0]).cuda()
    pv.cheb_propagate(lat, psi, 0.5, 2, a, b)
    assert not torch.isfinite(torch.linalg.vector_norm(psi)).item()
    # a clean potential restores everything, with no device error pending
    lat.set_potential(torch.from_numpy(V).cuda())
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V)
    mu = pv.kpm_moments(lat, 16, a, b, R=2, prec=pv.C128, seed=4).cpu().numpy()
    ref = O.kpm_moments(H, W.random_phase_block(4 * n, 2, 4), 16, a, b).real
    assert np.max(np.abs(mu - ref)) < 1e-12
    assert pv.device_error() == 0
