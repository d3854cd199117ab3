"""The two-band Weyl semimetal of Eq. TB_H_wsm on the GPU against the oracle."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pv = pytest.importorskip("paper_1708_09689_gb300")
pytestmark = pytest.mark.gpu

# boundary mixes, including periodic lengths 2 (bonds fold) and 1 (a site is its own neighbour)
CASES = [((8, 3, 4), (1, 1, 1)), ((6, 5, 3), (1, 0, 1)), ((2, 1, 3), (1, 1, 0)),
         ((4, 2, 2), (1, 1, 1)), ((2, 4, 1), (0, 1, 1)), ((10, 3, 2), (0, 0, 0))]


def _pair(dims, per, Wd=1.5, seed=6, k0=math.pi / 2):
    n = int(np.prod(dims))
    lat = pv.Lattice.wsm(dims, per, k0=k0, disorder=(Wd, seed))
    H = O.wsm_hamiltonian(dims, per, W.disorder_potential(n, Wd, seed), k0)
    return lat, H


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dims,per", CASES)
@pytest.mark.parametrize("R", [1, 2, 8])
@pytest.mark.parametrize("prec,tol", [(pv.C128, 1e-13), (pv.C64, 2e-6)])
def test_wsm_apply_H_matches_oracle(dims, per, R, prec, tol):
    lat, H = _pair(dims, per)
    assert lat.D == H.shape[0] == 2 * int(np.prod(dims))
    x = W.gaussian_block(H.shape[0], R, 1)
    cdt = torch.complex128 if prec == pv.C128 else torch.complex64
    y = pv.apply_H(lat, torch.from_numpy(x).to("cuda", cdt)).cpu().numpy().astype(np.complex128)
    xr = x.astype(np.complex64).astype(np.complex128) if prec == pv.C64 else x
    assert _rel(y, H @ xr) < tol


@pytest.mark.parametrize("dims,per", CASES[:3])
def test_wsm_cheb_step_and_dots(dims, per):
    lat, H = _pair(dims, per)
    R = 4
    x = W.gaussian_block(H.shape[0], R, 2)
    y0 = W.gaussian_block(H.shape[0], R, 3)
    yt = torch.from_numpy(y0).cuda()
    d = pv.cheb_step(lat, torch.from_numpy(x).cuda(), yt, [0.3] * R, [0.1] * R, [-1.0] * R, dots=7)
    yr, _, dr = O.cheb_step(H, x, y0, [0.3] * R, [0.1] * R, [-1.0] * R)
    assert _rel(yt.cpu().numpy(), yr) < 1e-12
    d = d.cpu().numpy()
    assert np.max(np.abs(d[1] - dr[:, 1].real)) < 1e-12 * np.abs(dr).max()


def test_wsm_bounds_kpm_and_propagation():
    dims, per = (8, 6, 4), (1, 1, 0)
    lat, H = _pair(dims, per, Wd=2.0)
    emin, emax, a, b = lat.spectral_bounds()
    ga, gb = O.gershgorin(H)
    assert abs(emin - ga) < 1e-12 and abs(emax - gb) < 1e-12
    ev = np.linalg.eigvalsh(H.toarray())
    assert emin <= ev[0] and ev[-1] <= emax
    r = W.random_phase_block(H.shape[0], 2, 5)
    mu = pv.kpm_moments(lat, 64, a, b, r0=torch.from_numpy(r).cuda()).cpu().numpy()
    assert np.max(np.abs(mu - O.kpm_moments(H, r, 64, a, b).real)) < 1e-12
    mu64 = pv.kpm_moments(lat, 64, a, b, r0=torch.from_numpy(r).cuda().to(torch.complex64)).cpu().numpy()
    assert np.max(np.abs(mu64 - O.kpm_moments(H, r, 64, a, b).real)) < 1e-4
    psi0 = W.gaussian_block(H.shape[0], 1, 7)
    psi0 /= np.linalg.norm(psi0)
    ref = O.propagate(H, psi0, 0.8, 3, a, b)
    psi = torch.from_numpy(psi0).cuda()
    pv.cheb_propagate(lat, psi, 0.8, 3, a, b)
    assert _rel(psi.cpu().numpy(), ref) < 1e-12


def test_wsm_clean_periodic_spectrum_through_the_gpu_stencil():
    # H applied on the GPU to the Bloch plane waves of one k gives the 2x2 band matrix
    # of Eq. band_h_wsm (Weyl nodes at (+-k0, 0, 0) have eigenvalue 0)
    dims = (8, 4, 4)
    lat = pv.Lattice.wsm(dims, (1, 1, 1))
    n = 128
    coords = np.stack(np.meshgrid(np.arange(8), np.arange(4), np.arange(4), indexing="ij"), -1)
    coords = coords.transpose(2, 1, 0, 3).reshape(n, 3)  # site = x + Lx (y + Ly z)
    for k in [(math.pi / 2, 0.0, 0.0), (-math.pi / 2, 0.0, 0.0), (math.pi / 4, math.pi / 2, math.pi)]:
        ph = np.exp(1j * coords @ np.array(k)) / math.sqrt(n)
        psi = np.zeros((2 * n, 2), dtype=np.complex128)
        psi[0::2, 0] = ph
        psi[1::2, 1] = ph
        Hpsi = pv.apply_H(lat, torch.from_numpy(psi).cuda()).cpu().numpy()
        Hk = psi.conj().T @ Hpsi
        kx, ky, kz = k
        dx = math.cos(kx) - math.cos(math.pi / 2) + math.cos(ky) + math.cos(kz) - 2.0
        ref = np.array([[math.sin(kz), dx - 1j * math.sin(ky)], [dx + 1j * math.sin(ky), -math.sin(kz)]])
        assert np.max(np.abs(Hk - ref)) < 1e-13
        if abs(abs(kx) - math.pi / 2) < 1e-15 and ky == 0 and kz == 0:
            assert np.max(np.abs(np.linalg.eigvalsh(Hk))) < 1e-13


def test_wsm_on_the_fly_potential_and_unsupported_paths():
    dims, per = (6, 4, 3), (1, 1, 1)
    lat_s = pv.Lattice.wsm(dims, per, disorder=(2.0, 3))
    lat_f = pv.Lattice.wsm(dims, per, disorder=(2.0, 3), on_the_fly=True)
    x = torch.from_numpy(W.gaussian_block(lat_s.D, 2, 1)).cuda()
    assert torch.equal(pv.apply_H(lat_s, x), pv.apply_H(lat_f, x))
    with pytest.raises(pv.PvscError):
        pv.Lattice.wsm((5, 4, 3), per)  # odd Lx: the sweep pairs sites along x
    _, _, a, b = lat_s.spectral_bounds()
    with pytest.raises(pv.PvscError):
        pv.kpm_moments(lat_s, 8, a, b, R=1, prec=pv.Q64)
    with pytest.raises(pv.PvscError):
        pv.kpm_moments_batched([lat_s], 8, [a], [b], R=1, prec=pv.C64, seeds=[1])


def test_wsm_bloch_states_and_spectral_function_on_gpu():
    dims = (8, 4, 4)
    lat = pv.Lattice.wsm(dims, (1, 1, 1))
    ks = [(math.pi / 2, 0.0, 0.0), (math.pi / 4, math.pi / 2, math.pi)]
    v = pv.bloch_vectors(lat, ks).cpu().numpy()
    ref = np.concatenate([O.bloch_vectors(dims, k, O=2) for k in ks], axis=1)
    assert v.shape == (256, 4) and np.max(np.abs(v - ref)) < 1e-15
    _, _, a, b = lat.spectral_bounds()
    E = np.linspace(b - a + 1e-9, b + a - 1e-9, 40001)
    A = pv.spectral_function(lat, ks, 512, a, b, E, prec=pv.C128).cpu().numpy()
    H = O.wsm_hamiltonian(dims, (1, 1, 1), np.zeros(128))
    for q, k in enumerate(ks):
        mu = O.kpm_moments(H, O.bloch_vectors(dims, k, O=2), 512, a, b).real
        refA = O.kpm_density(mu, E, a, b, O.jackson_kernel(512))
        assert np.max(np.abs(A[q] - refA)) < 1e-9 * np.max(refA)
        assert abs(np.trapezoid(A[q], E) - 2.0) < 1e-3


@pytest.mark.parametrize("shape", [dict(kernel=1, threads=128), dict(kernel=0, threads=128, zslab=2),
                                   dict(kernel=0, threads=64, zslab=0)])
@pytest.mark.parametrize("prec,tol", [(pv.C128, 1e-13), (pv.C64, 2e-6)])
def test_wsm_flat_and_marching_sweeps_match_oracle(shape, prec, tol):
    for dims, per in CASES:
        lat, H = _pair(dims, per)
        R = 4
        lat.set_tuning(R, prec, vpt=1, **shape)
        x = W.gaussian_block(H.shape[0], R, 4)
        cdt = torch.complex128 if prec == pv.C128 else torch.complex64
        y = pv.apply_H(lat, torch.from_numpy(x).to("cuda", cdt)).cpu().numpy().astype(np.complex128)
        xr = x.astype(np.complex64).astype(np.complex128) if prec == pv.C64 else x
        assert _rel(y, H @ xr) < tol, (dims, per)
