"""Spectral densities (Eq. DOS, Eq. ak) and Bloch start states on the GPU
against the oracle, and A(k, E) of a clean TI against its closed-form bands."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pv = pytest.importorskip("paper_1708_09689_gb300")
pytestmark = pytest.mark.gpu


def _g(kernel, M, lam):
    if kernel == pv.KERNEL_JACKSON:
        return O.jackson_kernel(M)
    if kernel == pv.KERNEL_LORENTZ:
        return O.lorentz_kernel(M, lam)
    return np.ones(M)


@pytest.mark.parametrize("M", [1, 7, 1024, 3001])
@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_density_matches_oracle(M, kernel):
    rng = np.random.default_rng(M + 10 * kernel)
    R, a, b, lam, scale = 3, 4.5, -0.2, 3.0, 1.7
    mu = rng.standard_normal((R, M)) / (1 + np.arange(M)) ** 0.5
    E = np.concatenate([np.linspace(b - a * 1.1, b + a * 1.1, 997), [b - a, b + a, b]])
    rho = pv.kpm_density(torch.from_numpy(mu).cuda(), torch.from_numpy(E).cuda(), a, b, kernel, lam,
                         scale).cpu().numpy()
    ref = O.kpm_density(mu, E, a, b, _g(kernel, M, lam), scale)
    assert np.array_equal(rho == 0.0, ref == 0.0)  # same support: |x| < 1
    assert np.max(np.abs(rho - ref)) < 1e-12 * np.max(np.abs(ref)) * max(1.0, M / 100)


def test_bloch_vectors_match_oracle():
    dims = (5, 4, 3)
    lat = pv.Lattice.ti(dims, (1, 1, 1))
    ks = [(0.3, -1.1, 2.0), (math.pi, 0.0, 0.5)]
    ref = np.concatenate([O.bloch_vectors(dims, k) for k in ks], axis=1)
    v = pv.bloch_vectors(lat, ks, pv.C128).cpu().numpy()
    assert np.max(np.abs(v - ref)) < 1e-15
    v64 = pv.bloch_vectors(lat, ks, pv.C64).cpu().numpy()
    assert np.max(np.abs(v64 - ref)) < 1e-7 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec,tol", [(pv.C128, 2e-3), (pv.C64, 3e-3)])
def test_spectral_function_of_clean_ti_on_gpu(prec, tol):
    # GPU KPM with the GPU Bloch states and density: peaks of weight 2 at the
    # closed-form +-E(k) of the clean periodic TI (reading of Eq. bloch_H_topi)
    dims = (8, 8, 8)
    lat = pv.Lattice.ti(dims, (1, 1, 1))
    _, _, a, b = lat.spectral_bounds()
    ks = [(2 * math.pi * 2 / 8, 0.0, 0.0), (2 * math.pi / 8, 2 * math.pi * 3 / 8, 2 * math.pi / 8)]
    E = np.linspace(b - a + 1e-9, b + a - 1e-9, 40001)
    A = pv.spectral_function(lat, ks, 512, a, b, E, prec=prec).cpu().numpy()
    H = O.ti_hamiltonian(dims, (1, 1, 1), 1.0, 2.0, np.zeros(512))
    for q, k in enumerate(ks):
        Ek = math.sqrt((2.0 - sum(math.cos(c) for c in k)) ** 2 + sum(math.sin(c) ** 2 for c in k))
        for e0 in (Ek, -Ek):
            m = (E > e0 - 0.4) & (E < e0 + 0.4)
            assert abs(E[m][np.argmax(A[q][m])] - e0) < 2e-3
            assert abs(np.trapezoid(A[q][m], E[m]) - 2.0) < tol
        if prec == pv.C128:  # the whole chain against the oracle's
            mu = O.kpm_moments(H, O.bloch_vectors(dims, k), 512, a, b).real
            ref = O.kpm_density(mu, E, a, b, O.jackson_kernel(512))
            assert np.max(np.abs(A[q] - ref)) < 1e-9 * np.max(ref)


def test_dos_of_random_vectors_integrates_to_D():
    dims = (12, 10, 8)
    lat = pv.Lattice.ti(dims, (1, 1, 0), disorder=(2.0, 3))
    _, _, a, b = lat.spectral_bounds()
    R, M = 8, 256
    mu = pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C64, seed=4)
    N = 4 * M
    x = np.cos(np.pi * (np.arange(N) + 0.5) / N)
    rho = pv.dos(lat, mu, b + a * x, a, b).cpu().numpy()
    integral = np.pi / N * np.sum(rho * a * np.sqrt(1 - x * x))  # exact Gauss-Chebyshev rule
    assert abs(integral - lat.D * mu[:, 0].mean().item()) < 1e-9 * lat.D
    assert rho.min() >= 0.0 or rho.min() > -1e-3 * rho.max()  # stochastic moments: nearly positive


def test_density_and_bloch_argument_errors():
    mu = torch.zeros((1, 4), dtype=torch.float64, device="cuda")
    E = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(pv.PvscError):
        pv.kpm_density(mu, E, 1.0, 0.0, kernel=7)
    with pytest.raises(pv.PvscError):
        pv.kpm_density(mu, E, 1.0, 0.0, kernel=pv.KERNEL_LORENTZ, lam=0.0)
    with pytest.raises(pv.PvscError):
        pv.kpm_density(mu, E, -1.0, 0.0)
    lat = pv.Lattice.ti((4, 4, 4), (1, 1, 1))
    with pytest.raises(pv.PvscError):
        pv.bloch_vectors(lat, [(0, 0, 0)] * 3)  # nk must be a power of two up to 16
    with pytest.raises(pv.PvscError):
        pv.bloch_vectors(pv.Lattice.graphene((4, 3), (1, 1)), [(0, 0, 0)])


def test_disorder_fills_the_bulk_gap_of_the_ti_dos():
    # the trend of the paper's disordered-TI DOS (Sec. 4.2): the clean m = 2
    # bulk has a gap |E| < 1; box disorder of growing width W puts states into
    # it.  Stochastic-trace KPM DOS of a periodic 14^3 lattice (no surfaces),
    # the same scaling for every W; the weight inside |E| < 0.5 grows with W
    # and is negligible without disorder
    dims, per = (14, 14, 14), (1, 1, 1)
    Ws = [0.0, 2.0, 4.0, 6.0]
    lats = [pv.Lattice.ti(dims, per, disorder=(Wd, 21)) if Wd else pv.Lattice.ti(dims, per) for Wd in Ws]
    _, _, a, b = lats[-1].spectral_bounds()   # the widest spectrum holds all of them
    M, R = 512, 16
    E = np.linspace(-0.5, 0.5, 201)
    inside = []
    for lat in lats:
        mu = pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C64, seed=7)
        rho = pv.dos(lat, mu, E, a, b).cpu().numpy()
        inside.append(float(np.sum(rho) * (E[1] - E[0])) / lat.D)
    assert inside[0] < 2e-3                       # the clean gap (KPM broadening leaks a little)
    assert all(x < y for x, y in zip(inside, inside[1:])), inside
    assert inside[-1] > 10 * max(inside[0], 1e-4)
