"""The on-site Delta_1 Gamma^5 + Delta_2 Gamma^15 terms of Eq. TB_H_topi on the
GPU against the oracle, in every TI sweep variant and in the spectral bounds."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pv = pytest.importorskip("paper_1708_09689_gb300")
pytestmark = pytest.mark.gpu

CASES = [((7, 5, 6), (1, 0, 1)), ((4, 4, 4), (1, 1, 1)), ((3, 2, 5), (0, 1, 0))]
DELTAS = [(0.4, 0.0), (0.0, -0.3), (0.35, 0.25)]


def _pair(dims, per, d1, d2, Wd=1.5, seed=4):
    n = int(np.prod(dims))
    lat = pv.Lattice.ti(dims, per, disorder=(Wd, seed), delta1=d1, delta2=d2)
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, W.disorder_potential(n, Wd, seed), d1, d2)
    return lat, H


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("dims,per", CASES)
@pytest.mark.parametrize("d1,d2", DELTAS)
@pytest.mark.parametrize("prec,tol", [(pv.C128, 1e-12), (pv.C64, 2e-6)])
def test_apply_H_with_delta_terms(dims, per, d1, d2, prec, tol):
    lat, H = _pair(dims, per, d1, d2)
    x = W.gaussian_block(H.shape[0], 4, 1)
    cdt = torch.complex128 if prec == pv.C128 else torch.complex64
    y = pv.apply_H(lat, torch.from_numpy(x).to("cuda", cdt)).cpu().numpy().astype(np.complex128)
    xr = x.astype(np.complex64).astype(np.complex128) if prec == pv.C64 else x
    assert _rel(y, H @ xr) < tol


@pytest.mark.parametrize("variant", [dict(kernel=0), dict(kernel=1), dict(kernel=2), dict(kernel=3),
                                     dict(tile_x=4, tile_y=4)])
def test_cheb_step_with_delta_terms_in_every_sweep_variant(variant):
    dims, per, d1, d2 = (6, 5, 7), (1, 1, 0), 0.35, 0.25
    lat, H = _pair(dims, per, d1, d2)
    R = 4
    shape = dict(threads=128, zslab=3, vpt=1)
    shape.update(variant)
    lat.set_tuning(R, pv.C128, **shape)
    x = W.gaussian_block(H.shape[0], R, 2)
    y0 = W.gaussian_block(H.shape[0], R, 3)
    yt = torch.from_numpy(y0).cuda()
    pv.cheb_step(lat, torch.from_numpy(x).cuda(), yt, [0.3] * R, [0.1] * R, [-1.0] * R)
    yr, _, _ = O.cheb_step(H, x, y0, [0.3] * R, [0.1] * R, [-1.0] * R)
    assert _rel(yt.cpu().numpy(), yr) < 1e-12


def test_kpm_and_bounds_with_delta_terms():
    dims, per = (6, 6, 6), (1, 1, 1)
    lat, H = _pair(dims, per, 0.5, -0.4)
    ev = np.linalg.eigvalsh(H.toarray())
    emin, emax, a, b = lat.spectral_bounds()
    ga, gb = O.gershgorin(H)
    assert abs(emin - ga) < 1e-12 and abs(emax - gb) < 1e-12  # same exact per-row bound
    assert emin <= ev[0] and ev[-1] <= emax
    r = W.random_phase_block(H.shape[0], 2, 5)
    mu = pv.kpm_moments(lat, 64, a, b, r0=torch.from_numpy(r).cuda()).cpu().numpy()
    ref = O.kpm_moments(H, r, 64, a, b).real
    assert np.max(np.abs(mu - ref)) < 1e-12
    with pytest.raises(pv.PvscError, match="Delta"):
        pv.kpm_moments(lat, 8, a, b, R=1, prec=pv.Q64)


def test_batched_kpm_with_delta_terms():
    specs = [((5, 5, 5), 0.3, 0.2), ((4, 6, 5), 0.0, 0.5)]
    lats, Hs, ab = [], [], []
    for dims, d1, d2 in specs:
        lat, H = _pair(dims, (1, 1, 1), d1, d2)
        lats.append(lat)
        Hs.append(H)
        ab.append(O.cheb_scale(*O.gershgorin(H)))
    mu = pv.kpm_moments_batched(lats, 32, [x[0] for x in ab], [x[1] for x in ab], R=2, prec=pv.C128,
                                seeds=[7, 8]).cpu().numpy()
    for i, (H, (a, b)) in enumerate(zip(Hs, ab)):
        ref = O.kpm_moments(H, W.random_phase_block(H.shape[0], 2, 7 + i), 32, a, b).real
        assert np.max(np.abs(mu[i] - ref)) < 1e-12
