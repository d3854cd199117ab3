"""Two KPM recurrence steps per sweep (temporal blocking) on the GPU.

The two-step sweep computes w_{k+1} and w_{k+2} with the single sweep's
arithmetic, so its vectors equal two single sweeps' bit for bit and its
moments differ from the single-step path only by the order of the fp64 dot
sums: they are compared to 1e-10 (mu_0 = 1), and to the oracle at the
complex64 tolerance of the KPM (1e-4 over the moments)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pv = pytest.importorskip("paper_1708_09689_gb300")
pytestmark = pytest.mark.gpu

# boundary mixes, lengths below and above the tile, partial tiles, periodic
# lengths 1 and 2 (the ring wraps onto the tile itself), open and periodic z
CASES = [((7, 5, 6), (1, 0, 1)), ((4, 4, 4), (1, 1, 1)), ((3, 2, 5), (0, 1, 0)),
         ((1, 3, 2), (1, 1, 1)), ((2, 1, 3), (1, 0, 0)), ((19, 14, 4), (1, 1, 0)),
         ((17, 25, 3), (0, 0, 1)), ((5, 6, 1), (1, 1, 1))]
TILES = [dict(), dict(tile_x=4, tile_y=3), dict(tile_x=2, tile_y=5, zslab=2),
         dict(tile_x=12, tile_y=12), dict(tile_x=1, tile_y=1, zslab=1)]


def _pair(dims, per, Wd=1.0, seed=3, **kw):
    n = int(np.prod(dims))
    lat = pv.Lattice.ti(dims, per, disorder=(Wd, seed), **kw)
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, W.disorder_potential(n, Wd, seed),
                         kw.get("delta1", 0.0), kw.get("delta2", 0.0))
    return lat, H


def _mu(lat, r, M, a, b, tuning):
    R = r.shape[1]
    if tuning is None:
        lat.set_tuning(R, pv.C64)  # default: single-step sweeps
    else:
        lat.set_tuning(R, pv.C64, kernel=4, **tuning)
    return pv.kpm_moments(lat, M, a, b, r0=r, prec=pv.C64).cpu().numpy()


@pytest.mark.parametrize("dims,per", CASES)
@pytest.mark.parametrize("tile", TILES)
def test_two_step_kpm_matches_single_steps_and_oracle(dims, per, tile):
    lat, H = _pair(dims, per)
    _, _, a, b = lat.spectral_bounds()
    R, M = 4, 40
    rh = W.random_phase_block(H.shape[0], R, 5)
    r = torch.from_numpy(rh).to("cuda", torch.complex64)
    mu1 = _mu(lat, r, M, a, b, None)
    mu2 = _mu(lat, r, M, a, b, tile)
    assert np.max(np.abs(mu2 - mu1)) < 1e-10
    ref = O.kpm_moments(H, r.cpu().numpy().astype(np.complex128), M, a, b).real
    assert np.max(np.abs(mu2 - ref)) < 1e-4


@pytest.mark.parametrize("M", [1, 2, 3, 4, 5, 6, 7, 8, 9, 33])
def test_two_step_kpm_every_moment_count(M):
    # M = 1..4: no double step; odd step counts end with one single step
    lat, H = _pair((6, 5, 7), (1, 1, 0))
    _, _, a, b = lat.spectral_bounds()
    r = torch.from_numpy(W.random_phase_block(H.shape[0], 2, 7)).to("cuda", torch.complex64)
    mu1 = _mu(lat, r, M, a, b, None)
    mu2 = _mu(lat, r, M, a, b, dict(tile_x=4, tile_y=4))
    assert mu2.shape == (2, M)
    assert np.max(np.abs(mu2 - mu1)) < 1e-10


@pytest.mark.parametrize("R", [2, 8, 16, 64])
def test_two_step_kpm_vector_blocks(R):
    lat, H = _pair((9, 7, 5), (1, 0, 1))
    _, _, a, b = lat.spectral_bounds()
    r = torch.from_numpy(W.random_phase_block(H.shape[0], R, 2)).to("cuda", torch.complex64)
    mu1 = _mu(lat, r, 24, a, b, None)
    for tile in [dict()] + ([dict(tile_x=5, tile_y=3)] if R <= 16 else []):
        mu2 = _mu(lat, r, 24, a, b, tile)
        assert np.max(np.abs(mu2 - mu1)) < 1e-10


def test_two_step_kpm_random_start_block_and_graph_replay():
    # start block generated on the device (seed): it occupies a work buffer
    # the two-step rotation must not overwrite
    lat, H = _pair((8, 8, 6), (1, 1, 1))
    _, _, a, b = lat.spectral_bounds()
    R, M = 8, 50
    mu1 = pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C64, seed=11).cpu().numpy()
    lat.set_tuning(R, pv.C64, kernel=4)
    mu2 = pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C64, seed=11).cpu().numpy()
    mu3 = pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C64, seed=11).cpu().numpy()
    assert np.array_equal(mu2, mu3)  # graph replay, fixed reduction order
    assert np.max(np.abs(mu2 - mu1)) < 1e-10
    r = pv.random_vectors(lat, R, pv.C64, 11).cpu().numpy().astype(np.complex128)
    ref = O.kpm_moments(H, r, M, a, b).real
    assert np.max(np.abs(mu2 - ref)) < 1e-4


def test_two_step_kpm_with_delta_terms_and_on_the_fly_potential():
    dims, per = (6, 7, 5), (1, 1, 0)
    lat, H = _pair(dims, per, Wd=2.0, seed=9, delta1=0.3, delta2=-0.2)
    lat_f = pv.Lattice.ti(dims, per, disorder=(2.0, 9), delta1=0.3, delta2=-0.2, on_the_fly=True)
    _, _, a, b = lat.spectral_bounds()
    r = torch.from_numpy(W.random_phase_block(H.shape[0], 4, 3)).to("cuda", torch.complex64)
    mu1 = _mu(lat, r, 30, a, b, None)
    mu2 = _mu(lat, r, 30, a, b, dict(tile_x=3, tile_y=4))
    mu3 = _mu(lat_f, r, 30, a, b, dict(tile_x=3, tile_y=4))
    assert np.max(np.abs(mu2 - mu1)) < 1e-10
    assert np.array_equal(mu2, mu3)
    ref = O.kpm_moments(H, r.cpu().numpy().astype(np.complex128), 30, a, b).real
    assert np.max(np.abs(mu2 - ref)) < 1e-4


def test_two_step_tuning_leaves_single_sweeps_and_rejects_other_paths():
    lat, H = _pair((5, 4, 3), (1, 1, 1))
    x = torch.from_numpy(W.gaussian_block(H.shape[0], 4, 1)).to("cuda", torch.complex64)
    y_def = pv.apply_H(lat, x)
    lat.set_tuning(4, pv.C64, kernel=4)
    assert torch.equal(pv.apply_H(lat, x), y_def)  # single sweeps keep the default kernel
    assert lat.get_tuning(4, pv.C64)["kernel"] == 4
    with pytest.raises(pv.PvscError, match="kernel 4"):
        lat.set_tuning(4, pv.C128, kernel=4)
    with pytest.raises(pv.PvscError, match="kernel 4"):
        lat.set_tuning(1, pv.C64, kernel=4)
    with pytest.raises(pv.PvscError, match="tile"):
        lat.set_tuning(4, pv.C64, kernel=4, tile_x=20, tile_y=20)
    gl = pv.Lattice.graphene((3, 2), (1, 1), V=W.disorder_potential(24, 0.5, 1))
    with pytest.raises(pv.PvscError, match="kernel 4"):
        gl.set_tuning(4, pv.C64, kernel=4)


def test_two_step_kpm_full_slab_against_single_steps():
    # the benchmark's lattice and launch configuration (default tile, whole columns)
    cfg = W.CONFIG_TI_SLAB
    lat = pv.Lattice.ti(cfg.dims, cfg.periodic, t=cfg.t, m=cfg.m, disorder=(cfg.W, cfg.seed_V))
    emin, emax, a, b = lat.spectral_bounds()
    R, M = 8, 24
    mu1 = pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C64, seed=5).cpu().numpy()
    lat.set_tuning(R, pv.C64, kernel=4)
    mu2 = pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C64, seed=5).cpu().numpy()
    assert np.allclose(mu2[:, 0], 1.0, atol=1e-6)
    assert np.max(np.abs(mu2)) <= 1.0 + 1e-6
    assert np.max(np.abs(mu2 - mu1)) < 1e-10


def test_two_step_work_buffer_follows_the_tuning():
    lat, H = _pair((6, 5, 4), (1, 1, 1))
    _, _, a, b = lat.spectral_bounds()
    R, M = 4, 16
    wb = lat.work_bytes(pv.OP_KPM, R, pv.C64, M)
    lat.set_tuning(R, pv.C64, kernel=4)
    wb4 = lat.work_bytes(pv.OP_KPM, R, pv.C64, M)
    vec = (lat.n_sites * 4 * R * 8 + 255) // 256 * 256  # one complex64 block, 256-byte aligned
    assert wb4 == wb + 2 * vec
    with pytest.raises(pv.PvscError, match="work buffer"):
        pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C64, seed=1, work=pv.work_buffer(wb))
    mu = pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C64, seed=1, work=pv.work_buffer(wb4))
    assert np.allclose(mu.cpu().numpy()[:, 0], 1.0, atol=1e-6)
