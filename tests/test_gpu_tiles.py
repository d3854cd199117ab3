"""The z-marching TI sweep over 2D column tiles (tuning kernel 5) against the
default row-segment grouping: the per-site arithmetic is the same, so the
vectors are bit-identical; moments differ only in the order of the dot sums."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pv = pytest.importorskip("paper_1708_09689_gb300")
pytestmark = pytest.mark.gpu

CASES = [((7, 5, 6), (1, 0, 1)), ((4, 4, 4), (1, 1, 1)), ((3, 2, 5), (0, 1, 0)),
         ((1, 3, 2), (1, 1, 1)), ((19, 13, 4), (1, 1, 0))]
# (R, precision, vpt, tile_x, tile_y): tile_x tile_y R / vpt threads, a multiple of 32
SHAPES = [(8, pv.C64, 2, 8, 4), (8, pv.C64, 2, 4, 4), (4, pv.C64, 2, 4, 8), (1, pv.C64, 1, 8, 4),
          (4, pv.C128, 1, 4, 2), (8, pv.C128, 1, 4, 8), (2, pv.C64, 2, 16, 2)]


@pytest.mark.parametrize("dims,per", CASES)
@pytest.mark.parametrize("R,prec,vpt,tx,ty", SHAPES)
def test_column_tiles_equal_the_default_sweep(dims, per, R, prec, vpt, tx, ty):
    n = int(np.prod(dims))
    lat = pv.Lattice.ti(dims, per, disorder=(1.5, 2))
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, W.disorder_potential(n, 1.5, 2))
    cdt = torch.complex128 if prec == pv.C128 else torch.complex64
    x = torch.from_numpy(W.gaussian_block(H.shape[0], R, 1)).to("cuda", cdt)
    y0 = pv.apply_H(lat, x)
    lat.set_tuning(R, prec, threads=tx * ty * R // vpt, vpt=vpt, tile_x=tx, tile_y=ty, kernel=5)
    y1 = pv.apply_H(lat, x)
    assert torch.equal(y0, y1)
    ref = H @ x.cpu().numpy().astype(np.complex128)
    tol = 1e-12 if prec == pv.C128 else 2e-6
    assert np.linalg.norm(y1.cpu().numpy() - ref) / np.linalg.norm(ref) < tol
    _, _, a, b = lat.spectral_bounds()
    mu1 = pv.kpm_moments(lat, 20, a, b, r0=x / torch.linalg.vector_norm(x, dim=0), prec=prec).cpu().numpy()
    lat.set_tuning(R, prec)
    mu0 = pv.kpm_moments(lat, 20, a, b, r0=x / torch.linalg.vector_norm(x, dim=0), prec=prec).cpu().numpy()
    assert np.max(np.abs(mu1 - mu0)) < 1e-10


def test_column_tile_shapes_are_checked():
    lat = pv.Lattice.ti((8, 8, 4), (1, 1, 1))
    with pytest.raises(pv.PvscError, match="kernel 5"):
        lat.set_tuning(8, pv.C64, vpt=2, tile_x=3, tile_y=3, kernel=5)  # 36 threads
    with pytest.raises(pv.PvscError, match="kernel 5"):
        lat.set_tuning(8, pv.C64, vpt=2, tile_x=16, tile_y=8, kernel=5)  # 512 threads
    gl = pv.Lattice.graphene((4, 4), (1, 1))
    with pytest.raises(pv.PvscError, match="kernel 5"):
        gl.set_tuning(1, pv.C64, tile_x=8, tile_y=4, kernel=5)


XCASES = CASES + [((2, 5, 3), (1, 1, 0)), ((1, 4, 3), (1, 0, 1)), ((24, 3, 2), (0, 1, 1))]


@pytest.mark.parametrize("dims,per", XCASES)
@pytest.mark.parametrize("R,prec,vpt,threads,xseg", [(8, pv.C64, 2, 128, 0), (8, pv.C64, 2, 64, 3),
                                                     (1, pv.C64, 1, 128, 0), (4, pv.C128, 1, 128, 5),
                                                     (64, pv.C64, 1, 128, 0)])
def test_march_along_x_equals_the_default_sweep(dims, per, R, prec, vpt, threads, xseg):
    n = int(np.prod(dims))
    lat = pv.Lattice.ti(dims, per, disorder=(1.5, 2), delta1=0.2)
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, W.disorder_potential(n, 1.5, 2), 0.2, 0.0)
    cdt = torch.complex128 if prec == pv.C128 else torch.complex64
    x = torch.from_numpy(W.gaussian_block(H.shape[0], R, 1)).to("cuda", cdt)
    y0 = pv.apply_H(lat, x)
    _, _, a, b = lat.spectral_bounds()
    r0 = x / torch.linalg.vector_norm(x, dim=0)
    mu0 = pv.kpm_moments(lat, 20, a, b, r0=r0, prec=prec).cpu().numpy()
    lat.set_tuning(R, prec, threads=threads, vpt=vpt, zslab=xseg, kernel=6)
    y1 = pv.apply_H(lat, x)
    assert torch.equal(y0, y1)  # same arithmetic in the same order
    ref = H @ x.cpu().numpy().astype(np.complex128)
    tol = 1e-12 if prec == pv.C128 else 2e-6
    assert np.linalg.norm(y1.cpu().numpy() - ref) / np.linalg.norm(ref) < tol
    mu1 = pv.kpm_moments(lat, 20, a, b, r0=r0, prec=prec).cpu().numpy()
    assert np.max(np.abs(mu1 - mu0)) < 1e-10


def test_march_along_x_needs_a_ti_lattice():
    gl = pv.Lattice.graphene((4, 4), (1, 1))
    with pytest.raises(pv.PvscError, match="kernel 6"):
        gl.set_tuning(1, pv.C64, kernel=6)


@pytest.mark.parametrize("kernel", [1, 2, 3, 6])
def test_kernels_without_tiles_reject_a_tile(kernel):
    # a tile selects the staged sweep of kernel 0 only; other kernels must not be
    # replaced by it silently
    lat = pv.Lattice.ti((8, 8, 4), (1, 1, 0))
    with pytest.raises(pv.PvscError, match="takes no tile"):
        lat.set_tuning(8, pv.C64, threads=128, tile_x=4, tile_y=4, kernel=kernel)


@pytest.mark.parametrize("prec,tol", [(pv.C128, 1e-12), (pv.C64, 1e-5)])
def test_march_along_x_series_propagation_and_step(prec, tol):
    # the accumulating (series) and fused-step features of the sweep marching along x
    dims, per = (9, 4, 3), (1, 0, 1)
    n = int(np.prod(dims))
    lat = pv.Lattice.ti(dims, per, disorder=(1.0, 6))
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, W.disorder_potential(n, 1.0, 6))
    R = 4
    lat.set_tuning(R, prec, threads=128, vpt=2 if prec == pv.C64 else 1, kernel=6)
    _, _, a, b = lat.spectral_bounds()
    x = W.gaussian_block(H.shape[0], R, 3)
    x /= np.linalg.norm(x, axis=0)
    psi = torch.from_numpy(x).cuda()
    pv.cheb_propagate(lat, psi, 0.6, 3, a, b, prec=prec)
    ref = O.propagate(H, x, 0.6, 3, a, b)
    assert np.linalg.norm(psi.cpu().numpy() - ref) / np.linalg.norm(ref) < tol
    cdt = torch.complex128 if prec == pv.C128 else torch.complex64
    xs = torch.from_numpy(x).to("cuda", cdt)
    y0 = W.gaussian_block(H.shape[0], R, 4)
    yt = torch.from_numpy(y0).to("cuda", cdt)
    pv.cheb_step(lat, xs, yt, [0.3] * R, [0.1] * R, [-1.0] * R)
    xr = xs.cpu().numpy().astype(np.complex128)
    yr, _, _ = O.cheb_step(H, xr, torch.from_numpy(y0).to(cdt).numpy().astype(np.complex128),
                           [0.3] * R, [0.1] * R, [-1.0] * R)
    got = yt.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - yr) / np.linalg.norm(yr) < (1e-12 if prec == pv.C128 else 2e-6)


@pytest.mark.parametrize("op", [pv.OP_SERIES, pv.OP_APPLY, pv.OP_KPM])
def test_autotune_per_operation_keeps_results(op):
    # the launch shape tuned on an operation's own sweeps changes no result:
    # the filter series and the moments against the oracle
    dims, per, R = (32, 16, 6), (1, 1, 0), 8
    n = int(np.prod(dims))
    lat = pv.Lattice.ti(dims, per, disorder=(1.0, 4))
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, W.disorder_potential(n, 1.0, 4))
    t = lat.autotune(R, pv.C64, op=op)
    assert t["time_ms"] > 0
    _, _, a, b = lat.spectral_bounds()
    x = W.gaussian_block(H.shape[0], R, 5)
    g = [1.0, 0.5, -0.25, 0.125, 0.3]
    y = pv.cheb_filter(lat, torch.from_numpy(x).cuda(), g, a, b, prec=pv.C64).cpu().numpy()
    ref = O.cheb_series(H, x, np.array(g, dtype=np.complex128), a, b)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-5
    mu = pv.kpm_moments(lat, 24, a, b, R=R, prec=pv.C64, seed=3).cpu().numpy()
    refm = O.kpm_moments(H, W.random_phase_block(4 * n, R, 3), 24, a, b).real
    assert np.max(np.abs(mu - refm)) < 1e-4
