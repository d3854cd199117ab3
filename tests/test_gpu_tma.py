"""The TI sweep with TMA-staged plane tiles (tuning kernel 7, complex64, R = 1 .. 64;
R = 1, 2 one thread per narrow site, R = 32 and 64 as slices of 16 vectors).

Its stencil arithmetic is the register z-march's, in the same order, so the
vectors it writes must equal the default sweep's bit for bit; they are also
checked against the oracle.  The cases cover every boundary mix, partial tiles
(Lx, Ly not multiples of the tile), periodic lengths 1 and 2 (a site is its own
or its double neighbour), one-plane z-chunks (every unit shorter than the copy
ring), the three potential sources and the Delta terms.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

pv = pytest.importorskip("paper_1708_09689_gb300")

CASES = [
    # dims, periodic, z-chunk depth
    ((32, 16, 6), (1, 1, 0), 0),
    ((20, 12, 5), (1, 1, 1), 2),      # partial tiles along x and y
    ((16, 8, 7), (0, 0, 0), 1),       # open everywhere, one-plane chunks
    ((4, 2, 3), (1, 1, 1), 0),        # x shorter than a tile, y of length 2
    ((8, 1, 4), (1, 1, 0), 3),        # y of length 1: its own neighbour
    ((36, 9, 1), (0, 1, 1), 0),       # one plane, periodic z of length 1
]


def _lattice(dims, per, vmode, delta):
    n = int(np.prod(dims))
    kw = dict(delta1=0.3, delta2=-0.2) if delta else {}
    if vmode == "stored":
        V = W.disorder_potential(n, 2.0, 7)
        return pv.Lattice.ti(dims, per, disorder=(2.0, 7), **kw), V
    if vmode == "fly":
        V = W.disorder_potential(n, 2.0, 7)
        return pv.Lattice.ti(dims, per, disorder=(2.0, 7), on_the_fly=True, **kw), V
    return pv.Lattice.ti(dims, per, **kw), np.zeros(n)


# the half tiles with three planes in flight (R = 32, 64: slices of 16 vectors on the tiles of R = 16)
DEEP_TILE = {1: (32, 16), 2: (32, 8), 4: (16, 8), 8: (16, 4), 16: (8, 4), 32: (8, 4), 64: (8, 4)}


def _variant(R, v):
    """Launch variants of kernel 7: the large tile on 8 warps (two items per
    thread) or on 16 warps (one item), and the half tile with the deeper rings."""
    if v == "deep":
        return dict(zip(("tile_x", "tile_y"), DEEP_TILE[R]))
    return dict(threads=512) if v == "wide" else {}


@pytest.mark.parametrize("dims,per,zs", CASES)
@pytest.mark.parametrize("R,variant", [(R, v) for R in (1, 2, 4, 8, 16, 32, 64) for v in ("large", "wide", "deep")])
def test_tma_sweep_equals_default_sweep_and_oracle(dims, per, zs, R, variant):
    lat, V = _lattice(dims, per, "stored", False)
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V)
    x = torch.from_numpy(W.gaussian_block(H.shape[0], R, 1)).to("cuda", torch.complex64)
    y0 = pv.apply_H(lat, x)
    lat.set_tuning(R, pv.C64, kernel=7, zslab=zs, **_variant(R, variant))
    y1 = pv.apply_H(lat, x)
    assert torch.equal(y0, y1)
    ref = H @ x.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(y1.cpu().numpy() - ref) / np.linalg.norm(ref) < 2e-6


@pytest.mark.parametrize("vmode,delta", [("stored", True), ("fly", False), ("zero", True)])
@pytest.mark.parametrize("R,variant", [(R, v) for R in (1, 2, 4, 8, 16, 32, 64) for v in ("large", "wide")])
def test_tma_fused_step_with_z_and_dots(vmode, delta, R, variant):
    dims, per = (24, 16, 5), (1, 0, 1)
    lat, V = _lattice(dims, per, vmode, delta)
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V, 0.3 if delta else 0.0, -0.2 if delta else 0.0)
    D = H.shape[0]
    x = torch.from_numpy(W.gaussian_block(D, R, 2)).to("cuda", torch.complex64)
    yin = torch.from_numpy(W.gaussian_block(D, R, 3)).to("cuda", torch.complex64)
    zin = torch.from_numpy(W.gaussian_block(D, R, 4)).to("cuda", torch.complex64)
    al = [0.2 + 0.01 * r for r in range(R)]
    be = [0.1 * (r - 2) for r in range(R)]
    ga = [-1.0 + 0.05 * r for r in range(R)]
    de = [0.5] * R
    ya, za = yin.clone(), zin.clone()
    da = pv.cheb_step(lat, x, ya, al, be, ga, z=za, delta=de, dots=7)
    lat.set_tuning(R, pv.C64, kernel=7, **_variant(R, variant))
    yb, zb = yin.clone(), zin.clone()
    db = pv.cheb_step(lat, x, yb, al, be, ga, z=zb, delta=de, dots=7)
    assert torch.equal(ya, yb) and torch.equal(za, zb)
    scale = da.abs().max().item()
    assert (da - db).abs().max().item() <= 1e-6 * scale
    xr = x.cpu().numpy().astype(np.complex128)
    yr, zr, dots = O.cheb_step(H, xr, yin.cpu().numpy().astype(np.complex128), al, be, ga,
                               zin.cpu().numpy().astype(np.complex128), de)
    assert np.linalg.norm(yb.cpu().numpy() - yr) / np.linalg.norm(yr) < 2e-6
    assert np.linalg.norm(zb.cpu().numpy() - zr) / np.linalg.norm(zr) < 2e-6
    got = db.cpu().numpy()
    # <x|x>, Re<y|x>, Im<y|x>, <y|y> of the written vectors, against the oracle's fp64 sums
    assert np.allclose(got[0], dots[:, 0].real, rtol=1e-5)
    assert np.allclose(got[1], dots[:, 1].real, rtol=1e-5, atol=1e-5 * np.abs(dots[:, 1]).max())
    assert np.allclose(got[2], dots[:, 1].imag, rtol=1e-5, atol=1e-5 * np.abs(dots[:, 1]).max())
    assert np.allclose(got[3], dots[:, 2].real, rtol=1e-5)


@pytest.mark.parametrize("dims,per,zs", CASES[:3])
@pytest.mark.parametrize("R,variant", [(R, v) for R in (1, 2, 4, 8, 16, 32, 64) for v in ("large", "wide", "deep")])
def test_tma_kpm_moments_match_oracle_and_default(dims, per, zs, R, variant):
    lat, V = _lattice(dims, per, "stored", False)
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V)
    a, b = O.cheb_scale(*O.gershgorin(H))
    M = 64
    r = W.random_phase_block(H.shape[0], R, 5)
    r0 = torch.from_numpy(r).to("cuda", torch.complex64)
    mu0 = pv.kpm_moments(lat, M, a, b, r0=r0).cpu().numpy()
    lat.set_tuning(R, pv.C64, kernel=7, zslab=zs, **_variant(R, variant))
    mu1 = pv.kpm_moments(lat, M, a, b, r0=r0).cpu().numpy()
    assert np.max(np.abs(mu1 - mu0)) < 1e-9
    ref = O.kpm_moments(H, r, M, a, b).real
    assert np.max(np.abs(mu1 - ref)) / ref[0, 0] < 1e-4


def test_tma_series_and_propagation():
    dims, per, R = (16, 16, 6), (1, 1, 0), 8
    lat, V = _lattice(dims, per, "stored", False)
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V)
    lat.set_tuning(R, pv.C64, kernel=7)
    _, _, a, b = lat.spectral_bounds()
    x = W.gaussian_block(H.shape[0], R, 3)
    x /= np.linalg.norm(x, axis=0)
    psi = torch.from_numpy(x).cuda()
    pv.cheb_propagate(lat, psi, 0.6, 3, a, b, prec=pv.C64)
    ref = O.propagate(H, x, 0.6, 3, a, b)
    assert np.linalg.norm(psi.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5


def test_tma_kernel_is_refused_where_it_does_not_apply():
    lat = pv.Lattice.ti((16, 8, 4), (1, 1, 0))
    for R, prec in ((8, pv.C128), (2, pv.C128), (1, pv.C128)):
        with pytest.raises(pv.PvscError, match="kernel 7"):
            lat.set_tuning(R, prec, kernel=7)
    with pytest.raises(pv.PvscError, match="kernel 7"):
        pv.Lattice.ti((18, 8, 4), (1, 1, 0)).set_tuning(8, pv.C64, kernel=7)  # Lx % 4 != 0
    with pytest.raises(pv.PvscError, match="kernel 7 takes no tile"):
        lat.set_tuning(8, pv.C64, kernel=7, tile_x=8, tile_y=8)
    gl = pv.Lattice.graphene((8, 8), (1, 1))
    with pytest.raises(pv.PvscError, match="kernel 7"):
        gl.set_tuning(8, pv.C64, kernel=7)


def test_tma_sweep_reports_no_device_error():
    lat = pv.Lattice.ti((32, 32, 8), (1, 1, 0), disorder=(1.0, 3))
    lat.set_tuning(8, pv.C64, kernel=7)
    x = pv.random_vectors(lat, 8, pv.C64, 1)
    pv.apply_H(lat, x)
    assert pv.device_error() == 0


# Weyl-semimetal cells (two x-adjacent sites) on the TMA-staged sweep: Lx a
# multiple of 4; periodic y of length 1 and 2, open and periodic z, partial tiles
WSM_CASES = [((16, 5, 4), (1, 1, 0)), ((36, 2, 3), (1, 1, 1)), ((8, 1, 5), (0, 1, 1)), ((12, 9, 2), (0, 0, 0))]


@pytest.mark.parametrize("dims,per", WSM_CASES)
@pytest.mark.parametrize("R", [1, 2, 4, 8, 16, 32, 64])
def test_tma_weyl_cells_equal_the_cell_sweeps_and_oracle(dims, per, R):
    n = int(np.prod(dims))
    V = W.disorder_potential(n, 1.5, 6)
    lat = pv.Lattice.wsm(dims, per, V=V)
    H = O.wsm_hamiltonian(dims, per, V)
    x = torch.from_numpy(W.gaussian_block(H.shape[0], R, 1)).to("cuda", torch.complex64)
    y_flat = pv.apply_H(lat, x)              # default: the flat cell sweep
    lat.set_tuning(R, pv.C64, threads=128, kernel=0)
    y_march = pv.apply_H(lat, x)             # the z-marching cell sweep
    if R >= 4:                                    # the cells marching along x (R >= 4)
        lat.set_tuning(R, pv.C64, kernel=8)
        assert torch.equal(pv.apply_H(lat, x), y_flat)
    lat.set_tuning(R, pv.C64, kernel=7, **_variant(R, "deep"))  # the half tile
    assert torch.equal(pv.apply_H(lat, x), y_flat)
    lat.set_tuning(R, pv.C64, kernel=7)
    y_tma = pv.apply_H(lat, x)
    assert torch.equal(y_tma, y_march) and torch.equal(y_tma, y_flat)
    ref = H @ x.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(y_tma.cpu().numpy() - ref) / np.linalg.norm(ref) < 2e-6
    # KPM moments and a fused step with z and dots
    a, b = O.cheb_scale(*O.gershgorin(H))
    r = W.random_phase_block(H.shape[0], R, 5)
    mu = pv.kpm_moments(lat, 24, a, b, r0=torch.from_numpy(r).to("cuda", torch.complex64)).cpu().numpy()
    refm = O.kpm_moments(H, r, 24, a, b).real
    assert np.max(np.abs(mu - refm)) < 1e-4
    yin = torch.from_numpy(W.gaussian_block(H.shape[0], R, 3)).to("cuda", torch.complex64)
    z0 = torch.from_numpy(W.gaussian_block(H.shape[0], R, 4)).to("cuda", torch.complex64)
    ya, za = yin.clone(), z0.clone()
    pv.cheb_step(lat, x, ya, [0.2] * R, [0.1] * R, [-1.0] * R, z=za, delta=[0.5] * R, dots=7)
    lat.set_tuning(R, pv.C64, threads=128, kernel=0)
    yb, zb = yin.clone(), z0.clone()
    pv.cheb_step(lat, x, yb, [0.2] * R, [0.1] * R, [-1.0] * R, z=zb, delta=[0.5] * R, dots=7)
    assert torch.equal(ya, yb) and torch.equal(za, zb)


# Kernel 8: the same tiles marching along x (tiles over the (y, z) columns), for
# lattices whose z columns are short; x is the march axis, so its length is free.
XM_CASES = [
    ((24, 16, 6), (1, 1, 0), 0),
    ((20, 12, 5), (1, 1, 1), 7),      # partial tiles along y and z, x-chunks of 7
    ((16, 9, 3), (0, 0, 0), 1),       # open everywhere, one-plane chunks
    ((8, 2, 1), (1, 1, 1), 0),        # z of length 1 (its own neighbour), y of length 2
    ((12, 1, 8), (1, 1, 0), 3),       # y of length 1
    ((4, 9, 10), (1, 0, 1), 0),       # x of length 4 (shorter than the columns)
]


@pytest.mark.parametrize("dims,per,zs", XM_CASES)
@pytest.mark.parametrize("R,variant", [(R, v) for R in (4, 8, 16, 32, 64) for v in ("large", "deep")])
def test_tma_x_march_equals_default_sweep_and_oracle(dims, per, zs, R, variant):
    lat, V = _lattice(dims, per, "stored", False)
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V)
    x = torch.from_numpy(W.gaussian_block(H.shape[0], R, 1)).to("cuda", torch.complex64)
    y0 = pv.apply_H(lat, x)
    lat.set_tuning(R, pv.C64, kernel=8, zslab=zs, **_variant(R, variant))
    y1 = pv.apply_H(lat, x)
    assert torch.equal(y0, y1)
    ref = H @ x.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(y1.cpu().numpy() - ref) / np.linalg.norm(ref) < 2e-6
    a, b = O.cheb_scale(*O.gershgorin(H))
    r = W.random_phase_block(H.shape[0], R, 5)
    r0 = torch.from_numpy(r).to("cuda", torch.complex64)
    mu1 = pv.kpm_moments(lat, 40, a, b, r0=r0).cpu().numpy()
    lat.set_tuning(R, pv.C64, threads=128, kernel=0)
    mu0 = pv.kpm_moments(lat, 40, a, b, r0=r0).cpu().numpy()
    assert np.max(np.abs(mu1 - mu0)) < 1e-9
    assert pv.device_error() == 0


@pytest.mark.parametrize("vmode,delta", [("stored", True), ("fly", False), ("zero", True)])
def test_tma_x_march_series_and_the_step_with_z(vmode, delta):
    dims, per, R = (24, 8, 6), (1, 0, 1), 16
    lat, V = _lattice(dims, per, vmode, delta)
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V, 0.3 if delta else 0.0, -0.2 if delta else 0.0)
    D = H.shape[0]
    _, _, a, b = lat.spectral_bounds()
    x = W.gaussian_block(D, R, 3)
    x /= np.linalg.norm(x, axis=0)
    psi0 = torch.from_numpy(x).cuda()
    outs = []
    for kernel in (0, 8):
        lat.set_tuning(R, pv.C64, threads=128 if kernel == 0 else 256, kernel=kernel)
        psi = psi0.clone()
        pv.cheb_propagate(lat, psi, 0.6, 3, a, b, prec=pv.C64)  # series sweeps with the accumulator
        xc = torch.from_numpy(W.gaussian_block(D, R, 2)).to("cuda", torch.complex64)
        yin = torch.from_numpy(W.gaussian_block(D, R, 4)).to("cuda", torch.complex64)
        zin = torch.from_numpy(W.gaussian_block(D, R, 6)).to("cuda", torch.complex64)
        pv.cheb_step(lat, xc, yin, [0.2] * R, [0.1] * R, [-1.0] * R, z=zin, delta=[0.5] * R, dots=7)
        outs.append((psi, yin, zin))
    assert torch.equal(outs[0][1], outs[1][1]) and torch.equal(outs[0][2], outs[1][2])
    assert torch.equal(outs[0][0], outs[1][0])
    ref = O.propagate(H, x, 0.6, 3, a, b)
    assert np.linalg.norm(outs[1][0].cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5


def test_tma_x_march_is_validated():
    lat = pv.Lattice.ti((16, 8, 4), (1, 1, 0))
    with pytest.raises(pv.PvscError, match="kernel 8"):
        lat.set_tuning(8, pv.C64, kernel=8, threads=512)
    with pytest.raises(pv.PvscError, match="kernel 8"):
        lat.set_tuning(8, pv.C128, kernel=8)
    with pytest.raises(pv.PvscError, match="kernel 8"):
        pv.Lattice.wsm((16, 4, 4), (1, 1, 0)).set_tuning(8, pv.C64, kernel=8, tile_x=16, tile_y=4)
    with pytest.raises(pv.PvscError, match="kernel 8"):
        pv.Lattice.graphene((8, 8), (1, 1)).set_tuning(8, pv.C64, kernel=8)
    with pytest.raises(pv.PvscError, match="kernel must be"):
        lat.set_tuning(8, pv.C64, kernel=9)
    lat.set_tuning(8, pv.C64, kernel=8, tile_x=16, tile_y=4)
    assert lat.get_tuning(8, pv.C64)["kernel"] == 8


@pytest.mark.parametrize("graphs", [True, False])
@pytest.mark.parametrize("model,R", [("ti", 8), ("ti", 64), ("wsm", 16)])
def test_programmatic_dependent_launch_changes_no_bit(monkeypatch, graphs, model, R):
    # The TMA-staged sweeps start the next sweep's blocks early (they wait for the
    # previous grid before touching global memory).  The KPM moments and a
    # filtered block (accumulating sweeps writing over their y_in) must be the
    # same bits with and without it, replayed from a graph or launched directly.
    monkeypatch.setenv("PVSC_NO_GRAPH", "0" if graphs else "1")
    dims, per = ((48, 40, 9), (1, 1, 0)) if model == "ti" else ((64, 24, 10), (1, 0, 1))
    out = {}
    for pdl in ("0", "1"):
        monkeypatch.setenv("PVSC_NO_PDL", "0" if pdl == "1" else "1")
        lat = (pv.Lattice.ti(dims, per, disorder=(2.0, 3)) if model == "ti"
               else pv.Lattice.wsm(dims, per, disorder=(1.0, 5)))  # a fresh handle: no cached graph
        lat.set_tuning(R, pv.C64, kernel=7)
        _, _, a, b = lat.spectral_bounds()
        mu = pv.kpm_moments(lat, 40, a, b, R=R, seed=6).cpu().numpy()
        x = pv.random_vectors(lat, R, pv.C128, 8)
        y = pv.cheb_filter(lat, x, [1.0 / (k + 1) for k in range(14)], a, b, prec=pv.C64).cpu().numpy()
        assert pv.device_error() == 0
        out[pdl] = (mu, y)
    assert np.array_equal(out["0"][0], out["1"][0])
    assert np.array_equal(out["0"][1], out["1"][1])


@pytest.mark.parametrize("dims,per,R,kernel", [
    ((32, 16, 12), (1, 1, 0), 8, 7),   # 8 tiles x chunks: fewer units than SMs, spread over all
    ((8, 8, 1), (1, 1, 1), 8, 7),      # one tile, one plane: almost every block has no plane
    ((16, 8, 3), (0, 1, 1), 64, 7),    # slices of 16 vectors, fewer planes than blocks
    ((32, 8, 4), (1, 1, 0), 1, 7),     # narrow sites
    ((48, 16, 8), (1, 0, 1), 16, 8),   # marching along x
])
def test_tma_sweep_spread_over_all_sms_equals_default(dims, per, R, kernel):
    # blocks_per_sm = 1 splits the planes over the whole grid even when there are
    # fewer units than SMs (blocks without a plane issue no copy); the filtered
    # vectors must be those of the default launch bit for bit, the moments equal
    # up to the order in which the blocks' fp64 dot partials are added.
    lat = pv.Lattice.ti(dims, per, disorder=(2.0, 9))
    _, _, a, b = lat.spectral_bounds()
    out = []
    for spread in (0, 1):
        lat.set_tuning(R, pv.C64, kernel=kernel, blocks_per_sm=spread)
        mu = pv.kpm_moments(lat, 24, a, b, R=R, seed=2).cpu().numpy()
        x = pv.random_vectors(lat, R, pv.C128, 5)
        y = pv.cheb_filter(lat, x, [0.5, -0.25, 0.125, 0.3, -0.2, 0.1, 0.05], a, b, prec=pv.C64).cpu().numpy()
        assert pv.device_error() == 0
        out.append((mu, y))
    assert np.max(np.abs(out[0][0] - out[1][0])) < 1e-12
    assert np.array_equal(out[0][1], out[1][1])


def test_tma_spread_tuning_is_validated():
    lat = pv.Lattice.ti((16, 8, 4), (1, 1, 0))
    with pytest.raises(pv.PvscError, match="blocks_per_sm"):
        lat.set_tuning(8, pv.C64, kernel=7, blocks_per_sm=2)
    lat.set_tuning(8, pv.C64, kernel=7, blocks_per_sm=1)
    assert lat.get_tuning(8, pv.C64)["blocks_per_sm"] == 1
