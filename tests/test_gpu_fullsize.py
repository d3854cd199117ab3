"""Parity at the full workload sizes, in the launch configuration the benchmark
times (autotuned shapes).  The oracle cannot run these lattices end to end, so
outputs are checked on sampled rows (the oracle assembles just those rows of
H from the model equations) and through properties that hold at any size:
mu_0 = 1 for random-phase vectors, |mu_k| <= mu_0, <x|x> and <y|x> recomputed
on the host from the same vectors, norm conservation of the propagation, and
complex64 against complex128 on the same inputs."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

pv = pytest.importorskip("paper_1708_09689_gb300")


def sample_sites(n, k, seed):
    rng = np.random.default_rng(seed)
    s = rng.choice(n, size=k, replace=False)
    return np.sort(np.concatenate([s, [0, n - 1]]))


@pytest.fixture(scope="module")
def ti_slab():
    cfg = W.CONFIG_TI_SLAB
    n = cfg.n_sites
    V = W.disorder_potential(n, cfg.W, cfg.seed_V)
    lat = pv.Lattice.ti(cfg.dims, cfg.periodic, t=cfg.t, m=cfg.m, disorder=(cfg.W, cfg.seed_V))
    rows = sample_sites(n, 3000, 1)
    Hs = O.ti_hamiltonian(cfg.dims, cfg.periodic, cfg.t, cfg.m, V, rows=rows)
    return cfg, lat, Hs, rows


@pytest.mark.parametrize("prec", [pv.C64, pv.C128])
def test_ti_slab_fused_step_sampled_rows_and_full_dots(ti_slab, prec):
    cfg, lat, Hs, rows = ti_slab
    R = 8
    lat.autotune(R, prec)
    x = pv.random_vectors(lat, R, prec, 3)
    y0 = pv.random_vectors(lat, R, prec, 4)
    y = y0.clone()
    a, b = 9.005, 0.0
    d = pv.cheb_step(lat, x, y, [2 / a] * R, [b] * R, [-1.0] * R, dots=7).cpu().numpy()
    xh = x.cpu().numpy().astype(np.complex128)
    yh = y.cpu().numpy().astype(np.complex128)
    y0h = y0.cpu().numpy().astype(np.complex128)
    idx = (rows[:, None] * 4 + np.arange(4)[None, :]).reshape(-1)
    ref = (2 / a) * (Hs @ xh)[idx] - (2 / a) * b * xh[idx] - y0h[idx]
    tol = 1e-12 if prec == pv.C128 else 2e-6
    assert np.linalg.norm(yh[idx] - ref) / np.linalg.norm(ref) < tol
    # the fused fp64 reductions against the host sums of the same vectors
    xx = np.sum(np.abs(xh) ** 2, axis=0)
    xy = np.sum(np.conj(yh) * xh, axis=0)
    yy = np.sum(np.abs(yh) ** 2, axis=0)
    rtol = 1e-12 if prec == pv.C128 else 1e-6
    assert np.allclose(d[0], xx, rtol=rtol, atol=0)
    assert np.allclose(d[1], xy.real, rtol=rtol, atol=rtol * np.abs(xy).max())
    assert np.allclose(d[3], yy, rtol=rtol, atol=0)


def test_ti_slab_kpm_properties_and_precisions(ti_slab):
    cfg, lat, Hs, rows = ti_slab
    R, M = 8, 64
    emin, emax, a, b = lat.spectral_bounds()
    mu64 = pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C64, seed=3).cpu().numpy()
    mu128 = pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C128, seed=3).cpu().numpy()
    assert np.allclose(mu128[:, 0], 1.0, atol=1e-12)
    assert np.max(np.abs(mu128)) <= 1.0 + 1e-12
    assert np.max(np.abs(mu64 - mu128)) < 1e-4
    # mu_1 = <r|H~|r> from one stencil application of the same start block
    r = pv.random_vectors(lat, R, pv.C128, 3)
    hr = pv.apply_H(lat, r).cpu().numpy()
    rh = r.cpu().numpy()
    mu1 = (np.sum(np.conj(rh) * hr, axis=0).real - b) / a
    assert np.max(np.abs(mu128[:, 1] - mu1)) < 1e-12


@pytest.fixture(scope="module")
def graphene_qd():
    cfg = W.CONFIG_GRAPHENE_QD
    V = cfg.potential()
    lat = pv.Lattice.graphene(cfg.cells, (0, 0), t=cfg.t, V=V)
    return cfg, lat, V


def test_graphene_qd_apply_sampled_rows(graphene_qd):
    cfg, lat, V = graphene_qd
    ncell = cfg.cells[0] * cfg.cells[1]
    cells = sample_sites(ncell, 3000, 2)
    Hs = O.graphene_hamiltonian(cfg.cells, (0, 0), cfg.t, V, rows=cells)
    idx = (cells[:, None] * 4 + np.arange(4)[None, :]).reshape(-1)
    psi = torch.from_numpy(cfg.packet()).cuda()
    for prec, tol in ((pv.C128, 1e-12), (pv.C64, 2e-6)):
        x = psi if prec == pv.C128 else psi.to(torch.complex64)
        lat.autotune(1, prec)
        y = pv.apply_H(lat, x).cpu().numpy().astype(np.complex128)
        xh = x.cpu().numpy().astype(np.complex128)
        ref = (Hs @ xh)[idx]
        assert np.linalg.norm(y[idx] - ref) / np.linalg.norm(ref) < tol


def test_graphene_qd_propagation_norm_and_precision(graphene_qd):
    cfg, lat, V = graphene_qd
    emin, emax, a, b = lat.spectral_bounds()
    assert len(pv.propagation_coeffs(a * cfg.dt, cfg.trunc)) == 20  # M = 19
    psi0 = torch.from_numpy(cfg.packet()).cuda()
    p128 = psi0.clone()
    p64 = psi0.clone()
    pv.cheb_propagate(lat, p128, cfg.dt, 4, a, b, cfg.trunc, prec=pv.C128)
    pv.cheb_propagate(lat, p64, cfg.dt, 4, a, b, cfg.trunc, prec=pv.C64)
    assert abs(torch.linalg.vector_norm(p128).item() - 1.0) < 1e-12
    assert abs(torch.linalg.vector_norm(p64).item() - 1.0) < 1e-5
    assert torch.linalg.vector_norm(p64 - p128).item() < 1e-4
    # the packet moved: overlap with the start state dropped below 1
    assert abs(torch.vdot(psi0, p128).item()) < 0.999


def test_batched_kpm_full_workload_properties():
    specs = W.batched_lattices()
    lats = [pv.Lattice.ti((L, L, L), (1, 1, 1), disorder=(Wd, s)) for L, Wd, s in specs]
    ab = [lat.spectral_bounds()[2:] for lat in lats]
    R, M = 16, 64
    seeds = list(range(100, 100 + len(lats)))
    mu = pv.kpm_moments_batched(lats, M, [x[0] for x in ab], [x[1] for x in ab], R=R, prec=pv.C64,
                                seeds=seeds).cpu().numpy()
    assert mu.shape == (64, R, M)
    assert np.allclose(mu[:, :, 0], 1.0, atol=1e-5)
    assert np.max(np.abs(mu)) <= 1.0 + 1e-5
    for i in (0, 17, 63):
        ref = pv.kpm_moments(lats[i], M, ab[i][0], ab[i][1], R=R, prec=pv.C64, seed=seeds[i]).cpu().numpy()
        assert np.max(np.abs(mu[i] - ref)) < 1e-5


def test_adjoint_full_lattice_against_central_differences():
    cfg = W.CONFIG_GRAPHENE_ADJ
    V = cfg.potential()
    lat = pv.Lattice.graphene(cfg.cells, (0, 0), V=V)
    emin, emax, a, b = lat.spectral_bounds()
    psi0 = torch.from_numpy(cfg.packet()).cuda()
    mask = torch.from_numpy(cfg.detector()).cuda()
    nsteps, every = 40, 20   # the full 200 steps run in bench.py's adjoint workload
    Vt = torch.tensor(V, dtype=torch.float64, device="cuda", requires_grad=True)
    psi = pv.propagate_with_grad(Vt, psi0, lat, cfg.dt, nsteps, a, b, every=every)
    loss = (psi.abs() ** 2 * mask).sum()
    loss.backward()
    g = Vt.grad.cpu().numpy()
    # central differences of the same loss at the sites of largest gradient and a few random ones
    order = np.argsort(-np.abs(g))
    rng = np.random.default_rng(W.ADJ_FD_SEED)
    sites = np.concatenate([order[:4], rng.choice(len(V), 4, replace=False)])
    h = W.ADJ_FD_H
    work = pv.work_buffer(lat.work_bytes(pv.OP_SERIES, 1, pv.C128, 20))

    def L(Vv):
        lat.set_potential(torch.from_numpy(Vv).cuda())
        p = psi0.clone()
        pv.cheb_propagate(lat, p, cfg.dt, nsteps, a, b, prec=pv.C128, work=work)
        return float((p.abs() ** 2 * mask).sum().item())

    for s in sites:
        Vp, Vm = V.copy(), V.copy()
        Vp[s] += h
        Vm[s] -= h
        fd = (L(Vp) - L(Vm)) / (2 * h)
        assert abs(fd - g[s]) <= 1e-5 * max(abs(g).max(), 1e-30) + 1e-5 * abs(fd), (s, fd, g[s])


def test_batched_kpm_full_workload_small_lattices_against_the_oracle():
    # the whole 64-lattice batch in the launch shape the benchmark tunes; the
    # first L = 24 lattice of the batch element by element against the oracle
    specs = W.batched_lattices()
    lats = [pv.Lattice.ti((L, L, L), (1, 1, 1), disorder=(Wd, s)) for L, Wd, s in specs]
    ab = [lat.spectral_bounds()[2:] for lat in lats]
    R, M = 16, 256
    seeds = list(range(300, 300 + len(lats)))
    args = ([x[0] for x in ab], [x[1] for x in ab])
    pv.autotune_batched(lats, 16, *args, R=R, prec=pv.C64, seeds=seeds)
    mu = pv.kpm_moments_batched(lats, M, *args, R=R, prec=pv.C64, seeds=seeds).cpu().numpy()
    i = next(k for k, (L, _, _) in enumerate(specs) if L == 24)
    L, Wd, s = specs[i]
    H = O.ti_hamiltonian((L, L, L), (1, 1, 1), 1.0, 2.0, W.disorder_potential(L ** 3, Wd, s))
    ref = O.kpm_moments(H, W.random_phase_block(H.shape[0], R, seeds[i]), M, *ab[i]).real
    assert np.max(np.abs(mu[i] - ref)) / ref[0, 0] < 1e-4
