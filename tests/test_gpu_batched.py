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


def test_batched_graph_follows_a_new_potential_on_a_later_lattice():
    # the batched graph is cached on lattice 0 but captures every lattice's geometry:
    # giving lattice 1 a potential between two calls with the same buffers must be seen
    dims0, dims1 = (5, 5, 5), (6, 4, 5)
    lat0 = pv.Lattice.ti(dims0, (1, 1, 1), disorder=(1.0, 51))
    lat1 = pv.Lattice.ti(dims1, (1, 1, 1))
    n1 = int(np.prod(dims1))
    H0 = O.ti_hamiltonian(dims0, (1, 1, 1), 1.0, 2.0, W.disorder_potential(125, 1.0, 51))
    V1 = W.disorder_potential(n1, 3.0, 52)
    ab0 = O.cheb_scale(*O.gershgorin(H0))
    H1 = O.ti_hamiltonian(dims1, (1, 1, 1), 1.0, 2.0, V1)
    ab1 = O.cheb_scale(*O.gershgorin(H1))   # holds the clean spectrum of lattice 1 too
    R, M = 2, 24
    work = pv.work_buffer(pv.batched_work_bytes([lat0, lat1], R, pv.C128, M))
    mu = torch.empty((2, R, M), dtype=torch.float64, device="cuda")
    args = ([ab0[0], ab1[0]], [ab0[1], ab1[1]])
    for _ in range(2):   # capture, then replay
        pv.kpm_moments_batched([lat0, lat1], M, *args, R=R, prec=pv.C128, seeds=[1, 2], work=work, mu=mu)
    clean = O.ti_hamiltonian(dims1, (1, 1, 1), 1.0, 2.0, np.zeros(n1))
    r1 = W.random_phase_block(4 * n1, R, 2)
    assert np.max(np.abs(mu[1].cpu().numpy() - O.kpm_moments(clean, r1, M, *ab1).real)) < 1e-12
    lat1.set_potential(torch.from_numpy(V1).cuda())
    pv.kpm_moments_batched([lat0, lat1], M, *args, R=R, prec=pv.C128, seeds=[1, 2], work=work, mu=mu)
    assert np.max(np.abs(mu[1].cpu().numpy() - O.kpm_moments(H1, r1, M, *ab1).real)) < 1e-12
    r0 = W.random_phase_block(4 * 125, R, 1)
    assert np.max(np.abs(mu[0].cpu().numpy() - O.kpm_moments(H0, r0, M, *ab0).real)) < 1e-12


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


STAGED_CASES = [((9, 11, 13), (0, 1, 1)), ((16, 8, 5), (1, 1, 0)), ((1, 2, 3), (1, 1, 1)),
                ((5, 1, 4), (1, 1, 0)), ((2, 7, 2), (1, 0, 1))]


@pytest.mark.parametrize("dims,per", STAGED_CASES)
@pytest.mark.parametrize("R", [1, 2, 8, 16])
@pytest.mark.parametrize("prec", [pv.C128, pv.C64])
def test_staged_sweep_matches_oracle(dims, per, R, prec):
    """The shared-memory staged sweep (bulk copies, halo tiles, ragged tiles,
    wrapped periodic halos, open edges) against the oracle, with dots."""
    n = int(np.prod(dims))
    V = W.disorder_potential(n, 2.0, 9)
    lat = pv.Lattice.ti(dims, per, disorder=(2.0, 9))
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V)
    cdt = torch.complex128 if prec == pv.C128 else torch.complex64
    tol = 1e-12 if prec == pv.C128 else 2e-6
    x = torch.from_numpy(W.gaussian_block(lat.D, R, 1)).to("cuda", cdt)
    y0 = torch.from_numpy(W.gaussian_block(lat.D, R, 2)).to("cuda", cdt)
    xh = x.cpu().numpy().astype(np.complex128)
    yh = y0.cpu().numpy().astype(np.complex128)
    yr, _, dr = O.cheb_step(H, xh, yh, [0.3] * R, [0.1] * R, [-1.0] * R)
    tried = 0
    for tile in [(4, 2), (3, 5), (8, 4), (2, 2)]:
        try:
            lat.set_tuning(R, prec, threads=128 if R <= 8 else 256, zslab=2, tile_x=tile[0],
                           tile_y=tile[1])
        except pv.PvscError as e:
            assert "shared memory" in str(e)  # tile too large for this R and precision
            continue
        tried += 1
        y = y0.clone()
        d = pv.cheb_step(lat, x, y, [0.3] * R, [0.1] * R, [-1.0] * R, dots=7).cpu().numpy()
        yy = y.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(yy - yr) / np.linalg.norm(yr) < tol, tile
        assert np.max(np.abs(d[0] - dr[:, 0].real)) < 10 * tol * np.abs(dr).max()
        assert np.max(np.abs(d[1] - dr[:, 1].real)) < 10 * tol * np.abs(dr).max()
        ya = pv.apply_H(lat, x).cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(ya - H @ xh) / np.linalg.norm(H @ xh) < tol
    assert tried >= 2
    flag = pv.ctypes.c_int()
    assert pv.lib().pvsc_device_error(pv.ctypes.byref(flag), 1) == 0 and flag.value == 0


def test_staged_kpm_and_series_match_oracle():
    dims, per = (12, 10, 9), (1, 1, 0)
    n = int(np.prod(dims))
    lat = pv.Lattice.ti(dims, per, disorder=(1.0, 4))
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, W.disorder_potential(n, 1.0, 4))
    a, b = O.cheb_scale(*O.gershgorin(H))
    for prec, tol in ((pv.C128, 1e-12), (pv.C64, 1e-4)):
        lat.set_tuning(8, prec, threads=256, zslab=3, tile_x=8, tile_y=4)
        mu = pv.kpm_moments(lat, 32, a, b, R=8, prec=prec, seed=3).cpu().numpy()
        ref = O.kpm_moments(H, W.random_phase_block(4 * n, 8, 3), 32, a, b).real
        assert np.max(np.abs(mu - ref)) < tol
        x = W.gaussian_block(4 * n, 8, 5)
        g = np.cos(0.3 * np.arange(9))
        y = pv.cheb_filter(lat, torch.from_numpy(x).cuda(), g, a, b, prec=prec).cpu().numpy()
        ref_y = O.cheb_series(H, x, g, a, b)
        assert np.linalg.norm(y - ref_y) / np.linalg.norm(ref_y) < (1e-12 if prec == pv.C128 else 1e-5)


@pytest.mark.parametrize("kernel", [1, 2, 3])
@pytest.mark.parametrize("dims,per", STAGED_CASES)
@pytest.mark.parametrize("R", [1, 2, 8, 64])
@pytest.mark.parametrize("prec", [pv.C128, pv.C64])
def test_flat_and_prefetching_sweeps_match_oracle(kernel, dims, per, R, prec):
    n = int(np.prod(dims))
    V = W.disorder_potential(n, 2.0, 9)
    lat = pv.Lattice.ti(dims, per, disorder=(2.0, 9))
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V)
    cdt = torch.complex128 if prec == pv.C128 else torch.complex64
    tol = 1e-12 if prec == pv.C128 else 2e-6
    x = torch.from_numpy(W.gaussian_block(lat.D, R, 1)).to("cuda", cdt)
    y0 = torch.from_numpy(W.gaussian_block(lat.D, R, 2)).to("cuda", cdt)
    xh = x.cpu().numpy().astype(np.complex128)
    yr, _, dr = O.cheb_step(H, xh, y0.cpu().numpy().astype(np.complex128), [0.3] * R, [0.1] * R,
                            [-1.0] * R)
    for th, zs in ((128, 2), (256, 0)):
        lat.set_tuning(R, prec, threads=th, zslab=zs, kernel=kernel)
        y = y0.clone()
        d = pv.cheb_step(lat, x, y, [0.3] * R, [0.1] * R, [-1.0] * R, dots=7).cpu().numpy()
        yy = y.cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(yy - yr) / np.linalg.norm(yr) < tol
        assert np.max(np.abs(d[1] - dr[:, 1].real)) < 10 * tol * np.abs(dr).max()


def test_new_tuning_replaces_captured_kpm_graph():
    # kpm_moments replays a captured CUDA graph; a later set_tuning must take
    # effect (the moments then equal those of a lattice tuned that way from the start)
    dims, R, M = (12, 10, 14), 4, 24
    shape_a = dict(threads=64, zslab=2, vpt=2)
    shape_b = dict(threads=256, zslab=0, vpt=1)

    def moments(lat, work, mu):  # same buffers on every call: the graph key repeats
        _, _, a, b = lat.spectral_bounds()
        pv.kpm_moments(lat, M, a, b, R=R, prec=pv.C64, seed=11, work=work, mu=mu)
        return mu.cpu().numpy()

    lat1 = pv.Lattice.ti(dims, (1, 1, 0), disorder=(1.0, 4))
    work = pv.work_buffer(lat1.work_bytes(pv.OP_KPM, R, pv.C64, M))
    mu = torch.empty((R, M), dtype=torch.float64, device="cuda")
    lat1.set_tuning(R, pv.C64, **shape_a)
    mu_a = moments(lat1, work, mu)
    lat1.set_tuning(R, pv.C64, **shape_b)
    mu_b1 = moments(lat1, work, mu)
    lat2 = pv.Lattice.ti(dims, (1, 1, 0), disorder=(1.0, 4))
    lat2.set_tuning(R, pv.C64, **shape_b)
    mu_b2 = moments(lat2, work, mu)
    assert np.array_equal(mu_b1, mu_b2)
    assert np.max(np.abs(mu_a - mu_b2)) < 1e-5


def test_explicit_tuning_shapes_all_agree():
    lat = pv.Lattice.ti((9, 11, 13), (0, 1, 1), disorder=(1.0, 8))
    x = torch.from_numpy(W.gaussian_block(lat.D, 16, 1)).cuda().to(torch.complex64)
    ref = pv.apply_H(lat, x)
    for th, bps, zs in [(64, 1, 1), (128, 2, 3), (256, 0, 13), (128, 0, 5)]:
        lat.set_tuning(16, pv.C64, th, bps, zs)
        assert torch.equal(pv.apply_H(lat, x), ref)
    with pytest.raises(pv.PvscError):
        lat.set_tuning(16, pv.C64, 100, 0, 0)  # not a multiple of 32


def test_batch_autotuner_picks_a_shape_and_results_hold():
    specs = [(6, 1.0, 61), ((9, 8, 12), 2.0, 62), (4, 0.5, 63), ((5, 7, 20), 3.0, 64)]
    lats, Hs, ab = _lattices(specs)
    R, M = 4, 24
    seeds = [70 + i for i in range(len(lats))]
    args = ([x[0] for x in ab], [x[1] for x in ab])
    t = pv.autotune_batched(lats, 8, *args, R=R, prec=pv.C64, seeds=seeds)
    assert t["threads"] in (128, 256) and t["time_ms"] > 0
    assert lats[0].get_tuning(R, pv.C64)["zslab"] == t["zslab"]
    mu = pv.kpm_moments_batched(lats, M, *args, R=R, prec=pv.C64, seeds=seeds).cpu().numpy()
    for i, (H, (a, b)) in enumerate(zip(Hs, ab)):
        ref = O.kpm_moments(H, W.random_phase_block(H.shape[0], R, seeds[i]), M, a, b).real
        assert np.max(np.abs(mu[i] - ref)) / ref[0, 0] < 1e-4, i


def test_per_lattice_batch_on_the_tma_sweep():
    # tuning kernel 7 on lats[0]: every lattice's KPM runs as its own chain of
    # TMA-staged sweeps on a few forked streams inside one graph; each chain
    # equals the single-lattice KPM with that kernel bit for bit
    specs = [((8, 5, 7), 1.0, 41), ((12, 6, 9), 3.0, 42), ((4, 4, 4), 0.5, 43), ((16, 9, 12), 2.0, 44),
             ((20, 8, 3), 1.5, 45)]
    lats, Hs, ab = _lattices(specs)
    R, M = 8, 40
    seeds = [200 + i for i in range(len(lats))]
    a_, b_ = [x[0] for x in ab], [x[1] for x in ab]
    mu_p = pv.kpm_moments_batched(lats, M, a_, b_, R=R, prec=pv.C64, seeds=seeds).cpu().numpy()
    lats[0].set_tuning(R, pv.C64, kernel=7)
    work = pv.work_buffer(pv.batched_work_bytes(lats, R, pv.C64, M))
    mu_t = pv.kpm_moments_batched(lats, M, a_, b_, R=R, prec=pv.C64, seeds=seeds, work=work)
    mu_t2 = pv.kpm_moments_batched(lats, M, a_, b_, R=R, prec=pv.C64, seeds=seeds, work=work)
    assert torch.equal(mu_t, mu_t2)  # the replayed graph
    assert pv.device_error() == 0
    mu_t = mu_t.cpu().numpy()
    assert np.max(np.abs(mu_t - mu_p)) < 1e-9  # same vectors as the persistent kernel's z-march
    for i, lat in enumerate(lats):
        lat.set_tuning(R, pv.C64, kernel=7)
        mu_s = pv.kpm_moments(lat, M, a_[i], b_[i], R=R, prec=pv.C64, seed=seeds[i]).cpu().numpy()
        assert np.array_equal(mu_t[i], mu_s), i
        r = W.random_phase_block(Hs[i].shape[0], R, seeds[i])
        ref = O.kpm_moments(Hs[i], r, M, a_[i], b_[i]).real
        assert np.max(np.abs(mu_t[i] - ref)) / ref[0, 0] < 1e-4, i


def test_per_lattice_batch_falls_back_where_the_tma_sweep_does_not_apply():
    # Lx = 6 (not a multiple of 4) has no TMA-staged sweep: the persistent kernel runs
    lats, Hs, ab = _lattices([((6, 4, 5), 1.0, 51), ((8, 4, 5), 2.0, 52)])
    R, M = 4, 24
    a_, b_ = [x[0] for x in ab], [x[1] for x in ab]
    lats[1].set_tuning(R, pv.C64, kernel=7)
    mu = pv.kpm_moments_batched(lats[::-1], M, a_[::-1], b_[::-1], R=R, prec=pv.C64, seeds=[3, 4]).cpu().numpy()
    for j, i in enumerate((1, 0)):
        r = W.random_phase_block(Hs[i].shape[0], R, [3, 4][j])
        ref = O.kpm_moments(Hs[i], r, M, a_[i], b_[i]).real
        assert np.max(np.abs(mu[j] - ref)) / ref[0, 0] < 1e-4
