"""Parity of the CUDA path (through the C ABI) with the CPU fp64 oracle.

Tolerances: complex128 paths <= 1e-12 relative (norm-wise), moments
max_k |d mu_k| / mu_0 <= 1e-12.  complex64 storage with fp32 stencil
arithmetic: one sweep <= 2e-6 relative (a sum of 13 fp32 terms, each
rounded at 2^-24 ~ 6e-8, plus the storage rounding of y), KPM moments
<= 1e-4 mu_0 over 256 moments, propagation <= 1e-4 after a few steps.
Indices, neighbour tables and the counter hash are compared bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

pv = pytest.importorskip("paper_1708_09689_gb300")

C128_TOL = 1e-12
C64_SWEEP_TOL = 2e-6


def dev(a, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


TI_CASES = [((7, 5, 6), (1, 0, 1)), ((4, 4, 4), (1, 1, 1)), ((3, 2, 5), (0, 1, 0)),
            ((1, 3, 2), (1, 1, 1)), ((2, 1, 3), (1, 0, 0))]
GR_CASES = [((5, 4), (1, 1)), ((6, 3), (0, 0)), ((1, 4), (1, 0)), ((3, 2), (0, 1))]


def ti_pair(dims, per, W_=1.0, seed=3, m=2.0, t=1.0):
    n = int(np.prod(dims))
    V = W.disorder_potential(n, W_, seed)
    lat = pv.Lattice.ti(dims, per, t=t, m=m, disorder=(W_, seed))
    H = O.ti_hamiltonian(dims, per, t, m, V)
    return lat, H, V


def gr_pair(cells, per, W_=0.5, seed=4, t=1.0):
    n = 4 * cells[0] * cells[1]
    V = W.disorder_potential(n, W_, seed)
    lat = pv.Lattice.graphene(cells, per, t=t, V=V)
    H = O.graphene_hamiltonian(cells, per, t, V)
    return lat, H, V


# ------------------------------------------------------------------ bit-exact parts
@pytest.mark.parametrize("dims,per", TI_CASES)
def test_ti_neighbour_table_bit_exact(dims, per):
    lat, H, _ = ti_pair(dims, per)
    nb = host(lat.neighbours())
    n = int(np.prod(dims))
    Hc = H.tocsr()
    for s in range(n):
        cols = Hc.indices[Hc.indptr[4 * s]:Hc.indptr[4 * s + 4]] // 4
        ref = set(cols.tolist()) - {s}
        got = set(x for x in nb[s, 1:].tolist() if x >= 0) - {s}
        assert got == ref, (s, got, ref)
        assert nb[s, 0] == s


@pytest.mark.parametrize("cells,per", GR_CASES)
def test_graphene_neighbour_table_bit_exact(cells, per):
    lat, H, _ = gr_pair(cells, per)
    nb = host(lat.neighbours())
    Hc = H.tocsr()
    for c in range(cells[0] * cells[1]):
        cols = Hc.indices[Hc.indptr[4 * c]:Hc.indptr[4 * c + 4]] // 4
        ref = set(cols.tolist()) - {c}
        got = set(x for x in nb[c, 1:5].tolist() if x >= 0) - {c}
        assert got == ref


def test_seeded_potential_bit_exact():
    for on_the_fly in (False, True):
        lat = pv.Lattice.ti((9, 7, 5), (1, 1, 0), disorder=(2.5, 77), on_the_fly=on_the_fly)
        V = host(lat.potential())
        ref = W.disorder_potential(9 * 7 * 5, 2.5, 77)
        assert np.array_equal(V.view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("dims,per", TI_CASES[:3])
def test_spectral_bounds_match_oracle_gershgorin(dims, per):
    lat, H, _ = ti_pair(dims, per, W_=2.0)
    emin, emax, a, b = lat.spectral_bounds(0.01)
    omin, omax = O.gershgorin(H)
    assert abs(emin - omin) < 1e-13 and abs(emax - omax) < 1e-13
    oa, ob = O.cheb_scale(omin, omax, 0.01)
    assert abs(a - oa) < 1e-13 and abs(b - ob) < 1e-13


@pytest.mark.parametrize("cells,per", GR_CASES)
def test_graphene_spectral_bounds(cells, per):
    lat, H, _ = gr_pair(cells, per)
    emin, emax, _, _ = lat.spectral_bounds()
    omin, omax = O.gershgorin(H)
    assert abs(emin - omin) < 1e-13 and abs(emax - omax) < 1e-13


# ------------------------------------------------------------------ apply H
@pytest.mark.parametrize("dims,per", TI_CASES)
@pytest.mark.parametrize("R", [1, 2, 4, 8, 16, 32, 64])
def test_ti_apply_H_c128(dims, per, R):
    lat, H, _ = ti_pair(dims, per)
    x = W.gaussian_block(H.shape[0], R, 11)
    y = pv.apply_H(lat, dev(x))
    assert relerr(host(y), H @ x) < C128_TOL


@pytest.mark.parametrize("dims,per", TI_CASES)
@pytest.mark.parametrize("R", [1, 2, 8, 32, 64])
def test_ti_apply_H_c64(dims, per, R):
    lat, H, _ = ti_pair(dims, per)
    x = W.gaussian_block(H.shape[0], R, 12).astype(np.complex64)
    y = pv.apply_H(lat, dev(x, torch.complex64))
    assert relerr(host(y).astype(np.complex128), H @ x.astype(np.complex128)) < C64_SWEEP_TOL


@pytest.mark.parametrize("cells,per", GR_CASES)
@pytest.mark.parametrize("R", [1, 2, 4, 16, 64])
def test_graphene_apply_H_c128_and_c64(cells, per, R):
    lat, H, _ = gr_pair(cells, per)
    x = W.gaussian_block(H.shape[0], R, 13)
    y = pv.apply_H(lat, dev(x))
    assert relerr(host(y), H @ x) < C128_TOL
    x32 = x.astype(np.complex64)
    y32 = pv.apply_H(lat, dev(x32, torch.complex64))
    assert relerr(host(y32).astype(np.complex128), H @ x32.astype(np.complex128)) < C64_SWEEP_TOL


def test_on_the_fly_disorder_matches_stored():
    dims, per = (6, 5, 7), (1, 1, 0)
    stored = pv.Lattice.ti(dims, per, disorder=(3.0, 9))
    fly = pv.Lattice.ti(dims, per, disorder=(3.0, 9), on_the_fly=True)
    x = dev(W.gaussian_block(4 * 210, 4, 5))
    a, b = pv.apply_H(stored, x), pv.apply_H(fly, x)
    assert torch.equal(a, b)


# ------------------------------------------------------------------ fused Chebyshev step
@pytest.mark.parametrize("prec", [pv.C128, pv.C64])
@pytest.mark.parametrize("model", ["ti", "gr"])
def test_cheb_step_with_z_and_dots(prec, model):
    R = 4
    if model == "ti":
        lat, H, _ = ti_pair((5, 6, 7), (1, 0, 1))
    else:
        lat, H, _ = gr_pair((7, 5), (0, 1))
    D = H.shape[0]
    x = W.gaussian_block(D, R, 1)
    y = W.gaussian_block(D, R, 2)
    z = W.gaussian_block(D, R, 3)
    cdt = np.complex128 if prec == pv.C128 else np.complex64
    tdt = torch.complex128 if prec == pv.C128 else torch.complex64
    x, y, z = x.astype(cdt), y.astype(cdt), z.astype(cdt)
    alpha, beta, gamma, delta = [0.3, 0.2, 0.25, 0.1], [0.1, -0.2, 0.0, 0.3], [-1.0, 0.5, 0.0, 1.0], [0.5, 1.0, -0.25, 2.0]
    xt, yt, zt = dev(x, tdt), dev(y, tdt), dev(z, tdt)
    dots = pv.cheb_step(lat, xt, yt, alpha, beta, gamma, z=zt, delta=delta, dots=7)
    yr, zr, dr = O.cheb_step(H, x.astype(np.complex128), y.astype(np.complex128), alpha, beta, gamma,
                             z.astype(np.complex128), delta)
    tol = C128_TOL if prec == pv.C128 else C64_SWEEP_TOL
    assert relerr(host(yt).astype(np.complex128), yr) < tol
    assert relerr(host(zt).astype(np.complex128), zr) < tol
    d = host(dots)
    scale = np.abs(dr).max()
    assert np.max(np.abs(d[0] - dr[:, 0].real)) < tol * 10 * scale
    assert np.max(np.abs(d[1] - dr[:, 1].real)) < tol * 10 * scale
    assert np.max(np.abs(d[2] - dr[:, 1].imag)) < tol * 10 * scale
    assert np.max(np.abs(d[3] - dr[:, 2].real)) < tol * 10 * scale


def test_cheb_step_dots_are_bitwise_reproducible():
    lat, H, _ = ti_pair((16, 16, 16), (1, 1, 1))
    x = dev(W.gaussian_block(H.shape[0], 8, 1))
    y0 = dev(W.gaussian_block(H.shape[0], 8, 2))
    outs = []
    for _ in range(2):
        y = y0.clone()
        outs.append(pv.cheb_step(lat, x, y, [0.2] * 8, [0.1] * 8, [-1.0] * 8, dots=7))
    assert torch.equal(outs[0], outs[1])


# ------------------------------------------------------------------ KPM
@pytest.mark.parametrize("prec,tol", [(pv.C128, 1e-12), (pv.C64, 1e-4)])
def test_kpm_moments_ti_cube(prec, tol):
    cfg = W.CONFIG_TI_CUBE
    lat, H, _ = ti_pair(cfg.dims, cfg.periodic, W_=cfg.W, seed=cfg.seed_V)
    omin, omax = O.gershgorin(H)
    a, b = O.cheb_scale(omin, omax)
    mu = host(pv.kpm_moments(lat, cfg.M, a, b, R=1, prec=prec, seed=cfg.seed_r))
    r = W.random_phase_block(cfg.D, 1, cfg.seed_r)
    ref = O.kpm_moments(H, r, cfg.M, a, b).real
    assert abs(mu[0, 0] - 1.0) < tol
    assert np.max(np.abs(mu - ref)) / ref[0, 0] < tol


@pytest.mark.parametrize("R", [2, 8])
@pytest.mark.parametrize("prec,tol", [(pv.C128, 1e-12), (pv.C64, 1e-4)])
def test_kpm_moments_with_given_start_block_and_odd_M(R, prec, tol):
    lat, H, _ = ti_pair((6, 7, 5), (1, 1, 0), W_=2.0, seed=2)
    a, b = O.cheb_scale(*O.gershgorin(H))
    r = W.random_phase_block(H.shape[0], R, 3)
    cdt = torch.complex128 if prec == pv.C128 else torch.complex64
    rt = dev(r, cdt)
    M = 41
    mu = host(pv.kpm_moments(lat, M, a, b, r0=rt))
    ref = O.kpm_moments(H, host(rt).astype(np.complex128), M, a, b).real
    assert np.max(np.abs(mu - ref)) / ref[0, 0] < tol
    assert torch.equal(rt, dev(r, cdt))  # start block untouched


def test_kpm_graphene_and_graph_replay():
    lat, H, _ = gr_pair((8, 6), (1, 0))
    a, b = O.cheb_scale(*O.gershgorin(H))
    work = pv.work_buffer(lat.work_bytes(pv.OP_KPM, 4, pv.C128, 64))
    mu1 = host(pv.kpm_moments(lat, 64, a, b, R=4, seed=5, work=work))
    mu2 = host(pv.kpm_moments(lat, 64, a, b, R=4, seed=5, work=work))  # replayed graph
    ref = O.kpm_moments(H, W.random_phase_block(H.shape[0], 4, 5), 64, a, b).real
    assert np.array_equal(mu1, mu2)
    assert np.max(np.abs(mu1 - ref)) < 1e-12


# ------------------------------------------------------------------ series, filter, propagation
def test_chebyshev_filter_matches_oracle():
    lat, H, _ = ti_pair((5, 4, 6), (1, 1, 0))
    a, b = O.cheb_scale(*O.gershgorin(H))
    g = np.cos(0.37 * np.arange(17)) / (1 + np.arange(17))
    x = W.gaussian_block(H.shape[0], 2, 7)
    ref = O.cheb_series(H, x, g, a, b)
    for prec, tol in ((pv.C128, C128_TOL), (pv.C64, 1e-5)):
        y = pv.cheb_filter(lat, dev(x), g, a, b, prec=prec)
        assert relerr(host(y), ref) < tol


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10])
@pytest.mark.parametrize("pattern", ["complex", "zeros"])
def test_cheb_series_short_and_in_place(K, pattern):
    lat, H, _ = gr_pair((4, 5), (0, 0))
    a, b = O.cheb_scale(*O.gershgorin(H))
    c = np.exp(1j * np.arange(K)) / (1 + np.arange(K))
    if pattern == "zeros":  # exact zeros, and purely real / imaginary weights in between
        c = np.where(np.arange(K) % 3 == 1, 0.0, np.where(np.arange(K) % 2 == 0, c.real, 1j * c.imag))
    x = W.gaussian_block(H.shape[0], 1, 8)
    ref = np.exp(0.3j) * O.cheb_series(H, x, c, a, b)
    for prec, tol in ((pv.C128, C128_TOL), (pv.C64, 1e-5)):
        xt = dev(x)
        y = pv.cheb_series(lat, xt, list(c), a, b, phase=np.exp(0.3j), y=xt, prec=prec)  # in place
        assert relerr(host(y), ref) < tol


def test_propagation_graphene_qd_small():
    cfg = W.GrapheneConfig(cells=(40, 24), ndots=2, R_dot=6.0, sigma=6.0, packet_offset=20.0)
    V = cfg.potential()
    psi0 = cfg.packet()
    lat = pv.Lattice.graphene(cfg.cells, (0, 0), V=V)
    H = O.graphene_hamiltonian(cfg.cells, (0, 0), 1.0, V)
    a, b = O.cheb_scale(*O.gershgorin(H))
    ref = O.propagate(H, psi0[:, None], 1.0, 5, a, b)
    for prec, tol in ((pv.C128, 1e-12), (pv.C64, 1e-4)):
        psi = dev(psi0[:, None])
        pv.cheb_propagate(lat, psi, 1.0, 5, a, b, prec=prec)
        assert relerr(host(psi), ref) < tol
        assert abs(np.linalg.norm(host(psi)) - 1) < (1e-12 if prec == pv.C128 else 1e-5)


def test_propagation_c64_norm_has_no_drift():
    # The exact propagator is unitary.  complex64 vectors add rounding that
    # varies with the data, so the norm error stays near the fp32 storage
    # level over many steps; a series coefficient rounded the same way on
    # every step would instead make it grow linearly (~1e-8 per step).
    cfg = W.GrapheneConfig(cells=(96, 64), ndots=2, R_dot=10.0, sigma=8.0, packet_offset=30.0)
    lat = pv.Lattice.graphene(cfg.cells, (0, 0), V=cfg.potential())
    _, _, a, b = lat.spectral_bounds()
    psi = dev(cfg.packet()[:, None])
    pv.cheb_propagate(lat, psi, 1.0, 400, a, b, prec=pv.C64)
    assert abs(torch.linalg.vector_norm(psi).item() - 1) < 5e-7


def test_propagation_ti_block():
    lat, H, _ = ti_pair((4, 5, 3), (1, 0, 1))
    a, b = O.cheb_scale(*O.gershgorin(H))
    x = W.gaussian_block(H.shape[0], 4, 9)
    x /= np.linalg.norm(x, axis=0)
    ref = O.propagate(H, x, 0.7, 3, a, b)
    psi = dev(x)
    pv.cheb_propagate(lat, psi, 0.7, 3, a, b)
    assert relerr(host(psi), ref) < 1e-12


# ------------------------------------------------------------------ adjoint
def test_adjoint_step_matches_oracle_gradient():
    cfg = W.GrapheneConfig(cells=(12, 10), ndots=2, R_dot=3.0, sigma=4.0, packet_offset=6.0)
    V = cfg.potential()
    psi0 = cfg.packet()
    H = O.graphene_hamiltonian(cfg.cells, (0, 0), 1.0, V)
    a, b = O.cheb_scale(*O.gershgorin(H))
    dt, S = 1.0, 4
    psiS = O.propagate(H, psi0, dt, S, a, b)
    mask = cfg.detector() | (np.arange(len(V)) % 7 == 0)
    G = 2.0 * mask * psiS
    ref, refG0 = O.propagate_adjoint(H, psi0, dt, S, a, b, G, O=1)
    lat = pv.Lattice.graphene(cfg.cells, (0, 0), V=V)
    Vt = torch.tensor(V, dtype=torch.float64, device="cuda", requires_grad=True)
    psi = pv.propagate_with_grad(Vt, dev(psi0), lat, dt, S, a, b, every=3)
    loss = (psi.abs() ** 2 * torch.tensor(mask, device="cuda")).sum()
    loss.backward()
    g = host(Vt.grad)
    assert np.max(np.abs(g - ref)) / np.max(np.abs(ref)) < 1e-9


@pytest.mark.parametrize("S,every", [(7, 3), (6, 6), (5, 1), (4, 10)])
def test_whole_propagation_adjoint_through_the_c_abi(S, every):
    # pvsc_cheb_propagate_checkpointed + pvsc_cheb_propagate_adjoint (one call each)
    # against the oracle's reverse sweep: dL/dV and dL/dpsi_0, segments of every
    # length (a last partial segment, one segment, one-step segments, every > S)
    cfg = W.GrapheneConfig(cells=(10, 8), ndots=2, R_dot=3.0, sigma=4.0, packet_offset=5.0)
    V = cfg.potential()
    psi0 = cfg.packet()
    H = O.graphene_hamiltonian(cfg.cells, (0, 0), 1.0, V)
    a, b = O.cheb_scale(*O.gershgorin(H))
    dt = 0.9
    psiS = O.propagate(H, psi0, dt, S, a, b)
    mask = cfg.detector() | (np.arange(len(V)) % 5 == 0)
    Gf = 2.0 * mask * psiS
    ref, refG0 = O.propagate_adjoint(H, psi0, dt, S, a, b, Gf, O=1)
    lat = pv.Lattice.graphene(cfg.cells, (0, 0), V=V)
    psi = dev(psi0)
    psi, ckpts = pv.cheb_propagate_checkpointed(lat, psi, dt, S, every, a, b)
    assert relerr(host(psi), psiS) < 1e-12
    assert ckpts.shape[0] == -(-S // every)
    assert relerr(host(ckpts[0]), psi0) == 0.0
    G = dev(Gf)
    dLdV = torch.zeros(len(V), dtype=torch.float64, device="cuda")
    pv.cheb_propagate_adjoint(lat, ckpts, G, dt, S, every, a, b, dLdV)
    g = host(dLdV)
    assert np.max(np.abs(g - ref)) / np.max(np.abs(ref)) < 1e-9
    assert relerr(host(G), refG0[:, 0]) < 1e-9


def test_whole_propagation_adjoint_rejects_bad_arguments():
    lat = pv.Lattice.graphene((4, 4), (0, 0))
    x = torch.zeros(64, dtype=torch.complex128, device="cuda")
    ck = torch.zeros((2, 64), dtype=torch.complex128, device="cuda")
    g = torch.zeros(16 * 4, dtype=torch.float64, device="cuda")
    with pytest.raises(pv.PvscError, match="every"):
        pv.cheb_propagate_adjoint(lat, ck, x, 1.0, 2, 0, 3.1, 0.0, g,
                                  work=pv.work_buffer(1 << 20))
    x2 = torch.zeros((64, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(pv.PvscError, match="R = 1"):
        pv.cheb_propagate_adjoint(lat, ck, x2, 1.0, 2, 1, 3.1, 0.0, g, work=pv.work_buffer(1 << 22))


def _rows_multisets(rowptr, col):
    return [sorted(col[rowptr[i]:rowptr[i + 1]].tolist()) for i in range(len(rowptr) - 1)]


@pytest.mark.parametrize("model,dims,per", [
    ("ti", (4, 3, 5), (1, 1, 0)), ("ti", (2, 1, 3), (1, 1, 1)), ("ti", (3, 2, 2), (0, 1, 1)),
    ("ti_delta", (3, 4, 2), (1, 0, 1)), ("graphene", (4, 3), (1, 0)), ("graphene", (2, 1), (1, 1)),
    ("wsm", (4, 3, 2), (1, 1, 0)), ("wsm", (2, 2, 1), (1, 1, 1))])
def test_exported_pattern_counts_every_stencil_term_of_the_oracle(model, dims, per):
    # the C ABI's CSR pattern (one entry per stencil term, duplicates kept) equals,
    # row by row as a multiset, the oracle's COO terms before they are summed;
    # periodic lengths 1 and 2 make coinciding neighbours, counted once per term
    n = int(np.prod(dims))
    if model.startswith("ti"):
        V = W.disorder_potential(n, 1.0, 4)
        kw = dict(delta1=0.3, delta2=0.2) if model == "ti_delta" else {}
        lat = pv.Lattice.ti(dims, per, V=V, **kw)
        r, c, _ = O.ti_hamiltonian(dims, per, 1.0, 2.0, V, kw.get("delta1", 0.0), kw.get("delta2", 0.0),
                                   terms=True)
        D = 4 * n
    elif model == "graphene":
        V = W.disorder_potential(4 * n, 1.0, 4)
        lat = pv.Lattice.graphene(dims, per, V=V)
        r, c, _ = O.graphene_hamiltonian(dims, per, 1.0, V, terms=True)
        D = 4 * n
    else:
        V = W.disorder_potential(n, 1.0, 4)
        lat = pv.Lattice.wsm(dims, per, V=V)
        r, c, _ = O.wsm_hamiltonian(dims, per, V, terms=True)
        D = 2 * n
    rowptr, col = lat.export_pattern()
    assert len(rowptr) == D + 1 and rowptr[-1] == len(c)
    order = np.lexsort((c, r))
    ref = [[] for _ in range(D)]
    for i, j in zip(r[order], c[order]):
        ref[i].append(int(j))
    assert _rows_multisets(rowptr, col) == ref
