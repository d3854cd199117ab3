"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these compare the oracle with itself: they use closed-form band
structures, dense diagonalisation, matrix exponentials, library Bessel
functions, finite differences and the paper's stated spectra.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla
from scipy.special import jv

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def facts():
    with open(os.path.join(GOLDEN, "paper_facts.json")) as f:
        return json.load(f)


# ---------------------------------------------------------------- Dirac algebra
def test_gamma_clifford_algebra():
    G = O.gamma_matrices()
    for a in range(1, 6):
        assert np.allclose(G[a], G[a].conj().T)
        for b in range(1, 6):
            anti = G[a] @ G[b] + G[b] @ G[a]
            assert np.allclose(anti, 2.0 * (a == b) * np.eye(4), atol=1e-15)
    assert np.allclose(G[1], np.diag([1, -1, 1, -1]))
    # Gamma^{ab} is Hermitian and anticommutes with Gamma^a
    G15 = O.gamma_commutator(G, 1, 5)
    assert np.allclose(G15, G15.conj().T)
    assert np.allclose(G15 @ G[1] + G[1] @ G15, 0)


# ---------------------------------------------------------------- TI Hamiltonian
def ti_bloch_energies(dims, m, t):
    """Closed-form bands E(k) = +-sqrt((m - t sum cos k_j)^2 + t^2 sum sin^2 k_j), each twice."""
    ks = [2 * np.pi * np.arange(L) / L for L in dims]
    KX, KY, KZ = np.meshgrid(*ks, indexing="ij")
    c = np.cos(KX) + np.cos(KY) + np.cos(KZ)
    s2 = np.sin(KX) ** 2 + np.sin(KY) ** 2 + np.sin(KZ) ** 2
    E = np.sqrt((m - t * c) ** 2 + t ** 2 * s2).reshape(-1)
    return np.sort(np.concatenate([E, E, -E, -E]))


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 5, 4), (6, 2, 3)])
@pytest.mark.parametrize("m", [0.5, 2.0, 3.5])
def test_ti_periodic_bands_match_closed_form(dims, m):
    n = int(np.prod(dims))
    H = O.ti_hamiltonian(dims, (1, 1, 1), 1.0, m, np.zeros(n))
    e = np.linalg.eigvalsh(H.toarray())
    assert np.max(np.abs(e - ti_bloch_energies(dims, m, 1.0))) < 1e-12


def test_ti_hopping_amplitude_t():
    dims = (4, 3, 5)
    n = int(np.prod(dims))
    H = O.ti_hamiltonian(dims, (1, 1, 1), 0.7, 1.3, np.zeros(n))
    e = np.linalg.eigvalsh(H.toarray())
    assert np.max(np.abs(e - ti_bloch_energies(dims, 1.3, 0.7))) < 1e-12


@pytest.mark.parametrize("dims,per", [((3, 4, 2), (1, 0, 1)), ((1, 2, 3), (1, 1, 0)),
                                      ((2, 1, 1), (1, 1, 1)), ((5, 3, 4), (0, 0, 0))])
def test_ti_hermitian_with_disorder(dims, per):
    n = int(np.prod(dims))
    V = W.disorder_potential(n, 2.0, 7)
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V)
    assert abs(H - H.conj().T).max() == 0.0
    assert np.allclose(H.diagonal().real.reshape(n, 4),
                       V[:, None] + 2.0 * np.array([1, -1, 1, -1])[None, :] +
                       _self_bond_diag(dims, per))


def _self_bond_diag(dims, per):
    # a periodic axis of length 1 bonds a site to itself: B + B^+ = -t Gamma^1
    g1 = np.array([1, -1, 1, -1], dtype=float)
    return sum(-g1 for L, p in zip(dims, per) if L == 1 and p)


def test_ti_bulk_gap_and_phase_boundaries():
    f = facts()
    dims = (6, 6, 6)
    n = 216
    H = O.ti_hamiltonian(dims, (1, 1, 1), 1.0, f["ti_clean_bulk_gap"]["m"], np.zeros(n))
    e = np.linalg.eigvalsh(H.toarray())
    assert abs(np.min(np.abs(e)) - f["ti_clean_bulk_gap"]["gap_edge"]) < 1e-12
    for m in f["ti_phase_boundaries"]["m_values"]:
        H = O.ti_hamiltonian(dims, (1, 1, 1), 1.0, m, np.zeros(n))
        assert np.min(np.abs(np.linalg.eigvalsh(H.toarray()))) < 1e-12
    for m in (0.5, 2.0, 3.5):   # gapped inside each phase
        H = O.ti_hamiltonian(dims, (1, 1, 1), 1.0, m, np.zeros(n))
        assert np.min(np.abs(np.linalg.eigvalsh(H.toarray()))) > 0.4


def test_ti_disordered_spectrum_in_paper_range():
    f = facts()["ti_spectrum_range"]
    dims = (6, 5, 6)
    n = int(np.prod(dims))
    V = W.disorder_potential(n, f["W"], 11)
    H = O.ti_hamiltonian(dims, (1, 1, 1), 1.0, f["m"], V)
    e = np.linalg.eigvalsh(H.toarray())
    lo, hi = f["interval"]
    assert e.min() >= lo and e.max() <= hi
    # and it is not trivially inside: the clean band edges are at +-5
    assert e.max() > 4.5 and e.min() < -4.5


def test_ti_open_boundary_drops_bonds():
    # a 1 x 1 x 2 open chain has exactly one bond along z
    H = O.ti_hamiltonian((1, 1, 2), (0, 0, 0), 1.0, 0.0, np.zeros(2)).toarray()
    G = O.gamma_matrices()
    B = -(1.0 / 2.0) * (G[1] - 1j * G[4])
    assert np.allclose(H[4:8, 0:4], B)
    assert np.allclose(H[0:4, 4:8], B.conj().T)
    assert np.allclose(H[0:4, 0:4], 0)


# ---------------------------------------------------------------- graphene
def graphene_paper_band(kx, ky):
    """|eps(k)| from Eq. graphene_e_k (a = 1)."""
    return np.sqrt(np.maximum(3 + 2 * np.cos(np.sqrt(3) * ky) +
                              4 * np.cos(np.sqrt(3) * ky / 2) * np.cos(1.5 * kx), 0.0))


@pytest.mark.parametrize("cells", [(6, 4), (5, 3), (4, 7)])
def test_graphene_periodic_bands_match_paper_formula(cells):
    Nx, Ny = cells
    H = O.graphene_hamiltonian(cells, (1, 1), 1.0, np.zeros(4 * Nx * Ny))
    assert abs(H - H.conj().T).max() == 0.0
    e = np.linalg.eigvalsh(H.toarray())
    ref = []
    for p in range(Nx):
        for q in range(Ny):
            # cell axis x spans physical Y (period sqrt3), cell axis y spans physical X (period 3)
            kX, kY = 2 * np.pi * q / (3 * Ny), 2 * np.pi * p / (np.sqrt(3) * Nx)
            for kx in (kX, kX + 2 * np.pi / 3):   # the 4-site cell folds two primitive k's
                E = graphene_paper_band(kx, kY)
                ref += [E, -E]
    assert np.max(np.abs(e - np.sort(ref))) < 1e-12


def test_graphene_bonds_have_unit_length():
    Nx, Ny = 5, 4
    H = O.graphene_hamiltonian((Nx, Ny), (0, 0), 1.0, np.zeros(4 * Nx * Ny)).tocoo()
    X, Y = W.graphene_positions(Nx, Ny)
    off = H.row != H.col
    d = np.hypot(X[H.row[off]] - X[H.col[off]], Y[H.row[off]] - Y[H.col[off]])
    assert np.allclose(d, 1.0)
    assert np.allclose(H.data[off], -1.0)
    # every interior site has exactly three neighbours
    deg = np.bincount(H.row[off], minlength=4 * Nx * Ny)
    assert deg.max() == 3


# Bonds of Eq. graphene_model as (dx, dy, site a of cell c + (dx, dy), site b of cell c):
# the chain 0-1-2-3 inside a cell, T_x (site 1 of cell n + x with site 0 of n, site 2
# of n + x with site 3 of n) and T_y (site 0 of cell n + y with site 3 of n).
EQ_BONDS = [(0, 0, 1, 0), (0, 0, 2, 1), (0, 0, 3, 2), (1, 0, 1, 0), (1, 0, 2, 3), (0, 1, 0, 3)]


def _mirrored_hamiltonian(Nx, Ny, periodic, V):
    """The honeycomb of the paper's DSL statement of the stencil (Sec. 3.2), which
    couples site 0 to site 1 of cell n - x where the equation uses n + x: the bonds
    of Eq. graphene_model with dx -> -dx, assembled bond by bond (hopping -1, on-site
    V), independently of the oracle's assembly."""
    import scipy.sparse as sp
    rows, cols, vals = list(range(4 * Nx * Ny)), list(range(4 * Nx * Ny)), list(V)
    for x in range(Nx):
        for y in range(Ny):
            c = x + Nx * y
            for dx, dy, sa, sb in EQ_BONDS:
                xx, yy = x - dx, y + dy
                if periodic[0]:
                    xx %= Nx
                if periodic[1]:
                    yy %= Ny
                if not (0 <= xx < Nx and 0 <= yy < Ny):
                    continue
                i, j = 4 * (xx + Nx * yy) + sa, 4 * c + sb
                rows += [i, j]
                cols += [j, i]
                vals += [-1.0, -1.0]
    D = 4 * Nx * Ny
    return sp.coo_matrix((vals, (rows, cols)), shape=(D, D)).tocsr()


@pytest.mark.parametrize("periodic", [(1, 1), (0, 0), (1, 0)])
def test_graphene_equation_equals_dsl_form_up_to_mirror(periodic):
    Nx, Ny = 5, 4
    V = W.disorder_potential(4 * Nx * Ny, 1.0, 3)
    Hd = _mirrored_hamiltonian(Nx, Ny, periodic, V).toarray()
    # mirror x -> Nx-1-x of the equation form (V mirrored along with it)
    perm = np.array([4 * ((Nx - 1 - (c % Nx)) + Nx * (c // Nx)) + nu
                     for c in range(Nx * Ny) for nu in range(4)])
    He = O.graphene_hamiltonian((Nx, Ny), periodic, 1.0, V[perm]).toarray()
    assert np.allclose(He[np.ix_(perm, perm)], Hd)
    assert np.allclose(np.linalg.eigvalsh(He), np.linalg.eigvalsh(Hd))


# ---------------------------------------------------------------- scaling
def test_gershgorin_matches_row_sums_and_brackets_spectrum():
    dims = (5, 4, 3)
    n = 60
    V = W.disorder_potential(n, 1.0, 1)
    H = O.ti_hamiltonian(dims, (1, 1, 1), 1.0, 2.0, V)
    emin, emax = O.gershgorin(H)
    # every TI bond block has unit row abs-sum per unit t: radius 6 t in the bulk
    assert abs(emin - (-2.0 - 6.0 + V.min())) < 1e-14 or abs(emin - (-2.0 - 6.0 + V[V < 0].min())) < 1e-14
    assert abs(emax - (2.0 + 6.0 + V.max())) < 1e-14
    e = np.linalg.eigvalsh(H.toarray())
    assert emin <= e.min() and e.max() <= emax
    a, b = O.cheb_scale(emin, emax)
    et = (e - b) / a
    assert et.min() > -1 and et.max() < 1
    # graphene: radius 3 t
    Hg = O.graphene_hamiltonian((4, 4), (1, 1), 1.0, np.full(64, 0.25))
    assert O.gershgorin(Hg) == (0.25 - 3.0, 0.25 + 3.0)


# ---------------------------------------------------------------- KPM
def _dense_Tk(H, a, b, kmax):
    e, U = np.linalg.eigh(H.toarray())
    et = np.clip((e - b) / a, -1, 1)
    return U, np.array([np.cos(k * np.arccos(et)) for k in range(kmax)])


def test_kpm_mu0_is_one_for_random_phase():
    dims = (3, 4, 5)
    n = 60
    H = O.ti_hamiltonian(dims, (1, 1, 0), 1.0, 2.0, W.disorder_potential(n, 1.0, 2))
    a, b = O.cheb_scale(*O.gershgorin(H))
    r = W.random_phase_block(4 * n, 3, 9)
    mu = O.kpm_moments(H, r, 16, a, b)
    assert np.allclose(mu[:, 0], 1.0, atol=1e-14)
    assert np.max(np.abs(mu.imag)) < 1e-13


def test_kpm_eigenvector_start_gives_chebyshev_of_energy():
    dims = (3, 3, 2)
    n = 18
    H = O.ti_hamiltonian(dims, (1, 1, 1), 1.0, 2.0, W.disorder_potential(n, 1.0, 4))
    a, b = O.cheb_scale(*O.gershgorin(H))
    e, U = np.linalg.eigh(H.toarray())
    l = [0, 17, 40]
    mu = O.kpm_moments(H, U[:, l], 64, a, b)
    ref = np.array([[math.cos(k * math.acos((e[j] - b) / a)) for k in range(64)] for j in l])
    assert np.max(np.abs(mu - ref)) < 1e-12


def test_kpm_exact_trace_equals_eigenvalue_sum():
    dims = (2, 2, 2)
    n = 8
    H = O.ti_hamiltonian(dims, (1, 1, 1), 1.0, 2.0, W.disorder_potential(n, 1.0, 5))
    a, b = O.cheb_scale(*O.gershgorin(H))
    D = 4 * n
    mu = O.kpm_moments(H, np.eye(D), 40, a, b).real.mean(axis=0)
    e = np.linalg.eigvalsh(H.toarray())
    ref = np.array([np.mean(np.cos(k * np.arccos((e - b) / a))) for k in range(40)])
    assert np.max(np.abs(mu - ref)) < 1e-12


def test_kpm_matches_dense_polynomial_graphene():
    H = O.graphene_hamiltonian((3, 4), (0, 1), 1.0, W.disorder_potential(48, 0.5, 6))
    a, b = O.cheb_scale(*O.gershgorin(H))
    r = W.random_phase_block(48, 2, 1)
    U, Tk = _dense_Tk(H, a, b, 30)
    ref = np.array([[np.vdot(r[:, j], U @ (Tk[k] * (U.conj().T @ r[:, j]))) for k in range(30)]
                    for j in range(2)])
    assert np.max(np.abs(O.kpm_moments(H, r, 30, a, b) - ref)) < 1e-12


def test_cheb_step_reproduces_recurrence_and_apply():
    H = O.ti_hamiltonian((3, 2, 4), (1, 0, 1), 1.0, 2.0, W.disorder_potential(24, 1.0, 8))
    x = W.gaussian_block(96, 2, 3)
    y, _, dots = O.cheb_step(H, x, np.zeros_like(x), [1, 1], [0, 0], [0, 0])
    e, U = np.linalg.eigh(H.toarray())
    assert np.allclose(y, U @ (e[:, None] * (U.conj().T @ x)), atol=1e-12)
    # <Hx|x> is the Rayleigh numerator, real for Hermitian H
    ray = np.sum(e[:, None] * np.abs(U.conj().T @ x) ** 2, axis=0)
    assert np.allclose(dots[:, 1], ray, atol=1e-12)
    assert np.allclose(dots[:, 0].real, np.sum(np.abs(x) ** 2, axis=0))
    a, b = O.cheb_scale(*O.gershgorin(H))
    w0 = x
    w1, _, _ = O.cheb_step(H, w0, np.zeros_like(x), [1 / a] * 2, [b] * 2, [0, 0])
    w2, z, _ = O.cheb_step(H, w1, w0, [2 / a] * 2, [b] * 2, [-1, -1], z=w0.copy(), delta=[0.5, 0.5])
    _, Tk = _dense_Tk(H, a, b, 3)
    assert np.allclose(w2, U @ (Tk[2][:, None] * (U.conj().T @ x)), atol=1e-12)
    assert np.allclose(z, w0 + 0.5 * w2)


# ---------------------------------------------------------------- propagation
def test_bessel_against_library_and_sum_rules():
    for x in (0.3, 3.05, 12.5):
        J = O.bessel_j(x, 80)
        assert np.max(np.abs(J - jv(np.arange(81), x))) < 2e-15
        assert abs(J[0] + 2 * J[2::2].sum() - 1) < 1e-15
        assert abs(J[0] ** 2 + 2 * np.sum(J[1:] ** 2) - 1) < 1e-14


def test_bessel_asymptotic_decay_from_paper():
    f = facts()["bessel_asymptotic"]
    x = f["x"]
    J = O.bessel_j(x, 60)
    prev = 0
    for k in f["k_values"]:
        ratio = J[k] / ((math.e * x / (2 * k)) ** k / math.sqrt(2 * math.pi * k))
        assert 0.85 < ratio < 1.0 and ratio > prev   # approaches 1 from below as k grows
        prev = ratio


def test_truncation_order_for_graphene_qd_workload():
    # open graphene, V in [0, 0.1]: Gershgorin [-3, 3.1], a = 3.055, dt = 1 -> M = 19
    a, b = O.cheb_scale(-3.0, 3.1)
    c = O.propagation_coeffs(a, 1.0, 1e-14)
    assert len(c) - 1 == 19
    J = O.bessel_j(a, 30)
    assert abs(J[19]) >= 1e-14 > abs(J[20])
    assert np.allclose(np.abs(c), np.abs(J[:20]))
    assert np.allclose(c[1], -1j * J[1]) and np.allclose(c[2], -J[2])


def test_propagation_matches_matrix_exponential():
    cells = (3, 4)
    V = W.disorder_potential(48, 0.6, 2)
    H = O.graphene_hamiltonian(cells, (0, 0), 1.0, V)
    a, b = O.cheb_scale(*O.gershgorin(H))
    psi0 = W.gaussian_block(48, 1, 4)[:, 0]
    psi0 /= np.linalg.norm(psi0)
    psi = O.propagate(H, psi0, 1.0, 3, a, b)
    U = sla.expm(-1j * H.toarray() * 1.0)
    ref = U @ (U @ (U @ psi0))
    assert np.linalg.norm(psi - ref) < 1e-12
    assert abs(np.linalg.norm(psi) - 1) < 1e-13


def test_propagation_eigenstate_picks_up_phase():
    H = O.ti_hamiltonian((2, 3, 2), (1, 1, 0), 1.0, 2.0, W.disorder_potential(12, 1.0, 3))
    a, b = O.cheb_scale(*O.gershgorin(H))
    e, U = np.linalg.eigh(H.toarray())
    psi = O.propagate(H, U[:, 5], 0.7, 4, a, b)
    assert np.linalg.norm(psi - np.exp(-1j * e[5] * 2.8) * U[:, 5]) < 1e-12


def test_filter_series_matches_dense_polynomial():
    H = O.ti_hamiltonian((2, 2, 3), (1, 1, 1), 1.0, 2.0, W.disorder_potential(12, 1.0, 1))
    a, b = O.cheb_scale(*O.gershgorin(H))
    g = np.cos(np.arange(12) * 0.3) / (1 + np.arange(12))
    x = W.gaussian_block(48, 2, 2)
    U, Tk = _dense_Tk(H, a, b, 12)
    ref = U @ ((g @ Tk)[:, None] * (U.conj().T @ x))
    assert np.allclose(O.cheb_series(H, x, g, a, b), ref, atol=1e-12)


# ---------------------------------------------------------------- adjoint
def _loss(H0diag_free, V, cells, psi0, dt, nsteps, a, b, mask):
    H = O.graphene_hamiltonian(cells, (0, 0), 1.0, V)
    psi = O.propagate(H, psi0, dt, nsteps, a, b)
    return O.detector_probability(psi, mask)


def test_adjoint_gradient_matches_central_differences():
    cells = (4, 3)
    n = 48
    V = W.disorder_potential(n, 0.4, 12)
    H = O.graphene_hamiltonian(cells, (0, 0), 1.0, V)
    a, b = O.cheb_scale(*O.gershgorin(H))
    psi0 = W.gaussian_block(n, 1, 3)[:, 0]
    psi0 /= np.linalg.norm(psi0)
    mask = np.zeros(n, dtype=bool)
    mask[[3, 7, 8, 20, 33]] = True
    dt, S = 0.8, 3
    psiS = O.propagate(H, psi0, dt, S, a, b)
    G = 2.0 * mask * psiS
    grad, _ = O.propagate_adjoint(H, psi0, dt, S, a, b, G, O=1)
    h = 1e-6
    for site in (0, 3, 17, 30, 47):
        Vp, Vm = V.copy(), V.copy()
        Vp[site] += h
        Vm[site] -= h
        fd = (_loss(None, Vp, cells, psi0, dt, S, a, b, mask) -
              _loss(None, Vm, cells, psi0, dt, S, a, b, mask)) / (2 * h)
        assert abs(fd - grad[site]) < 1e-8 * max(1.0, abs(fd)) + 1e-9


def test_adjoint_gradient_matches_daleckii_krein():
    # one exact step psi1 = exp(-i H dt) psi0: dU/dV_n = U_ev [F o (U_ev^+ P_n U_ev)] U_ev^+
    dims = (2, 2, 2)
    n = 8
    V = W.disorder_potential(n, 1.0, 21)
    H = O.ti_hamiltonian(dims, (1, 1, 0), 1.0, 2.0, V)
    a, b = O.cheb_scale(*O.gershgorin(H))
    dt = 0.9
    psi0 = W.random_phase_block(32, 1, 5)[:, 0]
    e, U = np.linalg.eigh(H.toarray())
    ph = np.exp(-1j * e * dt)
    de = e[:, None] - e[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        F = np.where(np.abs(de) > 1e-9, (ph[:, None] - ph[None, :]) / np.where(de == 0, 1, de),
                     -1j * dt * ph[:, None])
    psi1 = U @ (ph * (U.conj().T @ psi0))
    mask_rows = np.zeros(32, dtype=bool)
    mask_rows[4:12] = True
    G = 2.0 * mask_rows * psi1
    ref = np.zeros(n)
    for site in range(n):
        P = np.zeros(32)
        P[4 * site:4 * site + 4] = 1.0
        Pe = U.conj().T @ (P[:, None] * U)
        dU = U @ (F * Pe) @ U.conj().T
        ref[site] = np.real(np.vdot(G, dU @ psi0))
    grad, G0 = O.propagate_adjoint(H, psi0, dt, 1, a, b, G, O=4)
    assert np.max(np.abs(grad - ref)) < 1e-11
    # and the adjoint state is U^+ G
    Uf = U @ (ph[:, None] * U.conj().T)
    assert np.allclose(G0[:, 0], Uf.conj().T @ G, atol=1e-12)


# ---------------------------------------------------------------- inputs
def test_counter_hash_known_values_and_disorder_range():
    # SplitMix64 finaliser of 0 is 0 and of the golden gamma a published constant:
    # splitmix64 with state 0 yields 0xE220A8397B1DCDAF as its first output
    assert int(W.mix64(np.array([0], dtype=np.uint64))[0]) == 0
    assert int(W.mix64(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))[0]) == 0xE220A8397B1DCDAF
    V = W.disorder_potential(100000, 4.0, 2)
    assert V.min() >= -2.0 and V.max() < 2.0 and abs(V.mean()) < 0.02
    r = W.random_phase_block(1000, 3, 3)
    assert np.allclose(np.sum(np.abs(r) ** 2, axis=0), 1.0)


# ------------------------------------------------------------------ spectral densities (Eq. ak, Eq. DOS)
def test_jackson_kernel_small_cases_by_hand():
    # q = pi/(M+1); M = 2: g = (1, (2 cos q + sin q cot q)/3) = (1, 1/2);
    # M = 3: g_1 = (3 cos(pi/4) + sin(pi/4))/4 = 1/sqrt(2), g_2 = (0 + 1)/4 = 1/4
    assert np.allclose(O.jackson_kernel(2), [1.0, 0.5], atol=1e-15)
    assert np.allclose(O.jackson_kernel(3), [1.0, 1.0 / math.sqrt(2.0), 0.25], atol=1e-15)
    g = O.jackson_kernel(256)
    assert g[0] == 1.0 and np.all(np.diff(g) < 0) and g[-1] > 0


def test_lorentz_kernel_small_cases_by_hand():
    # M = 2: g_1 = sinh(lam / 2) / sinh(lam) = 1 / (2 cosh(lam / 2)) (sinh 2u = 2 sinh u cosh u);
    # M = 3: g_1 = sinh(2 lam / 3) / sinh(lam), g_2 = sinh(lam / 3) / sinh(lam), and with
    # u = lam / 3, sinh 3u = sinh u (4 cosh^2 u - 1), so g_2 = 1 / (4 cosh^2(lam / 3) - 1)
    for lam in (0.5, 2.0, 4.0):
        assert np.allclose(O.lorentz_kernel(2, lam), [1.0, 0.5 / math.cosh(lam / 2)], rtol=1e-14)
        g3 = O.lorentz_kernel(3, lam)
        assert abs(g3[2] - 1.0 / (4.0 * math.cosh(lam / 3) ** 2 - 1.0)) < 1e-14
        assert abs(g3[1] - 2.0 * math.cosh(lam / 3) * g3[2]) < 1e-14  # sinh 2u = 2 cosh u sinh u
    # the damping is a two-point boundary problem of the recurrence
    # g_{k+1} + g_{k-1} = 2 cosh(lam / M) g_k with g_0 = 1 and g_M = 0
    M, lam = 64, 4.0
    g = np.append(O.lorentz_kernel(M, lam), 0.0)
    assert abs(g[0] - 1.0) < 1e-15
    assert np.max(np.abs(g[2:] + g[:-2] - 2.0 * math.cosh(lam / M) * g[1:-1])) < 1e-14


def test_lorentz_damped_delta_peak_equals_geometric_series_closed_form():
    # One eigenvalue E0 has moments mu_k = T_k(x0).  With the Lorentz factors
    # g_k = [r^k - e^{-2 lam} r^{-k}] / (1 - e^{-2 lam}), r = e^{-lam/M} (the
    # exponential form of sinh(lam (1 - k/M)) / sinh(lam)), the damped series
    # sum_k (2 - delta_k0) g_k cos(k th0) cos(k th) is a combination of finite
    # geometric sums sum_{k<M} q^k cos(k phi) = Re[(1 - z^M) / (1 - z)], z = q e^{i phi},
    # at phi = th -+ th0: the Lorentzian peak of width ~lam/M in th of the KPM review
    # the paper cites (Weisse et al., Rev. Mod. Phys. 78, 275, Sec. II.C).
    M, lam, a, b = 200, 4.0, 3.0, 0.5
    E0 = 1.1
    x0 = (E0 - b) / a
    th0 = math.acos(x0)
    mu = np.cos(np.arange(M) * th0)[None, :]
    E = np.linspace(b - a + 1e-6, b + a - 1e-6, 4001)
    rho = O.kpm_density(mu, E, a, b, O.lorentz_kernel(M, lam))
    th = np.arccos((E - b) / a)

    def geo(q, phi):
        z = q * np.exp(1j * phi)
        return np.real((1.0 - z ** M) / (1.0 - z))

    def damped(q):
        return geo(q, th - th0) + geo(q, th + th0) - 1.0

    r = math.exp(-lam / M)
    series = (damped(r) - math.exp(-2 * lam) * damped(1.0 / r)) / (1.0 - math.exp(-2 * lam))
    ref = series / (math.pi * a * np.sin(th))
    assert np.max(np.abs(rho - ref)) < 1e-10 * np.max(np.abs(ref))
    # the peak sits at E0 and its half width in th is close to lam / M
    i = int(np.argmax(rho * np.sin(th)))
    assert abs(E[i] - E0) <= 2 * (E[1] - E[0])
    prof = rho * np.sin(th)
    half = th[prof >= 0.5 * prof[i]]
    assert abs((half.max() - half.min()) / 2 - lam / M) < 0.25 * lam / M


def test_kpm_density_normalisation_by_gauss_chebyshev_quadrature():
    # int rho dE = scale * sum_r g_0 mu_0^r, because int T_k(x) / (pi sqrt(1 - x^2)) dx = delta_k0;
    # Gauss-Chebyshev quadrature with N > M nodes is exact for the series
    rng = np.random.default_rng(3)
    mu = rng.standard_normal((3, 40))
    a, b = 2.5, 0.3
    g = O.jackson_kernel(40)
    N = 200
    x = np.cos(np.pi * (np.arange(N) + 0.5) / N)
    rho = O.kpm_density(mu, b + a * x, a, b, g, scale=0.7)
    integral = np.pi / N * np.sum(rho * a * np.sqrt(1 - x * x))
    assert abs(integral - 0.7 * g[0] * mu[:, 0].sum()) < 1e-12
    assert np.all(O.kpm_density(mu, np.array([b - a - 1e-3, b + a + 1e-3]), a, b, g) == 0.0)


def test_kpm_dos_counts_the_eigenvalues_of_dense_diagonalisation():
    # Eq. DOS from exact trace moments (all unit vectors) of a gapped periodic
    # disordered TI: integrated over windows whose ends lie in spectral gaps it
    # counts the eigenvalues of scipy/numpy's dense solver; Jackson damping keeps it >= 0
    dims = (4, 4, 4)
    V = W.disorder_potential(64, 1.0, 7)
    H = O.ti_hamiltonian(dims, (1, 1, 1), 1.0, 2.0, V)
    ev = np.linalg.eigvalsh(H.toarray())
    a, b = O.cheb_scale(*O.gershgorin(H))
    M = 512
    mu = O.kpm_moments(H, np.eye(H.shape[0], dtype=np.complex128), M, a, b).real
    E = np.linspace(b - a + 1e-9, b + a - 1e-9, 20001)
    rho = O.kpm_density(mu, E, a, b, O.jackson_kernel(M))
    assert rho.min() > 0
    assert not np.any(np.abs(ev) < 0.5)  # the window edge E = 0 sits in the bulk gap
    for lo, hi in ((b - a, 0.0), (0.0, b + a)):
        m = (E >= lo) & (E < hi)
        assert abs(np.trapezoid(rho[m], E[m]) - np.sum((ev >= lo) & (ev < hi))) < 1e-3


@pytest.mark.parametrize("k", [(2 * math.pi * 2 / 8, 0.0, 0.0),
                               (2 * math.pi / 8, 2 * math.pi * 3 / 8, 2 * math.pi / 8)])
def test_spectral_function_of_clean_ti_peaks_at_closed_form_bands(k):
    # Eq. ak on a clean periodic lattice: psi(k, nu) spans the Bloch block at k,
    # whose eigenvalues are +-E(k) (closed form, reading of Eq. bloch_H_topi),
    # each twice: A(k, E) = 2 delta(E - E(k)) + 2 delta(E + E(k)), total weight 4
    dims = (8, 8, 8)
    H = O.ti_hamiltonian(dims, (1, 1, 1), 1.0, 2.0, np.zeros(512))
    a, b = O.cheb_scale(*O.gershgorin(H))
    Ek = math.sqrt((2.0 - sum(math.cos(c) for c in k)) ** 2 + sum(math.sin(c) ** 2 for c in k))
    mu = O.kpm_moments(H, O.bloch_vectors(dims, k), 512, a, b).real
    E = np.linspace(b - a + 1e-9, b + a - 1e-9, 40001)
    A = O.kpm_density(mu, E, a, b, O.jackson_kernel(512))
    for e0 in (Ek, -Ek):
        m = (E > e0 - 0.4) & (E < e0 + 0.4)
        assert abs(E[m][np.argmax(A[m])] - e0) < 2e-3
        assert abs(np.trapezoid(A[m], E[m]) - 2.0) < 2e-3
    assert abs(np.trapezoid(A, E) - 4.0) < 1e-3


# ------------------------------------------------------------------ ChebFD (Sec. 5.3)
def _window_around_zero(ev, n):
    """[lo, hi] holding the n eigenvalues nearest 0, its ends at midpoints of spectral gaps."""
    idx = np.sort(np.argsort(np.abs(ev))[:n])
    i0, i1 = idx[0], idx[-1]
    return (ev[i0 - 1] + ev[i0]) / 2, (ev[i1] + ev[i1 + 1]) / 2


def test_chebfd_window_is_the_indicator_series():
    # undamped coefficients of the indicator reproduce it away from the edges
    # (quadrature check of c_k = (2 - delta_k0)/pi int chi(x) T_k(x)/sqrt(1-x^2) dx)
    lo, hi, a, b = -0.3, 0.5, 2.0, 0.1
    N = 4000
    x = np.cos(np.pi * (np.arange(N) + 0.5) / N)
    chi = ((b + a * x >= lo) & (b + a * x <= hi)).astype(float)
    ref = np.array([(1 if k == 0 else 2) / N * np.sum(chi * np.cos(k * np.arccos(x))) for k in range(60)])
    c = O.chebfd_window(lo, hi, a, b, 59) / O.jackson_kernel(60)
    assert np.max(np.abs(c - ref)) < 2e-3  # midpoint rule on a discontinuous integrand


def test_chebfd_finds_the_interior_eigenpairs_of_dense_diagonalisation():
    dims = (6, 6, 4)
    H = O.ti_hamiltonian(dims, (1, 1, 0), 1.0, 2.0, W.disorder_potential(144, 1.0, 3))
    ev = np.sort(np.linalg.eigvalsh(H.toarray()))
    a, b = O.cheb_scale(*O.gershgorin(H))
    lo, hi = _window_around_zero(ev, 16)
    th, X, res, it = O.chebfd(H, W.gaussian_block(H.shape[0], 32, 1), lo, hi, a, b, 400, 40, 1e-10)
    target = ev[(ev >= lo) & (ev <= hi)]
    assert len(th) == len(target) == 16
    assert np.max(np.abs(np.sort(th) - target)) < 1e-12
    assert np.all(res < 1e-10)
    assert np.allclose(X.conj().T @ X, np.eye(16), atol=1e-12)


@pytest.mark.parametrize("d1,d2", [(0.4, 0.0), (0.0, -0.3), (0.35, 0.25)])
def test_ti_delta_terms_match_the_bloch_spectrum(d1, d2):
    # Delta_1 Gamma^5 + Delta_2 Gamma^15 (Eq. TB_H_topi) on a clean periodic lattice: the
    # spectrum is the union over the lattice momenta of the eigenvalues of the 4x4 Bloch
    # matrix H(k) = E0 + sum_j (T_j e^{-i k_j} + T_j^+ e^{i k_j}), T_j = -(t/2)(Gamma^1 - i Gamma^{j+1})
    # the block from site n to n + e_j, with Gamma^15 = [Gamma^1, Gamma^5]/(2i)
    dims, t, m = (4, 3, 5), 1.0, 1.5
    H = O.ti_hamiltonian(dims, (1, 1, 1), t, m, np.zeros(60), d1, d2)
    ev = np.sort(np.linalg.eigvalsh(H.toarray()))
    G = O.gamma_matrices()
    G15 = (G[1] @ G[5] - G[5] @ G[1]) / 2j
    E0 = m * G[1] + d1 * G[5] + d2 * G15
    T = [-(t / 2) * (G[1] - 1j * G[j + 1]) for j in (1, 2, 3)]
    bloch = []
    for kx in 2 * np.pi * np.arange(dims[0]) / dims[0]:
        for ky in 2 * np.pi * np.arange(dims[1]) / dims[1]:
            for kz in 2 * np.pi * np.arange(dims[2]) / dims[2]:
                Hk = E0.copy()
                for Tj, kj in zip(T, (kx, ky, kz)):
                    Hk = Hk + Tj * np.exp(-1j * kj) + Tj.conj().T * np.exp(1j * kj)
                bloch.extend(np.linalg.eigvalsh(Hk))
    assert np.max(np.abs(np.sort(bloch) - ev)) < 1e-12
    a, b = O.cheb_scale(*O.gershgorin(H))
    assert b - a <= ev[0] and ev[-1] <= b + a


# ------------------------------------------------------------------ Weyl semimetal (Eq. TB_H_wsm)
@pytest.mark.parametrize("dims,k0", [((8, 3, 4), math.pi / 2), ((4, 4, 2), math.pi / 2), ((6, 5, 3), 1.1)])
def test_wsm_periodic_spectrum_is_the_closed_form_band(dims, k0):
    # Eq. band_h_wsm: eps(k) = sigma_x (cos kx - cos k0 + cos ky + cos kz - 2) + sigma_y sin ky
    # + sigma_z sin kz, eigenvalues +-|d(k)|, over the lattice momenta of a periodic cuboid
    H = O.wsm_hamiltonian(dims, (1, 1, 1), np.zeros(int(np.prod(dims))), k0)
    assert abs(H - H.conj().T).max() == 0
    ev = np.sort(np.linalg.eigvalsh(H.toarray()))
    band = []
    for kx in 2 * np.pi * np.arange(dims[0]) / dims[0]:
        for ky in 2 * np.pi * np.arange(dims[1]) / dims[1]:
            for kz in 2 * np.pi * np.arange(dims[2]) / dims[2]:
                d = np.array([math.cos(kx) - math.cos(k0) + math.cos(ky) + math.cos(kz) - 2.0,
                              math.sin(ky), math.sin(kz)])
                band += [np.linalg.norm(d), -np.linalg.norm(d)]
    assert np.max(np.abs(np.sort(band) - ev)) < 1e-12


def test_wsm_weyl_nodes_and_open_boundaries():
    # Weyl nodes at (+-k0, 0, 0), k0 = pi/2: a periodic cuboid with Lx = 8 contains both,
    # so E = 0 appears four times (two nodes, two bands each); an open axis drops the
    # bonds that leave the cuboid (the Hermitian matrix then differs only there)
    H = O.wsm_hamiltonian((8, 4, 4), (1, 1, 1), np.zeros(128))
    ev = np.linalg.eigvalsh(H.toarray())
    assert np.sum(np.abs(ev) < 1e-12) == 4
    Ho = O.wsm_hamiltonian((8, 4, 4), (1, 1, 0), np.zeros(128))
    diff = (H - Ho).tocoo()
    rows = diff.row // 2
    z = rows // 32
    assert set(np.unique(z)) == {0, 3}  # only the bonds across the z boundary differ


@pytest.mark.parametrize("k", [(math.pi / 2, 0.0, 0.0), (math.pi / 4, math.pi / 2, math.pi)])
def test_wsm_spectral_function_peaks_at_the_closed_form_band(k):
    # Eq. ak for the Weyl semimetal: the two states psi(k, nu) span the 2x2 Bloch block of
    # Eq. band_h_wsm with eigenvalues +-|d(k)|, one each; at the Weyl node both sit at E = 0
    dims = (8, 4, 4)
    H = O.wsm_hamiltonian(dims, (1, 1, 1), np.zeros(128))
    a, b = O.cheb_scale(*O.gershgorin(H))
    d = np.array([math.cos(k[0]) + math.cos(k[1]) + math.cos(k[2]) - 2.0 - math.cos(math.pi / 2),
                  math.sin(k[1]), math.sin(k[2])])
    e0 = float(np.linalg.norm(d))
    mu = O.kpm_moments(H, O.bloch_vectors(dims, k, O=2), 512, a, b).real
    E = np.linspace(b - a + 1e-9, b + a - 1e-9, 40001)
    A = O.kpm_density(mu, E, a, b, O.jackson_kernel(512))
    assert abs(np.trapezoid(A, E) - 2.0) < 1e-3
    for e in ((0.0,) if e0 < 1e-12 else (e0, -e0)):
        m = (E > e - 0.3) & (E < e + 0.3)
        assert abs(E[m][np.argmax(A[m])] - e) < 2e-3
        assert abs(np.trapezoid(A[m], E[m]) - (2.0 if e0 < 1e-12 else 1.0)) < 3e-3


def test_oracle_terms_count_the_couplings_of_every_row():
    # Eq. TB_H_topi per row: the diagonal plus, for each of the six neighbours,
    # the Gamma^1 entry and the one Gamma^{j+1} entry of the bond block: 13 terms.
    # On a periodic axis of length 2 both neighbours are the same site: the 13
    # terms fall on 11 distinct columns, and in the summed matrix the Gamma^{j+1}
    # parts of A_j and A_j^+ cancel (A_j + A_j^+ = -t Gamma^1), leaving 10.
    V = W.disorder_potential(27, 1.0, 3)
    r, c, _ = O.ti_hamiltonian((3, 3, 3), (1, 1, 1), 1.0, 2.0, V, terms=True)
    assert np.all(np.bincount(r) == 13)
    assert all(len(set(c[r == i])) == 13 for i in range(0, 108, 7))
    V = W.disorder_potential(18, 1.0, 3)
    r, c, _ = O.ti_hamiltonian((3, 2, 3), (1, 1, 1), 1.0, 2.0, V, terms=True)
    assert np.all(np.bincount(r) == 13)
    assert all(len(set(c[r == i])) == 11 for i in range(72))
    H = O.ti_hamiltonian((3, 2, 3), (1, 1, 1), 1.0, 2.0, V)
    assert np.all(np.diff(H.indptr) == 10)
    # open corner site of a 3x3x3 cube: the diagonal and three bonds
    r, c, _ = O.ti_hamiltonian((3, 3, 3), (0, 0, 0), 1.0, 2.0, W.disorder_potential(27, 1.0, 3), terms=True)
    assert np.bincount(r)[0] == 7
    # graphene (Eq. graphene_model): every site has three bonds plus its potential
    V = W.disorder_potential(48, 1.0, 2)
    r, _, _ = O.graphene_hamiltonian((4, 3), (1, 1), 1.0, V, terms=True)
    assert np.all(np.bincount(r) == 4)
