"""The gate-defined quantum-dot array (Eq. qdotarray) regenerated inside the
graphene sweeps, against the stored potential of the input generator.

complex128 sweeps and the spectral bounds evaluate the array in fp64 (equal to
the generator to ~1e-15 V0); complex64 sweeps evaluate it in fp32 from
dot-relative coordinates (within ~1e-7 V0), well inside the complex64 sweep
tolerance."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pv = pytest.importorskip("paper_1708_09689_gb300")
pytestmark = pytest.mark.gpu

# (cells, periodic, dots K, radius, V0, width, dV): overlapping cut-off discs
# (radius + 20 w above the spacing 4 radius), dots that reach the edges, a
# single dot, graded heights
CASES = [((48, 40), (0, 0), 3, 6.0, 0.3, 1.0, 0.0),
         ((40, 24), (1, 1), 2, 5.0, -0.2, 2.0, 0.05),
         ((33, 17), (1, 0), 1, 8.0, 0.5, 0.5, 0.0),
         ((64, 48), (0, 1), 4, 4.5, 0.1, 1.5, 0.02)]


def _pair(cells, per, K, Rd, V0, w, dV):
    V = W.qdot_potential(cells[0], cells[1], K, Rd, V0, w, dV)
    lat_q = pv.Lattice.graphene(cells, per, qdots=(K, Rd, V0, w, dV))
    lat_s = pv.Lattice.graphene(cells, per, V=V)
    H = O.graphene_hamiltonian(cells, per, 1.0, V)
    return lat_q, lat_s, H, V


@pytest.mark.parametrize("case", CASES)
def test_qdot_potential_and_bounds_match_the_generator(case):
    lat_q, lat_s, H, V = _pair(*case)
    Vq = lat_q.potential().cpu().numpy()
    assert np.max(np.abs(Vq - V)) < 1e-13 * max(1.0, np.max(np.abs(V)))
    assert np.count_nonzero(V) > 0
    bq, bs = lat_q.spectral_bounds(), lat_s.spectral_bounds()
    assert np.allclose(bq, bs, rtol=0, atol=1e-13)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec,tol", [(pv.C128, 1e-12), (pv.C64, 2e-6)])
def test_qdot_apply_H_matches_oracle(case, prec, tol):
    lat_q, lat_s, H, V = _pair(*case)
    x = W.gaussian_block(H.shape[0], 2, 4)
    cdt = torch.complex128 if prec == pv.C128 else torch.complex64
    y = pv.apply_H(lat_q, torch.from_numpy(x).to("cuda", cdt)).cpu().numpy().astype(np.complex128)
    xr = x.astype(np.complex64).astype(np.complex128) if prec == pv.C64 else x
    ref = H @ xr
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < tol


def test_qdot_propagation_and_kpm_match_the_stored_potential():
    cells, per = (48, 40), (0, 0)
    lat_q, lat_s, H, V = _pair(cells, per, 3, 6.0, 0.3, 1.0, 0.0)
    _, _, a, b = lat_s.spectral_bounds()
    psi0 = W.gaussian_block(H.shape[0], 1, 9)
    psi0 /= np.linalg.norm(psi0)
    ref = O.propagate(H, psi0, 0.7, 3, a, b)
    for prec, tol in ((pv.C128, 1e-12), (pv.C64, 1e-5)):
        out = {}
        for name, lat in (("q", lat_q), ("s", lat_s)):
            psi = torch.from_numpy(psi0).cuda()
            pv.cheb_propagate(lat, psi, 0.7, 3, a, b, prec=prec)
            out[name] = psi.cpu().numpy()
        assert np.linalg.norm(out["q"] - ref) < tol
        assert np.linalg.norm(out["q"] - out["s"]) < tol
    r = W.random_phase_block(H.shape[0], 2, 3)
    mu = pv.kpm_moments(lat_q, 40, a, b, r0=torch.from_numpy(r).cuda()).cpu().numpy()
    assert np.max(np.abs(mu - O.kpm_moments(H, r, 40, a, b).real)) < 1e-12


def test_qdot_rejects_other_models_bad_parameters_and_set_potential():
    with pytest.raises(pv.PvscError, match="graphene"):
        pv.Lattice.ti((4, 4, 4), (1, 1, 1), qdots=(2, 3.0, 0.1, 1.0))
    for bad in [(0, 3.0, 0.1, 1.0), (17, 3.0, 0.1, 1.0), (2, 0.0, 0.1, 1.0), (2, 3.0, 0.1, -1.0),
                (2, 3.0, float("nan"), 1.0)]:
        with pytest.raises(pv.PvscError):
            pv.Lattice.graphene((8, 8), (0, 0), qdots=bad)
    lat = pv.Lattice.graphene((8, 8), (0, 0), qdots=(2, 3.0, 0.1, 1.0))
    with pytest.raises(pv.PvscError, match="on the fly"):
        lat.set_potential(torch.zeros(lat.n_sites, dtype=torch.float64, device="cuda"))


def test_qdot_full_workload_potential_and_sampled_rows():
    # the propagation workload's 2^25-site lattice: the regenerated potential
    # equals the generator's, and a complex64 sweep agrees with the stored one
    cfg = W.CONFIG_GRAPHENE_QD
    V = cfg.potential()
    lat_q = pv.Lattice.graphene(cfg.cells, (0, 0), t=cfg.t, qdots=(cfg.ndots, cfg.R_dot, cfg.V0, cfg.w))
    Vq = lat_q.potential().cpu().numpy()
    assert np.max(np.abs(Vq - V)) < 1e-13
    lat_s = pv.Lattice.graphene(cfg.cells, (0, 0), t=cfg.t, V=V)
    x = torch.from_numpy(cfg.packet()).to("cuda", torch.complex64)
    yq = pv.apply_H(lat_q, x)
    ys = pv.apply_H(lat_s, x)
    assert (torch.linalg.vector_norm(yq - ys) / torch.linalg.vector_norm(ys)).item() < 1e-6
