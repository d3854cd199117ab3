"""The seeded input generators against brute force (no GPU).

The quantum-dot array potential (Eq. qdotarray) is an input of the graphene
workloads, stored by the stored-potential runs and regenerated inside the
sweep by PVSC_V_QDOT; both sides are compared with this generator, so its
per-dot bounding boxes are checked here against an evaluation of every dot at
every site."""
import math

import numpy as np
import pytest

import workloads as W


def _brute_qdot(Nx, Ny, K, R, V0, w, dV):
    X, Y = W.graphene_positions(Nx, Ny)
    Xe, Ye = W.graphene_extent(Nx, Ny)
    D, rcut = 4.0 * R, R + 20.0 * w
    V = np.zeros(X.shape)
    for l in range(K):
        for k in range(K):
            Rx = Xe / 2.0 + (l - (K - 1) / 2.0) * D
            Ry = Ye / 2.0 + (k - (K - 1) / 2.0) * D
            d = np.hypot(X - Rx, Y - Ry)
            V += np.where(d < rcut, (V0 + dV * abs(k - K / 2.0)) * 0.5 * (1.0 + np.tanh((R - d) / w)), 0.0)
    return V


@pytest.mark.parametrize("case", [((48, 40), 3, 6.0, 0.3, 1.0, 0.0), ((40, 24), 2, 5.0, -0.2, 2.0, 0.05),
                                  ((33, 17), 1, 8.0, 0.5, 0.5, 0.0), ((64, 48), 4, 4.5, 0.1, 1.5, 0.02),
                                  ((120, 60), 4, 7.0, 0.1, 5.0, 0.0)])
def test_qdot_potential_equals_every_dot_at_every_site(case):
    (Nx, Ny), K, R, V0, w, dV = case
    V = W.qdot_potential(Nx, Ny, K, R, V0, w, dV)
    ref = _brute_qdot(Nx, Ny, K, R, V0, w, dV)
    assert V.shape == (4 * Nx * Ny,)
    assert np.max(np.abs(V - ref)) < 1e-15 * max(1.0, np.max(np.abs(ref)))
    assert np.count_nonzero(ref) > 0


def test_qdot_potential_plateau_and_tail():
    # inside a dot far from its edge the step is ~1 (V ~ V0); beyond the cut-off it is 0
    Nx, Ny, K, R, V0, w = 96, 64, 1, 20.0, 0.25, 1.0
    V = W.qdot_potential(Nx, Ny, K, R, V0, w)
    X, Y = W.graphene_positions(Nx, Ny)
    Xe, Ye = W.graphene_extent(Nx, Ny)
    d = np.hypot(X - Xe / 2, Y - Ye / 2)
    assert np.allclose(V[d < R - 15 * w], V0, rtol=0, atol=V0 * 2e-13)
    assert np.all(V[d >= R + 20 * w] == 0.0)
    edge = np.abs(d - R) < 0.05
    assert np.allclose(V[edge], V0 / 2, atol=V0 * 0.05 / (2 * w))


def test_graphene_positions_bond_lengths_and_extent():
    X, Y = W.graphene_positions(5, 3)
    Xe, Ye = W.graphene_extent(5, 3)
    assert X.min() >= 0 and X.max() < Xe and Y.min() >= 0 and Y.max() < Ye
    # every site has its nearest neighbours at distance 1 (C-C distance)
    P = np.stack([X, Y], 1)
    dist = np.hypot(*(P[:, None, :] - P[None, :, :]).transpose(2, 0, 1))
    np.fill_diagonal(dist, np.inf)
    assert abs(dist.min() - 1.0) < 1e-12
    assert math.isclose(Ye / 5, math.sqrt(3.0)) and Xe / 3 == 3.0
