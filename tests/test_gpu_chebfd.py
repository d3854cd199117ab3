"""Chebyshev filter diagonalization on the GPU against dense diagonalisation
and the oracle's ChebFD (Sec. 5.3)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pv = pytest.importorskip("paper_1708_09689_gb300")
pytestmark = pytest.mark.gpu


def _case(dims, per, Wd, seed, n_target):
    n = int(np.prod(dims))
    lat = pv.Lattice.ti(dims, per, disorder=(Wd, seed))
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, W.disorder_potential(n, Wd, seed))
    ev = np.sort(np.linalg.eigvalsh(H.toarray()))
    idx = np.sort(np.argsort(np.abs(ev))[:n_target])
    lo, hi = (ev[idx[0] - 1] + ev[idx[0]]) / 2, (ev[idx[-1]] + ev[idx[-1] + 1]) / 2
    return lat, H, ev, lo, hi


@pytest.mark.parametrize("dims,per,n_search,n_target", [((6, 6, 4), (1, 1, 0), 32, 16),
                                                        ((8, 6, 4), (1, 1, 0), 64, 32),
                                                        ((5, 5, 5), (1, 1, 1), 32, 16)])
def test_chebfd_c128_finds_the_dense_eigenpairs(dims, per, n_search, n_target):
    lat, H, ev, lo, hi = _case(dims, per, 1.0, 3, n_target)
    _, _, a, b = lat.spectral_bounds()
    theta, res, X, n_in, iters = pv.chebfd(lat, lo, hi, a, b, n_search=n_search, degree=400,
                                           max_iter=40, tol=1e-10)
    inside = (theta >= lo) & (theta <= hi)
    target = ev[(ev >= lo) & (ev <= hi)]
    assert n_in == inside.sum() == len(target) == n_target
    assert iters < 40
    assert np.max(np.abs(theta[inside] - target)) < 1e-11
    assert np.all(res[inside] < 1e-10)
    Xh = X.cpu().numpy()
    assert np.max(np.abs(Xh.conj().T @ Xh - np.eye(n_search))) < 1e-11
    Xi = Xh[:, inside]
    assert np.max(np.linalg.norm(H @ Xi - Xi * theta[inside], axis=0)) < 1e-10  # residual on the CPU


def test_chebfd_agrees_with_the_oracle_chebfd():
    lat, H, ev, lo, hi = _case((6, 6, 4), (1, 1, 0), 1.0, 3, 16)
    _, _, a, b = lat.spectral_bounds()
    theta, res, X, n_in, iters = pv.chebfd(lat, lo, hi, a, b, n_search=32, degree=400, tol=1e-10)
    th_o, _, _, _ = O.chebfd(H, W.gaussian_block(H.shape[0], 32, 1), lo, hi, a, b, 400, 40, 1e-10)
    inside = (theta >= lo) & (theta <= hi)
    assert np.max(np.abs(np.sort(th_o) - theta[inside])) < 1e-11


def test_chebfd_with_complex64_filter():
    # the filter's recurrence vectors in complex64: Rayleigh-Ritz stays complex128,
    # residuals then settle near the fp32 rounding of the filtered block
    lat, H, ev, lo, hi = _case((6, 6, 4), (1, 1, 0), 1.0, 3, 16)
    _, _, a, b = lat.spectral_bounds()
    theta, res, X, n_in, iters = pv.chebfd(lat, lo, hi, a, b, n_search=32, degree=400, tol=1e-5,
                                           prec=pv.C64, max_iter=40)
    inside = (theta >= lo) & (theta <= hi)
    target = ev[(ev >= lo) & (ev <= hi)]
    assert n_in == len(target)
    assert np.all(res[inside] < 1e-5)
    assert np.max(np.abs(theta[inside] - target)) < 1e-9  # Ritz values are second order in the residual


def test_chebfd_argument_errors():
    lat = pv.Lattice.ti((4, 4, 4), (1, 1, 1))
    _, _, a, b = lat.spectral_bounds()
    with pytest.raises(pv.PvscError):
        pv.chebfd(lat, 0.5, -0.5, a, b)  # lo > hi
    with pytest.raises(pv.PvscError):
        pv.chebfd(lat, -0.5, 0.5, a, b, n_search=48)  # not a valid block width
