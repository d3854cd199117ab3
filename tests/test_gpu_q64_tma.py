"""The fixed-point (PVSC_Q64) KPM sweep: its integer arithmetic and its
TMA-staged form (tuning kernel 7 of that precision).

The sweeps form every update as floor((c1 x1 + c2 x2 + 2^59) / 2^60) and the
dot sums sum x^2, sum y x exactly, from 32-bit limb products.  Python integers
are exact, so the device routines (run through pvsc_debug_fx_arith) must equal
them bit for bit, over random operands and over the extremes of the ranges a
sweep meets.  The TMA-staged sweep writes the same integers as the z-marching
one (its moments then differ only in the order the exact per-thread sums are
converted and added in fp64) and must match the oracle's fp64 recurrence.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

pv = pytest.importorskip("paper_1708_09689_gb300")

C_MAX, X_MAX, T_MAX = 2 ** 61, 2 ** 59, 6 * 2 ** 59


def _edge_values(top):
    """Values at the ends of [-top, top] and around the 31-bit limb boundaries."""
    low = [0, 1, 2 ** 31 - 1, 2 ** 31, 2 ** 31 + 1, 2 ** 32 - 1, 2 ** 32]
    vals = {top, -top, top - 1, -top + 1, 0}
    for v in low:
        vals |= {v, -v, top - v, -top + v}
    return sorted(v for v in vals if -top <= v <= top)


def _mul2_exact(rec):
    c1, x1, c2, x2 = (int(v) for v in rec)
    return (c1 * x1 + c2 * x2 + 2 ** 59) >> 60  # Python's >> floors


def test_fixed_point_update_is_the_exactly_rounded_product_sum():
    rng = np.random.default_rng(11)
    n = 20000
    recs = np.stack([rng.integers(-C_MAX, C_MAX, n, endpoint=True), rng.integers(-X_MAX, X_MAX, n, endpoint=True),
                     rng.integers(-C_MAX, C_MAX, n, endpoint=True), rng.integers(-T_MAX, T_MAX, n, endpoint=True)],
                    axis=1).astype(np.int64)
    # every combination of edge values of the four operands (a sample of them)
    ec, ex, et = _edge_values(C_MAX), _edge_values(X_MAX), _edge_values(T_MAX)
    edge = np.array([(a, b, c, d) for a in ec[::2] for b in ex[::2] for c in ec[1::2] for d in et[::3]],
                    dtype=np.int64)
    # small magnitudes: the typical coefficient and entry sizes
    small = np.stack([rng.integers(-2 ** 40, 2 ** 40, 2000), rng.integers(-2 ** 50, 2 ** 50, 2000),
                      rng.integers(-2 ** 58, 2 ** 58, 2000), rng.integers(-2 ** 45, 2 ** 45, 2000)],
                     axis=1).astype(np.int64)
    allr = np.concatenate([recs, edge, small])
    got = pv.debug_fx_arith(0, torch.from_numpy(allr).cuda()).cpu().numpy()
    want = np.array([_mul2_exact(r) for r in allr], dtype=np.int64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, f"{bad.size} mismatches, first {allr[bad[0]].tolist()}: {got[bad[0]]} != {want[bad[0]]}"


def _dots_exact(recs):
    x = [int(v) for v in recs[:, :8].ravel()]
    y = [int(v) for v in recs[:, 8:].ravel()]
    xx = sum(v * v for v in x)
    xy = sum(a * b for a, b in zip(y, x))

    def pair(v):
        v %= 2 ** 128
        hi, lo = v >> 64, v & (2 ** 64 - 1)
        return [hi - 2 ** 64 if hi >= 2 ** 63 else hi, lo - 2 ** 64 if lo >= 2 ** 63 else lo]
    return pair(xx) + pair(xy)


def _unit_norm_records(rng, n, top_bits_low=False):
    """n records of two vectors with 2-norm <= 1 in Q4.59 (eight values each)."""
    x = rng.standard_normal((n, 8))
    y = rng.standard_normal((n, 8))
    x *= 0.999 / np.linalg.norm(x)
    y *= 0.999 / np.linalg.norm(y)
    xi = np.round(x * 2.0 ** 59).astype(np.int64)
    yi = np.round(y * 2.0 ** 59).astype(np.int64)
    if top_bits_low:  # low limbs at their extremes
        xi = (xi & ~np.int64(2 ** 31 - 1)) | np.int64(2 ** 31 - 1)
        yi = yi & ~np.int64(2 ** 31 - 1)
    return np.concatenate([xi, yi], axis=1)


@pytest.mark.parametrize("case", ["random", "one_record", "limb_edges", "one_value", "opposite", "empty"])
def test_fixed_point_dot_sums_are_exact(case):
    rng = np.random.default_rng(5)
    if case == "random":
        recs = _unit_norm_records(rng, 300)
    elif case == "one_record":
        recs = _unit_norm_records(rng, 1)
    elif case == "limb_edges":
        recs = _unit_norm_records(rng, 64, top_bits_low=True)
    elif case == "one_value":  # all of the norm in one entry, the largest value
        recs = np.zeros((3, 16), dtype=np.int64)
        recs[1, 5], recs[1, 13] = X_MAX, -X_MAX
    elif case == "opposite":  # y = -x: the cross sum is minus the square sum
        recs = _unit_norm_records(rng, 50)
        recs[:, 8:] = -recs[:, :8]
    else:
        recs = np.zeros((0, 16), dtype=np.int64)
    got = pv.debug_fx_arith(1, torch.from_numpy(recs).cuda()).cpu().numpy().tolist()
    assert got == _dots_exact(recs)


def test_fixed_point_arith_rejects_bad_arguments():
    with pytest.raises(pv.PvscError):
        pv.debug_fx_arith(2, torch.zeros((1, 4), dtype=torch.int64, device="cuda"))
    with pytest.raises(pv.PvscError):
        pv.debug_fx_arith(0, torch.zeros((1, 3), dtype=torch.int64, device="cuda"))


CASES = [
    # dims, periodic, z-chunk depth
    ((32, 16, 6), (1, 1, 0), 0),
    ((20, 12, 5), (1, 1, 1), 2),      # partial tiles along x and y
    ((16, 8, 7), (0, 0, 0), 1),       # open everywhere, one-plane chunks
    ((5, 2, 3), (1, 1, 1), 0),        # x shorter than a tile (and odd), y of length 2
    ((8, 1, 4), (1, 1, 0), 3),        # y of length 1: its own neighbour
    ((13, 9, 1), (0, 1, 1), 0),       # one plane, periodic z of length 1
]

# the half tiles of the layout of 2R complex64 vectors (R = 16, 32: slices of 8 vectors in the layout of 16)
DEEP_TILE = {1: (32, 8), 2: (16, 8), 4: (16, 4), 8: (8, 4), 16: (8, 4), 32: (8, 4)}


def _variant(R, v):
    if v == "deep":
        return dict(zip(("tile_x", "tile_y"), DEEP_TILE[R]))
    return dict(threads=512) if v == "wide" else {}


@pytest.mark.parametrize("dims,per,zs", CASES)
@pytest.mark.parametrize("R,variant", [(R, v) for R in (1, 2, 4, 8, 16, 32) for v in ("large", "wide", "deep")])
def test_q64_tma_sweep_matches_zmarch_and_oracle(dims, per, zs, R, variant):
    n = int(np.prod(dims))
    V = W.disorder_potential(n, 2.0, 7)
    lat = pv.Lattice.ti(dims, per, disorder=(2.0, 7))
    H = O.ti_hamiltonian(dims, per, 1.0, 2.0, V)
    _, _, a, b = lat.spectral_bounds()
    M = 41
    r = W.random_phase_block(H.shape[0], R, 17)
    rt = torch.from_numpy(r).cuda()
    lat.set_tuning(R, pv.Q64, threads=128, vpt=1, kernel=0)
    mu0 = pv.kpm_moments(lat, M, a, b, r0=rt, prec=pv.Q64).cpu().numpy()
    lat.set_tuning(R, pv.Q64, kernel=7, zslab=zs, **_variant(R, variant))
    assert lat.get_tuning(R, pv.Q64)["kernel"] == 7
    mu7 = pv.kpm_moments(lat, M, a, b, r0=rt, prec=pv.Q64).cpu().numpy()
    assert pv.device_error() == 0
    # the same integer vectors: the moments differ only by fp64 summation order
    assert np.max(np.abs(mu7 - mu0)) < 1e-14
    ref = O.kpm_moments(H, r, M, a, b).real
    assert np.max(np.abs(mu7 - ref)) < 1e-12


def test_q64_tma_sweep_with_on_the_fly_disorder_and_generated_block():
    dims, per = (24, 16, 9), (1, 0, 1)
    lat_s = pv.Lattice.ti(dims, per, disorder=(3.0, 8))
    lat_f = pv.Lattice.ti(dims, per, disorder=(3.0, 8), on_the_fly=True)
    _, _, a, b = lat_s.spectral_bounds()
    out = []
    for lat in (lat_s, lat_f):
        lat.set_tuning(8, pv.Q64, kernel=7)
        out.append(pv.kpm_moments(lat, 30, a, b, R=8, prec=pv.Q64, seed=4).cpu().numpy())
    assert np.array_equal(out[0], out[1])
    mu_d = pv.kpm_moments(lat_s, 30, a, b, R=8, prec=pv.C128, seed=4).cpu().numpy()
    assert np.max(np.abs(out[0] - mu_d)) < 1e-12


def test_q64_kernel7_tuning_is_validated():
    lat = pv.Lattice.ti((16, 8, 4), (1, 1, 0))
    for R in (64,):  # no fixed-point TMA layout for this block size
        with pytest.raises(pv.PvscError, match="kernel 7"):
            lat.set_tuning(R, pv.Q64, kernel=7)
    with pytest.raises(pv.PvscError, match="tile"):
        lat.set_tuning(8, pv.Q64, kernel=7, tile_x=4, tile_y=4)
    lat.set_tuning(8, pv.Q64, kernel=7, tile_x=8, tile_y=4)
    assert lat.get_tuning(8, pv.Q64)["tile_y"] == 4


@pytest.mark.parametrize("dims,R", [((16, 8, 3), 8), ((8, 4, 1), 2), ((16, 8, 2), 32)])
def test_q64_tma_sweep_spread_over_all_sms_equals_default(dims, R):
    # blocks_per_sm = 1: the planes split over every SM, most blocks without a
    # plane; the integer vectors are unchanged, and the moments differ only in
    # the order the blocks' fp64 conversions of the exact dot sums are added
    lat = pv.Lattice.ti(dims, (1, 1, 0), disorder=(2.0, 3))
    _, _, a, b = lat.spectral_bounds()
    out = []
    for spread in (0, 1):
        lat.set_tuning(R, pv.Q64, kernel=7, blocks_per_sm=spread)
        out.append(pv.kpm_moments(lat, 20, a, b, R=R, prec=pv.Q64, seed=3).cpu().numpy())
        assert pv.device_error() == 0
    assert np.max(np.abs(out[0] - out[1])) < 1e-14
