"""CPU fp64 oracle for the matrix-free Chebyshev stencil path (test infrastructure).

This package is test infrastructure.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it; the library never does, and it
never imports the library.  It is deliberately plain and slow: the Hamiltonian
is assembled as an explicit sparse matrix (COO triplets, duplicates summed,
converted to CSR) straight from the paper's equations, and every recurrence is
run in the order and notation of the paper, in complex128 throughout.

Vectors use the library's I/O layout: a block of R vectors is an array of
shape (D, R), D = n_sites * O (O = 4 orbitals for the topological insulator,
O = 1 for graphene sites), row index i = site * O + orbital.  Flattened in C
order this is element (site, orbital, r) at ((site * O + orbital) * R + r).

Contents and the passages they follow:
  gamma_matrices            Dirac matrices of Sec. 2.2 (Eq. TB_H_topi)
  ti_hamiltonian            Eq. TB_H_topi (cubic 4-band topological insulator)
  graphene_hamiltonian      Eq. graphene_model (4-site rectangular cell)
  wsm_hamiltonian           Eq. TB_H_wsm (two-band Weyl semimetal)
  gershgorin, cheb_scale    Sec. 4.1 (a = (Emax-Emin+eps)/2, b = (Emax+Emin)/2)
  cheb_step                 fused spMVM semantics of Listing graphenec (Sec. 3.2)
  kpm_moments               mu_k = <r|T_k(H~)|r> (Sec. 2.2, Sec. 4), direct recurrence
  bessel_j                  J_k by Miller's backward recurrence (Sec. 4.1 c_k)
  propagation_coeffs        c_k = (-i)^k J_k(a dt), truncation (Eq. U_1)
  cheb_series / propagate   Eq. U_1 with |w_k> from the Chebyshev recurrence
  propagate_adjoint         reverse-mode derivative of the propagated state
                            w.r.t. the on-site potential (not in the paper;
                            plain reverse sweep of the same recurrence)
  jackson_kernel, lorentz_kernel, kpm_density
                            DOS (Eq. DOS) and spectral function (Eq. ak) from
                            KPM moments, with the damping kernels of the KPM
                            method the paper cites
  bloch_vectors             the Bloch states psi(k, nu) of Eq. ak
  chebfd_window, chebfd     Chebyshev filter diagonalization (Sec. 5.3)
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

# ----------------------------------------------------------------------------
# Dirac matrices (Sec. 2.2, below Eq. TB_H_topi)
# ----------------------------------------------------------------------------
_S0 = np.eye(2, dtype=np.complex128)
_SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def gamma_matrices() -> list[np.ndarray]:
    """[Gamma^0, Gamma^1, ..., Gamma^5] as 4x4 complex matrices.

    Gamma^(1..5) = (1 (x) s_z, -sigma_y (x) s_x, sigma_x (x) s_x, -1 (x) s_y,
    sigma_z (x) s_x), sigma acting on spin (first Kronecker factor) and s on
    the orbital; Gamma^0 is the identity.
    """
    return [
        np.eye(4, dtype=np.complex128),
        np.kron(_S0, _SZ),
        -np.kron(_SY, _SX),
        np.kron(_SX, _SX),
        -np.kron(_S0, _SY),
        np.kron(_SZ, _SX),
    ]


def gamma_commutator(G: list[np.ndarray], a: int, b: int) -> np.ndarray:
    """Gamma^{ab} = [Gamma^a, Gamma^b] / (2i)."""
    return (G[a] @ G[b] - G[b] @ G[a]) / 2j


# ----------------------------------------------------------------------------
# Hamiltonian assembly
# ----------------------------------------------------------------------------
def _neighbour(coords: np.ndarray, axis: int, step: int, dims, periodic):
    """Coordinates moved by `step` along `axis`; returns (coords, valid mask)."""
    c = coords.copy()
    c[:, axis] += step
    if periodic[axis]:
        c[:, axis] %= dims[axis]
        valid = np.ones(len(c), dtype=bool)
    else:
        valid = (c[:, axis] >= 0) & (c[:, axis] < dims[axis])
    return c, valid


def _site_index(coords: np.ndarray, dims) -> np.ndarray:
    """n = x + Lx (y + Ly z) (x fastest)."""
    idx = coords[:, -1].copy()
    for ax in range(len(dims) - 2, -1, -1):
        idx = idx * dims[ax] + coords[:, ax]
    return idx


def _all_coords(dims) -> np.ndarray:
    """Coordinates of every site, site = x + Lx (y + Ly z), shape (n_sites, ndim)."""
    n = int(np.prod(dims))
    site = np.arange(n, dtype=np.int64)
    cols, stride = [], 1
    for L in dims:
        cols.append((site // stride) % L)
        stride *= L
    return np.stack(cols, axis=1)


def _assemble(dims, periodic, O, onsite_blocks, hop_blocks, rows=None, terms=False):
    """Generic block assembly of sum_n Psi_n^+ E_n Psi_n + sum_{n,j}(Psi_{n+e_j}^+ B_j Psi_n + h.c.).

    onsite_blocks: array (n_sites, O, O) of E_n.
    hop_blocks: list of (axis, B) with B an (O, O) matrix for the bond n -> n + e_axis.
    rows: optional array of site indices whose rows are wanted (others left empty).
    Duplicate (row, col) entries, which arise for lengths 1 and 2 with periodic
    boundaries, are summed when converting to CSR.  With terms=True the COO
    triplets are returned instead, before any summation: one (row, col, value)
    per nonzero entry of every on-site and bond block.
    """
    n_sites = int(np.prod(dims))
    D = n_sites * O
    coords = _all_coords(dims)
    sites = np.arange(n_sites, dtype=np.int64)
    want = np.ones(n_sites, dtype=bool) if rows is None else np.zeros(n_sites, dtype=bool)
    if rows is not None:
        want[np.asarray(rows, dtype=np.int64)] = True
    oo_r, oo_c = np.meshgrid(np.arange(O), np.arange(O), indexing="ij")
    oo_r, oo_c = oo_r.reshape(-1), oo_c.reshape(-1)
    R_list, C_list, V_list = [], [], []

    def emit(row_sites, col_sites, blocks):
        # blocks: (len(row_sites), O, O) per bond, or one (O, O) block for all
        keep = want[row_sites]
        if not np.any(keep):
            return
        b = blocks[keep] if blocks.ndim == 3 else np.broadcast_to(blocks, (int(keep.sum()), O, O))
        row_sites, col_sites = row_sites[keep], col_sites[keep]
        R_list.append((row_sites[:, None] * O + oo_r[None, :]).reshape(-1))
        C_list.append((col_sites[:, None] * O + oo_c[None, :]).reshape(-1))
        V_list.append(b.reshape(-1))

    emit(sites, sites, onsite_blocks)
    for axis, B in hop_blocks:
        nb, valid = _neighbour(coords, axis, +1, dims, periodic)
        n_from = sites[valid]
        n_to = _site_index(nb[valid], dims)
        emit(n_to, n_from, B)                       # Psi_{n+e}^+ B Psi_n
        emit(n_from, n_to, B.conj().T)              # its Hermitian conjugate
    if R_list:
        r = np.concatenate(R_list)
        c = np.concatenate(C_list)
        v = np.concatenate(V_list)
    else:
        r = c = np.zeros(0, dtype=np.int64)
        v = np.zeros(0, dtype=np.complex128)
    if terms:
        nz = v != 0
        return r[nz], c[nz], v[nz]
    H = sp.coo_matrix((v, (r, c)), shape=(D, D)).tocsr()
    H.sum_duplicates()
    H.eliminate_zeros()      # drop the structural zeros of the dense 4x4 blocks
    return H


def ti_hamiltonian(dims, periodic, t, m, V, delta1=0.0, delta2=0.0, rows=None, terms=False):
    """Eq. TB_H_topi on an Lx x Ly x Lz cuboid, as a (4N x 4N) CSR matrix.

    On-site block: m Gamma^1 + Delta1 Gamma^5 + Delta2 Gamma^15 + V_n Gamma^0.
    Bond n -> n + e_j (j = x, y, z): Psi_{n+e_j}^+ [-(t/2)(Gamma^1 - i Gamma^{j+1})] Psi_n
    plus its Hermitian conjugate.  The paper sets the transfer element t = 1;
    t is kept as an explicit prefactor of the hopping term.  Open axes drop the
    bonds that leave the cuboid; periodic axes wrap.
    """
    G = gamma_matrices()
    dims = tuple(int(d) for d in dims)
    n_sites = int(np.prod(dims))
    V = np.asarray(V, dtype=np.float64).reshape(n_sites)
    E0 = m * G[1] + delta1 * G[5] + delta2 * gamma_commutator(G, 1, 5)
    onsite = E0[None, :, :] + V[:, None, None] * G[0][None, :, :]
    hops = [(j, -(t / 2.0) * (G[1] - 1j * G[j + 2])) for j in range(3)]
    return _assemble(dims, periodic, 4, onsite, hops, rows, terms)


# Pauli matrices of the two-band Weyl semimetal (Eq. TB_H_wsm)
_PAULI = (np.array([[0, 1], [1, 0]], dtype=np.complex128),
          np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
          np.array([[1, 0], [0, -1]], dtype=np.complex128))


def wsm_hamiltonian(dims, periodic, V, k0=math.pi / 2, rows=None, terms=False):
    """Eq. TB_H_wsm on an Lx x Ly x Lz cuboid, as a (2N x 2N) CSR matrix.

    Two orbitals per site (row index = 2 site + orbital).  Bond n -> n + e_x:
    Psi_{n+x}^+ (sigma_x / 2) Psi_n; bond n -> n + e_j, j = y, z:
    Psi_{n+j}^+ ((sigma_x + i sigma_j) / 2) Psi_n; each plus its Hermitian
    conjugate.  On-site block V_n - sigma_x (2 + cos k0).  Transfer element 1.
    """
    sx, sy, sz = _PAULI
    dims = tuple(int(d) for d in dims)
    n_sites = int(np.prod(dims))
    V = np.asarray(V, dtype=np.float64).reshape(n_sites)
    onsite = V[:, None, None] * np.eye(2)[None, :, :] - (2.0 + math.cos(k0)) * sx[None, :, :]
    hops = [(0, sx / 2.0), (1, (sx + 1j * sy) / 2.0), (2, (sx + 1j * sz) / 2.0)]
    return _assemble(dims, periodic, 2, onsite, hops, rows, terms)


# The 4x4 matrices of Eq. graphene_model (entries in units of t)
GRAPHENE_TX = np.array([[0, 0, 0, 0], [-1, 0, 0, 0], [0, 0, 0, -1], [0, 0, 0, 0]], dtype=np.complex128)
GRAPHENE_TY = np.array([[0, 0, 0, -1], [0, 0, 0, 0], [0, 0, 0, 0], [0, 0, 0, 0]], dtype=np.complex128)
GRAPHENE_TN = np.array([[0, -1, 0, 0], [-1, 0, -1, 0], [0, -1, 0, -1], [0, 0, -1, 0]], dtype=np.complex128)


def graphene_hamiltonian(cells, periodic, t, V, rows=None, Tx=None, Ty=None, Tn=None, terms=False):
    """Eq. graphene_model on an Nx x Ny array of 4-site cells, as a (4NxNy)^2 CSR matrix.

    H = sum_n (Psi_{n+x}^+ T_x Psi_n + Psi_{n+y}^+ T_y Psi_n + h.c.)
        + sum_n Psi_n^+ (T_n + V_n) Psi_n,
    with V_n = diag(v_{n,0..3}) given per site (V has 4 Nx Ny entries).
    Site index = 4 c + nu with cell c = x + Nx y.  `rows` selects cells.
    Tx, Ty, Tn may be overridden (used to build a mirrored variant in tests).
    """
    Tx = GRAPHENE_TX if Tx is None else Tx
    Ty = GRAPHENE_TY if Ty is None else Ty
    Tn = GRAPHENE_TN if Tn is None else Tn
    dims = tuple(int(d) for d in cells)
    n_cells = dims[0] * dims[1]
    V = np.asarray(V, dtype=np.float64).reshape(n_cells, 4)
    onsite = t * Tn[None, :, :] + np.einsum("ca,ab->cab", V, np.eye(4))
    hops = [(0, t * Tx), (1, t * Ty)]
    return _assemble(dims, periodic, 4, onsite, hops, rows, terms)


# ----------------------------------------------------------------------------
# Spectral scaling (Sec. 4.1)
# ----------------------------------------------------------------------------
def gershgorin(H: sp.csr_matrix) -> tuple[float, float]:
    """Exact Gershgorin interval over all rows of H:
    Emin = min_i (Re H_ii - sum_{j != i} |H_ij|), Emax = max_i (Re H_ii + sum_{j != i} |H_ij|)."""
    H = H.tocsr()
    diag = H.diagonal().real
    absrow = np.asarray(abs(H).sum(axis=1)).reshape(-1)
    radius = absrow - np.abs(H.diagonal())
    return float(np.min(diag - radius)), float(np.max(diag + radius))


def cheb_scale(emin: float, emax: float, eps: float = 0.01) -> tuple[float, float]:
    """a = (Emax - Emin + eps)/2, b = (Emax + Emin)/2 so that H~ = (H - b)/a has spectrum in [-1, 1]."""
    return (emax - emin + eps) / 2.0, (emax + emin) / 2.0


# ----------------------------------------------------------------------------
# Fused Chebyshev step (semantics of Listing graphenec)
# ----------------------------------------------------------------------------
def apply_H(H, x):
    """y = H x for a block x of shape (D, R)."""
    return H @ x


def cheb_step(H, x, y, alpha, beta, gamma, z=None, delta=None):
    """Per vector r: y_new = alpha_r (H - beta_r) x + gamma_r y (the scale_h,
    shift_h, scale_z form of Listing graphenec), optionally z += delta_r y_new.

    Returns (y_new, z_new, dots) with dots[r] = (<x|x>, <y_new|x>, <y_new|y_new>)
    as complex numbers (<a|b> = sum conj(a) b), the partial dot products the
    listing fuses into the sweep.
    """
    alpha, beta, gamma = (np.asarray(v, dtype=np.float64) for v in (alpha, beta, gamma))
    y_new = alpha[None, :] * (H @ x - beta[None, :] * x) + gamma[None, :] * y
    z_new = None
    if z is not None:
        z_new = z + np.asarray(delta)[None, :] * y_new
    xx = np.sum(np.conj(x) * x, axis=0)
    xy = np.sum(np.conj(y_new) * x, axis=0)
    yy = np.sum(np.conj(y_new) * y_new, axis=0)
    return y_new, z_new, np.stack([xx, xy, yy], axis=1)


# ----------------------------------------------------------------------------
# Kernel polynomial method (Sec. 2.2, Sec. 4)
# ----------------------------------------------------------------------------
def kpm_moments(H, r, M, a, b):
    """Chebyshev moments mu_k = <r|T_k(H~)|r>, k = 0..M-1, for each column of r.

    Direct recurrence |w_0> = |r>, |w_1> = H~|w_0>, |w_{k+1}> = 2 H~|w_k> - |w_{k-1}>,
    with H~ = (H - b)/a, and mu_k = <r|w_k> taken for every k (no doubling
    identities).  Returns complex moments of shape (R, M); for Hermitian H they
    are real up to rounding.
    """
    r = np.asarray(r, dtype=np.complex128)
    if r.ndim == 1:
        r = r[:, None]
    Ht = lambda v: (H @ v - b * v) / a
    mu = np.zeros((r.shape[1], M), dtype=np.complex128)
    w_prev = r
    mu[:, 0] = np.sum(np.conj(r) * w_prev, axis=0)
    if M == 1:
        return mu
    w = Ht(r)
    mu[:, 1] = np.sum(np.conj(r) * w, axis=0)
    for k in range(2, M):
        w_next = 2.0 * Ht(w) - w_prev
        mu[:, k] = np.sum(np.conj(r) * w_next, axis=0)
        w_prev, w = w, w_next
    return mu


# ----------------------------------------------------------------------------
# Chebyshev time propagation (Sec. 4.1, Eq. U_1)
# ----------------------------------------------------------------------------
def bessel_j(x: float, kmax: int) -> np.ndarray:
    """J_0(x) .. J_kmax(x) by Miller's backward recurrence (Abramowitz & Stegun 9.12).

    J_{k-1} = (2k/x) J_k - J_{k+1} is run downward from an order well above
    both kmax and x with arbitrary start values, then normalised with the sum
    rule J_0 + 2 sum_{k>=1} J_{2k} = 1.
    """
    if x == 0.0:
        out = np.zeros(kmax + 1)
        out[0] = 1.0
        return out
    start = int(max(kmax, x) + 40 + 2 * math.sqrt(max(kmax, x) * 40))
    start += start % 2
    j = np.zeros(start + 2)
    j[start + 1] = 0.0
    j[start] = 1e-300
    for k in range(start, 0, -1):
        j[k - 1] = (2.0 * k / x) * j[k] - j[k + 1]
        if abs(j[k - 1]) > 1e250:       # rescale to avoid overflow
            j[k - 1:] *= 1e-250
    norm = j[0] + 2.0 * np.sum(j[2:start + 1:2])
    return j[: kmax + 1] / norm


def propagation_coeffs(a: float, dt: float, trunc: float = 1e-14) -> np.ndarray:
    """c_k(a dt) = (-i)^k J_k(a dt), k = 0..M, where M is the largest k with
    |J_k(a dt)| >= trunc (Sec. 4.1: truncate once the Bessel coefficients fall
    below the accuracy cutoff)."""
    x = a * dt
    kmax = int(2 * x + 60)
    J = bessel_j(x, kmax)
    ks = np.nonzero(np.abs(J) >= trunc)[0]
    M = int(ks.max())
    k = np.arange(M + 1)
    return ((-1j) ** k) * J[: M + 1]


def cheb_series(H, x, coeffs, a, b):
    """sum_k coeffs_k T_k(H~) x with H~ = (H - b)/a, w_k from the three-term recurrence.
    (coeffs are applied as given: no implicit factor 2.)"""
    Ht = lambda v: (H @ v - b * v) / a
    coeffs = np.asarray(coeffs)
    w_prev = np.asarray(x, dtype=np.complex128)
    acc = coeffs[0] * w_prev
    if len(coeffs) == 1:
        return acc
    w = Ht(w_prev)
    acc = acc + coeffs[1] * w
    for k in range(2, len(coeffs)):
        w_next = 2.0 * Ht(w) - w_prev
        acc = acc + coeffs[k] * w_next
        w_prev, w = w, w_next
    return acc


def series_weights(c: np.ndarray) -> np.ndarray:
    """Weights of Eq. U_1 in the form sum_k cw_k T_k: cw_0 = c_0, cw_k = 2 c_k (k >= 1)."""
    cw = 2.0 * np.asarray(c, dtype=np.complex128)
    cw[0] = c[0]
    return cw


def propagate(H, psi, dt, nsteps, a, b, trunc=1e-14, return_all=False):
    """psi(t + dt) = e^{-i b dt} [c_0 w_0 + 2 sum_{k=1}^{M} c_k w_k], repeated nsteps times (Eq. U_1)."""
    cw = series_weights(propagation_coeffs(a, dt, trunc))
    phase = np.exp(-1j * b * dt)
    psi = np.asarray(psi, dtype=np.complex128)
    states = [psi]
    for _ in range(nsteps):
        psi = phase * cheb_series(H, psi, cw, a, b)
        if return_all:
            states.append(psi)
    return states if return_all else psi


def site_projector_sum(u, w, O):
    """Per-site sum over orbitals of conj(u) w, for (D, R) blocks: shape (n_sites,)."""
    p = np.sum(np.conj(u) * w, axis=1)
    return p.reshape(-1, O).sum(axis=1)


def propagate_adjoint(H, psi0, dt, nsteps, a, b, G_final, O, trunc=1e-14):
    """Derivative of L w.r.t. the on-site potential V_n, for the propagated state.

    Given G_final with dL = Re <G_final | d psi_S> (the conjugate-Wirtinger
    gradient convention used by torch for a real loss), returns (dL/dV, G_0)
    where dL/dV has one entry per site (V_n enters H as V_n times the identity
    on the site's O orbitals) and G_0 = dL/dpsi_0 in the same convention.

    Forward: psi_{s+1} = phi sum_k cw_k w_k^{(s)}, w_0 = psi_s, w_1 = H~ w_0,
    w_{k+1} = 2 H~ w_k - w_{k-1}, phi = e^{-i b dt}; H~ = (H - b)/a with a, b
    held fixed.  Reverse, per step (all w_k of the step kept): with
    h = conj(phi) G_{s+1},
        u_M = conj(cw_M) h,  u_{M-1} = conj(cw_{M-1}) h + 2 H~ u_M,
        u_k = conj(cw_k) h + 2 H~ u_{k+1} - u_{k+2}    (1 <= k <= M-2)
        u_0 = conj(cw_0) h + H~ u_1 - u_2              (w_1 = H~ w_0 has no factor 2)
    G_s = u_0, and since d w_{k+1} holds (f_k/a) dV P w_k with f_0 = 1, f_k = 2,
        dL/dV_n += (1/a) Re sum_{k=0}^{M-1} f_k sum_{orbitals of n} conj(u_{k+1}) w_k.
    """
    cw = series_weights(propagation_coeffs(a, dt, trunc))
    M = len(cw) - 1
    phase = np.exp(-1j * b * dt)
    Ht = lambda v: (H @ v - b * v) / a
    psi = np.asarray(psi0, dtype=np.complex128)
    if psi.ndim == 1:
        psi = psi[:, None]
    # forward, storing every w_k of every step
    all_w = []
    for _ in range(nsteps):
        ws = [psi]
        if M >= 1:
            ws.append(Ht(psi))
        for k in range(1, M):
            ws.append(2.0 * Ht(ws[k]) - ws[k - 1])
        all_w.append(ws)
        acc = sum(cw[k] * ws[k] for k in range(M + 1))
        psi = phase * acc
    G = np.asarray(G_final, dtype=np.complex128)
    if G.ndim == 1:
        G = G[:, None]
    n_sites = psi.shape[0] // O
    grad = np.zeros(n_sites)
    for s in range(nsteps - 1, -1, -1):
        ws = all_w[s]
        h = np.conj(phase) * G
        u = [None] * (M + 3)
        zero = np.zeros_like(h)
        u[M + 1] = zero
        u[M + 2] = zero
        for k in range(M, 0, -1):
            u[k] = np.conj(cw[k]) * h + 2.0 * Ht(u[k + 1]) - u[k + 2]
        u0 = np.conj(cw[0]) * h + Ht(u[1]) - u[2] if M >= 1 else np.conj(cw[0]) * h
        for k in range(0, M):
            f = 1.0 if k == 0 else 2.0
            grad += (f / a) * site_projector_sum(u[k + 1], ws[k], O).real
        G = u0
    return grad, G


def detector_probability(psi, mask_sites, O=1):
    """L = sum over detector sites (and their orbitals) of |psi|^2."""
    p = np.abs(np.asarray(psi).reshape(-1, O)) ** 2
    return float(np.sum(p.sum(axis=1)[np.asarray(mask_sites, dtype=bool)]))


# ----------------------------------------------------------------------------
# Spectral densities from KPM moments (Eq. ak, Eq. DOS, Sec. 2.2; the kernel
# polynomial method the paper cites: A. Weisse, G. Wellein, A. Alvermann,
# H. Fehske, Rev. Mod. Phys. 78, 275 (2006), Sec. II)
# ----------------------------------------------------------------------------
def jackson_kernel(M: int) -> np.ndarray:
    """Jackson damping factors g_k, k = 0..M-1, for M moments:
    g_k = [(M - k + 1) cos(q k) + sin(q k) cot(q)] / (M + 1),  q = pi / (M + 1)."""
    k = np.arange(M, dtype=np.float64)
    q = math.pi / (M + 1)
    return ((M - k + 1) * np.cos(q * k) + np.sin(q * k) / math.tan(q)) / (M + 1)


def lorentz_kernel(M: int, lam: float) -> np.ndarray:
    """Lorentz damping factors g_k = sinh(lam (1 - k/M)) / sinh(lam), k = 0..M-1."""
    k = np.arange(M, dtype=np.float64)
    return np.sinh(lam * (1.0 - k / M)) / math.sinh(lam)


def kpm_density(mu, E, a, b, g, scale=1.0) -> np.ndarray:
    """Density from per-vector moments mu (R, M) on energies E:

        rho(E) = scale * sum_r [g_0 mu_0^r + 2 sum_{k>=1} g_k mu_k^r T_k(x)] / (pi a sqrt(1 - x^2)),

    x = (E - b)/a, T_k(x) = cos(k arccos x), rho = 0 for |x| >= 1.  With the
    stochastic-trace moments of R random vectors and scale = D/R this is the
    DOS of Eq. DOS; with the moments of the four Bloch vectors psi(k, nu) and
    scale = 1 it is A(k, E) of Eq. ak."""
    mu = np.atleast_2d(np.asarray(mu, dtype=np.float64))
    g = np.asarray(g, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    x = (E - b) / a
    inside = np.abs(x) < 1.0
    xs = np.where(inside, x, 0.0)
    theta = np.arccos(xs)
    c = g * mu.sum(axis=0)
    c[1:] *= 2.0
    k = np.arange(len(c))
    series = np.cos(np.outer(theta, k)) @ c
    rho = scale * series / (math.pi * a * np.sqrt(1.0 - xs * xs))
    return np.where(inside, rho, 0.0)


def bloch_vectors(dims, k, O=4) -> np.ndarray:
    """The states psi(k, nu), nu = 0..O-1, of Eq. ak on a cubic lattice with O
    orbitals per site (TI 4, Weyl semimetal 2): the plane wave
    exp(i k.r_n)/sqrt(N) on orbital nu of every site n (r_n = the site's integer
    coordinates), as an (O N, O) block in the library's layout."""
    coords = _all_coords(dims).astype(np.float64)
    N = coords.shape[0]
    kv = np.asarray(k, dtype=np.float64)[: coords.shape[1]]
    phase = np.exp(1j * (coords @ kv)) / math.sqrt(N)
    out = np.zeros((O * N, O), dtype=np.complex128)
    for nu in range(O):
        out[nu::O, nu] = phase
    return out


# ----------------------------------------------------------------------------
# Chebyshev filter diagonalization (Sec. 5.3 "Interior eigenvalues"; the
# ChebFD scheme of A. Pieper et al., J. Comput. Phys. 325, 226 (2016))
# ----------------------------------------------------------------------------
def chebfd_window(lo: float, hi: float, a: float, b: float, degree: int) -> np.ndarray:
    """Chebyshev coefficients c_0..c_degree of the indicator of [lo, hi] on the
    scaled axis x = (E - b)/a, damped by the Jackson kernel: with x = cos(theta),
    c_0 = (theta_lo - theta_hi)/pi, c_k = 2 (sin(k theta_lo) - sin(k theta_hi))/(pi k)."""
    tl = math.acos(max(-1.0, min(1.0, (lo - b) / a)))
    th = math.acos(max(-1.0, min(1.0, (hi - b) / a)))
    k = np.arange(1, degree + 1, dtype=np.float64)
    c = np.empty(degree + 1)
    c[0] = (tl - th) / math.pi
    c[1:] = 2.0 * (np.sin(k * tl) - np.sin(k * th)) / (math.pi * k)
    return c * jackson_kernel(degree + 1)


def chebfd(H, X0, lo, hi, a, b, degree, max_iter, tol):
    """Filter diagonalization in the paper's order: filter the block with the
    window polynomial, orthonormalize (QR), Rayleigh-Ritz on the filtered
    space, stop when every Ritz pair inside [lo, hi] has ||H x - theta x|| < tol.
    Returns (theta, X, residuals) of the pairs inside [lo, hi] and the number
    of iterations."""
    c = chebfd_window(lo, hi, a, b, degree)
    X = np.asarray(X0, dtype=np.complex128)
    for it in range(1, max_iter + 1):
        Y = cheb_series(H, X, c, a, b)
        Q, _ = np.linalg.qr(Y)
        HQ = H @ Q
        theta, W = np.linalg.eigh(Q.conj().T @ HQ)
        X = Q @ W
        res = np.linalg.norm(H @ X - X * theta, axis=0)
        inside = (theta >= lo) & (theta <= hi)
        if np.all(res[inside] < tol):
            break
    return theta[inside], X[:, inside], res[inside], it
