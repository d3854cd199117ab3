/*
 * pvsc.h -- C ABI of the GB300 matrix-free Chebyshev stencil library.
 *
 * The library applies the tight-binding Hamiltonians of Pieper, Hager and
 * Fehske (arXiv 1708.09689) to blocks of R complex vectors without storing a
 * matrix, and fuses that stencil into the Chebyshev recurrences that call it
 * (kernel polynomial method, Chebyshev filtering, Chebyshev time propagation).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Models.  PVSC_TI: Eq. TB_H_topi (Sec. 2.2), a cubic lattice with 4 orbitals
 *   per site, on-site m Gamma^1 + V_n, hopping -(t/2)(Gamma^1 - i Gamma^{j+1})
 *   from n to n + e_j plus its Hermitian conjugate (Delta_1 = Delta_2 = 0).
 *   PVSC_GRAPHENE: Eq. graphene_model (Sec. 2.1), an Nx x Ny array of 4-site
 *   cells with the 4x4 transfer matrices T_x, T_y, T_n (entries -t) and a
 *   per-site potential v_{n,j}.
 * Sites.  TI: n = x + Lx (y + Ly z).  Graphene: site = 4 c + nu, c = x + Nx y.
 * Vectors.  A block of R vectors is stored site-major with the vector index
 *   fastest (the interleaved layout of Sec. 3.1, Listing jacobi2d-r): element
 *   (site, orbital nu, vector r) sits at complex offset ((site O + nu) R + r),
 *   O = 4 (TI) or 1 (graphene site).  Complex numbers are (re, im) pairs:
 *   16 bytes for PVSC_C128, 8 bytes for PVSC_C64.  D = O * n_sites.
 * Precision.  PVSC_C128 stores and computes in fp64.  PVSC_C64 stores the
 *   recurrence vectors as complex64 and computes the stencil in fp32, while
 *   dot products, moments, the scaling (a, b), the Bessel coefficients and the
 *   propagation accumulator stay fp64.  Vectors the caller passes as
 *   "complex128" are complex128 in both precisions.  PVSC_Q64 (pvsc_kpm_moments
 *   on TI lattices only) keeps complex128-sized vectors as pairs of 64-bit
 *   fixed-point integers: each start vector is scaled by an exact power of two
 *   to 2-norm <= 1, values carry 59 fraction bits, stencil sums are exact
 *   integer additions and each update is rounded once at 2^-60; the dot
 *   products are exact integer sums converted to fp64.  Products are formed
 *   exactly from 32 x 32 -> 64-bit limb products (pvsc_debug_fx_arith runs
 *   them on given operands).  Moments agree with the fp64 path to ~1e-15.
 * R.  1, 2, 4, 8, 16, 32 or 64 vectors per block.
 * Memory.  Every vector, work buffer and output pointer is a DEVICE pointer
 *   owned by the caller, 16-byte aligned; the library owns only the lattice
 *   handle (geometry, parameters and its copy of V).  Work buffers are sized
 *   with pvsc_work_bytes.
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *   that launch kernels are asynchronous on that stream unless stated.
 * Threads.  A lattice handle is used by one host thread at a time (its
 *   tuning table and graph cache are not locked against concurrent tuning);
 *   distinct handles may be used from different threads concurrently.
 * Errors.  Every call returns PVSC_OK or a negative pvsc_status and leaves a
 *   message for pvsc_last_error() (thread-local).  Invalid arguments are
 *   reported before anything is launched; device-side waits are bounded and
 *   report PVSC_ERR_TIMEOUT; nothing aborts the process or traps the device.
 */
#ifndef PVSC_H
#define PVSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pvsc_lattice pvsc_lattice; /* opaque, library-owned */

typedef enum {
  PVSC_OK = 0,
  PVSC_ERR_ARG = -1,         /* invalid argument (null, size, alignment, range) */
  PVSC_ERR_CUDA = -2,        /* a CUDA runtime call failed */
  PVSC_ERR_OOM = -3,         /* a library-side allocation failed */
  PVSC_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up */
  PVSC_ERR_UNSUPPORTED = -5  /* valid but not implemented combination */
} pvsc_status;

enum { PVSC_TI = 1, PVSC_GRAPHENE = 2, PVSC_WSM = 3 };
enum { PVSC_C128 = 0, PVSC_C64 = 1, PVSC_Q64 = 2 };

/* Source of the on-site potential V (one fp64 value per site). */
enum {
  PVSC_V_ZERO = 0,       /* V = 0 */
  PVSC_V_HOST = 1,       /* copied from desc.V, a host array of n_sites doubles */
  PVSC_V_DEVICE = 2,     /* copied from desc.V, a device array of n_sites doubles */
  PVSC_V_SEED = 3,       /* V_n = W (u_n - 1/2), u_n from the counter hash, stored */
  PVSC_V_ON_THE_FLY = 4, /* same values, regenerated inside every stencil sweep */
  PVSC_V_QDOT = 5        /* graphene: gate-defined quantum-dot array (Eq. qdotarray), */
                         /* regenerated inside every sweep from the qd_* fields */
};

/* Damping kernels of pvsc_kpm_density. */
enum { PVSC_KERNEL_NONE = 0, PVSC_KERNEL_JACKSON = 1, PVSC_KERNEL_LORENTZ = 2 };

/* Dot-product selection for pvsc_cheb_step. */
enum { PVSC_DOT_XX = 1, PVSC_DOT_XY = 2, PVSC_DOT_YY = 4 };

/* Operations for pvsc_work_bytes. */
enum {
  PVSC_OP_APPLY = 0,
  PVSC_OP_CHEB_STEP = 1,
  PVSC_OP_KPM = 2,
  PVSC_OP_SERIES = 3,    /* pvsc_cheb_series, pvsc_cheb_filter, pvsc_cheb_propagate */
  PVSC_OP_ADJOINT = 4,   /* pvsc_cheb_adjoint_step; M = number of series terms */
  PVSC_OP_KPM_BATCHED = 5
};

/*
 * Lattice flags.  PVSC_LATTICE_Z_HALO_LO / _HI (TI only; the z axis open, at
 * least one plane besides the halo planes, the potential zero or given on the
 * host or device as the slab's part of the global potential, halo planes
 * included): the lattice is one z-slab of a larger lattice split along z (the
 * domain decomposition of Sec. 3.4).  With _LO plane 0, with _HI plane Lz-1 is
 * a halo plane that holds a copy of the neighbouring slab's boundary plane:
 * every sweep reads it as the z-neighbour of the plane next to it but updates,
 * writes and reduces (dot products, moments) the other planes only, the
 * spectral bounds cover the rows of those planes only, and the launch shape is
 * the default z-march whatever the tuning.  A slab at an open end of the
 * global lattice has no halo plane on that side.  The caller fills the halo
 * planes of every sweep input.  Not for the batched or fixed-point KPM.
 */
enum { PVSC_LATTICE_Z_HALO_LO = 1, PVSC_LATTICE_Z_HALO_HI = 2, PVSC_LATTICE_Z_HALO = 3 };

/*
 * Lattice description.  Defines H for one lattice: the model equation, the
 * cuboid and its boundary conditions (Sec. 3.4: per-dimension periodic or
 * open), the couplings and the on-site potential.  dims: TI (Lx, Ly, Lz)
 * sites; graphene (Nx, Ny, 1) cells.  periodic[d] != 0 wraps axis d; an open
 * axis drops the bonds that leave the cuboid.  Lengths 1 and 2 on a periodic
 * axis make a site its own or its double neighbour; the terms then add.
 * The counter hash is h = mix(mix(seed ^ (0 * 0x9E3779B97F4A7C15)) + n) with
 * mix the SplitMix64 finaliser, u_n = (h >> 11) 2^-53; the paper draws the
 * disorder from a box of width W (gamma), V_n in [-W/2, W/2) (Sec. 4.2).
 */
typedef struct {
  int32_t model;        /* PVSC_TI, PVSC_GRAPHENE or PVSC_WSM */
  int32_t periodic[3];
  int64_t dims[3];
  double t;             /* transfer integral (the paper's unit of energy) */
  double m;             /* TI mass parameter (ignored for graphene) */
  double delta1;        /* TI on-site Delta_1 Gamma^5 (Eq. TB_H_topi); 0 for graphene */
  double delta2;        /* TI on-site Delta_2 Gamma^15, Gamma^15 = [Gamma^1, Gamma^5]/2i */
  int32_t v_source;     /* PVSC_V_* */
  int32_t flags;        /* 0 or PVSC_LATTICE_Z_HALO_LO | PVSC_LATTICE_Z_HALO_HI */
  const double* V;      /* for PVSC_V_HOST / PVSC_V_DEVICE, else ignored */
  uint64_t seed;        /* for PVSC_V_SEED / PVSC_V_ON_THE_FLY */
  double W;             /* disorder width for PVSC_V_SEED / PVSC_V_ON_THE_FLY */
  double k0;            /* PVSC_WSM: Weyl nodes at (+-k0, 0, 0) (Eq. TB_H_wsm); else ignored */
  /* PVSC_V_QDOT (graphene): qd_count x qd_count dots of radius qd_radius on a
   * square grid of spacing 4 qd_radius centred in the sample; dot (l, k) at
   * physical (X_l, Y_k) = (X_c + (l - (K-1)/2) 4R, Y_c + (k - (K-1)/2) 4R),
   * (X_c, Y_c) = (3 Ny / 2, sqrt(3) Nx / 2), height V_k = qd_V0 + qd_dV |k - K/2|;
   * V(r) = sum_{l,k} V_k S(R - |r - (X_l, Y_k)|) with the step smoothed to
   * S(s) = (1 + tanh(s / qd_width)) / 2 within R + 20 qd_width of a centre and
   * 0 beyond.  Site nu of cell (x, y) sits at X = 3 y + {0, 1/2, 3/2, 2}[nu],
   * Y = sqrt(3) x + {sqrt(3)/2, 0, 0, sqrt(3)/2}[nu] (C-C distance 1).
   * complex64 sweeps evaluate it in fp32 (within ~1e-7 qd_V0 of the fp64
   * value), complex128 sweeps and the spectral bounds in fp64. */
  int32_t qd_count;     /* 1 .. 16 */
  int32_t qd_reserved;
  double qd_radius, qd_V0, qd_width, qd_dV;
} pvsc_lattice_desc;

/* Create a lattice handle.  Allocates the handle and its device copy of V,
 * copies or generates V on `stream` and synchronises it.  *out is set only
 * on success.  Errors: ARG (null, dims < 1, unknown model or v_source,
 * t, delta not finite; delta != 0 on graphene; PVSC_V_QDOT on another model
 * or with qd_count outside 1..16, qd_radius or qd_width not positive and
 * finite), OOM, CUDA. */
int pvsc_lattice_create(const pvsc_lattice_desc* desc, void* stream, pvsc_lattice** out);

/* Destroy a handle (NULL is accepted).  The caller must have synchronised
 * every stream that still uses it. */
int pvsc_lattice_destroy(pvsc_lattice* lat);

/* Host query: number of sites and orbitals per site (4 TI, 1 graphene). */
int pvsc_lattice_info(const pvsc_lattice* lat, int64_t* n_sites, int32_t* orbitals);

/* Replace the stored on-site potential from a device array of n_sites
 * doubles (for gradient loops over the gate potential).  Not allowed for
 * PVSC_V_ON_THE_FLY and PVSC_V_QDOT lattices (ARG).  Asynchronous on stream. */
int pvsc_set_potential(pvsc_lattice* lat, const double* V_dev, void* stream);

/* Write the potential the stencil uses (stored or regenerated) to a device
 * array of n_sites doubles.  Asynchronous on stream. */
int pvsc_get_potential(const pvsc_lattice* lat, double* V_out_dev, void* stream);

/* Exact Gershgorin interval over all rows of H (Sec. 4.1 needs the extreme
 * eigenvalues; this bound contains them): emin = min_i (H_ii - sum_{j!=i}
 * |H_ij|), emax = max_i (H_ii + sum_{j!=i}|H_ij|), evaluated on the device
 * per row, coinciding neighbours combined first.  Then a = (emax - emin +
 * eps)/2 and b = (emax + emin)/2, so that (H - b)/a has its spectrum inside
 * [-1, 1].  Any output pointer may be NULL.  Synchronous (host results).
 * A non-finite potential anywhere (a NaN or an infinity, e.g. a poisoned input)
 * is reported as PVSC_ERR_ARG instead of being dropped by the min / max.
 * `work` needs pvsc_work_bytes(lat, PVSC_OP_APPLY, 1, ...) bytes. */
int pvsc_spectral_bounds(const pvsc_lattice* lat, double eps, double* emin, double* emax,
                         double* a, double* b, void* work, size_t work_bytes, void* stream);

/* Random-phase start block (the stochastic trace vectors of the kernel
 * polynomial method, Sec. 4): out[i R + r] = exp(2 pi i u)/sqrt(D) with u from
 * the counter hash, stream 1, idx = r D + i, so <r|r> = 1.  The device-side
 * counterpart of the paper's pvsc_vector_from_func initialisation with a
 * random seed (Sec. 3.4).  out: device block of D*R complex in prec. */
int pvsc_random_vectors(const pvsc_lattice* lat, int R, int prec, uint64_t seed, void* out,
                        void* stream);

/* y = H x for a block of R vectors in precision prec (x, y: D*R complex).
 * x and y must not overlap.  No work buffer. */
int pvsc_apply_H(const pvsc_lattice* lat, int R, int prec, const void* x, void* y, void* stream);

/*
 * Fused Chebyshev step, the generated-kernel contract of Listing graphenec
 * (scale_h, shift_h, scale_z and the partial dot products xx, xy, yy):
 *   per vector r:  y <- alpha_r (H - beta_r) x + gamma_r y
 *   if z != NULL:  z <- z + delta_r y            (same precision as y)
 *   dots (device, 4 x R doubles, written when dot_flags != 0):
 *     dots[0 R + r] = <x|x>,   dots[1 R + r] = Re <y|x>,
 *     dots[2 R + r] = Im <y|x>, dots[3 R + r] = <y|y>   (y the new y)
 *   with <a|b> = sum_i conj(a_i) b_i accumulated in fp64 in a fixed order.
 * alpha, beta, gamma, delta: HOST arrays of R doubles (delta only with z;
 * gamma may be NULL for gamma = 0).  y is read (unless gamma is NULL) and
 * written in place; x must not overlap y or z.  dot_flags is a mask of
 * PVSC_DOT_*: unselected entries are left unspecified.
 * work: device scratch of pvsc_work_bytes(lat, PVSC_OP_CHEB_STEP, R, prec, 0).
 */
int pvsc_cheb_step(const pvsc_lattice* lat, int R, int prec, const void* x, void* y, void* z,
                   const double* alpha, const double* beta, const double* gamma,
                   const double* delta, int dot_flags, double* dots, void* work,
                   size_t work_bytes, void* stream);

/*
 * pvsc_cheb_step without a work buffer, for callers that cannot allocate
 * device memory (a fixed memory budget owned by another pool, callbacks that
 * must not call cudaMalloc because it can synchronise the device, hosts that
 * forbid allocation after start-up).  The paper has no counterpart: this is a
 * deployment variant of the fused step above, with identical arguments and
 * results except `work`.  Its dot-product scratch is a 2 MiB array inside the
 * library image; nothing is allocated.  Sizes that need more scratch than
 * that (on a 152-SM GB300: R >= 32 with dots) are rejected with PVSC_ERR_ARG.
 * Every call looks up the array's device address on the current device,
 * which must be the lattice's; the first call on a device also loads the
 * library's module there (make it before any stream capture).
 * All calls on a device share the array: calls whose kernels overlap on the
 * GPU race, so order them on one stream.  With dot_flags == 0 it needs no
 * scratch at all.
 */
int pvsc_cheb_step_noalloc(const pvsc_lattice* lat, int R, int prec, const void* x, void* y,
                           void* z, const double* alpha, const double* beta, const double* gamma,
                           const double* delta, int dot_flags, double* dots, void* stream);

/*
 * Kernel polynomial method moments (Sec. 2.2, Sec. 4): for each of the R
 * start vectors r, mu_k = <r|T_k(H~)|r>, k = 0..M-1, H~ = (H - b)/a, through
 * the recurrence w_0 = r, w_1 = H~ w_0, w_{k+1} = 2 H~ w_k - w_{k-1}, fused
 * with the dot products of each step and the doubling identities
 * mu_{2k} = 2<w_k|w_k> - mu_0, mu_{2k+1} = 2 Re<w_{k+1}|w_k> - mu_1
 * (ceil(M/2) stencil sweeps).  r0: device block in precision prec, or NULL
 * for random-phase vectors r_i = exp(2 pi i u)/sqrt(D) from the counter hash
 * with stream 1 and idx = r D + i.  mu: device array [R][M] of doubles.
 * M >= 1.  The step loop is captured once into a CUDA graph per argument set
 * and replayed; the first call for a new argument set captures.
 * prec == PVSC_Q64 (TI only): r0, if given, is complex128 and is not modified;
 * [b - a, b + a] must hold the Gershgorin interval of H (PVSC_ERR_ARG
 * otherwise).  The interval is computed by one pass over the potential that
 * synchronises the host with the stream, on the first PVSC_Q64 call after the
 * lattice is created or its potential is set, and kept in the handle; later
 * calls check against it and stay asynchronous.
 * complex64 on a TI lattice with tuning kernel 4: two recurrence steps per
 * sweep (dots <w_k|w_k>, Re<w_{k+1}|w_k>, <w_{k+1}|w_{k+1}>, Re<w_{k+2}|w_{k+1}>
 * give mu_2k .. mu_2k+3), the same vectors as the single sweeps; r0 is then
 * still read only.
 * work: pvsc_work_bytes(lat, PVSC_OP_KPM, R, prec, M).
 */
int pvsc_kpm_moments(const pvsc_lattice* lat, int R, int prec, const void* r0, uint64_t seed,
                     int M, double a, double b, double* mu, void* work, size_t work_bytes,
                     void* stream);

/*
 * Chebyshev series: y = phase * sum_{k=0}^{K-1} c_k T_k(H~) x, H~ = (H - b)/a,
 * with the |w_k> from the three-term recurrence (Sec. 4.1) and the weighted
 * sum accumulated in fp64.  x, y: device complex128 blocks (may be the same
 * buffer).  coeffs: HOST array of K complex values (re, im pairs), used as
 * given.  phase: HOST (re, im) or NULL for 1.  K >= 1.  The recurrence
 * vectors are stored in precision prec.  The accumulator is read and written
 * on every third sweep, which adds the three terms that sweep holds (its
 * y_in, input and output); with PVSC_C64 the three complex64 terms are summed
 * in fp32 with exact products and compensated additions, rounded once and
 * added in fp64 (weights carried as fp32 pairs, to about 2^-48).
 * work: pvsc_work_bytes(lat, PVSC_OP_SERIES, R, prec, K).
 */
int pvsc_cheb_series(const pvsc_lattice* lat, int R, int prec, const void* x, void* y,
                     const double* coeffs, int K, const double* phase, double a, double b,
                     void* work, size_t work_bytes, void* stream);

/* Host-only: the accumulator schedule of a series of K terms (for tests).
 * terms[j] (K ints, caller-owned) = the number of terms the recurrence sweep
 * j adds to the accumulator, ending with term j: 2 at j = 1, 3 on every third
 * sweep after it, the one to three left on the last sweep, 0 elsewhere;
 * K = 1: terms[0] = 1 (no sweep).  PVSC_ERR_ARG if K < 1 or terms is NULL. */
int pvsc_debug_series_plan(int K, int* terms);

/*
 * Chebyshev filter (the polynomial filter of ChebFD, Sec. 4.2):
 * y = sum_{k=0}^{K-1} g_k T_k(H~) x with real HOST coefficients g (window and
 * kernel factors already applied by the caller).  As pvsc_cheb_series.
 */
int pvsc_cheb_filter(const pvsc_lattice* lat, int R, int prec, const void* x, void* y,
                     const double* g, int K, double a, double b, void* work,
                     size_t work_bytes, void* stream);

/*
 * Chebyshev expansion coefficients of the time-evolution operator (Sec. 4.1,
 * Eq. U_1): c_k(a dt) = (-i)^k J_k(a dt), J_k by Miller's backward
 * recurrence normalised with J_0 + 2 sum J_2k = 1, truncated after the
 * largest k with |J_k(a dt)| >= trunc.  Writes the series weights
 * cw_0 = c_0, cw_k = 2 c_k (k >= 1) as (re, im) pairs to the HOST array
 * coeffs (capacity max_terms) and the number of terms M+1 to *n_terms.
 * Errors: ARG if max_terms is too small (*n_terms still set).  Host only.
 */
int pvsc_propagation_coeffs(double a_dt, double trunc, int max_terms, double* coeffs,
                            int* n_terms);

/*
 * Chebyshev time propagation (Sec. 4.1, Eq. U_1): nsteps times
 * psi <- e^{-i b dt} [c_0 w_0 + 2 sum_{k=1}^{M} c_k w_k],  w_k = T_k(H~) psi,
 * with c_k from pvsc_propagation_coeffs(a dt, trunc).  psi: device complex128
 * block (in/out).  Each time step is captured once into a CUDA graph and
 * replayed.  work: pvsc_work_bytes(lat, PVSC_OP_SERIES, R, prec, M+1).
 */
int pvsc_cheb_propagate(const pvsc_lattice* lat, int R, int prec, void* psi, double dt,
                        int nsteps, double a, double b, double trunc, void* work,
                        size_t work_bytes, void* stream);

/*
 * One time step of the adjoint of pvsc_cheb_propagate with respect to the
 * on-site potential (the paper has no adjoint; this is the reverse sweep of
 * the recurrence of Eq. U_1 with a, b held fixed).  Given the state psi_s
 * (device complex128, R vectors) and G = dL/dpsi_{s+1} in the convention
 * dL = Re <G|dpsi_{s+1}>, it recomputes w_0..w_M from psi_s, runs
 *   u_k = conj(cw_k) h + 2 H~ u_{k+1} - u_{k+2},  h = e^{+i b dt} G,
 *   u_0 = conj(cw_0) h + H~ u_1 - u_2,
 * adds (1/a) Re sum_k f_k sum_{orbitals, vectors} conj(u_{k+1}) w_k (f_0 = 1,
 * f_k = 2) to dLdV[n] for every site n, and overwrites G with u_0 =
 * dL/dpsi_s.  dLdV: device array of n_sites doubles (accumulated, not
 * cleared).  prec must be PVSC_C128.
 * work: pvsc_work_bytes(lat, PVSC_OP_ADJOINT, R, PVSC_C128, M+1).
 */
int pvsc_cheb_adjoint_step(const pvsc_lattice* lat, int R, int prec, const void* psi_s,
                           void* G, double dt, double a, double b, double trunc,
                           double* dLdV, void* work, size_t work_bytes, void* stream);

/*
 * KPM recurrence sweeps k_begin .. k_end-1 with caller-held vectors (the
 * recurrence and doubling identities of pvsc_kpm_moments, Sec. 2.2, Sec. 4):
 * resumable KPM (two calls over [0, K) and [K, K') give the moments and vectors
 * of one call over [0, K') bit for bit) and the per-sweep form that a
 * domain-decomposed lattice needs between halo exchanges.  Sweep k makes
 * w_{k+1} = 2 H~ w_k - w_{k-1} (k = 0: w_1 = H~ w_0) fused with the dot
 * products that give mu_{2k} = 2 <w_k|w_k> - mu_0 and mu_{2k+1} =
 * 2 Re <w_{k+1}|w_k> - mu_1 (k = 0: mu_0, mu_1), written to mu [R][M]
 * (device; sweeps k >= 1 read mu_0 and mu_1 from it).  w_j lives in wa for
 * even j and in wb for odd j: w_{k+1} overwrites w_{k-1} element by element.
 * On a lattice with halo planes (PVSC_LATTICE_Z_HALO_*) the dots (and so the
 * moments) cover the other planes only: summed over the slabs of a lattice
 * split along z they give the global moments.
 * 0 <= k_begin <= k_end <= ceil(M/2).  Direct launches (no CUDA graph).
 * work: pvsc_work_bytes(lat, PVSC_OP_CHEB_STEP, R, prec, 0).
 */
int pvsc_kpm_sweeps(const pvsc_lattice* lat, int R, int prec, int k_begin, int k_end, void* wa,
                    void* wb, double a, double b, double* mu, int M, void* work, size_t work_bytes,
                    void* stream);

/*
 * Chebyshev time propagation that also keeps checkpoints for the adjoint
 * (Sec. 4.1, Eq. U_1; the checkpoints are not in the paper): the same nsteps
 * time steps as pvsc_cheb_propagate on psi (device complex128, in/out), and
 * before segment s (steps s*every .. min((s+1)*every, nsteps) - 1) the state
 * psi_{s*every} is copied to ckpts + s * D * R complex128 values, for the
 * ceil(nsteps / every) segments.  ckpts: device, caller-owned, 16-byte
 * aligned, not overlapping psi or work.  every >= 1.
 * work: pvsc_work_bytes(lat, PVSC_OP_SERIES, R, prec, M+1).
 */
int pvsc_cheb_propagate_checkpointed(const pvsc_lattice* lat, int R, int prec, void* psi,
                                     double dt, int nsteps, int every, double a, double b,
                                     double trunc, void* ckpts, void* work, size_t work_bytes,
                                     void* stream);

/*
 * Adjoint of a whole checkpointed propagation with respect to the on-site
 * potential (the paper has no adjoint): given the checkpoints written by
 * pvsc_cheb_propagate_checkpointed (same lat, R, dt, nsteps, every, a, b,
 * trunc, potential) and G = dL/dpsi_nsteps (device complex128, convention
 * dL = Re <G|dpsi>), walks the segments in reverse: recomputes the states of a
 * segment from its checkpoint with the forward series, then applies
 * pvsc_cheb_adjoint_step from its last step to its first.  On return G holds
 * dL/dpsi_0 and dLdV (device, n_sites doubles) has dL/dV_n added (not
 * cleared).  a, b are held fixed.  R must be 1 and prec PVSC_C128.
 * Runs on the stream without a CUDA graph (the recomputed states differ in
 * every segment).  work: pvsc_propagate_adjoint_work_bytes.
 */
int pvsc_cheb_propagate_adjoint(const pvsc_lattice* lat, int R, int prec, const void* ckpts,
                                double dt, int nsteps, int every, double a, double b,
                                double trunc, void* G, double* dLdV, void* work,
                                size_t work_bytes, void* stream);

/* Work bytes of pvsc_cheb_propagate_adjoint: the states of one segment
 * (every vectors) plus the series and adjoint-step scratch; 0 on bad input. */
size_t pvsc_propagate_adjoint_work_bytes(const pvsc_lattice* lat, int R, int every, double a_dt,
                                         double trunc);

/*
 * Batched KPM: n independent TI lattices (uneven sizes allowed) x R
 * random-phase vectors each, M moments, in one persistent cooperative launch
 * that walks a device work list of (lattice, z-slab) units; a unit of step k
 * starts once every unit of its lattice has finished step k-1 (a per-lattice
 * phase counter, bounded spin waits), so the lattices advance independently.
 * Launch shape (threads per block, z-slab planes, blocks per SM): the tuning
 * entry (R, prec) of lats[0] if one is set, else 256 threads, whole columns
 * (one unit per column and step) and the occupancy maximum.  An entry with
 * kernel 7 (complex64, every lattice eligible for kernel 7) runs each
 * lattice's KPM instead as its own chain of TMA-staged sweeps (threads 256 or
 * 512: the large tile on 8 or 16 warps), the chains on a few streams forked
 * from `stream` inside one captured graph, the same moments as
 * pvsc_kpm_moments with that kernel and seed; that mode does not synchronise
 * and reports copy-wait timeouts through pvsc_device_error.
 * a, b: HOST arrays of n doubles.  Start vectors: counter hash, stream 1,
 * seed seeds[i] (HOST array of n).  mu: device [n][R][M] doubles.
 * Returns PVSC_ERR_TIMEOUT if a wait exceeded pvsc_set_wait_limit (the
 * kernel then stops cleanly; mu is undefined).
 * work: pvsc_batched_work_bytes (it depends on the launch shape: query it
 * after any pvsc_set_tuning on lats[0]).
 */
int pvsc_kpm_moments_batched(const pvsc_lattice* const* lats, int n, int R, int prec,
                             const uint64_t* seeds, int M, const double* a, const double* b,
                             double* mu, void* work, size_t work_bytes, void* stream);

/*
 * Spectral densities from KPM moments (Sec. 2.2: the DOS of Eq. DOS and the
 * momentum-resolved spectral function A(k, E) of Eq. ak), with the damping
 * kernels of the kernel polynomial method the paper cites:
 *   rho(E_j) = scale sum_r [g_0 mu_0^r + 2 sum_{k>=1} g_k mu_k^r T_k(x_j)]
 *              / (pi a sqrt(1 - x_j^2)),   x_j = (E_j - b)/a,
 * and rho(E_j) = 0 for |x_j| >= 1.  mu: device [R][M] doubles (as written by
 * pvsc_kpm_moments); E, rho: device arrays of NE doubles.  kernel:
 * PVSC_KERNEL_NONE (g_k = 1), PVSC_KERNEL_JACKSON (g_k = [(M-k+1) cos(q k)
 * + sin(q k) cot q]/(M+1), q = pi/(M+1)) or PVSC_KERNEL_LORENTZ (g_k =
 * sinh(lambda (1 - k/M))/sinh(lambda), lambda > 0).  DOS: random-phase
 * moments, scale = D/R (integrates to D); A(k, E): the moments of the O states
 * psi(k, nu) of pvsc_bloch_vectors, scale = 1 (integrates to O).
 */
int pvsc_kpm_density(int R, int M, const double* mu, int kernel, double lambda, double a, double b,
                     double scale, int NE, const double* E, double* rho, void* stream);

/*
 * The states psi(k, nu) of Eq. ak on a cubic lattice with O orbitals per site
 * (TI: O = 4, Weyl semimetal: O = 2), for nk k-points k[3 q .. 3 q + 2]
 * (HOST array of 3 nk doubles, components along x, y, z in radians per
 * lattice spacing; O nk a power of two <= 64, nk <= 16): vector r = O q + nu
 * of the block (R = O nk) is exp(i k_q . r_n)/sqrt(n_sites) on orbital nu of
 * every site n (r_n its integer coordinates) and zero on the other orbitals.
 * out: device block (D x R) in precision prec.  Phases are evaluated in fp64.
 */
int pvsc_bloch_vectors(const pvsc_lattice* lat, int nk, const double* k, int prec, void* out,
                       void* stream);

/*
 * Chebyshev filter diagonalization (ChebFD, Sec. 5.3 "Interior eigenvalues"):
 * the eigenpairs of H in [lo, hi] from a block of n_search <= 64 vectors.
 * Each iteration filters the block with the Jackson-damped Chebyshev series
 * of the indicator of [lo, hi] (degree `degree`, recurrence vectors in
 * `prec`), orthonormalizes it (shifted CholeskyQR3; Gram matrices by cuBLAS),
 * and performs Rayleigh-Ritz (the n_search x n_search projection by cuBLAS,
 * its eigen-decomposition by Jacobi rotations on the host); it stops when
 * every Ritz value inside [lo, hi] has ||H x - theta x|| < tol, or after
 * max_iter iterations.  The start block is the random-phase block of `seed`.
 * Outputs: X (device complex128 D x n_search, the Ritz vectors, orthonormal),
 * theta and resid (HOST arrays of n_search doubles, Ritz values ascending and
 * their residual norms), *n_inside (Ritz values inside [lo, hi]),
 * *iterations.  The search space should exceed the number of eigenvalues in
 * the interval (about 1.5-2x).  Synchronous (reads small matrices back every
 * iteration).  PVSC_ERR_ARG if the filtered block loses rank.
 * work: pvsc_chebfd_work_bytes.
 */
typedef struct {
  double lo, hi;   /* target interval (energies) */
  int32_t n_search;
  int32_t degree;  /* filter polynomial degree */
  int32_t max_iter;
  int32_t prec;    /* PVSC_C128 or PVSC_C64 for the filter's recurrence vectors */
  double tol;      /* residual bound */
  uint64_t seed;
} pvsc_chebfd_params;

int pvsc_chebfd(const pvsc_lattice* lat, const pvsc_chebfd_params* params, double a, double b,
                void* X, double* theta, double* resid, int* n_inside, int* iterations, void* work,
                size_t work_bytes, void* stream);
size_t pvsc_chebfd_work_bytes(const pvsc_lattice* lat, int n_search, int prec, int degree);

/* Host-only: eigen-decomposition of a Hermitian n x n matrix (column-major,
 * interleaved re/im) by the cyclic Jacobi method ChebFD uses; w ascending,
 * V (same layout as A) the eigenvectors.  For tests. */
int pvsc_debug_eigh(int n, const double* A, double* w, double* V);

/* Work bytes for pvsc_kpm_moments_batched over the given lattices. */
size_t pvsc_batched_work_bytes(const pvsc_lattice* const* lats, int n, int R, int prec, int M);

/* Device scratch bytes an operation needs (0 if none); M is the moment count
 * (KPM) or the number of series terms (series/adjoint).  0 on bad args. */
size_t pvsc_work_bytes(const pvsc_lattice* lat, int op, int R, int prec, int M);

/* Spin limit of every bounded device wait (persistent batched kernel); the
 * default allows several seconds.  A wait that exceeds it sets an error
 * word, the kernel returns, and the call reports PVSC_ERR_TIMEOUT. */
int pvsc_set_wait_limit(uint64_t spins);

/* Fault injection for tests of the bounded waits: while enabled, the first
 * dependency wait of every block in pvsc_kpm_moments_batched targets a phase
 * that is never published, so it runs out after the wait limit and the call
 * returns PVSC_ERR_TIMEOUT with the device context intact.  Host-side switch;
 * nothing faults, traps or hangs.  Off by default. */
int pvsc_debug_inject_stall(int enable);

/*
 * Launch tuning.  A tuning entry fixes, for (lattice, op, R, prec), the
 * threads per block, the blocks per SM of the persistent grid and the z-slab
 * depth of the TI z-marching sweep (0 = automatic).  pvsc_autotune times the
 * candidates on the device with CUDA events (synchronous; the vectors it
 * sweeps are allocated inside and freed) and stores the winner in the
 * handle; pvsc_get_tuning reads the entry in force.
 */
typedef struct {
  int32_t threads;
  int32_t blocks_per_sm; /* resident blocks per SM (0: from occupancy); kernels 7 and 8: 0 or 1, */
                         /* 1 spreading the planes over every SM when the sweep has fewer */
                         /* work units (tile x z-chunk) than SMs */
  int32_t zslab;
  float time_ms; /* measured time of one sweep, 0 if not measured */
  int32_t vpt;   /* vectors per thread: 1, or 2 (complex64 with R >= 2); 0 = automatic */
  int32_t tile_x; /* TI only: > 0 selects the shared-memory staged sweep (bulk-copy */
  int32_t tile_y; /* engine, 4-plane ring) with tiles of tile_x x tile_y columns */
  int32_t kernel; /* TI only: 0 z-marching in registers (or staged if tile_x > 0), */
                  /* 1 flat (one site per thread and pass, neighbours folded in turn), */
                  /* 2 z-marching with a cp.async ring of all six blocks of a plane, */
                  /* 3 z-marching with a deep cp.async ring of the two streamed blocks, */
                  /* 4 (complex64, R >= 2; pvsc_kpm_moments only, other calls keep the */
                  /* default sweep): two recurrence steps per sweep (temporal blocking), */
                  /* blocks of tile_x x tile_y columns plus a recomputed one-column ring, */
                  /* (tile_x tile_y + 2 (tile_x + tile_y)) R/2 <= 384 threads; 0 = the */
                  /* default tile of that R (16x12, 10x8, 8x8, 5x5, 3x3, 2x2 for R = 2..64); */
                  /* zslab = z-range of one block (0: whole columns).  Same vectors as */
                  /* two single sweeps bit for bit; needs a KPM work buffer of four */
                  /* vectors, which pvsc_work_bytes reports once this entry is set, */
                  /* 5 z-marching over tiles of tile_x x tile_y columns per block */
                  /* (threads = tile_x tile_y R/vpt, a multiple of 32, at most 256), */
                  /* 6 marching along x over lines (y, z), zslab = x-segment length, */
                  /* 7 (complex64, R = 1 .. 64, Lx a multiple of 4) TMA-staged */
                  /* plane tiles: one block per SM copies each z-plane of a tile of */
                  /* 32x32, 32x16, 16x16, 16x8 or 8x8 columns (R = 1, 2, 4, 8, 16; R = 1, */
                  /* 2: one thread per 32- or 64-byte site) with its one-site halo */
                  /* strips into a shared-memory ring (cp.async.bulk.tensor, */
                  /* mbarriers) for eight warps (threads 256, two (site, vector pair) */
                  /* items per thread) or sixteen (threads 512, one item); R = 32 and */
                  /* 64 run as 2 and 4 slices of 16 vectors on the 8x8 tiles, one slice */
                  /* per block; tile_x x tile_y = the half tile (32x16, 32x8, 16x8, 16x4, */
                  /* 8x4, 8x4, 8x4 for R = 1 .. 64) selects rings one plane deeper on eight warps */
                  /* (Weyl cells run eight warps, the large or the half tile); zslab = z-chunk */
                  /* depth (0: chosen from the grid size); vpt is ignored. */
                  /* 8 (as kernel 7) the same tiles marching along x over (y, z) columns, */
                  /* for lattices whose z columns are short; eight warps, the large or */
                  /* (TI) the half tile; zslab = x-chunk depth; same vectors as the */
                  /* z-march bit for bit; the fused step with z runs kernel 7. */
                  /* Kernels 7 and 8 are launched with programmatic dependent launch: */
                  /* the next sweep's blocks set up on free SMs and wait for the */
                  /* previous sweep to complete before touching global memory (same */
                  /* results; environment PVSC_NO_PDL=1 launches them plainly). */
                  /* PVSC_Q64 (KPM on TI lattices) takes kernels 0, 2, 3 (threads a */
                  /* multiple of R, one vector per thread, no tile) and 7 for R = 1 .. 32 */
                  /* (any Lx): the tiles, rings and variants of the complex64 layout */
                  /* of 2R vectors (a fixed-point value is 16 bytes; R = 16, 32 as */
                  /* slices of 8), one vector of one site per item.  Untuned it runs */
                  /* kernel 7 on sixteen warps for R = 2 .. 8 and on eight for R = 1, */
                  /* 16, 32, and kernel 2 for R = 64. */
} pvsc_tuning;

/* Device error word of the shared-memory staged sweeps: *flag = 1 if a copy
 * wait ran out since the last clear (the sweep then stopped early and its
 * outputs are invalid).  Synchronises the device.  clear != 0 resets it. */
int pvsc_device_error(int* flag, int clear);
int pvsc_set_tuning(pvsc_lattice* lat, int R, int prec, const pvsc_tuning* tuning);
int pvsc_get_tuning(const pvsc_lattice* lat, int R, int prec, pvsc_tuning* tuning);
int pvsc_autotune(pvsc_lattice* lat, int R, int prec, pvsc_tuning* best, void* stream);
/* pvsc_autotune timing the sweeps of one operation: PVSC_OP_KPM (what
 * pvsc_autotune times: the recurrence sweep with its dot products),
 * PVSC_OP_SERIES (one accumulating and two plain sweeps of pvsc_cheb_series,
 * pvsc_cheb_filter, pvsc_cheb_propagate and ChebFD's filter) or PVSC_OP_APPLY
 * (the plain sweep).  The winner replaces the (R, prec) tuning entry; the
 * on-disk cache keys on the operation too. */
int pvsc_autotune_op(pvsc_lattice* lat, int R, int prec, int op, pvsc_tuning* best, void* stream);

/* Launch-shape autotuner of the batched KPM over the whole batch (the batched
 * calls read the (R, prec) tuning entry of lats[0]): threads per block (128,
 * 256), z-segment length of the work units (whole columns, 16 .. 64 planes)
 * and blocks per SM (occupancy maximum, 1) are timed with CUDA events on the
 * batch itself running M moments, and the fastest becomes that entry.
 * Allocates and frees its own buffers; synchronises the stream.  Query
 * pvsc_batched_work_bytes again afterwards (it depends on the shape). */
int pvsc_autotune_batched(pvsc_lattice* const* lats, int n, int R, int prec, const uint64_t* seeds,
                          int M, const double* a, const double* b, pvsc_tuning* best, void* stream);

/* Neighbour table the stencil uses (debug/parity): for every site, 7 site
 * indices (TI: self, -x, +x, -y, +y, -z, +z) or, for graphene, per cell
 * (self, -x, +x, -y, +y) padded to 7 with -1, absent neighbours -1.
 * Computed by a device kernel into nbr_dev (int64, n_sites*7 or n_cells*7). */
int pvsc_debug_neighbours(const pvsc_lattice* lat, int64_t* nbr_dev, void* stream);

/* Sparsity pattern of H as the stencil applies it (debug/parity; Sec. 3.1:
 * the matrix the matrix-free stencil never stores), as CSR over the
 * D = n_sites * orbitals rows in the vector layout: one entry per stencil
 * term, so a neighbour that coincides with another (a periodic axis of
 * length 1 or 2) appears once per term and the entries of a row count the
 * terms that land on each column; terms whose block entry is structurally
 * zero (the zeros of the 4x4 Dirac and graphene blocks) are not listed.
 * Host only, no device work.  rowptr: HOST array of D + 1 (always written);
 * col: HOST array of rowptr[D] int32 column indices, or NULL to size it
 * first.  D at most 2^24 (PVSC_ERR_ARG otherwise). */
int pvsc_debug_export_pattern(const pvsc_lattice* lat, int64_t* rowptr, int32_t* col);

/* Fixed-point arithmetic of the PVSC_Q64 sweeps (debug/parity): runs the
 * device routines those sweeps use on caller-given 64-bit integers, so that
 * they can be checked against exact integer arithmetic.
 *   op 0: in holds n records (c1, x1, c2, x2); out[i] = floor((c1 x1 + c2 x2
 *         + 2^59) / 2^60), the once-rounded Q3.60 x Q4.59 update of a value.
 *         Valid for |c1|, |c2| <= 2^61, |x1| <= 2^59, |x2| <= 6 * 2^59 (the
 *         coefficients, vector entries and neighbour combinations a sweep
 *         meets under its scaling checks).
 *   op 1: in holds n records (x_0 .. x_7, y_0 .. y_7) (the eight values of a
 *         site block of two vectors); out[0..3] = the exact sums over all
 *         records of x_k^2 and of y_k x_k, each as a 128-bit two's-complement
 *         (hi, lo) pair.  Valid for |x_k|, |y_k| <= 2^59 with sum x_k^2 and
 *         sum y_k^2 <= 2^118 (two vectors of 2-norm <= 1).  One thread:
 *         meant for small n.
 * Outside those ranges the results are unspecified (no fault).  in, out:
 * DEVICE int64 arrays (in may be NULL when n = 0); n >= 0.  Asynchronous on
 * stream. */
int pvsc_debug_fx_arith(int op, const int64_t* in, int64_t n, int64_t* out, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* pvsc_last_error(void);

/* Library version string. */
const char* pvsc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PVSC_H */
