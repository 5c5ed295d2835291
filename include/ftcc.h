/*
 * ftcc.h -- C ABI of libftcc, a GB300 (sm_103a) implementation of the
 * finite-temperature CCSD imaginary-time amplitude sweep of
 * White & Chan, "Finite-temperature coupled cluster: efficient implementation
 * and application to prototypical systems" (arXiv:2004.01729).
 *
 * Conventions shared by every entry point
 *   - Return codes only: the library never aborts, traps or prints.  The text
 *     of the last failure of a context is returned by ftcc_last_error().
 *   - Host pointers are read (inputs) or written (outputs) only during the
 *     call; inputs are copied.  Device pointers named *_dev must be device
 *     memory of the context's device; the caller keeps ownership.
 *   - All device memory a context needs comes from the allocator given to
 *     ftcc_create (or cudaMalloc when it is NULL) and is released by
 *     ftcc_destroy.
 *   - Work runs on the CUDA stream given to ftcc_create (NULL = a
 *     non-blocking stream owned by the context; the legacy default stream
 *     cannot be captured into the per-iteration CUDA graph, so pass a created
 *     stream, never the handle of the legacy stream).  Entry points that
 *     return results on the host synchronise that stream before returning.
 *   - There is no CPU path: without a usable CUDA device every compute entry
 *     point returns FTCC_ERR_NO_DEVICE.
 *   - A context is not thread safe; distinct contexts are independent.
 *
 * Spin-orbital conventions: p = sigma * M + g (sigma = 0 up, 1 down, g the
 * spatial orbital), <pq||rs> = <pq|rs> - <pq|sr> in physicists' order,
 * dense row-major N^4.  Amplitudes are stored s1[x][i][a] and
 * s2[x][i][j][a][b] (x = tau point, i, j over the hole-like set O, a, b over
 * the particle-like set V, each in increasing orbital order).
 */
#ifndef FTCC_H
#define FTCC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ftcc_ctx ftcc_ctx;

typedef enum {
  FTCC_OK = 0,
  FTCC_ERR_INVALID_ARG = 1,   /* an argument is out of its documented range       */
  FTCC_ERR_NO_DEVICE = 2,     /* no CUDA device / driver                           */
  FTCC_ERR_OOM = 3,           /* the allocator returned NULL                        */
  FTCC_ERR_NOT_CONVERGED = 4, /* max_iter reached; outputs hold the last iterate   */
  FTCC_ERR_DIVERGED = 5,      /* NaN/Inf or runaway residual                        */
  FTCC_ERR_TIMEOUT = 6,       /* a bounded device wait gave up (error flag set)     */
  FTCC_ERR_UNSUPPORTED = 7,   /* valid request this build does not implement        */
  FTCC_ERR_STATE = 8,         /* call order violated (e.g. adjoint before solve)    */
  FTCC_ERR_CUDA = 9           /* a CUDA runtime call failed                         */
} ftcc_status;

/* Quadrature / propagation scheme (Sec. II.C).  SIMPSON is the implicit
 * integral method with the Simpson tensors g, G (Eq. smu, solved as one
 * fixed point over the grid).  RK1 / RK2 / RK4 march the differential form
 * ds/dtau = -(Delta s + S[s]) (Eq. smud) from s = 0 with one explicit step
 * per grid interval (Alg. 1; read as forward Euler, Heun's method and the
 * classical four-stage method, since the paper does not print the tableaux);
 * Omega_CC keeps the quadrature weights g.  The RK drivers run through
 * ft_ccsd_solve / ft_ccsd_solve_batched in FP64 without stream_tau
 * (otherwise FTCC_ERR_UNSUPPORTED); ft_ccsd_iterate and ft_ccsd_adjoint on
 * an RK solve return FTCC_ERR_UNSUPPORTED.  ftcc_result.iterations is then
 * the number of steps (ngrid - 1). */
typedef enum { FTCC_QUAD_SIMPSON = 0, FTCC_QUAD_RK1 = 1, FTCC_QUAD_RK2 = 2, FTCC_QUAD_RK4 = 3 } ftcc_quadrature;

/* Arithmetic of the contractions.  FP64: every tensor and GEMM in FP64.
 * TF32 / BF16X3: amplitudes and intermediates stored in FP32, contractions on
 * the tcgen05 tensor cores (kind::tf32, or a two-way bf16 split x = hi + lo
 * with the three kind::f16 products hi*hi + hi*lo + lo*hi), FP32
 * accumulation; occupations, orbital energies, the propagator factors
 * exp(-Delta h) (formed in FP64 per element, rounded once), quadrature
 * weights, the energy sums and the Omega accumulation stay FP64; the Simpson
 * recurrence runs in FP32 beside the FP32 amplitudes (option
 * fp64_propagation).
 * A TF32 solve runs three phases: TF32 iterations until Omega_CC changes by
 * less than tol_mixed or than the TF32 unit roundoff 2^-11 |Omega_CC|, or
 * stops improving; then up to polish_max_iter BF16X3 iterations from those
 * amplitudes, until |dOmega_CC| < tol_mixed or it stops improving; then up to
 * refine_max_iter FP64 residual corrections s <- s + (Phi(s) - s), each one
 * FP64 application of the fixed-point map.  A BF16X3 solve skips the TF32
 * phase. */
typedef enum { FTCC_PREC_FP64 = 0, FTCC_PREC_TF32 = 1, FTCC_PREC_BF16X3 = 2 } ftcc_precision;

typedef enum { FTCC_SYS_HUBBARD_1D = 0, FTCC_SYS_UEG = 1, FTCC_SYS_GENERIC = 2 } ftcc_system_kind;

/* Reference (orbitals and orbital energies) of the Hubbard ring (Sec. II.B:
 * at T > 0 both the orbitals and the reference energies define the theory;
 * Sec. IV.A uses the Neel state and zero-temperature UHF).
 *   KSPACE_RHF: restricted orbitals of crystal momentum k, eps = -2t cos k +
 *     U/2 (exact thermal HF at half filling of an even ring).
 *   NEEL_SITE: site orbitals (spin orbital sigma * L + i), eps_{i sigma} =
 *     h_ii + U n^Neel_{i,-sigma} with the Neel determinant spin up on even,
 *     spin down on odd sites: the diagonal of its zero-temperature Fock matrix.
 *   UHF_SITE: the zero-temperature unrestricted Hartree-Fock solution of the
 *     site-basis ring with L/2 up and L - L/2 down electrons, found from the
 *     Neel density by F_sigma = h + U diag(n_-sigma), filling the lowest
 *     orbitals and mixing old and new densities half and half until they
 *     change by less than 1e-12 (2000 iterations at most, else
 *     FTCC_ERR_NOT_CONVERGED); h and <pq||rs> are transformed to the UHF spin
 *     orbitals (sigma * L + k, k in ascending energy) and eps are the UHF
 *     orbital energies.  Built on the host (O(N^5)), then uploaded. */
typedef enum { FTCC_REF_KSPACE_RHF = 0, FTCC_REF_NEEL_SITE = 1, FTCC_REF_UHF_SITE = 2 } ftcc_reference;

/* Hamiltonian description for build_integrals.
 *   HUBBARD_1D: L-site ring (pbc must be 1), hopping t, on-site U, in the
 *     basis of its reference (ftcc_reference); the default k-space restricted
 *     orbitals phi_k, k = 2 pi m / L, give h_kk = -2 t cos k,
 *     <k1 k2|k3 k4> = U/L delta(k1 + k2 = k3 + k4), eps = h_kk + U/2
 *     (Sec. IV.A; the restricted reference at half filling).
 *   UEG: n_elec electrons at density rs in the n_pw lowest plane waves of a
 *     cubic cell (n_pw must close a shell), ordered by (|n|^2, nx, ny, nz);
 *     h_pp = k^2/2, <pq|rs> = 4 pi / (Vc |k_p - k_r|^2) with momentum and
 *     spin conservation, no q = 0 term; eps = zero-temperature HF energies of
 *     the n_elec/2 lowest plane waves per spin (Sec. IV.B, App. D).
 *   GENERIC: host FP64 arrays h[N*N], eri[N^4] (antisymmetrised <pq||rs>),
 *     eps[N]; copied.  Optionally charge[N*4] (host int): a conserved
 *     integer charge vector per spin orbital (momentum components, S_z ...),
 *     component k taken modulo charge_mod[k] when charge_mod is given and
 *     charge_mod[k] > 0; every h_pq and <pq||rs> that does not conserve it
 *     must vanish.  It enables the block_sparse option when all N charges
 *     differ.  NULL: none.
 * UEG and the k-space Hubbard ring (KSPACE_RHF) carry their momentum and
 * S_z as charges (ftcc_get_charges); the site-basis references carry none. */
typedef struct {
  int kind;
  int L; double t, U; int pbc;          /* HUBBARD_1D */
  int n_elec; double rs; int n_pw;      /* UEG */
  int N; const double* h; const double* eri; const double* eps; /* GENERIC */
  int reference;                        /* HUBBARD_1D: ftcc_reference (0 = KSPACE_RHF) */
  const int* charge; const int* charge_mod;   /* GENERIC: optional conserved charges [N*4], [4] */
} ftcc_system;

/* Solver options; pass NULL for the defaults in brackets.
 *   tol_omega  [1e-10]  stop when |dOmega_CC| < tol_omega ...
 *   tol_amp    [1e-8]   ... and max|ds| / max(1, max|s|) < tol_amp
 *   damping    [1.0]    s <- (1 - a) s + a Phi(s)
 *   trunc_thr  [0.0]    orbital kept hole-like if n >= thr, particle-like if 1 - n >= thr
 *   max_iter   [200]    iterations of the low-precision (or FP64) phase
 *   precision  [FP64]   ftcc_precision
 *   refine_max_iter [2] FP64 residual corrections after the low-precision
 *                       phases (0 = none); they stop early once tol_omega and
 *                       tol_amp hold
 *   tol_mixed  [1e-7]   |dOmega_CC| at which a low-precision phase hands over;
 *                       without FP64 corrections a mixed solve counts as
 *                       converged when its last iteration moved Omega_CC by
 *                       less than tol_mixed
 *   polish_max_iter [40] BF16X3 iterations after the TF32 phase of a TF32 solve
 *                       (0 = straight from TF32 to the FP64 corrections)
 *   fp64_propagation [1] arithmetic of the Simpson recurrence and the energy
 *                       sums of a TF32 / BF16X3 sweep (the ratios exp(-Delta h)
 *                       always come from FP64 factors): 2 = FP64 for both,
 *                       1 = FP32 recurrence with FP64 energy sums, 0 = FP32
 *   tol_refine [1e-6]   with FP64 corrections, a mixed solve counts as
 *                       converged when the FP64 tolerances hold or its last
 *                       correction moved Omega_CC by less than tol_refine
 *   mixed_adjoint [0]   1: ft_ccsd_adjoint after a mixed solve that ended in
 *                       a low-precision phase (refine_max_iter = 0) runs the
 *                       lambda sweep and the response on the FP32 solver
 *                       (FP32 multipliers, BF16X3 contractions, FP64 factors,
 *                       weights and sums), stopping when the multipliers
 *                       change by less than 1e-7 relative or stop falling;
 *                       0: the amplitudes are first refined in FP64 and the
 *                       sweep runs in FP64 (ftcc_rdm2 needs this one)
 *   tau_chunk  [0]      tau points per S-kernel pass (0 = all that fit)
 *   use_graph  [1]      replay one iteration as a CUDA graph
 *   stream_tau [0]      1: run the S kernel tau_chunk points at a time (0 picks
 *                       1), keep S only for the current propagation window
 *                       (max(3, tau_chunk) points) and advance the Simpson
 *                       propagation window by window, carrying five values per
 *                       amplitude element (the last two even-point integrals
 *                       and the last three S).  Same result as the unstreamed
 *                       iteration (in FP32 sweeps the carried values are
 *                       stored in FP32); amplitude-sized memory ~ ngrid + 5 +
 *                       max(3, tau_chunk) slices plus the S-kernel intermediates
 *                       of tau_chunk points, instead of 2 ngrid + intermediates.
 *                       Single instance only; ft_ccsd_adjoint then returns
 *                       FTCC_ERR_UNSUPPORTED.
 *   autotune   [1]      time the tensor-core tile width (32/64/128/256) and K split
 *                       of each contraction shape once, on the first (uncaptured)
 *                       iteration, and keep the fastest (0 = built-in choice)
 *   block_sparse [0]    1: exploit the conserved charge of every spin orbital
 *                       (crystal momentum and S_z) of the UEG and the k-space
 *                       Hubbard ring, whose orbitals all carry distinct charges:
 *                       one-index-pair factors become their diagonals, four-index
 *                       factors N^3 arrays with the fourth index implied, and
 *                       the contractions run over charge sectors only.  The same
 *                       equations and fixed point, with the work and memory of
 *                       one iteration cut by about the number of k-points.
 *                       precision FP64: FP64 throughout; TF32 or BF16X3: an FP32
 *                       sweep (FP32 storage and SIMT sector products, FP64
 *                       propagator factors and energy sums) handing over at
 *                       tol_mixed to at most refine_max_iter FP64 residual
 *                       corrections (no polishing phase).  Needs a single
 *                       instance of such a system (FTCC_ERR_INVALID_ARG
 *                       otherwise), no truncation (trunc_thr removes nothing)
 *                       and the Simpson integral form; stream_tau is ignored.
 *                       ft_ccsd_adjoint (the FP64 lambda sweep through the
 *                       transpose of the block-sparse S kernel; mixed_adjoint is
 *                       ignored), ftcc_rdm2 and
 *                       ftcc_mu_for_n work on it; ftcc_get_amplitudes,
 *                       ftcc_eval_s and ftcc_eval_s_vjp convert between the
 *                       dense layouts and the compressed one (inputs projected
 *                       onto the charge-conserving elements); ftcc_propagate,
 *                       ftcc_propagate_adjoint and ftcc_get_lambda take dense
 *                       layouts only (FTCC_ERR_UNSUPPORTED). */
typedef struct {
  double tol_omega, tol_amp, damping, trunc_thr;
  int max_iter, precision, refine_max_iter;
  double tol_mixed;
  int tau_chunk, use_graph;
  int stream_tau;
  int autotune;
  int polish_max_iter;
  int fp64_propagation;
  double tol_refine;
  int mixed_adjoint;
  int block_sparse;
} ftcc_options;

typedef struct {
  double omega;       /* Omega0 + Omega1 + Omega_CC                          */
  double omega0, omega1, omega_cc;
  double d_omega;     /* |Omega_CC change| in the last iteration              */
  double d_amp;       /* max|ds| / max(1, max|s|) in the last iteration       */
  int iterations;     /* total iterations, every phase                        */
  int refine_iterations; /* FP64 residual corrections of a mixed solve        */
  int converged;
  int n_occ, n_vir;   /* sizes of the hole-like / particle-like sets           */
  double ms_per_iter; /* mean device time of one iteration                    */
  int kernels_per_iter; /* kernel launches in one iteration (graph nodes)      */
  int polish_iterations; /* BF16X3 iterations after the TF32 phase             */
} ftcc_result;

typedef struct {
  double dOmega_dmu, dOmega_dbeta;
  double N, E, S;     /* N = -dOmega/dmu, E = Omega + beta dOmega/dbeta + mu N, S = beta^2 dOmega/dbeta */
  double trace_rdm1;
  int iterations;
} ftcc_adjoint_result;

typedef struct {
  void* (*alloc)(size_t bytes, void* user);   /* returns device memory or NULL */
  void (*release)(void* ptr, void* user);
  void* user;
} ftcc_allocator;

/* Create a context on CUDA device `device`, issuing work on `stream`
 * (a created cudaStream_t, or NULL for a stream owned by the context).  `alloc` may be NULL (cudaMalloc/cudaFree).
 * Returns FTCC_ERR_NO_DEVICE without a device, FTCC_ERR_UNSUPPORTED if the
 * device is not compute capability 10.3. */
ftcc_status ftcc_create(int device, void* stream, const ftcc_allocator* alloc, ftcc_ctx** out);

/* Release every resource of the context (NULL is ignored). */
void ftcc_destroy(ftcc_ctx* ctx);

const char* ftcc_status_string(ftcc_status s);
const char* ftcc_last_error(const ftcc_ctx* ctx);

/* Build the spin-orbital Hamiltonian (h, <pq||rs>, eps) in device memory
 * (layer below App. A).  Invalidates any previous solve.
 * FTCC_ERR_INVALID_ARG: L < 1, pbc != 1, U or t not finite, an unknown
 * reference, n_elec odd or < 2, rs <= 0, n_pw not a closed shell, N < 1, or
 * a NULL array. */
ftcc_status build_integrals(ftcc_ctx* ctx, const ftcc_system* sys);

/* Number of spin orbitals of the built system (0 before build_integrals). */
int ftcc_num_orbitals(const ftcc_ctx* ctx);

/* Copy the built eps[N], h[N*N] and, if eri != NULL, <pq||rs>[N^4] to host
 * buffers (any may be NULL). */
ftcc_status ftcc_get_system(ftcc_ctx* ctx, double* eps, double* h, double* eri);

/* Copy the conserved orbital charges of the built system: charge[N*4] and
 * charge_mod[4] (0 = not periodic); either may be NULL.  FTCC_ERR_STATE when
 * the system has none. */
ftcc_status ftcc_get_charges(ftcc_ctx* ctx, int* charge, int* charge_mod);

/* Chemical potential mu0 with sum_p n_p(beta, mu0) = n_elec for the
 * reference energies eps (the reference-system electron count used to fix
 * mu for the gas at fixed N, App. D).  FP64 bisection on the host, on a copy
 * of the device orbital energies, to 1e-15 relative. */
ftcc_status ftcc_reference_mu(ftcc_ctx* ctx, double beta, double n_elec, double* mu);

/* Chemical potential mu_CC of the coupled-cluster system at a fixed mean
 * electron number (App. D: the CC system and the reference each get their
 * own mu for N electrons; Sec. III.A fixes <N> for every grid):
 * N(mu) = -dOmega/dmu = n_target, with N(mu) from ft_ccsd_solve followed by
 * ft_ccsd_adjoint on this context (the lambda sweep, App. B).  Secant steps
 * from mu0 and mu0 + dmu (or mu0 - dmu when N(mu0) is above the target);
 * once two evaluations straddle the target, regula falsi with the Illinois
 * weighting (an end point kept twice in a row has its residual halved).
 * Stops when |N - n_target| < tol_n.  mu_out, n_out (may be NULL) and
 * evals_out (may be NULL) receive mu_CC, its N and the number of N
 * evaluations; out (may be NULL) the last solve; the context is left with
 * the last solve and its adjoint.  FTCC_ERR_NOT_CONVERGED after max_evals
 * evaluations (outputs hold the last point); FTCC_ERR_INVALID_ARG for beta,
 * dmu or tol_n not positive and finite, max_evals < 2, or n_target outside
 * (0, N); the errors of ft_ccsd_solve and ft_ccsd_adjoint pass through. */
ftcc_status ftcc_mu_for_n(ftcc_ctx* ctx, double beta, double n_target, int ngrid, ftcc_quadrature quad,
                          const ftcc_options* opt, double mu0, double dmu, double tol_n, int max_evals,
                          double* mu_out, double* n_out, int* evals_out, ftcc_result* out);

/* Set up a solve without iterating: Fermi-Dirac occupations, the thermal
 * Fock matrix f = h + sum_r n_r <pr||qr>, Omega0, Omega1 (Sec. II.A,
 * App. A-B), truncation sets, the Fermi-scaled integral blocks, the
 * quadrature tensors, and s = 0 at every tau point.
 * FTCC_ERR_INVALID_ARG: beta <= 0 or not finite, mu not finite, ngrid < 3,
 * options out of range or an unknown quadrature.  FTCC_ERR_UNSUPPORTED: an RK
 * quadrature with a precision other than FP64 or with stream_tau. */
ftcc_status ftcc_prepare(ftcc_ctx* ctx, double beta, double mu, int ngrid,
                         ftcc_quadrature quad, const ftcc_options* opt, ftcc_result* out);

/* Apply the discretised amplitude equations (Eq. smu, App. A) to every tau
 * point of the context's batch n_iter times without convergence checks: S
 * kernel (Eqs. ccS1, ccS2), propagation with exp(-Delta (tau_y - tau_x))
 * Simpson weights, E kernel (Eq. E) and Omega_CC (Eq. Ecc).  Requires
 * ftcc_prepare or a solve.  Precision is the prepared one.  `out` (may be
 * NULL) receives the state after the last iteration.  FTCC_ERR_UNSUPPORTED
 * when the prepared quadrature is an RK march (it is not iterated). */
ftcc_status ft_ccsd_iterate(ftcc_ctx* ctx, int n_iter, ftcc_result* out);

/* Full solve: ftcc_prepare, then fixed-point iterations from s = 0 until
 * converged (Alg. 2 run to self-consistency over the whole tau grid),
 * followed by FP64 refinement when the precision is TF32 / BF16X3; with an
 * RK quadrature, the explicit march of Eq. smud instead (ngrid - 1 steps,
 * FP64).  Returns FTCC_ERR_NOT_CONVERGED (with `out` filled) at the
 * iteration cap and FTCC_ERR_DIVERGED on NaN/Inf. */
ftcc_status ft_ccsd_solve(ftcc_ctx* ctx, double beta, double mu, int ngrid,
                          ftcc_quadrature quad, const ftcc_options* opt, ftcc_result* out);

/* Batched solve of n independent instances (one context each, systems
 * already built, same device): beta[i], mu[i] per instance, common ngrid,
 * quadrature and options.  Instances with equal spin-orbital counts (and
 * equal truncation sets) form one batch: every contraction, propagation and
 * reduction of an iteration covers the whole batch in one launch, and one
 * CUDA graph replays the iteration (with block_sparse every instance is a
 * batch of its own).  The batches advance together: fewer than eight each
 * keep one iteration in flight on their own home stream; eight or more,
 * once each has captured its iteration, step as one graph launch holding
 * every unfinished batch's iteration.  out[i] receives instance i.  Returns the first failure
 * (FTCC_ERR_DIVERGED before FTCC_ERR_NOT_CONVERGED); FTCC_ERR_INVALID_ARG for
 * a repeated context, mixed devices, or truncation sets that differ inside a
 * size class.  The batch's memory comes from the allocator of its first
 * context and its work runs on that context's stream. */
ftcc_status ft_ccsd_solve_batched(ftcc_ctx* const* ctx, int n, const double* beta, const double* mu, int ngrid,
                                  ftcc_quadrature quad, const ftcc_options* opt, ftcc_result* out);

/* Prepare the same batches without iterating (s = 0); ft_ccsd_iterate on any
 * member then advances its whole batch. */
ftcc_status ftcc_prepare_batched(ftcc_ctx* const* ctx, int n, const double* beta, const double* mu, int ngrid,
                                 ftcc_quadrature quad, const ftcc_options* opt);

/* Response of the converged solve (Eqs. Lagrangian, lmu, ltilde; App. B).
 * Solves the lambda equations in FP64 (the stationarity of the discrete
 * Lagrangian: the transposed propagation of Eq. ltilde and the transpose of
 * the S kernel, Eq. lmu, iterated from lambda = 0), then differentiates the
 * Lagrangian at fixed (s, lambda): through the Fermi factors and the thermal
 * Fock matrix of every integral block, the propagator (Delta and the grid,
 * both exact for the discrete scheme), and Omega0 + Omega1.  Fills `out`
 * (dOmega/dmu, dOmega/dbeta, N, E, S, trace of the 1-RDM) and, if rdm1 is not
 * NULL, the partially relaxed density p^cc (N*N host doubles, rdm1[q*N + p]
 * pairs with a perturbation X[p][q]; diagonal entries include the orbital
 * energy and occupation response).  A low-precision solve is first refined
 * in FP64, unless the solve's options set mixed_adjoint (then the sweep runs
 * in the mixed arithmetic).  FTCC_ERR_STATE without a converged solve;
 * FTCC_ERR_NOT_CONVERGED when the lambda iteration does not converge. */
ftcc_status ft_ccsd_adjoint(ftcc_ctx* ctx, ftcc_adjoint_result* out, double* rdm1);

/* ft_ccsd_adjoint for n contexts at once (without the 1-RDM): the batches
 * they belong to run their lambda sweeps and responses concurrently, each on
 * its home context's stream from its own host thread (at most as many threads
 * as host cores), the members of one batch one after another.  out[n] and
 * status[n] are caller-owned host arrays; status[i] is what ft_ccsd_adjoint
 * would return for ctx[i].  Returns FTCC_OK when every status is FTCC_OK,
 * else the first failing status in context order; FTCC_ERR_INVALID_ARG for
 * NULL arrays, a NULL context or n < 1 (nothing is run then). */
ftcc_status ft_ccsd_adjoint_batched(ftcc_ctx* const* ctx, int n, ftcc_adjoint_result* out, ftcc_status* status);

/* Unrelaxed normal-ordered two-particle density Gamma_N of the converged
 * solve (App. B), read as the derivative of the CC Lagrangian with respect
 * to the antisymmetrised integrals <pq||rs> that enter the CC equations and
 * the energy through the thermal blocks, at a fixed reference (occupations,
 * Fock matrix, orbital energies), projected onto the symmetries of the real
 * integrals (antisymmetric in (p, q) and in (r, s), symmetric under
 * (pq) <-> (rs)), the part a perturbation can see:
 * dOmega_CC = sum_pqrs Gamma[p][q][r][s] dV[p][q][r][s] for any dV with the
 * symmetries of <pq||rs>.  (The printed blocks
 * of App. B are garbled in places; this is what they are derived from.)
 * gamma: caller-owned host array of N^4 doubles.  Requires ft_ccsd_adjoint on
 * this context (FTCC_ERR_STATE otherwise). */
ftcc_status ftcc_rdm2(ftcc_ctx* ctx, double* gamma);

/* Copy the current amplitudes (FP64, layouts above) to host buffers of
 * ngrid*o*v and ngrid*o*o*v*v doubles (either may be NULL). */
ftcc_status ftcc_get_amplitudes(ftcc_ctx* ctx, double* s1, double* s2);

/* Evaluate the S kernel (Eqs. ccS1, ccS2) of the prepared problem for nx
 * caller amplitude slices.  t1_dev[nx*o*v], t2_dev[nx*o*o*v*v] are FP64
 * device inputs; s1_dev, s2_dev FP64 device outputs of the same shapes.
 * `precision` selects the arithmetic (FP64, TF32 or BF16X3; with
 * block_sparse, TF32 and BF16X3 both run the FP32 block-sparse kernels of the
 * mixed sweep on the inputs rounded to FP32).  Requires ftcc_prepare.  Used to
 * check the contraction schedule element by element. */
ftcc_status ftcc_eval_s(ftcc_ctx* ctx, int nx, int precision, const double* t1_dev,
                        const double* t2_dev, double* s1_dev, double* s2_dev);

/* Propagation with the prepared grid (Eq. smu, App. A) for one amplitude
 * block: s[y][mu] = -sum_x G[y,x] exp(Delta_mu (tau_x - tau_y)) S[x][mu]
 * with Delta from the slot classes `slots` ("ia" or "ijab": hole letters
 * i..n, particle letters a..h).  S_dev, s_dev: FP64 device [ngrid][size]. */
ftcc_status ftcc_propagate(ftcc_ctx* ctx, const char* slots, const double* S_dev, double* s_dev);

/* Vector-Jacobian product of the S kernel (the transpose that the lambda
 * equations, Eqs. lmu/ltilde, apply): t1bar = (dS1/ds1)^T w1 + (dS2/ds1)^T w2,
 * t2bar likewise, at the caller's amplitudes t1_dev/t2_dev for nx tau slices
 * of the prepared single-instance problem, in FP64.  Shapes as ftcc_eval_s;
 * all pointers FP64 device memory (w1/w2 are not modified). */
ftcc_status ftcc_eval_s_vjp(ftcc_ctx* ctx, int nx, const double* t1_dev, const double* t2_dev, const double* w1_dev,
                            const double* w2_dev, double* t1bar_dev, double* t2bar_dev);

/* Transpose of ftcc_propagate: u[x][mu] = sum_y G[y,x] exp(Delta_mu (tau_x - tau_y)) m[y][mu]
 * (the propagation of lambda-tilde in Eq. ltilde, App. A, up to the weights g). */
ftcc_status ftcc_propagate_adjoint(ftcc_ctx* ctx, const char* slots, const double* m_dev, double* u_dev);

/* Copy the converged weighted multipliers m_y = g_y lambda_y / beta of the
 * context's instance (layouts of s1 / s2) after ft_ccsd_adjoint. */
ftcc_status ftcc_get_lambda(ftcc_ctx* ctx, double* m1, double* m2);

/* Per-kernel timing of the iterations of a context's batch.  With enable = 1
 * every launch of an iteration is bracketed by CUDA events (recorded into
 * the per-iteration graph, which is captured again) and ft_ccsd_iterate /
 * ft_ccsd_solve accumulate, per kernel class, the device time, the number of
 * launches and the algorithmic bytes (elements read and written once each)
 * and flops of those launches.  Enabling or disabling resets the sums.
 * ftcc_profile_read fills up to max entries and returns how many.  Classes:
 * "gemm_tc_kernel" (tensor-core contractions), "gemm_simt_kernel" (FP64 and
 * skinny contractions), "layout:pack" (operand packs: permutes, bf16 hi/lo
 * splits, packs over unordered index pairs), "layout:scatter" (GEMM outputs
 * into the intermediates' layouts, block copies, the unpacking of pair-packed
 * results, the P(ij)P(ab) assembly of S2), "propagate_kernel" (Eq. smu and
 * the energy sums), "other" (tau, the remaining elementwise kernels). */
typedef struct {
  char name[32];
  long long launches;
  double ms, bytes, flops;
} ftcc_kernel_stats;
ftcc_status ftcc_profile(ftcc_ctx* ctx, int enable);
int ftcc_profile_read(ftcc_ctx* ctx, ftcc_kernel_stats* out, int max);

/* Dense GEMM on the tensor-core engine, exposed for testing:
 * C[b][m][n] = alpha * sum_k A[b][m][k] * B[b][n][k] (A, B, C FP32 for
 * TF32 / BF16X3, FP64 for FP64; row-major with leading dimensions lda,
 * ldb, ldc; batch strides sa, sb (0 = shared), sc).  lda and ldb must be
 * multiples of 4 elements and the base pointers 16-byte aligned for the
 * tensor-core kinds.  FTCC_ERR_INVALID_ARG otherwise.  When the output tiles
 * cannot fill the SMs the K loop is split over CTAs, with the partial sums
 * in scratch from the context's allocator (at most 64 MiB, released before
 * return) and reduced in a fixed order. */
ftcc_status ftcc_gemm(ftcc_ctx* ctx, int precision, int batch, int M, int N, int K, double alpha,
                      const void* A_dev, long long lda, long long sa,
                      const void* B_dev, long long ldb, long long sb,
                      void* C_dev, long long ldc, long long sc);

/* FP64 GEMM that allocates nothing (no paper counterpart: an engineering
 * entry point).  Same operation and layouts as ftcc_gemm with precision
 * FP64: C[b][m][n] = alpha * sum_k A[b][m][k] * B[b][n][k], all device
 * pointers, issued on `stream` (a cudaStream_t; NULL = legacy stream), no
 * context needed.  The K dimension is split across blocks when the output
 * is small, and the partial sums live in a 16 MiB static device array held
 * by every GPU that loads the library until the process exits; no
 * cudaMalloc, cudaFree or allocating library routine is called.  For callers
 * that cannot allocate device memory where they call it: code running inside
 * a device-memory allocator's own callback (allocating there would re-enter
 * the allocator), or programs that fix their device-memory footprint at
 * start-up and may not grow it afterwards.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the array: calls that overlap on the GPU (different
 *     streams, or different host threads) race and give wrong results.
 *     Every partial sum a call reads was written earlier in the same call,
 *     so nothing in the array has to start at zero.
 *   - batch * M * N must not exceed 2^20 (half the array, so that at least
 *     two K splits fit).  The limit covers every call, including outputs
 *     large enough to run without a K split: larger outputs return
 *     FTCC_ERR_INVALID_ARG.
 * Returns FTCC_ERR_INVALID_ARG for bad sizes or NULL pointers,
 * FTCC_ERR_NO_DEVICE without a GPU, FTCC_ERR_CUDA if a launch fails. */
ftcc_status ftcc_gemm_f64_static(void* stream, int batch, int M, int N, int K, double alpha, const double* A_dev,
                                 long long lda, long long sa, const double* B_dev, long long ldb, long long sb,
                                 double* C_dev, long long ldc, long long sc);

/* Device error flag set by bounded in-kernel waits (0 = none); reading it
 * synchronises the stream and clears it. */
int ftcc_device_error(ftcc_ctx* ctx);

/* Host-side fault injection (no paper counterpart; failure-handling tests):
 * write `code` (> 0) into the context's device error flag, as a bounded
 * device wait that gave up would.  The next entry point that checks the flag
 * (every solve does, before returning) returns FTCC_ERR_TIMEOUT and clears
 * it.  No kernel is made to fault or wait.  FTCC_ERR_INVALID_ARG for a NULL
 * context or code <= 0. */
ftcc_status ftcc_inject_device_error(ftcc_ctx* ctx, int code);

#ifdef __cplusplus
}
#endif
#endif /* FTCC_H */
