/*
 * wd.h -- C ABI of libwd, a B300 (sm_103a) engine for the data-parallel hot
 * path of stochastic trace estimation with the Wilson-Dirac operator:
 * many-right-hand-side Krylov solves with D, torus-colouring probing with
 * spin-colour dilution, and two-level multigrid multilevel Monte Carlo.
 *
 * Paper: "Variance reduction with probing and Multilevel Monte Carlo in
 * Lattice QCD" (Frommer, Jimenez-Merchan, Lang, Papace, Ramirez-Hidalgo).
 * Equations are cited in order of appearance: Eq. 1 noise moments,
 * Eq. 3 Hutchinson estimator, Eq. 4 its variance, Eq. 7 Galerkin coarse
 * operator, Eqs. 9-12 level splitting and the multigrid MLMC estimator,
 * Eqs. 13-14 probing vectors and estimator, Eq. 15 torus colouring,
 * Eq. 21 the disconnected loop O(t).
 *
 * Conventions shared by every entry point
 *   dims[4] = {X, Y, Z, T}; every extent must be even (even-odd ordering).
 *   Site index = x + X*(y + Y*(z + Z*t)).
 *   Gauge field (host, caller owned, read once): complex128 interleaved
 *     [4][T][Z][Y][X][3][3], entry [mu][t][z][y][x][a][b] = U_mu(x)_{ab},
 *     mu = 0..3 <-> x, y, z, t.
 *   Spinor fields (caller owned, DEVICE memory unless stated): complex
 *     interleaved [nrhs][T][Z][Y][X][4][3] (spin before colour),
 *     complex128 for WD_FP64 and complex64 for WD_MIXED_FP32 where a
 *     precision selects the element type; complex128 everywhere else.
 *   Operator (reading of Sec. 1, which fixes only "12x12 blocks on a
 *     nearest-neighbour torus"): Wilson hopping form
 *       D psi(x) = psi(x) - kappa sum_mu [(1-g_mu) U_mu(x) psi(x+mu)
 *                                        + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)]
 *     with Hermitian chiral gammas (g5 = diag(1,1,-1,-1)) and a factor bc[mu]
 *     on hops that wrap around the lattice in direction mu.
 *   All work is queued on the CUDA stream given to wd_create; entry points
 *   that return host results synchronise that stream before returning.
 *   Every entry point returns a wd_status; on failure wd_last_error() gives
 *   a message (thread-local, valid until the next call on that thread).
 *   No entry point is safe to call concurrently on the same context;
 *   different contexts (each with its own stream) may be driven from
 *   different host threads at once.
 *   Launch shapes: the first stencil launch of each (input precision, output
 *   precision, RHS-count bucket) on a context times the kernel's launch-shape
 *   candidates on that context's stream and keeps the fastest.  Work of other
 *   streams running meanwhile distorts that choice, so make the first call of
 *   each shape on an otherwise idle GPU.  WD_NO_AUTOTUNE=1 (read at
 *   wd_create) keeps the default shapes; WD_HOP_R / WD_DD_R pin one.  For a
 *   fixed shape every result is bit-reproducible; shapes whose FP32 sums run
 *   in another order can differ in the last bits.
 */
#ifndef WD_H
#define WD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wd_ctx wd_ctx;

typedef enum {
    WD_OK = 0,
    WD_EINVAL = -1,      /* bad argument (null pointer, odd extent, nrhs < 0, ...) */
    WD_ENOMEM = -2,      /* device or host allocation failed */
    WD_ECUDA = -3,       /* a CUDA call failed (message has the CUDA error string) */
    WD_ENOCONV = -4,     /* a solve hit max_iter; outputs hold the best iterate */
    WD_EBREAKDOWN = -5,  /* Krylov breakdown (rho, omega ~ 0 or non-finite) */
    WD_ETIMEOUT = -6,    /* a bounded device wait ran out */
    WD_ENOTSUP = -7      /* feature not available for these arguments */
} wd_status;

typedef enum {
    WD_FP64 = 0,         /* FP64 storage and arithmetic throughout */
    WD_MIXED_FP32 = 1,   /* FP32 inner Krylov solve inside FP64 defect correction */
    WD_MIXED_BF16 = 2,   /* BF16 storage, FP32 arithmetic inner solve, FP64 outer */
    WD_FP64_DD = 3       /* wd_apply only: FP64 fields, double-float arithmetic */
} wd_prec;

/* trace_estimate methods */
enum { WD_HUTCH = 0, WD_PROBE = 1, WD_MLMC2 = 2, WD_MLMC2_PROBE = 3 };
/* trace_estimate operators B in tr[B D^{-1}(t,t)] */
enum { WD_TR_DINV = 0, WD_TR_G5_DINV = 1 };
/* dilution flags: low byte = spin-colour dilution (1 or 12); OR in
   WD_DIL_TIME to also dilute in time (one timeslice per right-hand side);
   OR in WD_COLOR_3D (with WD_DIL_TIME) to probe with the 3D colouring of
   one timeslice (Eq. 15 with n_D = 3: c(x) = sum_{j<3} sigma_j x_j mod n_c) */
enum { WD_DIL_TIME = 0x100, WD_COLOR_3D = 0x200 };

/* Create a context: uploads the gauge field, folds the boundary factors
 * into the wrap-around links and builds FP64/FP32/BF16 even-odd copies.
 * stream: a cudaStream_t (NULL = legacy default stream).  The context owns
 * every device buffer it allocates; `gauge` is not retained. */
int wd_create(wd_ctx **out, const int dims[4], const double *gauge, double kappa,
              const int bc[4], void *stream);
int wd_destroy(wd_ctx *ctx);

/* y = D x (dagger = 0) or D^dag x (dagger = 1) on nrhs fields (Sec. 1).
 * in/out: device, complex128 for WD_FP64, complex64 for WD_MIXED_FP32
 * (then the stencil runs in FP32); WD_MIXED_BF16 takes complex64 fields,
 * rounds them and the links to BF16 and accumulates in FP32.  WD_FP64_DD
 * takes complex128 fields and computes with pairs of FP32 numbers
 * (double-float: error-free products and sums), agreeing with WD_FP64 to about
 * 2^-44 normwise; inputs below 2^-103 in magnitude count as zero.  It is the
 * stencil of the FP64 steps of the mixed-precision solves. */
int wd_apply(wd_ctx *ctx, const void *in, void *out, int nrhs, int prec, int dagger);

/* x = D^{-1} b for nrhs right-hand sides (the D^{-1} eta products of Sec. 1),
 * even-odd preconditioned BiCGStab.  rhs, x: device complex128.  prec selects
 * the inner arithmetic (WD_FP64, WD_MIXED_FP32, WD_MIXED_BF16); for the mixed
 * modes the outer loop is defect correction on FP64 fields whose stencil steps
 * (source, residuals, odd-site reconstruction) use WD_FP64_DD arithmetic, so
 * tol (relative residual ||b - D x|| / ||b|| per RHS) can be 1e-10 or below;
 * a tol under 1e-12 runs those steps in FP64 arithmetic instead.  iters_out[nrhs] (host, nullable): inner iterations summed
 * over outer steps; true_resid_out[nrhs] (host, nullable): final FP64 relative
 * residual.  Returns WD_ENOCONV if some RHS missed tol within max_iter inner
 * iterations (x still holds the best iterate). */
int wd_solve(wd_ctx *ctx, const double *rhs, double *x, int nrhs, double tol, int prec,
             int max_iter, int *iters_out, double *true_resid_out);

/* Torus colouring (Sec. 3, Eq. 15): smallest n_c and the lexicographically
 * first sigma such that c(x) = sum_j sigma_j x_j mod n_c gives different
 * colours to all sites within torus L1 distance d.  Host only, exact integer
 * search (n_c ascending, sigma lexicographic, sigma_1 most significant).
 * dims[nD] (nD = 3 uses X, Y, Z of a timeslice).  colors (host, nullable):
 * [prod dims] per-site colours, first coordinate fastest.
 * Returns WD_ENOTSUP if no colouring with n_c <= 4096 exists. */
int probe_color(const int *dims, int nD, int d, int *n_colors, int *sigma, int32_t *colors);

/* Stochastic trace estimate of tr[B D^{-1}(t,t)] per timeslice (Eq. 21 for
 * B = g5), B = 1 (WD_TR_DINV) or g5 (WD_TR_G5_DINV).
 *   WD_HUTCH: Eq. 3 with Rademacher vectors (Sec. 1).
 *   WD_PROBE: Eqs. 13-14; vectors are Rademacher on one colour of the
 *             distance-d torus colouring (Eq. 15), times the dilution.
 *   WD_MLMC2: two-level multigrid MLMC (Eqs. 9-12, L = 2); needs wd_mg_setup.
 *             N is the level-1 sample count, n2 the level-2 count.
 *   WD_MLMC2_PROBE: WD_MLMC2 with the level-1 term tr(B M_1) estimated by the
 *             probing x dilution vectors of WD_PROBE (d, dilution) -- the
 *             combination of both methods the paper proposes in its outlook
 *             (Sec. 6); level 2 as WD_MLMC2.  N level-1 samples (each N *
 *             n_c * dilution fine and as many coarse solves), n2 level-2.
 * Noise: entry j of sample i is 1 - 2*(top bit of splitmix64(seed ^ (i<<40) ^ j)),
 * j = 12*site + 3*spin + colour; coarse noise uses sample | 2^23.
 * dilution: 1 or 12, optionally | WD_DIL_TIME.  batch: RHS solved together
 * (0 = automatic).  prec, tol: as wd_solve.
 * Outputs (host): estimate[2*(T+1)] complex mean per timeslice then the total;
 * sample_var[T+1] sample variance sum |X_i - mean|^2 / (N-1) of the per-sample
 * values (for WD_MLMC2 / WD_MLMC2_PROBE: the variance of the two-level
 * estimate itself, s_1^2/N + s_2^2/n2, per timeslice and total);
 * n_solves_out: number of fine plus coarse solves; samples_out (nullable):
 * [N][T][2] per-sample values (the level-1 values for the MLMC methods). */
int trace_estimate(wd_ctx *ctx, int method, int dilution, int N, int n2, int d, uint64_t seed,
                   int op, int prec, int batch, double tol, double *estimate, double *sample_var,
                   int64_t *n_solves_out, double *samples_out);

/* Pseudoscalar correlator from point sources: C(t) = sum_{x in t} sum over the
 * 12 x 12 spin-colour entries |D^{-1}(x; x0)|^2, from the 12 columns of D^{-1}
 * with the source at site x0 = src[4] (x, y, z, t), solved as 12 RHS with the
 * precision / tolerance semantics of wd_solve.  C: host [T], absolute
 * timeslice index.  The connected observable of Sec. 4 at one source, without
 * the multilevel splitting. */
int wd_point_correlator(wd_ctx *ctx, const int src[4], int prec, double tol, double *C);

/* Two-level MLMC with probing on both levels (the combination of the
 * outlook, Sec. 6): level 1 as WD_MLMC2_PROBE (fine probing at distance d
 * with `dilution`); level 2, tr(B P D_c^{-1} P^dag), with probing vectors of
 * the coarse lattice: the coarse noise of each sample (as WD_MLMC2) masked to
 * one colour of the distance-d2 torus colouring of the coarse lattice (d2 = 0:
 * one colour) and, for coarse_dil = 2*nv, to one coarse dof of the site
 * (coarse_dil = 1: none).  N1 fine samples (N1 * n_c * dilution fine and as
 * many coarse solves), N2 coarse samples (N2 * n_c2 * coarse_dil coarse
 * solves).  Outputs as trace_estimate for WD_MLMC2; samples1 [N1][T][2] and
 * samples2 [N2][T][2] (host, nullable) are the level values per sample. */
int trace_estimate_mlmc_probe(wd_ctx *ctx, int dilution, int d, int N1, int coarse_dil, int d2, int N2,
                              uint64_t seed, int op, int prec, int batch, double tol, double *estimate,
                              double *sample_var, int64_t *n_solves_out, double *samples1, double *samples2);

/* Per-sample level values of the last WD_MLMC2 / WD_MLMC2_PROBE estimate:
 * level 2 samples [n2][T][2] (host). */
int wd_mlmc_level2_samples(wd_ctx *ctx, double *samples_out, int n2);

/* Connected pseudoscalar two-point function with the two-level multigrid
 * decomposition (Sec. 4, Eqs. 16-20, L = 2; needs wd_mg_setup):
 * G(t) = (1/T) sum_t' tr[D^{-1}(t+t',t') g5 D^{-1}(t',t+t') g5] = sum_ij G_ij(t)
 * with B_1 = D^{-1} - P D_c^{-1} P^dag and B_2 = P D_c^{-1} P^dag.  Estimated
 * with time-diluted Rademacher noise eta on each source timeslice t' and
 * y_k = B_k eta: sample_ij(t) = (1/T) sum_t' sum_{x in t+t'} y_j(x)^dag y_i(x).
 * Level 1: N1 samples (noise samples 0..N1-1; T fine and T coarse solves
 * each) give (1,1), (1,2), (2,1); the (2,2) term takes N2 samples of its own
 * (noise samples i | 2^21; T coarse solves each).  N1, N2 >= 2.  The (2,2)
 * term on the level-1 noise also gives the plain (undecomposed) estimator
 * |y_1 + y_2|^2 on the same samples, for comparison.
 * Outputs (host): G[6][T][2] complex means of (1,1), (1,2), (2,1), (2,2), the
 * total and the plain estimator; var[6][T] variances of those means (total:
 * var of the level-1 sum / N1 + var(2,2) / N2); samples1 (nullable)
 * [N1][4][T][2] ((1,1), (1,2), (2,1), (2,2) on the level-1 noise);
 * samples2 (nullable) [N2][T][2]; n_solves_out (nullable): fine + coarse
 * solves.  prec, tol, batch as trace_estimate. */
int wd_connected_mlmc(wd_ctx *ctx, int N1, int N2, uint64_t seed, int prec, double tol, int batch, double *G,
                      double *var, double *samples1, double *samples2, int64_t *n_solves_out);

/* ---- third multigrid level (Sec. 2 with L = 3) ----------------------- */

/* Aggregates the coarse lattice of wd_mg_setup again (agg2[4] coarse sites per
 * direction, dividing the coarse extents) and builds P_2 (level-2 test vectors
 * restricted to each level-3 aggregate and chirality half, orthonormalised by
 * modified Gram-Schmidt in test-vector order) and D_3 = P_2^dag D_c P_2 (Eq. 7
 * with l = 2), a 9-point block stencil with 2 nv2 dofs per level-3 site.
 * tv2 (host, nullable): [nv2][Vc][2 nv] complex level-2 test vectors; NULL
 * builds them by tv_iters inverse iterations with the coarse solver from
 * random coarse vectors (seed).  nv2: positive multiple of 6.  wd_mg_setup
 * discards the third level. */
int wd_mg3_setup(wd_ctx *ctx, const double *tv2, int nv2, const int agg2[4], int tv_iters, uint64_t seed);
/* y = D_3 x on level-3 vectors [nrhs][Vcc][2 nv2] (device complex128, FP64). */
int wd_coarse3_apply(wd_ctx *ctx, const double *in, double *out, int nrhs);
/* y3 = P_2^dag y2 and y2 = P_2 y3 (device complex128; level-2 vectors
 * [nrhs][Vc][2 nv], level-3 vectors [nrhs][Vcc][2 nv2]). */
int wd_restrict2(wd_ctx *ctx, const double *y2, double *y3, int nrhs);
int wd_prolong2(wd_ctx *ctx, const double *y3, double *y2, int nrhs);
/* Three-level MLMC estimate of tr[B D^{-1}(t,t)] (Eq. 12 with L = 3):
 *   X_1 = eta^dag B (D^{-1} - P_1 D_2^{-1} P_1^dag) eta              (N1 fine noise samples),
 *   X_2 = (P_1 xi)^dag B P_1 (D_2^{-1} - P_2 D_3^{-1} P_2^dag) xi     (N2 coarse samples | 2^23),
 *   X_3 = (P_1 P_2 zeta)^dag B P_1 P_2 D_3^{-1} zeta                 (N3 level-3 samples | 2^24).
 * Level-3 solves run in FP64 to min(tol, 1e-12).  Outputs as trace_estimate
 * for WD_MLMC2 (variance: sum_l s_l^2 / N_l); samples1..3 (host, nullable)
 * [N_l][T][2].  N1, N2, N3 >= 2. */
int trace_estimate_mlmc3(wd_ctx *ctx, int N1, int N2, int N3, uint64_t seed, int op, int prec, int batch,
                         double tol, double *estimate, double *sample_var, int64_t *n_solves_out,
                         double *samples1, double *samples2, double *samples3);

/* Samples per level of a multilevel estimator (Sec. 2, Eq. 6): the N_l that
 * minimise the total cost sum_l N_l C_l for a target variance eps^2 of the
 * estimate, N_l = eps^-2 sqrt(V_l / C_l) sum_i sqrt(V_i C_i), rounded up (at
 * least 1), so that sum_l V_l / N_l <= eps^2.  V[L]: per-sample variance of
 * level l (>= 0), C[L]: cost of one level-l sample (> 0), eps > 0; N_out[L]
 * (host).  Host only.  WD_EINVAL for bad arguments or a count beyond 2^62. */
int mlmc_allocate(int L, const double *V, const double *C, double eps, int64_t *N_out);

const char *wd_last_error(void);

/* ---- multigrid (Sec. 2) ---------------------------------------------- */

/* Build the aggregation prolongator P and D_c = P^dag D P (Eq. 7).
 * tv: host complex128 [nv][T][Z][Y][X][4][3] test vectors (nullable: then
 * nv vectors are generated on the GPU as wd_mg_test_vectors does).
 * agg[4]: aggregate extents (must divide dims).  Each test vector is restricted
 * to each aggregate and chirality half (spins {0,1} / {2,3}) and
 * orthonormalised by modified Gram-Schmidt in test-vector order; coarse dof
 * index = 2*nv*Xc + nv*h + k.  Requires nv a positive multiple of 6 with
 * nv <= 6 * prod(agg) (else WD_EINVAL); WD_ENOTSUP when the 2nv x 2nv blocks
 * exceed the assembly kernel's shared memory. */
int wd_mg_setup(wd_ctx *ctx, const double *tv, int nv, const int agg[4], int tv_iters,
                uint64_t seed);

/* The test vectors wd_mg_setup(tv = NULL) builds (Sec. 2: the near-null space
 * that P is built from; the paper takes the setup from DD-alpha-AMG): start k
 * (k < nv) is the Rademacher vector of noise sample 2^22 + k of `seed` (the
 * generator of trace_estimate), and each of `iters` inverse iterations
 * replaces v by x / ||x|| with x = D^{-1} v from a mixed-precision solve to a
 * relative residual of 1e-6 (norm over the whole lattice).  tv_out: device
 * complex128 [nv][T][Z][Y][X][4][3], owned by the caller.  WD_EINVAL for
 * nv < 1, iters < 0 or a null pointer. */
int wd_mg_test_vectors(wd_ctx *ctx, int nv, int iters, uint64_t seed, double *tv_out);

/* y_c = D_c x_c on the coarse lattice: device complex128 [nrhs][Vc][2nv].
 * prec WD_FP64 uses FP64 blocks.  The mixed precisions run the 9-point block
 * stencil on the tensor cores (2nv in {48, 96}; FP32 accumulate): WD_MIXED_BF16
 * with the blocks and x rounded to BF16 (~2^-8 per product), WD_MIXED_FP32
 * with both as BF16 pairs hi + lo (~2^-16 per product, the operator of the
 * mixed coarse solves).  Other shapes take the FP32 blocks on the CUDA cores. */
int wd_coarse_apply(wd_ctx *ctx, const double *in, double *out, int nrhs, int prec);

/* Restriction P^dag and prolongation P: fine device complex128
 * [nrhs][T][Z][Y][X][4][3] <-> coarse [nrhs][Vc][2nv]. */
int wd_restrict(wd_ctx *ctx, const double *fine, double *coarse, int nrhs);
int wd_prolong(wd_ctx *ctx, const double *coarse, double *fine, int nrhs);

/* x_c = D_c^{-1} b_c (coarse BiCGStab; FP64 defect correction around a
 * mixed inner solve when prec != WD_FP64).  Device complex128 [nrhs][Vc][2nv]. */
int wd_coarse_solve(wd_ctx *ctx, const double *b, double *x, int nrhs, double tol, int prec,
                    int max_iter, double *true_resid_out);

/* ---- adjoint (derivatives of the estimates) -------------------------- */

/* Link force of X = sum_i w_i^dag ... : for device complex128 fields w, z
 * [nrhs][T][Z][Y][X][4][3] writes (device, complex128) G and H, each
 * [4][T][Z][Y][X][3][3], summed over the nrhs fields:
 *   G_mu(x) = kappa b sum_s z(x+mu)_s [(1-g_mu) w(x)]_s^dag
 *   H_mu(x) = kappa b sum_s [(1+g_mu) w(x+mu)]_s z(x)_s^dag
 * (b = bc[mu] on wrapping links, else 1), so that for U -> U + h Delta
 *   d/dh sum_i (-w_i^dag dD z_i) = sum tr(Delta G) + conj(tr(Delta H)).
 * accumulate = 1 adds to G, H instead of overwriting. */
int wd_link_force(wd_ctx *ctx, const double *w, const double *z, int nrhs, double *G, double *H,
                  int accumulate);

/* Derivatives of the estimate of L = Re sum_t weights[t] * mean_i X_i(t) for
 * the Hutchinson / probing estimators of trace_estimate (same method,
 * dilution, N, d, seed, op, prec, batch, tol; weights host [T], nullable =
 * all ones).  Writes dkappa (host) and the link force G, H (device complex128
 * [4][T][Z][Y][X][3][3], overwritten) so that for U -> U + h Delta,
 * dL/dh = Re sum tr(Delta (G + H)); i.e. the gradient in PyTorch's convention
 * is (G + H)^dagger per link.  One extra solve per RHS unless op = g5 with
 * equal weights (then w = g5 z by gamma5-hermiticity). */
int trace_gradient(wd_ctx *ctx, int method, int dilution, int N, int d, uint64_t seed, int op, int prec,
                   int batch, double tol, const double *weights, double *dkappa, double *G, double *H);

/* Replace the links / kappa of an existing context (same dims and bc).
 * gauge: host or device pointer (unified addressing), layout as wd_create. */
int wd_update_gauge(wd_ctx *ctx, const double *gauge, double kappa);

/* ---- batched solves over several lattices ------------------------------ */

typedef struct wd_batch wd_batch;

/* Group 1..8 contexts (lattices of any even extents, distinct contexts) that
 * were created on the same CUDA stream. */
int wd_batch_create(wd_batch **out, wd_ctx *const *ctxs, int n);
int wd_batch_destroy(wd_batch *b);

/* Solve D_j x_j = b_j for every lattice j of the batch in lockstep, mixed
 * precision only (WD_MIXED_FP32 or WD_MIXED_BF16 inner, FP64 defect
 * correction).  Each inner BiCGStab iteration applies all lattices' even-odd
 * operators with two persistent batched stencil launches (one static work
 * list over all lattices' site and RHS tiles).  use_graph = 1 captures the
 * inner iterations between convergence checks into a CUDA graph and replays
 * it.  rhs[j], x[j]: device complex128 [nrhs[j]][T][Z][Y][X][4][3] of lattice j.
 * iters_out (host, nullable) [n]: inner iterations of the slowest RHS per
 * lattice; resid_out (host, nullable) [sum nrhs]: final FP64 relative residual
 * ||b - D x|| / ||b|| per RHS (the even-site Schur residual, which equals the
 * full residual since the odd sites are reconstructed exactly). */
int wd_batch_solve(wd_batch *b, const double *const *rhs, double *const *x, const int *nrhs, double tol, int prec,
                   int max_iter, int use_graph, int *iters_out, double *resid_out);

/* ---- allocation-free variant ------------------------------------------ */

/* The paper has no counterpart to this entry point.
 * Same result as wd_apply (same arguments, same layouts; precisions WD_FP64,
 * WD_MIXED_FP32 and WD_MIXED_BF16), but
 * the call allocates no memory: for callers that cannot allocate device memory
 * while running -- services that reserve their whole device-memory budget at
 * start-up, and frameworks whose caching allocator must own every byte of
 * device memory.  The even-odd staging fields live in one static device array
 * of 64 MiB per GPU; a call needing more staging (2 input + 2 output
 * half-fields for nrhs fields; e.g. FP64: 384 bytes per site and right-hand
 * side) is rejected with WD_EINVAL.  The array comes into being on a GPU when
 * the first context is created there: wd_create (which allocates anyway)
 * loads the code that holds it and resolves its address, with the context's
 * device current, and the array then stays until the process exits.  A call
 * stages on its context's device whichever device is current.  All calls on
 * one GPU share the array and leave its contents behind: calls whose work
 * overlaps on the GPU (other streams, other host threads) race on it. */
int wd_apply_noalloc(wd_ctx *ctx, const void *in, void *out, int nrhs, int prec, int dagger);

/* ---- instrumentation ------------------------------------------------- */

/* Kernel timing with CUDA events on the context stream.  kernel ids:
   WD_K_HOP fine stencil in FP32/BF16 storage, WD_K_HOP64 fine stencil in FP64,
   WD_K_COARSE coarse block stencil, WD_K_FORCE link force, WD_K_BLAS unused. */
enum { WD_K_HOP = 0, WD_K_BLAS = 1, WD_K_COARSE = 2, WD_K_FORCE = 3, WD_K_HOP64 = 4, WD_K_COUNT = 5 };
int wd_profile(wd_ctx *ctx, int enable);            /* 1 = start (clears), 0 = stop */
/* launches, summed event time (ms) and summed algorithmic bytes (or flops for
   WD_K_COARSE) of the launches of one kernel family since wd_profile(ctx, 1). */
int wd_profile_get(wd_ctx *ctx, int kernel, int64_t *launches, double *ms, double *bytes);
/* Number of kernels this context launched since creation (all families). */
int64_t wd_launch_count(wd_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* WD_H */
