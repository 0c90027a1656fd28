/*
 * laph.h -- C ABI of the GB300 (sm_103a) stochastic-LapH quark-line library.
 *
 * The library computes, on one GPU, the four steps of the stochastic LapH
 * method of Morningstar et al., "Improved stochastic estimation of quark
 * propagation with Laplacian Heaviside smearing in lattice QCD"
 * (arXiv:1104.3870):
 *   (a) the lowest N_v eigenpairs of the 3D gauge-covariant Laplacian on every
 *       time slice (Sec. II, Laplacian and LapH smearing; Sec. IV, KSRL with
 *       Chebyshev acceleration)                                   laph_eigvecs
 *   (b) Z4 noise in the LapH subspace, diluted sources
 *       varrho = V_s P^(b) rho (Sec. II, Eq. (varrhodef); Sec. IV noise)
 *                                                            laph_make_sources
 *   (c) solves of Omega x = y, Omega = gamma_4 K, for every diluted source
 *       (Sec. II quark line; Sec. IV solver)               dirac_solve_batch
 *   (d) sink coefficients V_s^dag x (Sec. IV) and meson / two-pion
 *       correlators (Sec. III, Eqs. (mesonfunc), (mesoncorr))  laph_sinks,
 *                                                                 correlate
 * plus the gauge preparation (stout smearing, Sec. II) in laph_stout_smear.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  * Every array argument is a plain pointer to caller-owned memory, either
 *    device memory of the context's GPU or host memory (pageable or pinned);
 *    the library detects which with cudaPointerGetAttributes and stages host
 *    arrays through its own device workspace.  The library never frees or
 *    retains caller memory past the call.
 *  * Complex numbers are interleaved (re, im) doubles ("c128").
 *  * Sites are ordered lexicographically with x fastest:
 *      site = ((t * ns + z) * ns + y) * ns + x,  V3 = ns^3, V = V3 * nt.
 *    Gauge links:   [V][mu = x,y,z,t][3][3]  c128 (row index first).
 *    Spinor fields: [V][spin 4][colour 3]    c128.
 *    Eigenvectors:  [nt][nv][V3][colour 3]   c128 (orthonormal per slice).
 *    Z4 noise:      uint8 code v[nt][spin 4][nv], rho = i^v.
 *    Coefficients:  [nrhs][nt][spin 4][nv]   c128.
 *  * Dirac matrices are in the chiral basis (gamma_5 = diag(1,1,-1,-1)).
 *  * ns and nt must be even (even-odd ordering); ns >= 2, nt >= 2.
 *  * Calls are issued on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream).  A call returns after its work is queued unless it writes host
 *    memory or a report, in which case it synchronises `stream` first; the
 *    eigensolver and the solvers also synchronise `stream` for their
 *    host-side convergence checks.  Nothing is issued on any other stream.
 *  * A context (its workspace and autotune cache) serves one host thread at a
 *    time; separate contexts may run concurrently on separate streams of the
 *    same GPU (the measurement helpers below are shared and thread-safe).
 *  * Return value: LAPH_OK or an error code; laph_last_error() then gives a
 *    message (thread-local).  No C++ exception crosses the ABI.
 */
#ifndef LAPH_H
#define LAPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LAPH_OK = 0,
    LAPH_ERR_ARG = 1,            /* invalid argument (sizes, dilution, pointers)      */
    LAPH_ERR_CUDA = 2,           /* a CUDA runtime call failed                         */
    LAPH_ERR_NOT_CONVERGED = 3,  /* outputs written but above tolerance (see report)   */
    LAPH_ERR_TIMEOUT = 4,        /* a bounded device wait gave up                      */
    LAPH_ERR_NOMEM = 5           /* workspace allocation failed                        */
};

typedef struct laph_ctx laph_ctx;

typedef struct {
    int ns;        /* spatial extent L (lattice L^3 x nt), even */
    int nt;        /* temporal extent, even                      */
    double xi;     /* anisotropy a_s / a_t                        */
} laph_lattice;

/* Creates a context on CUDA device `device` (workspace, autotune cache). */
int laph_ctx_create(int device, laph_ctx **out);
void laph_ctx_destroy(laph_ctx *ctx);
/* Message of the last error on this thread ("" if none). */
const char *laph_last_error(void);
/* Library version string. */
const char *laph_version(void);

/* Measurement helpers (not part of the paper's method).
 * laph_launch_count: number of kernels the library has launched so far.
 * laph_profile_enable(level): 0 off; 1 time every Dirac-stencil launch with
 *   CUDA events on its stream; 2 time every instrumented kernel family.
 * laph_profile_read: launches, total milliseconds, algorithmic bytes and
 *   flops accumulated for one family (e.g. "dslash_fp32"); synchronises on
 *   the recorded events.  laph_profile_families writes the comma-separated
 *   family names into buf (returns the full length).  laph_profile_reset
 *   clears the table. */
long laph_launch_count(void);
void laph_profile_enable(int level);
void laph_profile_reset(void);
int laph_profile_families(char *buf, int len);
int laph_profile_read(const char *family, long *launches, double *ms, double *bytes, double *flops);

/* ------------------------------------------------------------------------
 * Gauge preparation: stout smearing (Sec. II: spatial links smeared with
 * the stout recipe, only spatial staples, temporal links not smeared).
 *   links        [V][4][3][3] c128, smeared in place.
 *   rho          staple weight (0.1 in the paper).
 *   nsteps       number of stout steps.
 *   spatial_only 1: staples and updates over spatial directions only (the
 *                paper's 3D smearing); 0: all four directions (4D).
 * Each step computes C_mu = rho sum_{nu != mu} staples, Omega = C_mu U_mu^dag,
 * Q = (i/2)(Omega^dag - Omega) - (i/6) Tr(Omega^dag - Omega),
 * U_mu <- exp(iQ) U_mu for all links at once.  Errors: LAPH_ERR_ARG for bad
 * sizes or a null pointer.
 * ------------------------------------------------------------------------ */
int laph_stout_smear(laph_ctx *ctx, const laph_lattice *lat, void *links, double rho,
                     int nsteps, int spatial_only, void *stream);

/* ------------------------------------------------------------------------
 * (a) Laplacian eigenvectors (Sec. II: V_s holds the eigenvectors of the N_v
 * lowest eigenvalues of -Delta on each time slice; Sec. IV: Krylov-spectral
 * restarted Lanczos with Chebyshev acceleration A = T_n(B),
 * B = 1 + 2 (Delta + lambda_C)/(lambda_L - lambda_C), full
 * reorthogonalisation repeated while the norm drops by 1/sqrt(2), at most 4).
 *   links3d  [V][4][3][3] c128: stout-smeared links (slots x,y,z used).
 *   nv       number of eigenpairs per slice, 1 <= nv <= 3 V3 / 2.
 *   evals    [nt][nv] doubles, ascending eigenvalues of -Delta.
 *   evecs    [nt][nv][V3][3] c128; each vector has the phase convention
 *            applied: its largest-modulus component (the first in storage
 *            order among those within a relative 1e-8 of the largest) is real
 *            and positive.
 *   params   NULL for defaults (lambda_L = 15, lambda_C chosen per slice from a
 *            short Lanczos run refined by one filtered cycle: 1.5 times the
 *            largest Rayleigh quotient of the wanted Ritz vectors plus 0.02,
 *            raised until the filter's gain over the wanted range is <= 1e3;
 *            Chebyshev order 16, Krylov dimension
 *            max(2 nv + 16, nv + 32), tolerance 1e-13 on ||(-Delta) v - lambda v||
 *            relative to ||-Delta|| <= 12, at most 50 restarts).
 *   report   optional (may be NULL).
 * Returns LAPH_ERR_NOT_CONVERGED (outputs still written) if some pair misses
 * the tolerance after max_restarts.
 * ------------------------------------------------------------------------ */
typedef struct {
    double lambda_L;      /* upper bound of the spectrum of -Delta (<= 0: 15)     */
    double lambda_C;      /* cutoff mapped to 1 (<= 0: automatic)                 */
    int cheb_order;       /* n of T_n (<= 0: 16)                                  */
    int krylov_dim;       /* Krylov space dimension m (<= 0: automatic)           */
    int max_restarts;     /* (<= 0: 50)                                           */
    double tol;           /* residual tolerance relative to 12 (<= 0: 1e-13)      */
    uint64_t seed;        /* start vector seed (0: the all-equal start vector)    */
} laph_eig_params;

typedef struct {
    int restarts;         /* restarts performed                                   */
    int matvecs;          /* Laplacian applications per slice                     */
    int nconv;            /* minimum over slices of converged pairs               */
    double max_resid;     /* max over slices/pairs of ||Lv - lambda v||           */
    double lambda_C;      /* cutoff used                                          */
} laph_eig_report;

int laph_eigvecs(laph_ctx *ctx, const laph_lattice *lat, const void *links3d, int nv,
                 const laph_eig_params *params, double *evals, void *evecs,
                 laph_eig_report *report, void *stream);

/* ------------------------------------------------------------------------
 * (b) Z4 noise and diluted sources (Sec. II, Eq. (varrhodef) with D = 1 and
 * the dilution projectors P^(b) = P_T (x) P_S (x) P_L; Sec. IV noise).
 * Noise: rho(t, alpha, n) = i^v with v the low two bits of word 0 of
 * Philox4x32-10(counter = ((t*4 + alpha)*nv + n, 0, 0, 0),
 *               key = ((config_id << 16) | noise_id, 0x4C415048)).
 * Dilution type codes per index space (N = nt, 4, nv): 0 none (1 projector),
 * 1 full (N), 2 block-J (J; P^(b)_ii = [floor(J i / N) == b]),
 * 3 interlace-J (J; P^(b)_ii = [i mod J == b]); N must be divisible by J.
 * Flat projector index b = (b_T * n_S + b_S) * n_L + b_L.
 *   b_list   nb projector indices to build (host or device int array).
 *   rhs      [nb][V][4][3] c128 output: gamma_4 V_s P^(b) rho, i.e. the
 *            right-hand side of K x = gamma_4 y for Omega x = y.
 *   noise    optional [nt][4][nv] uint8 output of the codes v (may be NULL).
 * Errors: LAPH_ERR_ARG for a bad dilution (J not dividing N) or b out of range.
 * ------------------------------------------------------------------------ */
typedef struct { int type; int J; } laph_dil1;
typedef struct { laph_dil1 T, S, L; } laph_dilution;

int laph_make_sources(laph_ctx *ctx, const laph_lattice *lat, const void *evecs, int nv,
                      uint16_t noise_id, uint16_t config_id, const laph_dilution *dil,
                      const int *b_list, int nb, void *rhs, uint8_t *noise, void *stream);

/* ------------------------------------------------------------------------
 * (c) Solves of K x = b for nrhs right-hand sides (Sec. II: Omega = gamma_4 K;
 * Sec. IV: even-odd preconditioned BiCGStab, CG on the normal equations
 * when it fails).  K is the anisotropic Wilson-clover matrix
 *   K psi(x) = (m0 + 3/xi + 1) psi(x)
 *     - 1/2 sum_mu w_mu [(1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)]
 *     - (c_sw/2) sum_{mu<nu} w_{mu nu} sigma_{mu nu} F_{mu nu}(x) psi(x),
 * w = 1/xi (space), 1 (time); w_{k4} = (1 + 1/xi)/2, w_{jk} = 1/xi; F the
 * traceless clover-leaf field strength; sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu];
 * periodic in space, antiperiodic in time for the fermion.
 *   links  [V][4][3][3] c128 (the Dirac links, not the 3D-smeared ones).
 *   rhs    [nrhs][V][4][3] c128 right-hand sides b.
 *   sol    [nrhs][V][4][3] c128 solutions x (written).
 *   params solver choice; NULL = MIXED_FP32, tol 1e-10.
 *   report optional [nrhs] array.
 * Convergence is judged by the FP64 true residual ||b - K x|| / ||b|| on the
 * full (not even-odd) operator.  Modes:
 *   LAPH_SOLVE_PLAIN_FP64  FP64 even-odd BiCGStab, rhs_block RHS per launch
 *                          (rhs_block = 1 is the one-at-a-time baseline).
 *   LAPH_SOLVE_MIXED_FP32  FP64 defect correction around FP32 even-odd
 *                          BiCGStab, all RHS of a block in one launch.
 *   LAPH_SOLVE_MIXED_BF16  the same defect correction around an inner BiCGStab whose
 *                          spinors and Krylov vectors are stored in BF16 (FP32
 *                          arithmetic, FP32 links, clover and iterate; default
 *                          inner_tol 1e-2); blocks of 32, 64, 128 or 256 RHS, a
 *                          block of another size runs the FP32 inner solver.
 *   LAPH_SOLVE_LEARNED     FP64 defect correction around FP32 flexible GCR
 *                          with the learned right preconditioner `weights`
 *                          (layout of laph_precond_train).
 * Sec. IV: where BiCGStab does not converge, a CG solve of the normal
 * equations finishes the system.  Here (params->fallback nonzero, PLAIN and
 * MIXED modes) a right-hand side still above tol when the inner budget
 * (maxiter) or 100 defect-correction cycles are spent, or whose true residual
 * fell by less than 2x in each of three consecutive cycles, is finished by
 * FP64 CG on K^dag K e = K^dag r (K^dag = gamma_5 K gamma_5); report[i].iters
 * then includes the CG iterations and report[i].fallback_used = 1.  In
 * LEARNED mode a stalled flexible-GCR cycle hands the right-hand side to the
 * MIXED solver instead (fallback_used = 1).
 * ------------------------------------------------------------------------ */
enum {
    LAPH_SOLVE_PLAIN_FP64 = 0,
    LAPH_SOLVE_MIXED_FP32 = 1,
    LAPH_SOLVE_MIXED_BF16 = 2,
    LAPH_SOLVE_LEARNED = 3
};

typedef struct {
    double m0;    /* bare mass                */
    double csw;   /* clover coefficient       */
} laph_dirac_params;

typedef struct {
    double tol;            /* FP64 true relative residual target (<= 0: 1e-10)     */
    int maxiter;           /* total inner iterations per RHS (<= 0: 100000)        */
    int mode;              /* LAPH_SOLVE_*                                          */
    int rhs_block;         /* RHS per launch (<= 0: PLAIN 1, LEARNED min(nrhs, 64),
                              MIXED autotuned, see laph_tuned_block)                */
    double inner_tol;      /* inner relative tolerance per cycle (<= 0: 3e-4)      */
    int fallback;          /* 1: finish stalled RHS with the fallback solver        */
    const float *weights;  /* LEARNED only: preconditioner weights (device/host)   */
    int gcr_restart;       /* LEARNED only: FGCR restart length (<= 0: 16)         */
    int check_every;       /* iterations between host convergence checks (<= 0: 5) */
} laph_solver_params;

typedef struct {
    int iters;             /* inner iterations (Schur-operator applications / 2)   */
    int outer;             /* defect-correction cycles                              */
    int status;            /* LAPH_OK or LAPH_ERR_NOT_CONVERGED                     */
    int fallback_used;     /* 1 if the fallback solver ran for this RHS            */
    double true_resid;     /* final ||b - K x|| / ||b|| in FP64                     */
} laph_solve_report;

int dirac_solve_batch(laph_ctx *ctx, const laph_lattice *lat, const void *links,
                      const laph_dirac_params *dirac, const void *rhs, void *sol, int nrhs,
                      const laph_solver_params *params, laph_solve_report *report, void *stream);

/* RHS block the mixed solver's autotuner chose for a lattice of vh = V/2 sites, where nmax is
 * the largest candidate block that fitted (16, 32, 64 or 128, at most nrhs); 0 if no mixed
 * solve with rhs_block <= 0 has needed it in this context yet.  The tuner times t = M s with
 * the inner products <t, s>, <t, t> (the solver's own kernels) at each candidate on scratch
 * fields once and keeps the block with the lowest time per right-hand side (ties within 3 %
 * go to the larger block). */
int laph_tuned_block(laph_ctx *ctx, int vh, int nmax);

/* ------------------------------------------------------------------------
 * Learned preconditioner for LAPH_SOLVE_LEARNED (the paper has no learned
 * component; the network is this library's addition).  A linear,
 * gauge-covariant network of 4 layers with 1 -> 4 -> 4 -> 4 -> 1 complex
 * channels:
 *   out_c(x) = sum_{c'} sum_{d=0..8} W[d][c][c'] (T_d in_{c'})(x),
 *   T_0 = 1, T_{1+mu} psi(x) = s U_mu(x) psi(x+mu), T_{5+mu} psi(x) = s U_mu(x-mu)^dag psi(x-mu),
 * s = -1 for hops across the time boundary; W[d][c][c'] is a 4x4 complex
 * spin matrix acting as the identity on colour (so N(G psi; U^G) = G N(psi; U)).
 * Weights: float array of laph_precond_size() entries, layers in order, each
 * [9][c_out][c_in][4][4] complex as (re, im).  Training minimises
 * (1/B) sum_i ||N(rho_i) - phi_i||^2 / ||phi_i||^2 over pairs with K phi_i = rho_i
 * (Adam on the real and imaginary parts, FP32 network, FP64 gradient sums).
 * All arrays may be host or device memory; rho/phi are [npairs][V][4][3] c128.
 * ------------------------------------------------------------------------ */
int laph_precond_size(void);
/* Seeded start: channel 0 carries the identity (1/diag in the last layer), other weights small. */
int laph_precond_init(uint64_t seed, double diag, float *weights);
/* epochs over the pairs in batches of `batch`; weights and adam ([2][size] floats,
 * first then second moments, zero at the start) are updated in place; step0 counts
 * the Adam steps already taken; loss (optional) receives the mean batch loss. */
int laph_precond_train(laph_ctx *ctx, const laph_lattice *lat, const void *links, const laph_dirac_params *dirac,
                       const void *rho, const void *phi, int npairs, int epochs, int batch, double lr, int step0,
                       float *weights, float *adam, double *loss, void *stream);
/* Loss over all pairs (one batch, npairs <= 256) and its gradient dL/d conj(W) as c128
 * in the weight layout. */
int laph_precond_grad(laph_ctx *ctx, const laph_lattice *lat, const void *links, const laph_dirac_params *dirac,
                      const float *weights, const void *rho, const void *phi, int npairs, double *loss, void *grad,
                      void *stream);
/* out = N(in) for nrhs fields (c128). */
int laph_precond_apply(laph_ctx *ctx, const laph_lattice *lat, const void *links, const laph_dirac_params *dirac,
                       const float *weights, const void *in, void *out, int nrhs, void *stream);
/* The same network with its layers on the tensor cores (tcgen05; transported inputs and
 * weights rounded to BF16, FP32 accumulation), as the learned solver applies it inside FGCR
 * (LAPH_NN_FP32=1 in the environment keeps that solver on the FP32 layers).  nrhs a multiple
 * of 32 (LAPH_ERR_ARG otherwise). */
int laph_precond_apply_tc(laph_ctx *ctx, const laph_lattice *lat, const void *links, const laph_dirac_params *dirac,
                          const float *weights, const void *in, void *out, int nrhs, void *stream);

/* Applies K (FP64) to nrhs fields: out = K in (layouts as dirac_solve_batch). */
int laph_dirac_apply(laph_ctx *ctx, const laph_lattice *lat, const void *links,
                     const laph_dirac_params *dirac, const void *in, void *out, int nrhs,
                     void *stream);

/* One even-odd hopping call with its fused site term, on half-lattice fields (the
 * even-odd splitting of K used by the solvers, Sec. II; D = -1/2 sum_mu w_mu [...] as in
 * laph_dirac_apply).  For output parity p (0 even, 1 odd) and q = 1 - p:
 *   LAPH_HOP_CLOVINV       out = A_pp^{-1} D_pq in
 *   LAPH_HOP_CLOVINV_XPAY  out = z - A_pp^{-1} D_pq in
 *   LAPH_HOP_APPLY         out = A_pp z + D_pq in      (= (K x)_p with x_p = z, x_q = in)
 * Half-lattice layout: [cb][spin*3 + colour][nrhs] complex, where cb = (lexicographic
 * site index) / 2 runs over the Vh = V/2 sites of the field's parity and the right-hand
 * side index is innermost.  precision LAPH_PREC_FP64: c128 fields, the FP64 kernel;
 * LAPH_PREC_FP32: c64 fields, the packed-FP32 kernel of the mixed solver (links and
 * clover rounded to FP32); LAPH_PREC_BF16: fields of bfloat16 pairs (re, im), the same kernel
 * reading and writing BF16 spinors with FP32 links, clover and arithmetic (the inner operator of
 * LAPH_SOLVE_MIXED_BF16; nrhs 32, 64, 128 or 256).  `z` may be NULL for LAPH_HOP_CLOVINV.  Host or device
 * pointers; links [V][4][3][3] c128.  Returns after the stream has drained, so that a
 * copy wait that gave up is reported (LAPH_ERR_TIMEOUT).  Errors: LAPH_ERR_ARG for a bad parity, mode or
 * precision, nrhs < 1 or a missing pointer. */
enum { LAPH_HOP_CLOVINV = 0, LAPH_HOP_CLOVINV_XPAY = 1, LAPH_HOP_APPLY = 2 };
enum { LAPH_PREC_FP64 = 0, LAPH_PREC_FP32 = 1, LAPH_PREC_BF16 = 2 };
int laph_dslash_eo(laph_ctx *ctx, const laph_lattice *lat, const void *links, const laph_dirac_params *dirac,
                   int parity, int mode, int precision, const void *in, const void *z, void *out, int nrhs,
                   void *stream);

/* ------------------------------------------------------------------------
 * (d) Sink coefficients (Sec. IV: the quark-propagation coefficients
 * V_s^dag Omega^{-1} V_s P^(b) rho, N_t N_v per spin):
 *   coef[i][t][alpha][n] = sum_{x in slice t, c} conj(V(t,n,x,c)) sol[i](t,x,alpha,c)
 *   evecs [nt][nv][V3][3], sol [nrhs][V][4][3], coef [nrhs][nt][4][nv], all c128.
 * ------------------------------------------------------------------------ */
int laph_sinks(laph_ctx *ctx, const laph_lattice *lat, const void *evecs, int nv,
               const void *sol, int nrhs, void *coef, void *stream);

/* ------------------------------------------------------------------------
 * (d) Correlators in coefficient space (Sec. III, meson function
 * Eq. (mesonfunc) at zero momentum without displacement, correlator
 * Eq. (mesoncorr) first term, gamma_5-swapped line Eq. (laphpropg5)).
 * With c = gamma_4 Gamma (q-bar = psi-bar gamma_4):
 *   M^[b1 b2](a, b; t) = sum_n sum_{alpha beta} conj(a^[b1](t,alpha,n)) c_{alpha beta} b^[b2](t,beta,n)
 *   meson:  C(dt) = - sum_{b1 b2} M(phibar_1, phi_2; t0+dt) conj(M(rhobar_1, rho_2; t0))
 *   I=2 pi pi: C = Cpi(1,2) Cpi(3,4) - X,
 *     X = sum M^[b1 b4](phibar_1, phi_4; tF) M^[b3 b2](phibar_3, phi_2; tF)
 *               conj(M^[b1 b2](rhobar_1, rho_2; t0)) conj(M^[b3 b4](rhobar_3, rho_4; t0))
 * where phi = coef, rho^[b] = P^(b) rho (LapH coordinates), phibar = gamma_5 gamma_4 phi,
 * rhobar = -gamma_5 gamma_4 rho.  Channels: pion (Gamma = gamma_5), rho
 * (gamma_k, the three averaged), scalar (1), I=2 pi pi.
 *   spec->nlines quark lines (2 for mesons, 4 for pi pi); line k has
 *   coef[k] = [nb][nt][4][nv] c128 (the sinks of its nb solved projectors,
 *   in the order of b_list[k]) and noise[k] = [nt][4][nv] uint8 codes.
 *   corr  [nt] c128 output, indexed by dt = (tF - t0) mod nt.
 * All lines of one call share nb, b_list and the dilution scheme.
 * ------------------------------------------------------------------------ */
enum { LAPH_CH_PION = 0, LAPH_CH_RHO = 1, LAPH_CH_SCALAR = 2, LAPH_CH_PIPI_I2 = 3 };

typedef struct {
    int channel;              /* LAPH_CH_*                                          */
    int t0;                   /* source time                                        */
    int nv;
    laph_dilution dil;        /* dilution of every line                             */
    int nb;                   /* projectors per line                                */
    const int *b_list;        /* [nb] flat projector indices (host)                 */
} laph_corr_spec;

int correlate(laph_ctx *ctx, const laph_lattice *lat, const laph_corr_spec *spec,
              const void *const *coef, const uint8_t *const *noise, void *corr, void *stream);

/* ------------------------------------------------------------------------
 * Momentum and same-time pieces of the meson correlators (Sec. III: the phase
 * e^{-ip.x} of Eq. (mesonfunc) without displacement; the second term of
 * Eq. (mesoncorr), the isoscalar "smt" diagram of Sec. V).  Momenta are integer
 * triples (px, py, pz), p = 2 pi (px, py, pz) / ns; x is the site's spatial
 * position (x fastest).  All arithmetic FP64; arrays host or device.
 *
 * laph_mom_overlaps: Phi_p(t)[n][n'] = sum_{x,c} conj(V(t,n,x,c)) e^{-ip.x} V(t,n',x,c)
 *   for nmom momenta (mom: host [nmom][3] ints); phi [nmom][nt][nv][nv] c128.
 *   Phi_0 is the identity for orthonormal eigenvectors.
 *
 * correlate_mom: the meson channels of correlate() (pion, rho, scalar) at momentum p:
 *   both meson functions of Eq. (mesoncorr) take e^{-ip.x}, which in LapH
 *   coordinates puts phi = Phi_p [nt][nv][nv] between the two lines:
 *   M^[b1 b2](a, b; t) = sum conj(a^[b1](t,alpha,n)) W_{alpha beta} Phi_p(t)[n][n'] b^[b2](t,beta,n').
 *   spec, coef, noise, corr as in correlate() with two lines.
 *
 * laph_meson_loops: same-time line of one noise closed on every slice,
 *   loops[c][t] = sum_b M^[bb](varrho, varphi; t)           (reverse = 0)
 *   loops[c][t] = sum_b M^[bb](varphi, varrho; t)           (reverse = 1)
 *   with the channel's c = gamma_4 Gamma (no gamma_5 swap), one row per component
 *   (nc = 3 for the rho, else 1), phi = Phi_p or NULL for p = 0.  coef
 *   [nb][nt][4][nv] and noise [nt][4][nv] of one line whose projectors
 *   (spec->b_list) cover every slice to be used (time interlacing, all solved).
 *   loops [nc][nt] c128.
 *
 * correlate_disconnected: corr[dt] = (1/nc) sum_c loops1[c][(t0+dt) mod nt]
 *   conj(loops2[c][t0]) - vev, with loops1 forward and loops2 reversed lines of
 *   two independent noises.  For the two degenerate light flavours the isoscalar
 *   correlator is corr_connected + 2 corr_disconnected (flavour weights of
 *   (u-bar Gamma u + d-bar Gamma d)/sqrt 2); vev = <L_1> conj(<L_2>) for the scalar.
 * ------------------------------------------------------------------------ */
int laph_mom_overlaps(laph_ctx *ctx, const laph_lattice *lat, const void *evecs, int nv, int nmom, const int *mom,
                      void *phi, void *stream);
int correlate_mom(laph_ctx *ctx, const laph_lattice *lat, const laph_corr_spec *spec, const void *const *coef,
                  const uint8_t *const *noise, const void *phi, void *corr, void *stream);
int laph_meson_loops(laph_ctx *ctx, const laph_lattice *lat, const laph_corr_spec *spec, const void *coef,
                     const uint8_t *noise, const void *phi, int reverse, void *loops, void *stream);
int correlate_disconnected(laph_ctx *ctx, const laph_lattice *lat, int t0, int nc, const void *loops1,
                           const void *loops2, double vev_re, double vev_im, void *corr, void *stream);

/* ------------------------------------------------------------------------
 * Displaced overlaps (Sec. II: the quark line D^(j) S Omega^{-1} S D^(k)dag of
 * Eq. (quarkdef); Sec. III: the phase e^{-ip.(x + (d_j + d_k)/2)} of Eq. (mesonfunc)):
 *   (D psi)(x) = U_{s1}(x) U_{s2}(x+s1) ... psi(x + s1 + ... + sL), a step -mu
 *   through U_mu(y - mu)^dag, steps s = +-1, +-2, +-3 (x, y, z), at most 64;
 *   Phi_{p,jk}(t)[n][n'] = e^{-ip.(d_j+d_k)/2} sum_{x,c} conj((D^(j) V_n)(x,c)) e^{-ip.x} (D^(k) V_n')(x,c)
 * for qbar displaced along path_bar (j) and q along path (k); d the net displacements.
 *   links3d [V][4][3][3] c128 (the Laplacian's smeared links), evecs as laph_eigvecs,
 *   mom host int[3], paths host int arrays (empty: no displacement), phi [nt][nv][nv] c128.
 * correlate_mom with phi = Phi_{p,jk} gives the connected correlator of the displaced
 * elemental (c, p, j, k) (the sink and the source function take the same (c, p, j, k)).
 * ------------------------------------------------------------------------ */
int laph_displaced_overlaps(laph_ctx *ctx, const laph_lattice *lat, const void *links3d, const void *evecs, int nv,
                            const int *mom, int len_bar, const int *path_bar, int len, const int *path, void *phi,
                            void *stream);

/* ------------------------------------------------------------------------
 * Two-pion correlators of isospin I = 0, 1, 2 (Sec. III two-meson diagrams,
 * Sec. V two-pion operators): the state |I, I3> of a pion of momentum p and
 * one of -p (pi+ = ubar d, pi0 = (dbar d - ubar u)/sqrt 2, pi- = -dbar u,
 * coupled by the Clebsch-Gordan coefficients of 1 x 1; c = gamma_4 gamma_5),
 * its source partner at t0, and every Wick contraction of the four bilinears
 * (direct, crossed, box and vacuum diagrams), each propagator a line estimate:
 *   - antiquark end at the source: forward line k, sum_b phi^[b] rho^[b]dag;
 *   - sink to source: forward line k through gamma_5 Hermiticity,
 *     G' (sum_b phi^[b] rho^[b]dag)^dag G', G' = gamma_4 gamma_5;
 *   - sink to sink: same-time line k.
 * A term's propagators take forward lines 0, 1, 2, 3 and same-time lines 0, 1
 * in the order its cycles are visited (cycles started from the lowest unvisited
 * bilinear, sink bilinears 0 (p) and 1 (-p), source bilinears 2 and 3).  At
 * t_F = t0 the sink bilinears keep the sink rules.
 *   coef_fwd[4] [nb_fwd][nt][4][nv], noise_fwd[4] [nt][4][nv]: lines sourced at
 *     t0 (b_fwd: the projectors whose time support holds t0);
 *   coef_smt[2] [nb_smt][nt][4][nv], noise_smt[2]: same-time lines, every
 *     projector of dil_smt solved, each slice covered by equally many
 *     projectors; needed (non-null) only where a diagram uses them (I < 2 or
 *     I3 < I);
 *   phi_p, phi_mp [nt][nv][nv] c128: Phi_p and Phi_-p (laph_mom_overlaps), or
 *     both NULL for p = 0;
 *   corr [nt] c128, corr[dt] = <pipi(t0 + dt) pipi-bar(t0)> (no vacuum
 *     subtraction).  Scratch about (nt nb^2) complex doubles per distinct
 *     meson function, nb the larger of nb_fwd and the projectors per slice.
 * ------------------------------------------------------------------------ */
typedef struct {
    int iso, iso3;            /* total isospin I and I3 (0 <= I3 <= I <= 2)         */
    int t0;
    int nv;
    laph_dilution dil_fwd;    /* forward lines                                      */
    int nb_fwd;
    const int *b_fwd;         /* [nb_fwd] host                                      */
    laph_dilution dil_smt;    /* same-time lines                                    */
    int nb_smt;
    const int *b_smt;         /* [nb_smt] host (NULL when nb_smt = 0)               */
} laph_pipi_spec;

int correlate_pipi(laph_ctx *ctx, const laph_lattice *lat, const laph_pipi_spec *spec, const void *const *coef_fwd,
                   const uint8_t *const *noise_fwd, const void *const *coef_smt, const uint8_t *const *noise_smt,
                   const void *phi_p, const void *phi_mp, void *corr, void *stream);

/* ------------------------------------------------------------------------
 * Baryons (Sec. III: three-quark elemental operators, Eq. (baryonfunc) and
 * Eq. (baryoncorr)).  All arithmetic FP64; arrays host or device.
 *
 * laph_baryon_tensor: T_p(t)[n1][n2][n3] = sum_x e^{-ip.x} eps_abc
 *   V(t,n1,x,a) V(t,n2,x,b) V(t,n3,x,c), antisymmetric in (n1, n2, n3);
 *   evecs as laph_eigvecs, mom host int[3], T [nt][nv][nv][nv] c128, nv <= 512.
 *
 * correlate_baryon: the correlator of Eq. (baryoncorr) for one source time,
 *   corr[dt] = sum_{b1 b2 b3} B^[b1 b2 b3](phi_1, phi_2, phi_3; t0 + dt)
 *              conj( sum_pi sgn(pi) B^[b_pi0 b_pi1 b_pi2](rho_pi0, rho_pi1, rho_pi2; t0) ),
 *   B^[b1 b2 b3](f1, f2, f3; t) = c_{alpha beta gamma} sum_{n1 n2 n3} T_p(t)[n1][n2][n3]
 *                                 f1^[b1](t,alpha,n1) f2^[b2](t,beta,n2) f3^[b3](t,gamma,n3)
 *   (c_snk at the sink, c_src at the source); pi runs over the orderings of the
 *   three lines for which sink quark pi(s) has the flavour of source slot s.
 *   coef[k] = [nb][nt][4][nv] and noise[k] = [nt][4][nv] of line k (three lines,
 *   one noise each, the same nb, b_list and dilution), T from laph_baryon_tensor.
 *   corr [nt] c128.  Scratch: 16 nt nv nb^2 + 4 nt nv^2 nb + nt nb^3 complex doubles
 *   (LAPH_ERR_NOMEM when the device cannot hold it).
 * ------------------------------------------------------------------------ */
typedef struct {
    int t0;                   /* source time                                        */
    int nv;
    laph_dilution dil;        /* dilution of every line                             */
    int nb;                   /* projectors per line (<= 1024)                      */
    const int *b_list;        /* [nb] flat projector indices (host)                 */
    const double *c_snk;      /* [4][4][4] complex, re/im interleaved (host)        */
    const double *c_src;      /* [4][4][4] complex, re/im interleaved (host)        */
    int flav_snk[3];          /* flavour labels of the sink quarks (A, B, C)        */
    int flav_src[3];          /* flavour labels of the source slots                 */
} laph_baryon_spec;

int laph_baryon_tensor(laph_ctx *ctx, const laph_lattice *lat, const void *evecs, int nv, const int *mom, void *T,
                       void *stream);
int correlate_baryon(laph_ctx *ctx, const laph_lattice *lat, const laph_baryon_spec *spec, const void *const *coef,
                     const uint8_t *const *noise, const void *T, void *corr, void *stream);

/* ------------------------------------------------------------------------
 * correlate_noalloc: the same correlators as correlate(), for callers that
 * cannot allocate GPU memory (no counterpart in the paper; it exists for
 * callers such as code running inside a caller-owned memory pool or arena,
 * processes whose device memory is reserved up front, or loops that must not
 * stall on an allocation).  It calls no cudaMalloc/cudaFree and no allocating
 * library routine and needs no laph_ctx.
 *   - coef[k], noise[k] and corr must be device pointers of one device
 *     (LAPH_ERR_ARG otherwise: host arrays would need staging memory); the
 *     call runs on that device (made current for the call, the caller's
 *     current device restored on return), and a stream other than the
 *     default ones must belong to it.  spec->b_list is a host array of at
 *     most 512 entries, passed to the device as a kernel argument.
 *   - Scratch comes from one fixed 16 MiB __device__ array inside the
 *     library, held by every GPU that loads it until the process exits.  A
 *     problem needing more (about nt nb^2 complex doubles for a meson
 *     channel, 5 nt nb^2 for pi pi) is rejected with LAPH_ERR_ARG and a
 *     message giving the size.
 *   - Each call looks up the array's device address (cudaGetSymbolAddress)
 *     on its device; the first call on a device also loads the library's
 *     kernels there, so make that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents: calls
 *     that overlap on the GPU (unordered streams or threads) race on it.
 * ------------------------------------------------------------------------ */
int correlate_noalloc(const laph_lattice *lat, const laph_corr_spec *spec, const void *const *coef,
                      const uint8_t *const *noise, void *corr, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LAPH_H */
