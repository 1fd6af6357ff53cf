/*
 * tw.h -- C ABI of the GB300 online Bayesian inversion library (libtw.so).
 *
 * The library implements the online phase (Phase 4) of the offline-online
 * inversion of arXiv 2504.16344, "Real-time Bayesian inference at extreme
 * scale: a digital twin for tsunami early warning":
 *
 *   posterior mean   m = Gamma_pr F* (Gamma_n + F Gamma_pr F*)^{-1} d
 *   forecast         q = F_q m
 *
 * where F (p2o map) and F_q (p2q map) are block lower-triangular Toeplitz in
 * time (Sec. "FFT-based Hessian matvecs", Eq. ShiftInvariance) and are
 * applied by zero-padding time to 2 Nt, a batched real FFT along time, one
 * complex matrix-vector product per frequency and an inverse FFT.
 *
 * Conventions (all entry points):
 *  - Vectors are time-major and row-major: a parameter vector m is
 *    [Nt][Nm] (m_j = m[j*Nm .. j*Nm+Nm-1]), a data vector d is [Nt][Nd], a
 *    QoI vector q is [Nt][Nq]; Nm = Nx*Ny with flat grid index a*Ny + b.
 *    Several right-hand sides are stacked: [nrhs][Nt][...].
 *  - Every vector argument is a DEVICE pointer owned by the caller unless the
 *    comment says host.  Work is enqueued on `stream` (a cudaStream_t passed
 *    as void*, NULL = legacy default stream) and is stream-ordered: outputs
 *    are valid once the stream reaches that point.  The context owns every
 *    other buffer (the frequency-domain operators, K's factor, workspaces);
 *    online calls allocate nothing.
 *  - User-facing values are IEEE binary64.
 *  - Every call returns a tw_status; no C++ exception crosses the ABI.  On
 *    error tw_last_error() gives a message.  Errors raised by kernels (a
 *    non-positive pivot, a wait that ran out) are recorded on the device and
 *    reported by tw_check() after the stream has been synchronised.
 *  - A context is not thread-safe: one host thread at a time.
 */
#ifndef TW_H
#define TW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tw_ctx tw_ctx;

typedef enum {
  TW_OK = 0,
  TW_ERR_ARG = 1,            /* invalid argument (size, pointer, enum)          */
  TW_ERR_OOM = 2,            /* device allocation failed or budget exceeded     */
  TW_ERR_CUDA = 3,           /* a CUDA runtime call failed                      */
  TW_ERR_STATE = 4,          /* call out of order (e.g. infer before factor)    */
  TW_ERR_NOT_SPD = 5,        /* Cholesky met a non-positive pivot               */
  TW_ERR_NOT_CONVERGED = 6,  /* iterative refinement did not reach its tolerance*/
  TW_ERR_TIMEOUT = 7         /* a bounded device wait ran out                   */
} tw_status;

/* Which Toeplitz map: the p2o map F (Nd rows) or the p2q map F_q (Nq rows). */
typedef enum { TW_MAP_F = 0, TW_MAP_FQ = 1 } tw_map;

/* Storage / arithmetic of the frequency-domain operator in an apply.
 *  TW_PREC_FP64   : F^ held as float pairs (hi + lo, 48-bit significand,
 *                   16 bytes per complex entry, the size of complex128);
 *                   arithmetic in double-float (error-free FP32 transforms).
 *                   This is the library's FP64-class path.
 *  TW_PREC_C64    : F^ held as complex64.  Adjoint applies (F^T y, the
 *                   posterior mean's product) take y's spectrum as float
 *                   pairs and sum without rounding loss, so the result
 *                   carries the operator's own rounding only (y is large
 *                   against m and F^T y cancels; an FP32 sum would lose
 *                   digits by that cancellation): one right-hand side with
 *                   exact products and double-float running sums, batches
 *                   on the tensor cores with both sides cut into exact
 *                   fixed-point bf16 slices (per-row / per-column power-of-
 *                   two scales, the leading terms accumulated exactly;
 *                   batched adjoints need rows <= 512, TW_ERR_CUDA beyond).
 *                   Forward applies, inverse FFTs and the prior run in FP32.
 *  TW_PREC_BF16X2 : F^ held as bf16 hi + bf16 lo per real (8 bytes per
 *                   complex entry, 16-17 significant bits); arithmetic as
 *                   TW_PREC_C64.                                             */
typedef enum { TW_PREC_FP64 = 0, TW_PREC_C64 = 1, TW_PREC_BF16X2 = 2 } tw_prec;

/* Storage kept by the context (bit mask for tw_create's `keep`). */
#define TW_KEEP_FP64   1u
#define TW_KEEP_C64    2u
#define TW_KEEP_BF16X2 4u
/* TW_KEEP_G: tw_factor_K also forms G^ = F^ C per frequency in every kept
 * format -- the block Toeplitz G* = Gamma_pr F* of Phase 2 (Sec. "Real-time
 * Bayesian inference and prediction framework") -- and tw_infer's adjoint
 * applies use it, so the online posterior mean needs no prior filter.
 * Formed in the FP64 and complex64 storages (bf16 hi+lo would round G^ at
 * 2^-18, which reaches m unsmoothed: the TW_PREC_BF16X2 path keeps F^ and
 * the prior filter).  Adds the storage of F's FP64 and complex64 operators;
 * needs TW_KEEP_FP64. */
#define TW_KEEP_G      8u
/* TW_KEEP_FACTOR64: tw_factor_K forms only the FP64 factor of K, also in a
 * context that keeps no FP64 operator (the mixed operator paths then solve
 * with it, as they do by default when both are present), and skips the FP32
 * factor.  Lets a complex64 / bf16x2 context run the FP64-factor solves
 * without the memory of the FP64 operator or of the FP32 factor. */
#define TW_KEEP_FACTOR64 16u

/*
 * tw_create -- allocate a context for Nd sensors, Nq forecast points, an
 * Nx x Ny periodic parameter grid over [0,Lx) x [0,Ly) and Nt time steps.
 * `keep` selects which operator storages are filled (TW_KEEP_*).  `device`
 * is the CUDA device ordinal.  Allocates the frequency-domain operators
 * (Nt+1 frequencies x rows x Nm per kept format) and online workspaces.
 * Errors: TW_ERR_ARG for non-positive sizes, TW_ERR_OOM, TW_ERR_CUDA.
 */
tw_status tw_create(tw_ctx **out, int Nd, int Nq, int Nx, int Ny, int Nt,
                    double Lx, double Ly, unsigned keep, int device);

/* Free everything the context owns.  Safe on NULL. */
void tw_destroy(tw_ctx *ctx);

/* Last error message of this context (static storage of the context). */
const char *tw_last_error(const tw_ctx *ctx);

/*
 * tw_set_block_column -- load rows [row0, row0+nrows) of the first block
 * column of F (which = TW_MAP_F, rows are sensors) or F_q (TW_MAP_FQ, rows
 * are forecast points): col is a device array [Nt][nrows][Nm] in FP64 with
 * col[l][r][k] = (F_l)[row0+r, k], l the 0-based time lag (Sec. "FFT-based
 * Hessian matvecs": only the first block column is stored, O(Nm Nd Nt)).
 * The call computes the rows' frequency-domain blocks F^(w), w = 0..Nt, by a
 * real FFT of length 2Nt along the lag and stores them in every kept format.
 * `col` is only read during the call (stream-ordered).  Rows may be loaded
 * in any order and chunking; all rows must be loaded before an apply.
 * When tw_set_prior came first, the call also keeps G = Phi C^{1/2} for
 * these rows of F (computed in FP64 from `col`, Nt*nrows*Nm float pairs of
 * device memory until tw_factor_K consumes them): K is then formed from the
 * exact input rather than from the stored frequency-domain operator.
 */
tw_status tw_set_block_column(tw_ctx *ctx, tw_map which, int row0, int nrows,
                              const double *col, void *stream);

/*
 * tw_set_prior -- Matern prior Gamma_pr = I_Nt (x) C (Sec. "State of the
 * art": block diagonal in time, each block a Matern covariance).  C is the
 * stationary covariance on the periodic grid with Fourier eigenvalues
 * lambda_k = var * N * s(k) / sum s, s(k) = (kappa^2 + |k|^2)^-(nu+1),
 * kappa = sqrt(2 nu)/ell, k = 2 pi (p/Lx, q/Ly): the pointwise variance is
 * exactly var.  Errors: TW_ERR_ARG for non-positive nu, ell or var.
 */
tw_status tw_set_prior(tw_ctx *ctx, double nu, double ell, double var);

/*
 * tw_p2o_apply -- out = F x (which = TW_MAP_F, out [nrhs][Nt][Nd]) or
 * out = F_q x (TW_MAP_FQ, out [nrhs][Nt][Nq]) for x [nrhs][Nt][Nm]:
 * out_i = sum_{j<=i} F_{i-j} x_j (Eq. ShiftInvariance), computed as
 * irfft_2Nt( F^(w) rfft_2Nt(x)(w) ) truncated to Nt steps.
 * prec selects the operator storage (must have been kept).
 */
tw_status tw_p2o_apply(tw_ctx *ctx, tw_map which, tw_prec prec, int nrhs,
                       const double *x, double *out, void *stream);

/*
 * tw_p2o_adjoint -- x = F^T y (Euclidean adjoint; y [nrhs][Nt][Nd], x
 * [nrhs][Nt][Nm]) or F_q^T y: x_j = sum_{i>=j} F_{i-j}^T y_i, computed as
 * irfft( F^(w)^H rfft(y)(w) ) truncated to Nt steps.  With a reduced
 * precision, several right-hand sides and a reserved batch
 * (tw_reserve_batch), they run as batches of the per-frequency matrix
 * product on the tensor cores.
 */
tw_status tw_p2o_adjoint(tw_ctx *ctx, tw_map which, tw_prec prec, int nrhs,
                         const double *y, double *x, void *stream);

/*
 * tw_prior_apply -- y = Gamma_pr^power x for x, y [nrhs][Nt][Nm], power 1
 * or 0.5 (the square root used to draw prior samples).  2D real FFT per time
 * step, scaling by lambda^power, inverse FFT.  x and y may alias.
 */
tw_status tw_prior_apply(tw_ctx *ctx, double power, int nrhs, const double *x,
                         double *y, void *stream);

/*
 * tw_factor_K -- form and factor the data-space Hessian of Phase 2,
 *   K = Gamma_n + F Gamma_pr F^T,  Gamma_n = noise_var * I,
 * (Sec. "Real-time Bayesian inference and prediction framework": the
 * Sherman-Morrison-Woodbury rewrite moves the inverse to data space).  K is
 * (Nd*Nt) x (Nd*Nt), time-major (index t*Nd + sensor).  It is formed from the
 * time-domain block column as K_(i,j) = noise_var delta_ij I +
 * sum_{s<=min(i,j)} F_{i-s} C F_{j-s}^T (a product G G^T with
 * G = Phi C^{1/2}, then prefix sums along block diagonals; the product runs
 * on the tensor cores from exact fixed-point bf16 slices of G with integer-
 * exact sums, one FP64 rounding per 8,192-column panel), then Cholesky-
 * factored: in FP64 if TW_KEEP_FP64 or TW_KEEP_FACTOR64 was kept (the
 * trailing updates as exact tensor-core products; the single-vector and
 * batched solves then stream its blocks, pre-multiplied by the diagonal-block
 * inverses, as float pairs in double-float arithmetic), and in
 * FP32 if TW_KEEP_C64 or TW_KEEP_BF16X2 was kept without TW_KEEP_FACTOR64.  K itself is kept as
 * packed double-float blocks (refinement residuals, tw_apply_K).  Needs
 * tw_set_prior, and either the FP64 operator of F or F's block column loaded
 * after tw_set_prior (TW_ERR_STATE otherwise).  The dense K is released as
 * soon as it has been factored.
 * Set-up call: allocates, synchronises `stream`, and returns TW_ERR_NOT_SPD
 * (pivot row in tw_last_error) if K is not numerically positive definite.
 * Best accuracy: tw_set_prior, then the block column of F, then this call
 * (G is then exact to FP64; it is released after use, so a second call, for
 * another noise level, rebuilds Phi from the stored operator).
 */
tw_status tw_factor_K(tw_ctx *ctx, double noise_var, void *stream);

/*
 * Phase-2 checkpoint.  The offline-online split of the paper (Sec. "Real-time
 * Bayesian inference and prediction framework": Phases 1-3 run once, Phase 4
 * reuses their results) lets one context form and factor K and another,
 * created later or elsewhere with the same sizes, prior and block column,
 * load the factor instead of forming K again.
 *
 * tw_factor_bytes -- size in bytes of the checkpoint of the context's FP64
 *   factor; 0 when there is none.
 * tw_save_factor  -- writes the checkpoint to `host` (bytes >= tw_factor_bytes;
 *   host memory, pageable or pinned, owned by the caller): a 96-byte header
 *   (magic "TWLFAC01", Nd, Nt, Nx, Ny, block count, block size, noise
 *   variance, prior parameters, domain size), then the packed lower-triangular
 *   64x64 blocks of the FP64 Cholesky factor (block (I,J), J <= I, at
 *   I(I+1)/2 + J, row-major) and the inverses of the diagonal blocks.
 *   Synchronises `stream`.  TW_ERR_STATE without an FP64 factor, TW_ERR_ARG
 *   for a short buffer.
 * tw_load_factor  -- reads such a checkpoint into a context with the same
 *   Nd, Nt, Nx, Ny, Lx, Ly and prior (tw_set_prior first; TW_ERR_ARG on any
 *   mismatch, a bad magic or a truncated buffer), then prepares the solves
 *   exactly as tw_factor_K does after its factorisation (chain blocks,
 *   single-vector solve tables, G^ when TW_KEEP_G, batch copies).  The
 *   caller guarantees that the block column of F is the one the factor was
 *   formed from.  K itself is not part of the checkpoint: afterwards
 *   tw_apply_K returns TW_ERR_STATE, tw_infer_stats.resid_rel reads -1, and
 *   the solves use the FP64 factor whatever tw_set_solver selected (no FP32
 *   factor is held).  Any G held for forming K is released.
 *   Synchronises the device.
 */
size_t tw_factor_bytes(const tw_ctx *ctx);
tw_status tw_save_factor(tw_ctx *ctx, void *host, size_t bytes, void *stream);
tw_status tw_load_factor(tw_ctx *ctx, const void *host, size_t bytes, void *stream);

/* Statistics of the last right-hand side of tw_infer (optional output). */
typedef struct {
  int ir_iters;      /* refinement steps taken (mixed path; 0 for FP64)   */
  double resid_rel;  /* |d' - K' y| / |d'| with the stored K; -1 without K */
} tw_infer_stats;

/*
 * tw_infer -- posterior mean (MAP point) of Phase 4 with m_prior = 0:
 *   m = Gamma_pr F'^T (Gamma_n + F' Gamma_pr F'^T)^{-1} d'
 * for each right-hand side r, where the observation window Nt' =
 * nt_window[r] (host array, NULL = Nt for all) keeps the leading Nt' time
 * blocks of the data: d' = d[r][0..Nt'-1][.], F' = the leading Nt' block
 * rows of F, and K' = K[:Nd Nt', :Nd Nt'] (Cholesky factors nest, so the
 * one factor serves every window).  Rows t >= Nt' of m are 0 (the prior
 * mean; data before Nt' do not inform them).
 * d: device [nrhs][Nt][Nd] FP64 (rows >= Nt' ignored); m: device
 * [nrhs][Nt][Nm] FP64.  prec TW_PREC_FP64 uses the FP64 factor and the
 * double-float operator; TW_PREC_C64 / TW_PREC_BF16X2 use the FP32 operator for F'^T and
 * the prior, and solve K' y = d' as tw_set_solver selects (double-float
 * factor, or FP32 factor + FP64-residual refinement).
 * stats may be NULL; when given, the call synchronises `stream` once.
 */
tw_status tw_infer(tw_ctx *ctx, tw_prec prec, int nrhs, const int *nt_window, const double *d,
                   double *m, tw_infer_stats *stats, void *stream);

/*
 * tw_solve_K -- the data-space solve of Phase 4 alone: y = K'^{-1} d' for
 * each right-hand side (window Nt' = nt_window[r], NULL = Nt), with the
 * solver tw_infer would use for `prec`.  d, y: device [nrhs][Nt][Nd] FP64;
 * rows t >= Nt' of y are 0.
 */
tw_status tw_solve_K(tw_ctx *ctx, tw_prec prec, int nrhs, const int *nt_window, const double *d,
                     double *y, void *stream);

/*
 * tw_apply_K -- out = K' x with the stored K (double-float, packed lower
 * blocks; K' = leading Nd Nt' rows and columns).  For residual
 * certificates |d - K y|.  x, out: device [nrhs][Nt][Nd] FP64.
 */
tw_status tw_apply_K(tw_ctx *ctx, int nrhs, const int *nt_window, const double *x, double *out,
                     void *stream);

/*
 * tw_sample_posterior -- posterior samples by perturb-then-condition, exact
 * for the linear-Gaussian model: for each sample k with window Nt'
 * (nt_window[k], NULL = Nt),
 *   m_pr = Gamma_pr^{1/2} z_m,
 *   s    = m_pr + Gamma_pr F'^T K'^{-1} (d' - F' m_pr - sigma z_n),
 * whose covariance is Gamma_post = Gamma_pr - G* K^{-1} G (the Woodbury form
 * of Phase 2) and whose mean is the posterior mean; this realises the paper's
 * Gamma_post^{1/2} z draws.  The random draws are inputs: z_m [ns][Nt][Nm]
 * and z_n [ns][Nt][Nd] (rows >= Nt' unused), d [ns][Nt][Nd] the data of each
 * sample (rows >= Nt' unused), sigma the noise standard deviation used in K.
 * samples [ns][Nt][Nm]; rows t >= Nt' hold the prior draw m_pr.  FP64 path.
 */
tw_status tw_sample_posterior(tw_ctx *ctx, int ns, const int *nt_window, const double *d,
                              const double *z_m, const double *z_n, double sigma,
                              double *samples, void *stream);

/*
 * tw_forecast -- QoI forecast q = F_q m (Phase 4, q_map = F_q m_map):
 * m [nrhs][Nt][Nm] -> q [nrhs][Nt][Nq], the Toeplitz apply of the p2q map.
 */
tw_status tw_forecast(tw_ctx *ctx, tw_prec prec, int nrhs, const double *m, double *q,
                      void *stream);

/*
 * tw_infer_forecast -- tw_infer followed by tw_forecast of its result in one
 * call (Phase 4: m_map, then q_map = F_q m_map): m [nrhs][Nt][Nm] and
 * q [nrhs][Nt][Nq] as those two calls give them; arguments and errors as
 * theirs.  With G^ kept (TW_KEEP_G) and one right-hand side at a time (no
 * reserved batch or nrhs = 1), the inverse time FFT that produces m also
 * takes m's forward time FFT for the forecast in the same kernel, from shared
 * memory: the forecast then does not read m back.  The FP64 path's q may
 * differ from tw_forecast's in the last bits (m's spectrum is taken from the
 * double-float m before its rounding to FP64); the reduced-precision paths
 * give the same bits.
 */
tw_status tw_infer_forecast(tw_ctx *ctx, tw_prec prec, int nrhs, const int *nt_window, const double *d,
                            double *m, double *q, tw_infer_stats *stats, void *stream);

/* Number of iterative-refinement steps of the mixed-precision tw_infer
 * (range 0..50).  tw_factor_K picks it by refining a probe right-hand side
 * until the FP64 residual stops falling; this call overrides that choice. */
tw_status tw_set_refinement(tw_ctx *ctx, int steps);

/* How the mixed-precision tw_infer (TW_PREC_C64 / TW_PREC_BF16X2) solves
 * K y = d.  TW_SOLVE_FACTOR64 (default): the FP64 factor (needs
 * TW_KEEP_FP64 at set-up); only the operator applies run in FP32.
 * TW_SOLVE_FP32_IR: the FP32 factor plus iterative refinement with the FP64
 * residual r = d - K y (the number of steps: tw_set_refinement). */
typedef enum { TW_SOLVE_FACTOR64 = 0, TW_SOLVE_FP32_IR = 1 } tw_solver;
tw_status tw_set_solver(tw_ctx *ctx, tw_solver solver);

/* Refinement steps the mixed-precision tw_infer currently takes (-1 if ctx
 * is NULL). */
int tw_refinement_steps(const tw_ctx *ctx);

/* Phases of the online calls, for per-phase device timing. */
typedef enum {
  TW_PH_TRSV_FWD = 0,   /* L z = d (forward substitution, persistent kernel)  */
  TW_PH_TRSV_BWD,       /* L^T y = z                                           */
  TW_PH_RESIDUAL,       /* r = d - K x (refinement residual, FP64 K)           */
  TW_PH_RFFT_DATA,      /* time FFT of a data-space vector (Nd or Nq series)   */
  TW_PH_GEMV_ADJ,       /* x^(w) = F^(w)^H y^(w), all frequencies              */
  TW_PH_IRFFT_PARAM,    /* inverse time FFT of a parameter vector (Nm series)  */
  TW_PH_PRIOR,          /* Matern filter (three passes)                        */
  TW_PH_RFFT_PARAM,     /* time FFT of a parameter vector                      */
  TW_PH_GEMV_FWD,       /* y^(w) = F^(w) x^(w) incl. the chunk reduction       */
  TW_PH_IRFFT_DATA,     /* inverse time FFT of a data-space vector             */
  TW_PH_FORM_K,         /* set-up: K = sigma^2 I + prefix sums of G G^T        */
  TW_PH_CHOLESKY,       /* set-up: FP64 Cholesky of K and packing              */
  TW_PH_CHOLESKY32,     /* set-up: FP32 factor and its refinement probe        */
  TW_PH_SOLVE_SETUP,    /* set-up: chain blocks, block-scaled factor, tables   */
  TW_PH_FORM_GSTAR,     /* set-up: G^ = F^ C per frequency (TW_KEEP_G)         */
  TW_PH_COUNT
} tw_phase;

/* Record CUDA events around every phase of later calls (on the stream the
 * phase is launched on).  Off by default; costs two event records a phase. */
tw_status tw_profile_enable(tw_ctx *ctx, int on);

/* Synchronise on the recorded events and return, per phase, the summed
 * device time in ms and the number of timed launches since the last reset
 * (host arrays of TW_PH_COUNT entries; either may be NULL).  reset != 0
 * clears the totals. */
tw_status tw_profile_read(tw_ctx *ctx, double *ms, long long *calls, int reset);

/* Number of CUDA kernels this library has enqueued in this process. */
long long tw_kernel_launches(void);

/*
 * tw_p2o_apply_noalloc -- the same result as tw_p2o_apply, from a call that
 * allocates nothing (the paper has no counterpart: this serves callers that
 * must not allocate device memory after start-up, such as a real-time loop
 * with a fixed footprint).  The per-chunk partial sums of the frequency GEMV,
 * which tw_p2o_apply keeps in the context, live in a fixed 32 MiB device
 * array inside the library; every GPU that loads the library holds it until
 * the process exits.  Sizes whose partial sums exceed it,
 * (Nt+1) * ceil(Nm/1024) * rows * (16 bytes FP64 path, 8 bytes FP32 paths),
 * return TW_ERR_ARG with a message.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress), so make that first call
 * before any stream capture.  All calls share the one array: calls that
 * overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller.  Nothing in the array needs clearing between
 * calls; each call overwrites what it reads.
 */
tw_status tw_p2o_apply_noalloc(tw_ctx *ctx, tw_map which, tw_prec prec, int nrhs,
                               const double *x, double *out, void *stream);

/*
 * ---- Batches of right-hand sides (Phase 4 serving many events and
 * posterior samples at once).  With B right-hand sides the solves become
 * block products L_IJ x Z_J(64 x 8 columns) and each frequency's product
 * F^(w)^H Y^(w) a matrix-matrix product, so the factor and the operator
 * are streamed once per column slice instead of once per right-hand side.
 *
 * tw_reserve_batch -- allocate the workspaces of batches of up to bmax
 * right-hand sides (about bmax * (Nt+1) * Nm * 16 bytes, plus float-pair
 * copies of the factor's diagonal-block inverses); bmax = 0 frees them.
 * Needs tw_factor_K (the FP64 factor); a later tw_factor_K or tw_load_factor
 * refreshes the copies.  Set-up call: synchronises the device.  Once a batch is reserved,
 * tw_infer (FP64 path, or mixed path with TW_SOLVE_FACTOR64), tw_forecast and
 * tw_sample_posterior with several right-hand sides run as batches of up to
 * bmax columns.
 */
tw_status tw_reserve_batch(tw_ctx *ctx, int bmax);

/* Reserved batch size (0 if none, -1 if ctx is NULL). */
int tw_batch_capacity(const tw_ctx *ctx);

/*
 * tw_infer_batch -- posterior means of nrhs <= bmax right-hand sides, and
 * their forecasts when q != NULL, with the windows in DEVICE memory:
 * nt_window_dev[r] in [0, Nt] (0: an empty slot, m and q come out zero).
 * d [nrhs][Nt][Nd], m [nrhs][Nt][Nm], q [nrhs][Nt][Nq]; same results as
 * tw_infer / tw_forecast.  prec TW_PREC_FP64 solves with the FP64 factor;
 * the mixed precisions solve with its float-pair copy (48-bit), whatever
 * tw_set_solver selected.  The call allocates nothing and never
 * synchronises: it can be captured into a CUDA graph (tw_capture_begin)
 * and relaunched after new data and windows are written to the same
 * buffers.
 */
tw_status tw_infer_batch(tw_ctx *ctx, tw_prec prec, int nrhs, const int *nt_window_dev,
                         const double *d, double *m, double *q, void *stream);

/*
 * Tiles of the batched per-frequency products.  tw_reserve_batch times the
 * legal candidates on the context's operator and workspaces (CUDA events,
 * one warm-up launch, the mean of two) and keeps the fastest; the choice is
 * cached for the process by shape (Nd, Nq, Nx, Ny, Nt, bmax, keep), so a
 * later context of the same shape takes it without measuring.  The
 * environment variable TW_AUTOTUNE=0 keeps the built-in rules instead.
 *   adj_tile  : right-hand sides per tensor-core tile of the reduced-
 *               precision adjoint (multiple of 8, <= 80; more tiles re-read
 *               the operator, fewer leave the MMA narrow)
 *   adj_rw    : right-hand sides per warp of the FP64-class adjoint (1, 2, 4;
 *               0 = by batch size)
 *   fwd_lanes : lanes per right-hand side of the forward products (1, 2)
 * A column's result never depends on its batch mates for any choice; it
 * can differ in the last bits between choices (fwd_lanes changes the order
 * of its sums), so every lane of a context uses the same tiles.
 */
typedef struct {
  int adj_tile, adj_rw, fwd_lanes;
  double adj_tile_ms, adj_rw_ms, fwd_lanes_ms;  /* time of each choice; -1 if not measured */
  int tuned;            /* 1 measured (now or by an earlier context), 0 built-in
                           rules, 2 set by tw_set_batch_tiles                  */
} tw_tiles;

/* The tiles the reserved batch uses (TW_ERR_STATE without tw_reserve_batch). */
tw_status tw_batch_tiles(const tw_ctx *ctx, tw_tiles *out);
/* Use these tiles instead (validated; the *_ms fields are ignored). */
tw_status tw_set_batch_tiles(tw_ctx *ctx, const tw_tiles *tiles);
/* The selection rule: index of the smallest positive time among n (-1 if
 * none; ties keep the earlier candidate).  Host only. */
int tw_autotune_pick(int n, const double *ms);
/* Forget the process-wide cache of measured tiles. */
void tw_autotune_clear_cache(void);

/* tw_sample_posterior for ns <= bmax samples with windows in DEVICE memory
 * (values in [0, Nt]); prec as tw_infer_batch.  No allocation, no
 * synchronisation (capturable). */
tw_status tw_sample_posterior_batch(tw_ctx *ctx, tw_prec prec, int ns, const int *nt_window_dev,
                                    const double *d, const double *z_m, const double *z_n,
                                    double sigma, double *samples, void *stream);

/* q = F_q m for nrhs <= bmax parameter vectors; rows t >= nt_window_dev[r]
 * of m are taken as zero (NULL: all rows).  Capturable. */
tw_status tw_forecast_batch(tw_ctx *ctx, tw_prec prec, int nrhs, const int *nt_window_dev,
                            const double *m, double *q, void *stream);

/*
 * CUDA graphs of batched calls.  tw_capture_begin starts capturing `stream`
 * (a created stream, not NULL); the batched calls above then only record
 * their work; tw_capture_end ends the capture and instantiates the graph.
 * tw_graph_launch replays it on any stream: the recorded calls run again
 * with whatever the captured buffers (data, windows) hold at that time.
 * Make one uncaptured call of the same kind first, so every kernel's
 * shared-memory attribute is already set.
 */
typedef struct tw_graph tw_graph;
tw_status tw_capture_begin(tw_ctx *ctx, void *stream);
tw_status tw_capture_end(tw_ctx *ctx, void *stream, tw_graph **out);
tw_status tw_graph_launch(tw_graph *graph, void *stream);
/* Kernel nodes in the graph (-1 on error). */
int tw_graph_kernel_count(const tw_graph *graph);
void tw_graph_destroy(tw_graph *graph);

/*
 * ---- Serving (Phase 4 under a stream of requests).
 * A request names an event (a data vector in a device-resident bank) and an
 * observation window Nt'; it is served when its posterior mean and
 * forecast are computed and the forecast is in host memory.  Continuous
 * batching over "lanes": a lane is one set of batch workspaces and slot
 * buffers with its own stream, holding a batch of up to max_batch requests.
 * Requests queue in arrival order; whenever a lane is free and requests
 * wait, the oldest min(waiting, max_batch) start in that lane at once, while
 * the other lanes' batches are still running, so requests that arrive during
 * a batch start as soon as any lane frees up and their kernels overlap the
 * running batches' on the device.  Lane 0 is the context's reserved batch
 * (tw_reserve_batch); the session adds lanes while device memory allows
 * (cudaMemGetInfo, 2 GB margin), up to the requested count.
 */
typedef struct {
  int batches;         /* batches launched                                   */
  int max_batch;       /* largest batch                                      */
  double mean_batch;   /* requests per batch                                 */
  double makespan_s;   /* first arrival to last completion                   */
  double busy_s;       /* summed start-to-completion time of the batches
                          (batches that overlap count in full)               */
  int lanes;           /* lanes the session used                             */
  int max_in_flight;   /* most batches in flight at once                     */
} tw_serve_stats;

/*
 * tw_serve_replay -- replay a trace in real time: request i arrives
 * arrival_s[i] seconds (host, sorted) after the call starts its clock,
 * with event[i] in [0, nevents) and window[i] in [1, Nt] (host arrays).
 * event_data: device [nevents][Nt][Nd].  lanes: batches in flight at most
 * (1..4; 0 = as many as device memory allows, up to 4).  Outputs (host):
 * latency_ms[i] = completion - arrival; q_out [nreq][Nt][Nq] and m_out
 * [nreq][Nt][Nm] (either may be NULL; copying m_out is outside the timed path
 * but slows the replay).  stats may be NULL.  Needs tw_reserve_batch
 * (max_batch <= the reserved batch); allocates the extra lanes' workspaces,
 * each lane's slot buffers (max_batch x (Nt Nm + Nt Nd + Nt Nq) doubles) and
 * streams before the clock starts, and frees them on return.  `stream` (lane
 * 0's) must be a created stream.  A result does not depend on the lane or on
 * the batch it ran in (bitwise).
 */
tw_status tw_serve_replay(tw_ctx *ctx, tw_prec prec, int nreq, const double *arrival_s,
                          const int *event, const int *window, int nevents,
                          const double *event_data, int max_batch, int lanes, double *latency_ms,
                          double *q_out, double *m_out, tw_serve_stats *stats, void *stream);

/*
 * tw_serve_simulate -- the same admission policy on a virtual clock, each
 * lane a server whose batch takes cost_ms + cost_ms_per_req * batch size
 * (host only, no device use; the lanes of the model do not slow each other):
 * latency_ms[i] and the batch index batch_of[i] (may be NULL; batches are
 * numbered in start order) of each request.  Returns TW_ERR_ARG for
 * unsorted arrivals, max_batch < 1, lanes < 1 or NULL arrays.
 */
tw_status tw_serve_simulate(int nreq, const double *arrival_s, int max_batch, int lanes,
                            double cost_ms, double cost_ms_per_req, double *latency_ms,
                            int *batch_of);

/*
 * ---- Phase 3 / Phase 4 for the QoI (Sec. "Real-time Bayesian inference and
 * prediction framework").  Phase 3 precomputes, from Nq*Nt actions on QoI
 * unit vectors e_j (QoI entry j = t*Nq + i),
 *   the data-to-QoI map       Q = F_q Gamma_post F^T Gamma_n^{-1} = F_q Gamma_pr F^T K^{-1}
 *   the QoI posterior covariance  F_q Gamma_post F_q^T = C - W^T K^{-1} W,
 *     C = F_q Gamma_pr F_q^T, W = F Gamma_pr F_q^T,
 * so that Phase 4 forecasts q = Q d directly from data (full observation
 * window; windowed forecasts go through tw_infer + tw_forecast).
 *
 * tw_qoi_build -- the Phase 3 pass (FP64 path: double-float applies, FP64
 * factor), in batches of min(96, reserved batch) unit vectors; needs
 * tw_reserve_batch.  Keeps Q and W ((Nq Nt) x (Nd Nt) doubles each), C and
 * the variances on the device.  Set-up call: allocates, synchronises.
 */
tw_status tw_qoi_build(tw_ctx *ctx, void *stream);

/* q = Q d for nrhs data vectors: d device [nrhs][Nt][Nd], q device
 * [nrhs][Nt][Nq] (FP64).  Equals tw_forecast of the full-window tw_infer. */
tw_status tw_qoi_apply(tw_ctx *ctx, int nrhs, const double *d, double *q, void *stream);

/* Variances of the QoI posterior (diagonal of F_q Gamma_post F_q^T), device
 * [Nt][Nq]; the 95% credible interval of q_j is q_j +- 1.96 sqrt(var_j). */
tw_status tw_qoi_variance(tw_ctx *ctx, double *var, void *stream);

/* The dense QoI posterior covariance, device [Nq Nt][Nq Nt] (row-major),
 * C - W^T (K^{-1} W) as one FP64 GEMM over Nd*Nt terms. */
tw_status tw_qoi_covariance(tw_ctx *ctx, double *cov, void *stream);

/* Synchronise `stream` and report errors recorded by kernels (TW_OK,
 * TW_ERR_NOT_SPD, TW_ERR_TIMEOUT, TW_ERR_CUDA).  Clears the record. */
tw_status tw_check(tw_ctx *ctx, void *stream);

/* Device bytes held by the context. */
size_t tw_device_bytes(const tw_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* TW_H */
