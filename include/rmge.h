/*
 * rmge.h -- C ABI of librmge, a single-GPU (GB300, sm_103a) implementation of the
 * randomized-multiplier GENP solve of Pan, Qian and Yan, "Random multipliers numerically
 * stabilize Gaussian and block Gaussian elimination" (arXiv:1406.5802).
 *
 * The method (Fact 4.1 with F = I, H = G): to solve A X = B, draw a random multiplier G
 * (Def. 4.1 Gaussian, or a circulant of Sec. 5), form M = A G, factor M = L U by Gaussian
 * elimination with no pivoting (GENP, eq. (3.1) applied recursively, Sec. 3), solve
 * L U Y = B, and return X = G Y; refine X by residual correction (Sec. 1.2, Sec. 7.1).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are row-major with an explicit leading dimension (elements between rows),
 *   ld >= number of columns.  Element (i, j) of a matrix P with leading dimension ldp is
 *   P[i * ldp + j].
 * - Unless a parameter says otherwise, every pointer is caller-owned DEVICE memory (or
 *   host memory the device can address, e.g. pinned), must stay valid until the work
 *   enqueued on `stream` has completed, and is never freed or retained by the library.
 * - The library allocates no memory.  Scratch comes from a caller buffer `ws` of at least
 *   rmge_workspace_size(...) bytes, 256-byte aligned.  Its contents need not be initialised
 *   and are undefined after the call.  Two calls that run concurrently need two buffers.
 * - Every call only validates its arguments and enqueues kernels on `stream` (a
 *   cudaStream_t; NULL = legacy default stream).  It returns RMGE_OK when all launches were
 *   accepted.  Numerical outcomes (breakdown step, growth, backward errors, sweep count)
 *   are written by the kernels to caller memory and are valid once the stream has been
 *   synchronised; none of them changes the return value.  The one exception is an _ex call
 *   with rmge_options.sync set, which synchronises the stream and returns the outcome.
 * - No call prints, aborts, throws, or traps on the device.  Argument errors return
 *   RMGE_ERR_INVALID_ARG and enqueue nothing; a failed launch returns RMGE_ERR_CUDA.
 * - n >= 1, nrhs >= 1; n <= RMGE_MAX_N.
 */
#ifndef RMGE_H
#define RMGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RMGE_MAX_N 65536

/* Opaque CUDA stream (identical to cudaStream_t), so this header needs no CUDA headers. */
typedef struct CUstream_st* rmge_stream_t;

typedef enum {
    RMGE_OK = 0,
    RMGE_ERR_INVALID_ARG = 1,   /* bad size, leading dimension, pointer or enum; nothing enqueued */
    RMGE_ERR_BREAKDOWN = 2,     /* a zero or non-finite pivot (Cor. 3.1) */
    RMGE_ERR_GROWTH = 3,        /* pivot growth above rmge_options.growth_tol (Thm 3.2, Remark 3.2) */
    RMGE_ERR_NOT_CONVERGED = 4, /* refinement stopped above be_tol */
    RMGE_ERR_CUDA = 5,          /* a CUDA launch or copy failed */
    RMGE_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    RMGE_ERR_WORKSPACE = 7,     /* ws is NULL, too small or misaligned */
    RMGE_ERR_UNSUPPORTED = 8,   /* valid request the library does not implement (e.g. circulant n not 2^p) */
    RMGE_ERR_NONFINITE = 9      /* a result (factors, X) holds an Inf or NaN */
} rmge_status;

/* Random multiplier G (Sec. 4-5). */
typedef enum {
    RMGE_GAUSSIAN = 0,           /* dense n x n, i.i.d. N(0,1) entries (Def. 4.1) */
    RMGE_CIRCULANT_GAUSSIAN = 1, /* circulant whose first column is i.i.d. N(0,1) (Sec. 5) */
    RMGE_CIRCULANT_UNIFORM = 2,  /* circulant whose first column is i.i.d. U[-1,1) (Ex. 5.1) */
    RMGE_CIRCULANT_UNITARY = 3,  /* unitary circulant of Ex. 5.2: spectrum u_j = exp(2 pi phi_j sqrt(-1)),
                                    phi_j i.i.d. U[0,1), drawn Hermitian-symmetric (u_{n-j} = conj(u_j),
                                    u_0, u_{n/2} = +-1) so that C is real orthogonal; c = Omega^{-1} u */
    RMGE_TOEPLITZ_GAUSSIAN = 4,  /* Toeplitz multiplier: the leading n x n block of the 2n x 2n circulant
                                    with an i.i.d. N(0,1) first column (Sec. 7.2's leading blocks of
                                    random circulants), applied by 2n-point FFTs */
    RMGE_TOEPLITZ_UNIFORM = 5    /* the same from an i.i.d. U[-1,1) first column (Ex. 5.1) */
} rmge_mult_kind;

/* Precision of the working matrix M and of its factorization. */
typedef enum {
    RMGE_F64 = 0,    /* FP64 everywhere */
    RMGE_F32 = 1,    /* FP32 working matrix and FP32 SIMT trailing updates */
    RMGE_BF16_TC = 2,/* FP32 working matrix; trailing updates on tcgen05 tensor cores, BF16 operands, FP32 accumulation */
    RMGE_F16_TC = 3, /* as RMGE_BF16_TC with FP16 operands (power-of-two operand scaling for range) */
    RMGE_BF16X3_TC = 4, /* as RMGE_BF16_TC, each FP32 operand split x = x_hi + x_lo into two BF16 terms and the
                           product formed as x_hi y_hi + x_hi y_lo + x_lo y_hi (three tensor-core passes) */
    RMGE_F16X3_TC = 5,  /* the three-pass split with FP16 terms */
    RMGE_F64X_TC = 6    /* FP64 working matrix, factors and refinement; M = A G and GENP's Schur-complement
                           updates are FP64 products emulated on the BF16 tensor cores (7 balanced base-256
                           digits per entry, 28 digit-pair products in exact FP32 chunks, 64-bit fixed-point
                           sums; the updates first balance column k of L21 against row k of U12 by a power
                           of two; while 4096 or more rows remain, pivot steps go in pairs with one step of
                           look-ahead, one 128-deep update per pair); pivot blocks, panels, solves and
                           residuals run on the FP64 pipe */
} rmge_prec;

/*
 * Options of the _ex entry points.  rmge_options_init fills the defaults, which are what the calls
 * without _ex use; a NULL options pointer means the defaults too.
 * - growth_tol (default 0 = no gate): rmge_factor_ex reports RMGE_ERR_GROWTH when the pivot growth
 *   max|U_ij| / max|M_ij| exceeds it.  Thm 3.2 bounds the pivots of GENP on a Gaussian-multiplied
 *   matrix and Remark 3.2 ties the stability of GENP to that growth; growth near 1/u of the factor
 *   precision means the factors carry no correct digits.
 * - spin_limit (default 2^22, about a second): polls of each bounded device-side wait of the
 *   triangular solves (a row block waits for the blocks it depends on) and of the batched solve (a
 *   system waits for the CTAs that share its FP64 fallback product) before the wait gives up: the
 *   solve then records RMGE_ERR_TIMEOUT and its CTAs return without writing; the batched system gets
 *   info -1.  0 gives up at the first unmet poll.  The tensor-core kernels keep their own
 *   time-based limit.
 * - gmres_m (default 16, at most 256): restart length of the FGMRES cycles that refinement runs
 *   with reduced-precision factors (see rmge_refine).  The workspace grows with it
 *   (rmge_workspace_size_ex).  A cycle also ends once every column's residual estimate has fallen by
 *   a factor 1e-6.
 * - apply_digits (default 7, from 1 to 7): balanced base-256 digits per entry that
 *   rmge_apply_multiplier_ex keeps for RMGE_F64X_TC with a Gaussian multiplier.  7 digit planes (28
 *   digit-pair products, 55 bits per operand) reproduce FP64 rounding; d digits keep d (d + 1) / 2
 *   products and 8 d - 1 bits, which is M = A G with a relative error near (d + 5) 2^(-8 d) of the row
 *   and column maxima per term.  Refinement with FP64 residuals wins that back while kappa(A G) times
 *   that error stays well below 1 (a sweep more for each factor of about 1e4 lost); the factorization
 *   itself is unchanged.
 * - factor_digits (default 7, from 4 to 7): the same for GENP's Schur updates in rmge_factor_ex with
 *   RMGE_F64X_TC (d (d + 1) / 2 digit-pair products per update).  Fewer digits give factors of about
 *   8 d - 1 bits: the growth g of GENP multiplies their error, so refinement to FP64 accuracy needs
 *   kappa(A G) g 2^(-8 d) well below 1, and then takes a sweep for each factor of that product lost.
 * - status (device int32, may be NULL): receives the call's outcome, RMGE_OK or the first of
 *   RMGE_ERR_TIMEOUT, RMGE_ERR_BREAKDOWN, RMGE_ERR_NONFINITE, then RMGE_ERR_GROWTH (factor) or
 *   RMGE_ERR_NOT_CONVERGED (refine) that applies; valid once the stream is synchronised.
 * - sync (default 0): nonzero makes the call synchronise `stream` after enqueuing its work and return
 *   that outcome instead of RMGE_OK (not for use inside stream capture).
 */
typedef struct rmge_options {
    double growth_tol;
    int64_t spin_limit;
    int32_t* status;
    int32_t gmres_m;
    int32_t apply_digits;
    int32_t sync;
    int32_t factor_digits;
} rmge_options;

void rmge_options_init(rmge_options* opts);

/*
 * Multiplier storage (what `G` points to in every call below):
 * - RMGE_GAUSSIAN: n x n row-major, leading dimension n; FP64 for RMGE_F64 and RMGE_F64X_TC, FP32
 *   for the other precisions.
 * - circulant kinds: 3n FP64 values: the first column c[0..n-1], then its DFT u = Omega c
 *   (Theorem 5.1; Omega = (w^{ij}), w = exp(2 pi sqrt(-1) / n)) stored as n interleaved
 *   (re, im) pairs.  n must be a power of two, 4 <= n <= 16384.
 * - Toeplitz kinds: 6n FP64 values, the same for the 2n x 2n circulant whose leading n x n block
 *   is the multiplier: c2[0..2n-1], then its 2n-point DFT.  n a power of two, 2 <= n <= 8192.
 *   (No square Toeplitz multiplier is cut from a unitary circulant: that block is singular exactly
 *   when u_0 u_n = -1.)
 * rmge_multiplier_bytes returns the size (0 for an invalid request).
 */
size_t rmge_multiplier_bytes(rmge_mult_kind kind, int64_t n, rmge_prec prec);

/*
 * Scratch bytes needed by any of the calls below for this (n, nrhs, kind, prec); one buffer of
 * this size serves all of them.  0 for an invalid request.
 */
size_t rmge_workspace_size(int64_t n, int64_t nrhs, rmge_mult_kind kind, rmge_prec prec);

/* rmge_workspace_size for the _ex calls with these options (the FGMRES basis grows with gmres_m). */
size_t rmge_workspace_size_ex(int64_t n, int64_t nrhs, rmge_mult_kind kind, rmge_prec prec, const rmge_options* opts);

/*
 * The smaller scratch size that rmge_solve, and rmge_solve_backward without refinement, need
 * (no tensor-core operand buffers and no refinement work).  0 for an invalid request.
 */
size_t rmge_solve_workspace_size(int64_t n, int64_t nrhs, rmge_mult_kind kind, rmge_prec prec);

/*
 * Draw the multiplier (Def. 4.1; Ex. 5.1; Theorem 5.1 for the spectrum).
 * Entries come from the counter-based generator Philox4x32-10 (Salmon et al., SC'11) with
 * key = seed and the 64-bit counter words (2,3) = subsequence; entry e of the stream uses
 * counter words (0,1) = e / 2.  Gaussian entries use Box-Muller on two 53-bit uniforms;
 * uniform entries are 2 m / 2^53 - 1 for a 53-bit integer m.  Identical (seed, subsequence)
 * give identical multipliers on every call.  Writes rmge_multiplier_bytes(kind, n, prec)
 * bytes at G.  The circulant spectrum is computed by an O(n log n) FFT.
 */
rmge_status rmge_make_multiplier(rmge_mult_kind kind, int64_t n, uint64_t seed, uint64_t subsequence,
                                 rmge_prec prec, void* G, rmge_stream_t stream);

/*
 * M = A G (post-multiplication, Fact 4.1).  A: n x n FP64 (lda).  M: n x n (ldm), FP64 for
 * RMGE_F64, FP32 otherwise.  Dense G: 2n^3 - n^2 flops (Sec. 5 cost statement).  Circulant G:
 * each row of A G is the circular cross-correlation of the row of A with c, computed by FFT
 * (Theorem 5.1), O(n^2 log n).  M must not overlap A.
 */
rmge_status rmge_apply_multiplier(rmge_mult_kind kind, int64_t n, const double* A, int64_t lda,
                                  const void* G, void* M, int64_t ldm, rmge_prec prec,
                                  void* ws, size_t ws_bytes, rmge_stream_t stream);
/* rmge_apply_multiplier with options (apply_digits for RMGE_F64X_TC; the other fields do not apply). */
rmge_status rmge_apply_multiplier_ex(rmge_mult_kind kind, int64_t n, const double* A, int64_t lda,
                                     const void* G, void* M, int64_t ldm, rmge_prec prec, const rmge_options* opts,
                                     void* ws, size_t ws_bytes, rmge_stream_t stream);

/*
 * In-place blocked GENP of M (eq. (3.1) with pivot blocks of nb columns; by Sec. 3 every
 * blocking yields the same Schur complements, hence the same L and U as unblocked GENP).
 * On exit M holds the unit lower factor L strictly below the diagonal and U on and above it.
 * info (device int32): 0, or the 1-based step of the first zero or non-finite pivot (Cor. 3.1:
 * a leading block of M is singular); after a breakdown the remaining steps are skipped and M is
 * partially factored.  growth (device double, may be NULL): max|U_ij| / max|M_ij| over the input
 * M (the pivot-growth quantity bounded by Thm 3.2 / Remark 3.2); +Inf/NaN if non-finite values
 * appeared.  prec selects the trailing-update engine and M's type (FP64 or FP32).
 */
rmge_status rmge_factor(int64_t n, void* M, int64_t ldm, rmge_prec prec, int32_t* info, double* growth,
                        void* ws, size_t ws_bytes, rmge_stream_t stream);
/* rmge_factor with options: growth gate (RMGE_ERR_GROWTH), status and sync as described there. */
rmge_status rmge_factor_ex(int64_t n, void* M, int64_t ldm, rmge_prec prec, int32_t* info, double* growth,
                           const rmge_options* opts, void* ws, size_t ws_bytes, rmge_stream_t stream);

/*
 * X = G U^{-1} L^{-1} B (Fact 4.1: x = H y with (A H) y = b), nrhs right-hand sides.
 * LU: packed factors from rmge_factor (FP64 for RMGE_F64, FP32 otherwise).  B, X: n x nrhs FP64;
 * X must not overlap B.  For reduced precisions B is rounded to FP32 for the triangular solves
 * and X = G Y is accumulated in FP32 then widened.
 */
rmge_status rmge_solve(rmge_mult_kind kind, int64_t n, int64_t nrhs, const void* LU, int64_t ldlu,
                       const void* G, const double* B, int64_t ldb, double* X, int64_t ldx, rmge_prec prec,
                       void* ws, size_t ws_bytes, rmge_stream_t stream);
/* rmge_solve with options: the spin limit of the triangular solves' waits, and a status of RMGE_ERR_TIMEOUT
 * or RMGE_ERR_NONFINITE (X holds an Inf or NaN, e.g. from factors that broke down). */
rmge_status rmge_solve_ex(rmge_mult_kind kind, int64_t n, int64_t nrhs, const void* LU, int64_t ldlu,
                          const void* G, const double* B, int64_t ldb, double* X, int64_t ldx, rmge_prec prec,
                          const rmge_options* opts, void* ws, size_t ws_bytes, rmge_stream_t stream);

/*
 * Iterative refinement of X (Sec. 1.2 and Sec. 7.1: one or more sweeps of residual
 * correction).  A sweep computes R = B - A X in FP64 and a correction D with A D ~= R, then
 * X <- X + D.  With RMGE_F64 factors D = G U^{-1} L^{-1} R (classical refinement).  With
 * reduced-precision factors (every other rmge_prec) classical refinement diverges once
 * kappa(A G) times the factorization error exceeds one -- and kappa(A G) grows like kappa(A) n for a
 * Gaussian G -- so each sweep instead runs one restarted cycle of flexible GMRES in FP64 on
 * A D = R, right-preconditioned by G U^{-1} L^{-1} applied in the factor precision (GMRES-based
 * refinement, Carson and Higham 2017).  Before each sweep and after the last one the normwise
 * backward error
 *   eta = max_c ||b_c - A x_c||_inf / (||A||_inf ||x_c||_inf + ||b_c||_inf)
 * is computed in FP64 on the device; sweeping stops when eta <= be_tol, after max_iters sweeps,
 * or when eta fails to halve over two sweeps (stagnation).  0 <= max_iters <= 64.
 * berr (device double[max_iters + 1], may be NULL): eta before sweep 0, 1, ...; entries after
 * the last evaluated one are set to -1.  iters (device int32, may be NULL): sweeps performed.
 * The sweep loop runs on the device state only: every sweep's kernels are enqueued and skip
 * their work once the stopping test has fired, so the call never synchronises the stream.
 * Returns RMGE_OK once enqueued; whether eta <= be_tol is read from berr/iters afterwards.
 */
rmge_status rmge_refine(rmge_mult_kind kind, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                        const void* LU, int64_t ldlu, const void* G, const double* B, int64_t ldb,
                        double* X, int64_t ldx, rmge_prec prec, int32_t max_iters, double be_tol,
                        double* berr, int32_t* iters, void* ws, size_t ws_bytes, rmge_stream_t stream);
/* rmge_refine with options: FGMRES restart length, spin limit, and a status of RMGE_ERR_TIMEOUT,
 * RMGE_ERR_NONFINITE (the last backward error is not finite) or RMGE_ERR_NOT_CONVERGED (it is above be_tol).
 * ws: rmge_workspace_size_ex bytes for these options. */
rmge_status rmge_refine_ex(rmge_mult_kind kind, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                           const void* LU, int64_t ldlu, const void* G, const double* B, int64_t ldb,
                           double* X, int64_t ldx, rmge_prec prec, int32_t max_iters, double be_tol,
                           double* berr, int32_t* iters, const rmge_options* opts, void* ws, size_t ws_bytes,
                           rmge_stream_t stream);

/*
 * Adjoint of X = A^{-1} B for a loss L with dX = dL/dX given (n x nrhs): reusing the factors of
 * A G = L U, A^{-T} = L^{-T} U^{-T} G^T, so
 *   dB = L^{-T} U^{-T} (G^T dX)   (n x nrhs, FP64 out)
 *   dA = -dB X^T                   (n x n, FP64 out, ldda; may be NULL to skip)
 * X: the solution (n x nrhs FP64).  dB must not overlap dX.  With max_iters > 0 and A given, dB is
 * then refined on the transposed system A^T dB = dX exactly as rmge_refine refines X (FP64
 * residuals; classical sweeps for FP64 factors, FGMRES sweeps otherwise), with berr / iters as
 * there; max_iters = 0 skips refinement (A, berr, iters may be NULL).  The scratch needed is
 * rmge_solve_workspace_size without refinement and rmge_workspace_size with it.  (The paper has no
 * gradients; this is the adjoint of the linear solve its method computes.)
 */
rmge_status rmge_solve_backward(rmge_mult_kind kind, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                                const void* LU, int64_t ldlu, const void* G, const double* X, int64_t ldx,
                                const double* dX, int64_t lddx, double* dB, int64_t lddb, double* dA, int64_t ldda,
                                rmge_prec prec, int32_t max_iters, double be_tol, double* berr, int32_t* iters,
                                void* ws, size_t ws_bytes, rmge_stream_t stream);

/*
 * Pre-multiplied and two-sided forms (Fact 4.1: A^{-1} = (F A)^{-1} F and A^{-1} = H (F A H)^{-1} F,
 * so F A H y = F b and x = H y; Remark 5.1 proposes random pre- and post-multipliers together).
 * F (pre-multiplier) and H (post-multiplier) are multipliers drawn by rmge_make_multiplier, with
 * kinds kindF and kindH and the storage above; either pointer may be NULL, meaning the identity
 * (H = NULL is pre-multiplication alone; F = NULL is the post-multiplied solve of the calls above).
 * Data precision FP64 only: RMGE_F64, or RMGE_F64X_TC (dense products emulated on the tensor cores);
 * other precisions return RMGE_ERR_UNSUPPORTED, as do FFT kinds with an unsupported n.
 *
 * rmge_workspace_size_two_sided: scratch bytes for any of the three calls with these kinds (pass the
 * kind of an absent side as RMGE_GAUSSIAN); 0 for an invalid request.
 * rmge_apply_two_sided: M = F A H (n x n, FP64, row-major).  With both F and H, T (n x n, leading
 * dimension ldt >= n, caller-owned FP64 device memory) receives A H first; T may be NULL otherwise.
 * The FFT kinds apply F to the columns (circular convolution) and H to the rows (correlation).
 * rmge_solve_two_sided: X = H U^{-1} L^{-1} F B from the factors of M (rmge_factor).
 * rmge_refine_two_sided: sweeps X <- X + H U^{-1} L^{-1} F (B - A X), residuals in FP64, with the
 * stopping rule, berr and iters of rmge_refine.
 * Errors as for the one-sided calls; every call is asynchronous on `stream`.
 */
size_t rmge_workspace_size_two_sided(int64_t n, int64_t nrhs, rmge_mult_kind kindF, rmge_mult_kind kindH,
                                     rmge_prec prec);
rmge_status rmge_apply_two_sided(rmge_mult_kind kindF, const void* F, rmge_mult_kind kindH, const void* H, int64_t n,
                                 const double* A, int64_t lda, double* M, int64_t ldm, double* T, int64_t ldt,
                                 rmge_prec prec, void* ws, size_t ws_bytes, rmge_stream_t stream);
rmge_status rmge_solve_two_sided(rmge_mult_kind kindF, const void* F, rmge_mult_kind kindH, const void* H, int64_t n,
                                 int64_t nrhs, const void* LU, int64_t ldlu, const double* B, int64_t ldb, double* X,
                                 int64_t ldx, rmge_prec prec, void* ws, size_t ws_bytes, rmge_stream_t stream);
rmge_status rmge_refine_two_sided(rmge_mult_kind kindF, const void* F, rmge_mult_kind kindH, const void* H, int64_t n,
                                  int64_t nrhs, const double* A, int64_t lda, const void* LU, int64_t ldlu,
                                  const double* B, int64_t ldb, double* X, int64_t ldx, rmge_prec prec,
                                  int32_t max_iters, double be_tol, double* berr, int32_t* iters, void* ws,
                                  size_t ws_bytes, rmge_stream_t stream);

/*
 * Randomized low-rank approximation (Sec. 6, Algorithm 6.1, after Halko, Martinsson and Tropp): for
 * A (m x n, FP64 row-major) and an n x l multiplier H, Q (m x l) is an orthonormal basis of the range
 * of A H and Z = Q^T A (l x n), so that A ~ Q Z = Q Q^T A (rank <= l).  The paper shows that l equal
 * to the numerical rank r (no oversampling) suffices with Gaussian H.
 * Multipliers: RMGE_GAUSSIAN, H is n x l FP64 (leading dimension l); the circulant kinds
 * (RMGE_CIRCULANT_GAUSSIAN, _UNIFORM, _UNITARY; n a power of two, 4 <= n <= 16384), H is the n x l leading block
 * of the circulant stored as by rmge_make_multiplier (3n FP64; Sec. 7.2's Toeplitz multipliers),
 * applied by FFT.  1 <= l <= 64, l <= m, l <= n.
 * rmge_lowrank_multiplier draws H (the Gaussian entries are the first n l of the stream of
 * rmge_make_multiplier's Gaussian kind).  rmge_lowrank_basis computes B = A H, then Q by CholeskyQR2
 * (two passes of Q^T Q = R^T R, Q <- Q R^{-1}; R has a positive diagonal, so Q is the unique thin QR
 * factor of a full-rank B); it needs B well-conditioned enough for the Cholesky of its Gram matrix
 * (kappa(A H) well below 1e8).  *info (device int32, may be NULL) is 0, or j > 0 when the Cholesky met
 * a non-positive pivot at column j (Q is then not orthonormal).  ws: rmge_lowrank_workspace_size bytes,
 * 256-byte aligned.  rmge_lowrank_project computes Z = Q^T A.  Errors: RMGE_ERR_INVALID_ARG,
 * RMGE_ERR_WORKSPACE; all calls are asynchronous on `stream`.
 */
size_t rmge_lowrank_workspace_size(rmge_mult_kind kind, int64_t m, int64_t n, int32_t l);
rmge_status rmge_lowrank_multiplier(rmge_mult_kind kind, int64_t n, int32_t l, uint64_t seed, uint64_t subsequence,
                                    double* H, rmge_stream_t stream);
rmge_status rmge_lowrank_basis(rmge_mult_kind kind, int64_t m, int64_t n, int32_t l, const double* A, int64_t lda,
                               const double* H, double* Q, int64_t ldq, int32_t* info, void* ws, size_t ws_bytes,
                               rmge_stream_t stream);
rmge_status rmge_lowrank_project(int64_t m, int64_t n, int32_t l, const double* Q, int64_t ldq, const double* A,
                                 int64_t lda, double* Z, int64_t ldz, rmge_stream_t stream);

/*
 * rmge_solve for callers that cannot allocate device memory.  The paper has no counterpart: this is
 * a deployment convenience.  Some callers must not call cudaMalloc at the point where they solve:
 * a serving loop with latency guarantees (a device allocation can synchronise the whole device),
 * or a plugin whose host process owns all device memory and passes it only inputs and outputs.
 * This call takes the same inputs and outputs as rmge_solve but no workspace: its scratch is one
 * file-scope device array of rmge_noalloc_capacity() bytes (16 MiB).  The call itself allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine); it looks up the array's device
 * address with cudaGetSymbolAddress on the current device at every call.  The module that holds the
 * array loads lazily: the first call on each device loads it, which places the array in device
 * memory (held until the process exits) and may synchronise the device, so make one call per device
 * at start-up, before any stream capture or latency-bound loop.  Requests whose
 * rmge_solve_workspace_size exceeds the capacity return RMGE_ERR_WORKSPACE and enqueue nothing (FP64
 * with nrhs = 16 fits n up to about 43 000).  Every call shares the array and leaves its contents
 * behind; each call clears what must start at zero (the control block and the solve flags) on its
 * stream before use, so calls that follow one another on a stream are safe, but calls that overlap
 * on the GPU (other streams, other host threads) race.
 */
rmge_status rmge_solve_noalloc(rmge_mult_kind kind, int64_t n, int64_t nrhs, const void* LU, int64_t ldlu,
                               const void* G, const double* B, int64_t ldb, double* X, int64_t ldx, rmge_prec prec,
                               rmge_stream_t stream);

/* Bytes of the device array rmge_solve_noalloc uses as its scratch. */
size_t rmge_noalloc_capacity(void);

/*
 * Batched solve: count independent systems A_i x_i = b_i (one right-hand side each) of uneven sizes
 * n[i] <= nmax, each by the whole method with FP32 factors (Def. 4.1 multiplier G_i, M_i = A_i G_i,
 * blocked GENP, x_i = G_i U^{-1} L^{-1} b_i) and FP64 refinement sweeps (residual b - A x in FP64,
 * stop at normwise backward error <= be_tol or after max_sweeps), in ONE persistent kernel launch:
 * each CTA takes the next system from a queue in the order given (pass decreasing n), so uneven sizes
 * balance across SMs.  G_i is the FP32 Gaussian multiplier stream (seed, subsequence i) of
 * rmge_make_multiplier.  Sweeps are classical while each halves the backward error, then
 * right-preconditioned GMRES cycles in FP64; when a GMRES cycle fails to halve it (or a pivot is zero)
 * the system starts again with a fresh multiplier from subsequence i + d * count, d = 1, 2 (the method
 * succeeds with probability close to 1 per draw).  max_sweeps bounds the sweeps of each draw; sweeps[i]
 * counts them over all draws.  Device arrays: n[count]; offA[count] element offsets of A_i (n_i x n_i, FP64,
 * row-major, ld n_i) in A; offv[count] element offsets of b_i, x_i in b, x (FP64); order[count] a
 * permutation of 0..count-1; outputs info[i] (0, the first breakdown step, or -1 if the system's wait for
 * other CTAs' share of its FP64 fallback product timed out, which does not happen in a healthy launch),
 * berr[i], sweeps[i].
 * config selects the compiled tile shape (0: 256 threads, 32x32 tiles; 1: 256 threads, 64x64;
 * 2: 1024 threads, 64x64) and ctas the number of persistent CTAs -- both chosen by the autotuner of
 * the Python binding.  ws: rmge_batched_workspace_size(nmax, ctas) bytes, 256-byte aligned (per-CTA
 * scratch for G_i, M_i and vectors).  The launch (one memset of the queue head + one kernel) can be
 * captured in a CUDA graph and replayed.  rmge_solve_batched_ex takes options: spin_limit bounds the
 * waits of the shared fallback product (its owner's wait for the other CTAs' blocks is 16 spin_limit
 * polls of 1 us; an idle CTA offers help for spin_limit polls); status and sync report
 * RMGE_ERR_TIMEOUT if any system's wait gave up (info -1).
 */
size_t rmge_batched_workspace_size(int64_t nmax, int32_t ctas);
rmge_status rmge_solve_batched(int64_t count, const int32_t* n, const int64_t* offA, const int64_t* offv,
                               const int32_t* order, const double* A, const double* b, double* x, int32_t* info,
                               double* berr, int32_t* sweeps, uint64_t seed, int32_t max_sweeps, double be_tol,
                               int64_t nmax, int32_t config, int32_t ctas, void* ws, size_t ws_bytes,
                               rmge_stream_t stream);
rmge_status rmge_solve_batched_ex(int64_t count, const int32_t* n, const int64_t* offA, const int64_t* offv,
                                  const int32_t* order, const double* A, const double* b, double* x, int32_t* info,
                                  double* berr, int32_t* sweeps, uint64_t seed, int32_t max_sweeps, double be_tol,
                                  int64_t nmax, int32_t config, int32_t ctas, const rmge_options* opts, void* ws,
                                  size_t ws_bytes, rmge_stream_t stream);

/*
 * Uniform batches: count independent systems of one order n, each with its own dense Gaussian multiplier
 * G_i (Def. 4.1; drawn per system, e.g. by rmge_make_multiplier), solved by the same method as the calls
 * above -- M_i = A_i G_i (Fact 4.1), blocked GENP of M_i (eq. (3.1), Sec. 3) -- with one launch per kernel
 * and per pivot-block step covering all of them, so that the short latency-bound steps of many small
 * systems run side by side instead of one system after another.  The triangular solves, X_i = G_i Y_i and
 * the refinement then use rmge_solve / rmge_refine per system on the factors left in M_i.
 * Precision RMGE_F64X_TC only (the emulated-FP64 products; other precisions return RMGE_ERR_UNSUPPORTED).
 * Matrices are row-major with leading dimensions lda, ldm >= n; system i's A, G and M start strideA,
 * strideG (G has leading dimension n) and strideM elements after system i-1's, and must not overlap
 * (stride >= (n - 1) ld + n).  1 <= count <= 65535.
 * rmge_batched_uniform_workspace_size: scratch bytes for both calls (count control blocks, per-system digit
 * planes of A and G, exponents and per-step maxima); 0 for an invalid request.
 * rmge_apply_multiplier_batched: M_i = A_i G_i; opts may be NULL (apply_digits applies as for
 * rmge_apply_multiplier_ex).
 * rmge_factor_batched: in-place GENP of every M_i, as rmge_factor; info[i] and growth[i] (device arrays of
 * count entries; growth may be NULL) as rmge_factor reports them; opts may be NULL (factor_digits and
 * spin_limit apply as for rmge_factor_ex; growth_tol, status and sync are not used here: info and growth
 * carry every system's outcome).  A breakdown of one system does not stop the others.
 */
size_t rmge_batched_uniform_workspace_size(int64_t count, int64_t n, rmge_prec prec);
rmge_status rmge_apply_multiplier_batched(int64_t count, int64_t n, const double* A, int64_t lda, int64_t strideA,
                                          const double* G, int64_t strideG, double* M, int64_t ldm, int64_t strideM,
                                          rmge_prec prec, const rmge_options* opts, void* ws, size_t ws_bytes,
                                          rmge_stream_t stream);
rmge_status rmge_factor_batched(int64_t count, int64_t n, double* M, int64_t ldm, int64_t strideM, rmge_prec prec,
                                int32_t* info, double* growth, const rmge_options* opts, void* ws, size_t ws_bytes,
                                rmge_stream_t stream);

/*
 * The rest of a uniform batch, with the FP64 factors that rmge_factor_batched leaves (RMGE_F64 or
 * RMGE_F64X_TC; other precisions return RMGE_ERR_UNSUPPORTED) and dense Gaussian multipliers (leading
 * dimension n): the calls rmge_solve, rmge_refine and rmge_solve_backward make for one system, for all
 * count systems at once, each kernel launched once for all of them.  System i's LU, G, A, B, X, dX, dB and
 * dA start stride* elements after system i-1's (leading dimensions as the single calls take them); berr
 * holds count consecutive arrays of max_iters + 1 entries and iters count entries, as rmge_refine fills
 * them per system.  The refinement is the classical FP64 correction of FP64 factors; each system stops on
 * its own test.  ws: rmge_uniform_solve_workspace_size bytes, 256-byte aligned (one single-system block
 * per system).  Errors as for the single calls.
 */
size_t rmge_uniform_solve_workspace_size(int64_t count, int64_t n, int64_t nrhs, rmge_prec prec);
rmge_status rmge_solve_uniform_batched(int64_t count, int64_t n, int64_t nrhs, const double* LU, int64_t ldlu,
                                       int64_t strideLU, const double* G, int64_t strideG, const double* B,
                                       int64_t ldb, int64_t strideB, double* X, int64_t ldx, int64_t strideX,
                                       rmge_prec prec, void* ws, size_t ws_bytes, rmge_stream_t stream);
rmge_status rmge_refine_uniform_batched(int64_t count, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                                        int64_t strideA, const double* LU, int64_t ldlu, int64_t strideLU,
                                        const double* G, int64_t strideG, const double* B, int64_t ldb,
                                        int64_t strideB, double* X, int64_t ldx, int64_t strideX, rmge_prec prec,
                                        int32_t max_iters, double be_tol, double* berr, int32_t* iters, void* ws,
                                        size_t ws_bytes, rmge_stream_t stream);
rmge_status rmge_solve_backward_uniform_batched(int64_t count, int64_t n, int64_t nrhs, const double* A, int64_t lda,
                                                int64_t strideA, const double* LU, int64_t ldlu, int64_t strideLU,
                                                const double* G, int64_t strideG, const double* X, int64_t ldx,
                                                int64_t strideX, const double* dX, int64_t lddx, int64_t stridedX,
                                                double* dB, int64_t lddb, int64_t stridedB, double* dA, int64_t ldda,
                                                int64_t stridedA, rmge_prec prec, int32_t max_iters, double be_tol,
                                                double* berr, int32_t* iters, void* ws, size_t ws_bytes,
                                                rmge_stream_t stream);

/* Number of kernel launches this process has enqueued through the library so far (host-side
 * counter; lets a caller count the kernels of a timed region). */
unsigned long long rmge_kernel_launches(void);

/* Launch timing of GENP's emulated Schur updates (Sec. 3's E -= L21 U12 on the BF16 tensor cores), a
 * measurement aid.  These launches happen inside rmge_factor*, out of the caller's reach, and they take
 * the largest share of the RMGE_F64X_TC solve's time.
 *   RMGE_TIMED_UPDATE128  the 128-deep update of two paired pivot steps (oz_update128_kernel);
 *   RMGE_TIMED_UPDATE     the 64-deep update of one step, and the two thin strips of a paired step
 *                         (oz_update_kernel).
 * rmge_launch_timing(1) clears the records and starts recording: each later launch of these kernels
 * records a CUDA event pair around itself on its own stream, with its BF16 MMA work, digit pairs
 * s(s+1)/2 x 2 M N K per system.  rmge_launch_timing(0) stops recording.  Launches on a stream that is
 * being captured into a CUDA graph are not recorded, and neither are launches beyond the 65536th.
 * Returns RMGE_OK, or RMGE_ERR_INVALID_ARG for `enable` other than 0 or 1.
 * rmge_launch_timing_read waits for the recorded launches of `kernel` to finish.  It writes their count,
 * their summed device time in ms and their summed MMA flops.  Returns RMGE_ERR_INVALID_ARG for an unknown
 * kernel or a null pointer, and RMGE_ERR_CUDA if an event fails.  Both calls take a lock; factorizations
 * in several host threads at once interleave their records.  Each event is created on the device current
 * at the time and reused until the next rmge_launch_timing(1), which destroys them: a process that moves
 * to another device calls it again there, or launches on that device go unrecorded. */
typedef enum { RMGE_TIMED_UPDATE128 = 0, RMGE_TIMED_UPDATE = 1 } rmge_timed_kernel;
rmge_status rmge_launch_timing(int32_t enable);
rmge_status rmge_launch_timing_read(int32_t kernel, int64_t* launches, double* ms, double* mma_flops);

/* Human-readable name of a status code (static string). */
const char* rmge_status_string(rmge_status s);

#ifdef __cplusplus
}
#endif

#endif /* RMGE_H */
