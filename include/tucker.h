/*
 * tucker.h -- C ABI of the GB300 (sm_103a) ST-HOSVD library.
 *
 * The library computes the sequentially-truncated HOSVD of Algorithm 1
 * (Sec. 2.2): for each mode n in turn it forms the Gram matrix
 * S = Y_(n) Y_(n)^T of the current tensor, eigendecomposes it, keeps the
 * R_n leading eigenvectors with R_n chosen by the error rule
 * sum_{r>R} lambda_r <= eps^2 ||X||^2 / N, and shrinks the tensor with the
 * mode-n product Y <- Y x_n U_n^T.  Every step runs in this library's own
 * CUDA kernels on one GPU; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Tensors are dense and stored in *natural layout*: element
 *   (i_1, ..., i_N) (0-based) sits at offset i_1 + I_1 (i_2 + I_2 (i_3 + ...)),
 *   i.e. the mode-1 unfolding is column-major (Sec. 4.1).  At mode n the
 *   library views a tensor of current dimensions J_1..J_N as the 3-D array
 *   (L, J_n, B) with L = prod_{m<n} J_m (fastest) and B = prod_{m>n} J_m;
 *   entry (l, j, b) is at l + L (j + J_n b).  This is the unfolding of
 *   Sec. 2.1 read in place: no data is moved.
 * - Matrices (factors, Gram matrices, eigenvector matrices) are column-major.
 * - Sizes are int64_t; mode numbers and mode orders are 0-based.
 * - "device" pointers are CUDA global-memory pointers on the current device;
 *   "host" pointers are ordinary (ideally pinned) host memory.
 * - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Every call is stream-ordered on it; calls that return results on the host
 *   synchronise that stream before returning.
 * - Inputs are never modified.  Errors are reported only through the returned
 *   tucker_status (never by exceptions, exit() or a device trap); the text of
 *   the last error of the calling thread is available from tucker_last_error().
 * - Device kernels contain no unbounded waits: the Jacobi eigensolver stops
 *   after a fixed number of sweeps (TUCKER_ENOCONV), and every wait of the
 *   tensor-core kernels gives up after a bounded time, sets an error flag and
 *   returns (TUCKER_ETIMEOUT).
 */
#ifndef TUCKER_GB300_H
#define TUCKER_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define TUCKER_API __attribute__((visibility("default")))
#else
#define TUCKER_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define TUCKER_MAX_MODES 16
/* Largest mode length the eigensolver accepts (the paper assumes I_n <= 2000,
 * Sec. 2.2; the Gram-plus-eigensolver route is the paper's choice there). */
#define TUCKER_MAX_DIM 1024

typedef enum {
  TUCKER_OK = 0,
  TUCKER_EINVAL = -1,      /* invalid argument (null pointer, size, NaN eps, bad order) */
  TUCKER_ENOMEM = -2,      /* device or pinned host allocation failed */
  TUCKER_ECUDA = -3,       /* a CUDA runtime call or kernel launch failed */
  TUCKER_ENOCONV = -4,     /* Jacobi eigensolver hit its sweep cap */
  TUCKER_ETIMEOUT = -5,    /* a bounded device wait of a tensor-core kernel expired */
  TUCKER_ENONFINITE = -6,  /* input holds Inf/NaN (||X||^2 is not finite) */
  TUCKER_EUNSUPPORTED = -7 /* valid request the library does not implement */
} tucker_status;

/* Element type of an input tensor.  Internal tensors are always float64. */
typedef enum { TUCKER_F64 = 0, TUCKER_F32 = 1 } tucker_dtype;

/* Arithmetic of the Gram and mode-product steps.  TUCKER_PREC_FP64 is the
 * plain method.  TUCKER_PREC_BF16X4 ("BF16 digits") runs both on the BF16
 * tensor cores with exact integer digits: the Gram rounds every entry to 21
 * bits below the power of two above its row's largest magnitude in a group
 * of 512 columns and splits it into three balanced 7-bit digits (see
 * tucker_gram_split); the mode product rounds each column of the unfolding
 * and of U_n to 28 bits and splits them into four digits (see
 * tucker_ttm_split).  Digit products accumulate exactly in FP32 tensor
 * memory and are reduced in float64; ||X||^2, the eigensolver and the rank
 * rule stay float64.  The name counts the four digit tiles each operand
 * stage holds.  It needs I_n <= 128 at every mode. */
typedef enum {
  TUCKER_PREC_FP64 = 0,
  TUCKER_PREC_BF16X4 = 1,
  /* The Gram on the FP8 tensor cores (tcgen05 kind::f8f6f4): every entry is
   * rounded to 15 bits below its (row, 512-column group) power of two and
   * split into four balanced base-16 digits that E4M3 holds exactly (see
   * tucker_gram_split_e4m3); ||X||^2 comes from a float64 pass over X and the
   * mode product is that of TUCKER_PREC_BF16X4.  16 bits per entry instead
   * of 22: its error against float64 is measured, not bounded to the float64
   * path's. */
  TUCKER_PREC_E4M3X4 = 2
} tucker_precision;

/* Which eigensolver produced a mode's eigenpairs (tucker_result.eig_path). */
typedef enum {
  TUCKER_EIG_MIXED = 0,          /* mixed-precision solver, result verified on the device */
  TUCKER_EIG_JACOBI = 1,         /* float64 Jacobi (J outside the mixed-precision range, or forced) */
  TUCKER_EIG_JACOBI_FALLBACK = 2 /* float64 Jacobi after the mixed-precision result failed its check */
} tucker_eig_path;

/* Result of an ST-HOSVD (Algorithm 1's output (G, {U_n}) plus diagnostics).
 * Owned by the library; release with tucker_result_free(). */
typedef struct tucker_result {
  int N;                              /* number of modes */
  int on_host;                        /* 0: core/factors are device pointers; 1: host */
  int64_t dims[TUCKER_MAX_MODES];     /* I_n */
  int64_t ranks[TUCKER_MAX_MODES];    /* R_n chosen by the error rule */
  int mode_order[TUCKER_MAX_MODES];   /* order in which the modes were processed */
  int sweeps[TUCKER_MAX_MODES];       /* Jacobi sweeps used per mode */
  double *core;                       /* prod(R_n) float64, natural layout, mode positions as in X */
  double *factors[TUCKER_MAX_MODES];  /* U_n: I_n x R_n float64, column-major, orthonormal columns */
  double *eigvals[TUCKER_MAX_MODES];  /* host: the I_n eigenvalues of S_n, descending.  Past the
                                         rank cut, a cluster of eigenvalues whose sum with all
                                         smaller ones is within the threshold may be left
                                         unresolved (Algorithm 1 needs only the leading R_n
                                         eigenvectors and the discarded sum): its entries are
                                         then Rayleigh quotients of a basis of its invariant
                                         subspace, and every sum from the cut on stays exact */
  double tail[TUCKER_MAX_MODES];      /* discarded eigenvalue sum per mode (clamped at 0) */
  double norm2_x;                     /* ||X||^2 */
  double threshold;                   /* eps^2 ||X||^2 / N (0 when eps <= 0) */
  int eig_path[TUCKER_MAX_MODES];     /* tucker_eig_path of each mode's eigensolve */
  int eig_resolved[TUCKER_MAX_MODES]; /* leading eigenvalues of mode n resolved one by one (I_n unless a
                                         tail cluster was left unresolved; eigvals past this count are
                                         Rayleigh quotients whose sum is exact) */
  void *priv;                         /* library bookkeeping; do not touch */
} tucker_result;

/*
 * tucker_sthosvd -- Algorithm 1 (ST-HOSVD), Sec. 2.2.
 *   X          device, prod(dims) elements of type dt, natural layout; read only.
 *   dims, N    I_1..I_N, 1 <= N <= TUCKER_MAX_MODES, 1 <= I_n <= TUCKER_MAX_DIM.
 *   eps        relative error target (not squared).  eps <= 0 keeps every index
 *              (R_n = I_n); NaN is rejected.  R_n is the smallest R in [1, J_n]
 *              with sum_{r>R} max(lambda_r, 0) <= eps^2 ||X||^2 / N, where ||X|| is
 *              the norm of the original X (Algorithm 1; Sec. 7.2).
 *   mode_order 0-based permutation of 0..N-1 giving the processing order, or NULL
 *              for 0..N-1 ("the modes can be processed in any arbitrary order",
 *              Sec. 2.2).  The core keeps the original mode positions.
 *   prec       arithmetic of the Gram step (TUCKER_PREC_FP64).
 *   out        filled on success with device-resident core and factors
 *              (stream-ordered allocations) and host eigenvalues.
 * Synchronises `stream` once per mode (the rank decides the next launch shape).
 * Returns TUCKER_OK, EINVAL, ENOMEM, ECUDA, ENOCONV or ENONFINITE; on error
 * `out` holds nothing that needs freeing.
 */
TUCKER_API int tucker_sthosvd(const void *X, tucker_dtype dt, const int64_t *dims, int N, double eps,
                   const int *mode_order, tucker_precision prec, void *stream, tucker_result *out);

/*
 * tucker_sthosvd_host -- the same computation for a tensor in host memory.
 * Copies X_host (pinned memory recommended) to the device, runs
 * tucker_sthosvd, and returns the core and factors in library-allocated host
 * memory (out->on_host = 1).  Device buffers are released before returning.
 * With TUCKER_PREC_BF16X4 and mode 1 processed first, the copy goes in up to
 * eight chunks of columns of the mode-1 unfolding on a stream of the
 * library's own, and mode 1's Gram runs chunk by chunk as they land (the
 * chunks' Grams are summed), so the copy hides that pass; the result then
 * equals tucker_sthosvd's up to the rounding of that sum (ranks and
 * discarded sums to ~1e-15 relative).  Otherwise one copy, also on the
 * library's stream, before the compute.  Synchronises `stream`.
 */
TUCKER_API int tucker_sthosvd_host(const void *X_host, tucker_dtype dt, const int64_t *dims, int N, double eps,
                        const int *mode_order, tucker_precision prec, void *stream, tucker_result *out);

/*
 * tucker_sthosvd_host_many -- tucker_sthosvd_host on `count` host tensors of
 * one shape and dtype, in order, through two device buffers: the copy of
 * tensor k + 1 runs while tensor k is compressed, so a stream of tensors
 * costs about the longer of the two per tensor instead of their sum.  Each
 * result is what tucker_sthosvd_host returns for that tensor alone.
 *   X_hosts  count host pointers, prod(dims) elements each (pinned memory
 *            recommended: a pageable copy cannot overlap).
 *   out      count results, filled in order (out->on_host = 1).
 * count = 0 does nothing.  On error every result is released and zeroed.
 * Device memory: two copies of X at a time.  Synchronises `stream`.
 */
TUCKER_API int tucker_sthosvd_host_many(const void *const *X_hosts, int count, tucker_dtype dt, const int64_t *dims,
                                        int N, double eps, const int *mode_order, tucker_precision prec,
                                        void *stream, tucker_result *out);

/*
 * tucker_reconstruct -- X~ = G x_1 U_1 ... x_N U_N (Eq. reconstruct, Sec. 2.3).
 *   r     a device-resident result (r->on_host == 0).
 *   Xhat  device, caller-allocated, prod(r->dims) float64, natural layout.
 * Uses stream-ordered temporaries for the partial expansions.
 */
TUCKER_API int tucker_reconstruct(const tucker_result *r, double *Xhat, void *stream);

/*
 * tucker_reconstruct_sub -- the subtensor X~[lo_1:hi_1, ..., lo_N:hi_N) of
 * Eq. reconstruct without forming X~: G x_1 U_1[lo_1:hi_1, :] ... x_N
 * U_N[lo_N:hi_N, :], i.e. the same product with subsets of rows of the factor
 * matrices (Sec. 2.3; e.g. one variable, a few time steps or a subgrid).
 *   lo, hi  host arrays of r->N indices, 0 <= lo[n] < hi[n] <= r->dims[n].
 *   Xsub    device, caller-allocated, prod(hi - lo) float64, natural layout
 *           (index lo fastest in mode 1).
 * Returns TUCKER_OK, EINVAL (bad ranges or result), ENOMEM or ECUDA.
 * Synchronises `stream`.
 */
TUCKER_API int tucker_reconstruct_sub(const tucker_result *r, const int64_t *lo, const int64_t *hi, double *Xsub,
                                      void *stream);

/*
 * tucker_hooi -- Algorithm 2 (HOOI, Sec. 2.2), started from Algorithm 1.
 *   X, dt, dims, N, eps, prec  as for tucker_sthosvd (identity mode order); the
 *              ST-HOSVD fixes the ranks R_n and gives the starting factors.
 *   max_iters  >= 0 iterations at most (0 returns the ST-HOSVD result).
 *   tol        >= 0: stop after an iteration that lowers ||X||^2 - ||G||^2 by
 *              at most tol ||X||^2 (the fit test of Algorithm 2).
 *   out        as for tucker_sthosvd; eigvals and tail stay those of the
 *              starting ST-HOSVD.
 *   iters      host int: the iterations run.
 *   fit        NULL or a host array of max_iters + 1 doubles: ||X||^2 - ||G||^2
 *              at the start and after each iteration (a difference of nearly
 *              equal numbers: meaningful while it is well above the rounding
 *              of ||G||^2, ~1e-16 ||X||^2 in float64 and ~1e-8 ||X||^2 with
 *              the split-precision mode products).
 * One iteration: for n = 1..N, Y = X x {U_m^T}_{m != n} with the factors
 * updated so far, U_n = the leading R_n eigenvectors of Y_(n) Y_(n)^T; then
 * G = Y x_N U_N^T.  With prec = TUCKER_PREC_BF16X4 the mode products run on
 * the split-precision kernels and the (small) Grams of Y in float64.
 * Returns the codes of tucker_sthosvd; on error `out` holds nothing.
 */
TUCKER_API int tucker_hooi(const void *X, tucker_dtype dt, const int64_t *dims, int N, double eps, int max_iters,
                           double tol, tucker_precision prec, void *stream, tucker_result *out, int *iters,
                           double *fit);

/*
 * tucker_sthosvd_batched -- Algorithm 1 on `count` independent tensors (the
 * many-small-tensors workload), identity mode order.
 *   When every I_n <= 128 the batch runs as one device pipeline in float64
 *   (the plain method, whatever `prec`): per mode, one launch per phase for
 *   all tensors -- a planner kernel that builds the work list of (tensor,
 *   column range) items from the ranks already chosen on the device, a
 *   persistent Gram over the items, a per-tensor reduction (the first mode's
 *   trace gives ||X_t||^2), one Jacobi CTA per tensor, the rank rule on the
 *   device, a persistent mode product -- captured in one CUDA graph, with no
 *   host round trip until the results are collected.  The columns per item
 *   and the persistent grid come from a small autotuner run on the first call
 *   for a batch shape (see tucker_batched_tuning).  The results' cores and
 *   factors share one device block, released with the last of them.
 *   Otherwise each tensor's ST-HOSVD runs as tucker_sthosvd, the tensors
 *   spread over `workers` host threads, each driving its own stream
 *   (TUCKER_BATCH=threads forces this path).
 *   X        host array of `count` device pointers (type dt, natural layout).
 *   dims     host array of count x N sizes: row i holds tensor i's I_1..I_N.
 *   eps, prec  as for tucker_sthosvd, shared by all tensors.
 *   workers  host threads (0: 8), at most 64.
 *   stream   the workers start after the work already queued on it.
 *   out      host array of `count` results, filled on success; on error all
 *            are released and zeroed, and the first failing tensor's status
 *            and message are returned.
 * Returns when every result is ready.
 */
TUCKER_API int tucker_sthosvd_batched(const void *const *X, tucker_dtype dt, const int64_t *dims, int N, int count,
                                      double eps, tucker_precision prec, int workers, void *stream,
                                      tucker_result *out);

/* Mode-order rules for tucker_mode_order (Sec. 8.3). */
typedef enum {
  TUCKER_ORDER_GREEDY_FLOPS = 0, /* at each step the mode whose step costs the fewest flops */
  TUCKER_ORDER_GREEDY_RATIO = 1, /* at each step the mode with the largest I_n / R_n */
  TUCKER_ORDER_EXHAUSTIVE = 2    /* the order of fewest total flops, every permutation tried (N <= 9) */
} tucker_order_rule;

/*
 * tucker_order_flops -- flops of Algorithm 1 in a mode order, by the cost model
 * of Sec. 6.1 with one process: the step on mode n, with J the product of the
 * current dimensions, costs 2 I_n J (Gram) + 2 R_n J (TTM) + 10/3 I_n^3
 * (eigenvectors), and then J_n becomes R_n.
 *   dims, ranks  host, N values, 1 <= R_n <= I_n (ranks known or estimated).
 *   order        0-based permutation or NULL (0..N-1).  flops: host double.
 * Host only (no device work).  Returns TUCKER_OK or EINVAL.
 */
TUCKER_API int tucker_order_flops(const int64_t *dims, const int64_t *ranks, int N, const int *order,
                                  double *flops);

/*
 * tucker_mode_order -- a processing order for tucker_sthosvd by one of the
 * heuristics of Sec. 8.3 (rule: tucker_order_rule; ties keep the lower mode
 * index, and the exhaustive search keeps the lexicographically first of
 * equal-cost orders).  order: host, N ints (0-based).  Host only.
 * Returns TUCKER_OK or EINVAL.
 */
TUCKER_API int tucker_mode_order(const int64_t *dims, const int64_t *ranks, int N, int rule, int *order);

/*
 * tucker_rel_error -- ||X - X~|| / ||X|| (the normalised RMS error of Sec. 7.2).
 * X~ is never materialised: the last mode's expansion is fused with reading X
 * and accumulating (x - x~)^2 in float64.  rel_out is a host double.
 * Returns 0 for X = 0 = X~, +Inf for X = 0 != X~.  Synchronises `stream`.
 */
TUCKER_API int tucker_rel_error(const void *X, tucker_dtype dt, const tucker_result *r, double *rel_out, void *stream);

/* Release everything a tucker_result owns (device and host) and zero it.
 * Safe on a zeroed struct.  Synchronises the device if device memory is freed. */
TUCKER_API void tucker_result_free(tucker_result *r);

/* ---------------------------------------------------------------------------
 * The steps of Algorithm 1 as separate calls (same kernels as tucker_sthosvd).
 * ------------------------------------------------------------------------- */

/* ||X||^2 = sum of squares of n elements (Sec. 2.1), float64 accumulation in a
 * fixed order (run-to-run identical).  X may be NULL when n == 0.  out is a
 * host double; synchronises. */
TUCKER_API int tucker_norm2(const void *X, tucker_dtype dt, int64_t n, double *out, void *stream);

/* Gram step of Algorithm 1: S = Y_(n) Y_(n)^T for Y viewed as (L, J, B):
 * S[i + J j] = sum_{b<B} sum_{l<L} Y[l + L(i + J b)] Y[l + L(j + J b)].
 *   Y  device, L*J*B elements of type dt.   S  device, J*J float64, written in
 *   full (both triangles, exactly symmetric).  J <= TUCKER_MAX_DIM. */
TUCKER_API int tucker_gram(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *S, void *stream);

/* Eigenvector step of Algorithm 1: all eigenpairs of the symmetric J x J matrix S
 * (device, column-major; only its upper triangle is read) by cyclic Jacobi in
 * float64 with a parallel (round-robin) rotation order.
 *   lam  device, J values, descending (ties keep the lower index first).
 *   V    device, J*J column-major; column r is the eigenvector of lam[r], signed so
 *        that its largest-magnitude entry is positive (lowest row on ties).
 *   sweeps  host int (may be NULL): sweeps used.  Synchronises; returns
 *   TUCKER_ENOCONV after the sweep cap. */
TUCKER_API int tucker_eig(const double *S, int64_t J, double *lam, double *V, int *sweeps, void *stream);

/* Rank step of Algorithm 1: smallest R in [1, J] with sum_{r>R} max(lam[r], 0) <=
 * threshold, tails summed from the smallest eigenvalue upward; keep_all != 0
 * returns R = J.  lam is device (descending); R and tail are host; synchronises. */
TUCKER_API int tucker_rank_cut(const double *lam, int64_t J, double threshold, int keep_all, int64_t *R, double *tail,
                    void *stream);

/* Split-precision Gram step: the Gram of tucker_gram (same view, layout and
 * output) computed on the BF16 tensor cores (tcgen05, accumulators in tensor
 * memory).  Columns are taken in groups of 512; with 2^E_ig the smallest
 * power of two above row i's largest magnitude in group g, each entry is
 * rounded to the integer v = round(y 2^(21 - E_ig)) and split into three
 * balanced digits (|s1| <= 128, |s2|, |s3| <= 64) that BF16 holds exactly;
 * digit products of levels 2..5 are accumulated exactly in FP32 and drained
 * into double-float sums every 512 columns, the level-6 squares of the
 * diagonal are added exactly, and the float64 result is symmetrised.  The
 * difference from the float64 Gram is the rounding of Y to 21 bits below
 * each local power of two, plus zero-mean level-6 off-diagonal terms of
 * relative size ~2^-28.  The exponents come from a pass over Y on the device
 * (no host round trip besides the final synchronisation).
 *   J <= 128 (else TUCKER_EUNSUPPORTED).  An Inf or NaN in Y makes every
 *   entry of S NaN.  Synchronises `stream`; returns TUCKER_ETIMEOUT if a
 *   bounded tensor-core wait expired.  No counterpart in the paper (its Gram
 *   is float64, Sec. 5.3); this is the split-precision reading of the Gram
 *   step of Algorithm 1. */
TUCKER_API int tucker_gram_split(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *S,
                                 void *stream);

/* The Gram of tucker_gram_split (same arguments, view, output and error
 * codes) from E4M3 digits on the FP8 tensor cores: each entry is rounded to
 * the integer v = round(y 2^(15 - E_ig)) (|v| <= 2^15) and split into four
 * balanced base-16 digits (|d| <= 8, exact in E4M3); the seven digit-product
 * levels accumulate exactly in FP32 tensor memory (four accumulators, scaled
 * digit tiles folding pairs of levels) and are reduced in float64.  The only
 * difference from the float64 Gram is the rounding of Y to 15 bits below each
 * local power of two (radius 2^(E_ig - 16)).  J <= 128.  No counterpart in
 * the paper (its Gram is float64, Sec. 5.3). */
TUCKER_API int tucker_gram_split_e4m3(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *S,
                                      void *stream);

/* Split-precision TTM step: Z = Y x_n U^T for Y viewed as (L, J, B) and Z as
 * (L, R, B), i.e. Z[l + L(r + R b)] = sum_j U[j + J r] Y[l + L(j + J b)], on the
 * BF16 tensor cores.  Each column of U is rounded to 28 bits below the power of
 * two above its largest magnitude, and so is each column (l, b) of Y (its J
 * entries); both are split into four exact BF16 digits; digit products of
 * levels 2..5 accumulate exactly in FP32 tensor memory (levels 6..8 are
 * dropped), and every output is assembled exactly in int64 before the
 * float64 store.  The difference from the float64 product is bounded by
 * h_r |y_c|_1 + |u_r|_1 h_c + J h_r h_c + 2^-26 (|U|^T |Y|)_rc with h the
 * rounding radii 2^(e - 29).
 *   U  device, J x R float64 column-major; R <= J <= 128 (else
 *   TUCKER_EUNSUPPORTED).  Synchronises; TUCKER_ETIMEOUT if a bounded
 *   tensor-core wait expired. */
TUCKER_API int tucker_ttm_split(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, const double *U,
                                int64_t R, double *Z, void *stream);

/* TTM step of Algorithm 1 (Sec. 2.1 mode-n product): Z = Y x_n M with Y viewed as
 * (L, J, B) and Z as (L, K, B): Z[l + L(k + K b)] = sum_j M[k, j] Y[l + L(j + J b)].
 *   M is given column-major as either K x J (trans_m == 0, M[k,j] = Mp[k + K j]) or
 *   J x K and used transposed (trans_m != 0, M[k,j] = Mp[j + J k]; pass U_n with
 *   trans_m = 1 for the shrinking product Y x_n U_n^T).
 *   Y device (dt), M device float64, Z device float64 with L*K*B elements. */
TUCKER_API int tucker_ttm(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, const double *M, int64_t K,
               int trans_m, double *Z, void *stream);

/* tucker_gram_noalloc -- the Gram step of tucker_gram, for callers that cannot
 * allocate device memory.  The paper has no counterpart: it is an addition for
 * callers such as a process whose framework has already reserved nearly all
 * of the GPU's memory for its own pool, or code that must not trigger the
 * device-wide synchronisation that cudaMalloc/cudaFree can cause.
 *   Same arguments, layout and result as tucker_gram (the caller passes Y and S).
 *   The split-K partial sums live in a static device array of
 *   TUCKER_NOALLOC_SCRATCH_BYTES that each GPU loading the library holds until
 *   the process exits; the call allocates nothing.  Requests whose partial sums
 *   cannot fit (J > TUCKER_MAX_DIM) return TUCKER_EINVAL with a message.
 *   The first call on a device looks up the array's device address (once per
 *   device); make that first call before any stream capture.
 *   All calls on a device share the array: calls whose kernels overlap on the
 *   GPU (different streams or host threads) race and must be serialised.
 *   Stream-ordered; does not synchronise. */
#define TUCKER_NOALLOC_SCRATCH_BYTES (16ll << 20)
TUCKER_API int tucker_gram_noalloc(const void *Y, tucker_dtype dt, int64_t L, int64_t J, int64_t B, double *S,
                                   void *stream);

/* ---------------------------------------------------------------------------
 * Diagnostics.
 * ------------------------------------------------------------------------- */

TUCKER_API const char *tucker_status_string(int status);
/* Message of the last failing call on this thread ("" if none). */
TUCKER_API const char *tucker_last_error(void);
/* Number of kernels this library has launched in this process. */
TUCKER_API int64_t tucker_launch_count(void);

/* Memory held between calls, for monitoring a long-running process.  Any
 * pointer may be NULL.
 *   pool_used      bytes in use in the current device's default stream-ordered
 *                  pool: every live device-resident result and any temporary a
 *                  call on another thread holds (other users of that pool count
 *                  too).  Back at its earlier value once the results made since
 *                  are freed.
 *   pool_reserved  bytes that pool holds from the driver; up to 64 GiB stay
 *                  reserved between calls so repeated ST-HOSVDs do not map
 *                  memory again.
 *   host_cached    bytes of pinned host blocks kept after tucker_result_free of
 *                  host results, for the next host result (at most 4 GiB).
 * Returns TUCKER_OK or TUCKER_ECUDA. */
TUCKER_API int tucker_memory_stats(int64_t *pool_used, int64_t *pool_reserved, int64_t *host_cached);

/* Returns the cached pinned host blocks to the driver and trims the current
 * device's default pool to what is in use.  Synchronises the device.
 * Returns TUCKER_OK or TUCKER_ECUDA. */
TUCKER_API int tucker_memory_trim(void);

/* The tuning of the last batched device pipeline: columns per work item,
 * persistent CTAs, and the six candidates' times in ms (512 / 2048 / 8192
 * columns x 2 / 4 CTAs per SM, the first mode's Gram).  Any pointer may be
 * NULL.  Host only. */
TUCKER_API void tucker_batched_tuning(int64_t *cols_per_item, int *ctas, float *candidate_ms);

/* Float64 throughput of the current GPU: a register-resident loop of
 * independent fused multiply-adds (no memory traffic) over every SM, timed
 * with CUDA events on `stream` after one untimed launch.  The float64 phases
 * of Algorithm 1 (Gram, mode products, eigensolver refinement) are bound by
 * this rate, so it is the roofline peak they are reported against.
 *   tflops  host double: 2 x fused multiply-adds / time, in TFLOP/s.
 *   ms      host double (may be NULL): duration of the timed launch.
 * Synchronises `stream`.  No counterpart in the paper (a measurement aid). */
TUCKER_API int tucker_fp64_peak(double *tflops, double *ms, void *stream);

/* Per-phase device timing with CUDA events recorded on the caller's stream. */
typedef enum {
  TUCKER_PHASE_NORM = 0,
  TUCKER_PHASE_GRAM = 1,   /* the Gram split-K kernel (partials) */
  TUCKER_PHASE_GRAM_REDUCE = 2,
  TUCKER_PHASE_EIG = 3,
  TUCKER_PHASE_RANK = 4,
  TUCKER_PHASE_TTM = 5,
  TUCKER_PHASE_SCALE = 6,   /* exponent-table pass of the split-precision Gram */
  TUCKER_PHASE_TTM_L1 = 7,  /* split-precision TTM of a mode with L == 1 (contiguous columns) */
  TUCKER_PHASE_COUNT = 8
} tucker_phase;

typedef struct tucker_profile {
  double ms[TUCKER_PHASE_COUNT];       /* summed kernel time per phase */
  int64_t launches[TUCKER_PHASE_COUNT];
  double flops[TUCKER_PHASE_COUNT];    /* algorithmic flops (Gram: J(J+1) L B, symmetric count;
                                          TTM: 2 J K L B) */
  double bytes[TUCKER_PHASE_COUNT];    /* algorithmic bytes (inputs read once + outputs written once) */
} tucker_profile;

/* Enable (1) or disable (0) phase timing for calls made afterwards on this process;
 * enabling resets the counters. */
TUCKER_API void tucker_profile_enable(int on);
/* Copy the accumulated counters (phases of completed calls only). */
TUCKER_API void tucker_profile_read(tucker_profile *p);

#ifdef __cplusplus
}
#endif

#endif /* TUCKER_GB300_H */
