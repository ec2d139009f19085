/* nufft.h -- C ABI of the GB300 low-rank NUFFT library (libnufft.so).
 *
 * The transform is the nonuniform DFT of type II of Ruiz-Antolin and Townsend,
 * "A nonuniform fast Fourier transform based on low rank approximation"
 * (arXiv:1701.04492), eq. (1.2):
 *
 *     f_j = sum_{k=0}^{N-1} c_k exp(-2 pi i x_j k),      j = 0..M-1,
 *
 * computed by the method of section 2.2: each sample is rounded to the nearest of
 * L grid points (eqs. (2.8)-(2.9)), the perturbation matrix is replaced by its
 * rank-K Chebyshev/Bessel approximation (eq. (2.6), Theorem A.2), and f is the
 * sum of K diagonally scaled FFTs of length L (eq. (2.11), section 2.3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex arrays are interleaved (re, im), contiguous: float2 for NUFFT_F32
 *   (torch.complex64), double2 for NUFFT_F64 (torch.complex128), as the plan's
 *   precision says.  Real arrays (x, gx) are double for the plan, and of the
 *   plan's precision for gx.
 * - Pointers named *_dev are device pointers owned by the caller; *_host are
 *   host pointers (pinned memory gives the fastest copies).  The library keeps no
 *   reference to any caller pointer after a call returns.
 * - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *   stream).  Exec calls are asynchronous on that stream: they enqueue kernels,
 *   allocate nothing and do not synchronise.
 * - Frequencies are k = 0..N-1 (not centred), with the negative exponent, as in
 *   the paper.  Samples x_j may be any finite reals; they are wrapped by
 *   periodicity (section 2.2 allows samples outside [0, 1)).
 * - Return value: NUFFT_OK (0) or a negative NUFFT_E* code; nufft_strerror()
 *   names it.  No C++ exception crosses this boundary.  A plan stays valid after
 *   an exec call fails.
 * - A plan may be used from one stream at a time: its work buffer is shared by
 *   all exec calls on it.
 */
#ifndef NUFFT_H
#define NUFFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nufft_plan_s *nufft_plan;

enum nufft_prec { NUFFT_F32 = 0, NUFFT_F64 = 1 };

enum nufft_status {
    NUFFT_OK = 0,
    NUFFT_EINVAL = -1,        /* bad argument: size, eps, null pointer, non-finite x */
    NUFFT_ENOMEM = -2,        /* device or host allocation failed */
    NUFFT_ECUDA = -3,         /* a CUDA call failed (no device, launch error, ...) */
    NUFFT_EUNSUPPORTED = -4,  /* a size or mode beyond the library's limits */
    NUFFT_ESTATE = -5,        /* call needs a plan option that was not set */
    NUFFT_ETIMEOUT = -6,      /* a bounded device-side wait gave up (see nufft2_check) */
    NUFFT_ECHECK = -7         /* an index check failed (builds with NUFFT_CHECK; see nufft2_check) */
};

/* Plan flags. */
#define NUFFT_PLAN_UNFUSED 1u  /* also build the materialised factors U (M x K) and
                                  V (N x K) used by nufft2_exec_unfused */
#define NUFFT_PLAN_TIMING 2u   /* record a CUDA event around every kernel the exec
                                  calls launch (see nufft_kernel_times) */
#define NUFFT_PLAN_AUTOTUNE 4u /* with L = 0 (and no NUFFT_PLAN_LONG_COLUMNS): time the
                                  candidate layouts -- the default grid L0 and the
                                  oversampled 2 L0 (section 2.3), each with either
                                  four-step split when log2 L is odd and either pass-1
                                  tile (NUFFT_PLAN_HALF_TILE) -- by one forward
                                  and one adjoint exec each (CUDA events, best of 3
                                  after a warm-up), and keep the fastest.  Choices are
                                  cached per process by (device, N, M rounded up to a
                                  power of two, eps, prec, K), so a repeated shape
                                  plans once.  Synchronises `stream` per candidate. */
#define NUFFT_PLAN_HALF_TILE 64u /* pass 1 (the column pass) takes half as many
                                  columns per CTA: twice the CTAs of half the threads (the
                                  autotuners' tile axis).  Results agree to rounding. */
#define NUFFT_PLAN_LONG_COLUMNS 16u /* for odd log2 L: the four-step split
                                  L = L1 L2 takes the longer FFT on the columns
                                  (L2 = 2 L1) instead of the rows (L1 = 2 L2).
                                  Results agree to rounding; speeds differ. */

/* Planning stage (section 2.3, "Planning the transform").
 *
 * Computes s = rint(L x), t = s mod L, delta = L x - s (eqs. (2.8)-(2.9)) and the
 * scaled perturbation d = delta * N / L in FP64 on the device, then
 * gamma = max |d| (section 2.1.2 "always compute gamma"), the rank K (the smallest
 * rank whose dropped Chebyshev/Bessel terms sum to <= eps, capped by Table 2.1's
 * double-precision row), the coefficients a_pr of eq. (2.6), a bucketing of the
 * samples by grid point, and twiddle tables.
 *
 *   out    receives the plan handle (set to NULL on failure).
 *   N      number of frequencies, 1 <= N <= 2^22.
 *   M      number of samples, 0 <= M < 2^31.
 *   x_dev  M doubles on the device; read during the call only.  Must be finite
 *          with |L x| < 2^52.
 *   eps    working accuracy, 0 < eps < 1.
 *   prec   NUFFT_F32 or NUFFT_F64: the arithmetic of the exec calls.
 *   L      grid size: 0 picks the smallest power of two >= max(N, 1024); a
 *          nonzero value must be a power of two with max(N, 1024) <= L <= 2^22
 *          (L > N is the oversampling variant of section 2.3 and lowers K).
 *   flags  0 or a combination of NUFFT_PLAN_UNFUSED and NUFFT_PLAN_TIMING.
 *
 * Allocates all device memory the exec calls need.  Synchronises `stream` once
 * (to read gamma and validate x).  Errors: NUFFT_EINVAL, NUFFT_EUNSUPPORTED,
 * NUFFT_ENOMEM, NUFFT_ECUDA.
 */
int nufft2_plan(nufft_plan *out, int64_t N, int64_t M, const double *x_dev, double eps,
                int prec, int64_t L, unsigned flags, void *stream);

/* The planner's rank rule, on the host (no GPU call): the smallest K whose
 * dropped terms of eq. (2.6), summed with the weights of the primes (the
 * triangle-inequality bound in the proof of Lemma A.1), are <= eps; capped at Table
 * 2.1's double-precision row; K = 1 for gamma = 0 (section 2.1.2).  gamma is the
 * largest |delta_j| of eq. (2.9), in [0, 1/2].  NUFFT_EINVAL for eps outside (0, 1),
 * gamma outside [0, 1/2] (or NaN), or K NULL. */
int nufft_rank(double eps, double gamma, int *K);

/* The coefficients of eq. (2.6) (Lemma A.1, eq. (A.1)), on the host: alpha[p*K + r]
 * for 0 <= p, r < K, with a_pr = i^r alpha_pr,
 *     alpha_pr = 4 J_{(p+r)/2}(-gamma pi / 2) J_{(r-p)/2}(-gamma pi / 2)   (p - r even),
 * 0 otherwise; J_n by its power series.  alpha: K*K doubles, caller-owned.
 * NUFFT_EINVAL for K outside 1..64, gamma outside [0, 1/2], or alpha NULL. */
int nufft_lowrank_coeffs(int K, double gamma, double *alpha);

/* The autotuner's table (NUFFT_PLAN_AUTOTUNE) across processes.  The choices the
 * tuner has made in this process -- (device, N, M rounded up to a power of two, eps,
 * prec, K) -> (L, four-step split, pass-1 tile) -- can be written to a text file and
 * read back in a later process, whose NUFFT_PLAN_AUTOTUNE plans then take the stored
 * layouts without timing candidates.  A table is only meaningful on the GPU type that
 * wrote it.  No GPU call is made.
 *   nufft_tune_save   writes every entry to `path` (replacing the file).
 *   nufft_tune_load   merges the entries of a file written by nufft_tune_save (an
 *                     entry for a key already present replaces it).  A file that is
 *                     not such a table, or holds an invalid entry (a grid that is not a
 *                     power of two in range, eps outside (0, 1), ...), merges nothing.
 *   nufft_tune_clear  empties the table.
 * entries (may be NULL): the number of entries written, read or present before the
 * clear.  Returns NUFFT_OK, or NUFFT_EINVAL for a NULL path, a file that cannot be
 * opened or written, or a malformed table. */
int nufft_tune_save(const char *path, int64_t *entries);
int nufft_tune_load(const char *path, int64_t *entries);
int nufft_tune_clear(int64_t *entries);

/* Plan facts.  Any output pointer may be NULL.  K = rank, gamma = max |d_j|,
 * L = grid size, work_bytes = device memory the plan owns. */
int nufft2_plan_info(nufft_plan p, int *K, double *gamma, int64_t *L, int64_t *work_bytes);

/* Copy the plan's FP64 rounding results and coefficients out (for checking).
 *   t_dev      M int32 on the device: t_j = mod(rint(L x_j), L)     (eq. (2.9)); may be NULL
 *   d_dev      M doubles on the device: d_j = (L x_j - s_j) N / L   (the scaled
 *              perturbation of eq. (2.10)); may be NULL
 *   alpha_host K*K doubles on the host, [p*K + r] = alpha_pr with the eq. (2.6)
 *              coefficient a_pr = i^r alpha_pr; may be NULL
 * Synchronises `stream`. */
int nufft2_plan_export(nufft_plan p, int32_t *t_dev, double *d_dev, double *alpha_host, void *stream);

/* Release the plan and all device memory it owns.  Safe on NULL.  The caller must
 * make sure no exec on the plan is still running (synchronise its stream). */
int nufft_destroy(nufft_plan p);

/* Online stage, forward (eq. (2.11); the two-step form of section 2.3):
 * f = sum_r D_{u_r} I_L(t,:) F_L D_{v_r} c.
 *   c_dev  N complex coefficients.   f_dev  M complex values (written).
 * c and f must not overlap.  Error bound: |f - f_exact|_inf <= eps ||c||_1 plus
 * rounding of the plan's precision. */
int nufft2_exec(nufft_plan p, const void *c_dev, void *f_dev, void *stream);

/* Adjoint: c = A^H g, the conjugate transpose of nufft2_exec's operator, i.e.
 * c_k = sum_j g_j exp(+2 pi i x_j k).  Section 3.1 gives the transpose (the
 * paper's NUFFT-I) as the same factors with F^T in place of F; the adjoint is
 * its complex conjugate: F~2^T g = conj(A^H conj(g)).
 *   g_dev  M complex values.   c_dev  N complex coefficients (written). */
int nufft1_exec(nufft_plan p, const void *g_dev, void *c_dev, void *stream);

/* Derivative with respect to the samples (not in the paper; the chain rule of
 * eq. (1.2)): gx_j (+)= Re(conj(g_j) f'_j) with f'_j = sum_k (-2 pi i k) c_k
 * exp(-2 pi i x_j k), computed as a second NUFFT-II of (-2 pi i k) o c on the same
 * plan.  This is d/dx_j of Re(sum_j conj(g_j) f_j).
 *   c_dev   N complex, g_dev M complex, gx_dev M reals of the plan's precision.
 *   accumulate  0: gx = ..., 1: gx += ... */
int nufft2_exec_dx(nufft_plan p, const void *c_dev, const void *g_dev, void *gx_dev,
                   int accumulate, void *stream);

/* The forward transform and its derivative with respect to the samples in one
 * call: f = A c and fprime_j = d f_j / d x_j = sum_k (-2 pi i k) c_k exp(-2 pi i x_j k).
 * With k = N (z + 1)/2 and z T_r(z) = (T_{r+1}(z) + T_{r-1}(z))/2 (z = 2k/N - 1),
 * the rank-r factor of A_K((-2 pi i k) o c) is a combination of ranks r - 1, r and
 * r + 1 of the forward, so both come from K + 1 FFTs of length L (eq. (2.11) with
 * one more rank); the result equals nufft2_exec applied to (-2 pi i k) o c.
 *   c_dev N complex; f_dev and fprime_dev M complex (written). */
int nufft2_exec_deriv(nufft_plan p, const void *c_dev, void *f_dev, void *fprime_dev, void *stream);

/* gx_j (+)= Re(conj(g_j) fprime_j): the x-gradient of Re(sum_j conj(g_j) f_j) from
 * the fprime of nufft2_exec_deriv.  g_dev, fprime_dev M complex; gx_dev M reals of
 * the plan's precision; accumulate 0: gx = ..., 1: gx += ... */
int nufft2_grad_x(nufft_plan p, const void *g_dev, const void *fprime_dev, void *gx_dev, int accumulate,
                  void *stream);

/* Reserve what the batch calls and nufft2_step_host need, so that those exec calls
 * allocate nothing and do not synchronise (and can be captured in a CUDA graph).  Not in
 * the paper: part of the planning stage for these entry points.
 *   B_max  the largest batch (B) the batch calls on this plan will be given.  FP32 plans
 *          on grids of up to 2^18 points get a workspace for B_max members (each member's
 *          slice of the rank intermediate, partial sums, pass B's partials) and the
 *          members' kernel arguments, built here once; a larger B_max replaces them.  Other
 *          plans run batch members in turn and need nothing (B_max is then ignored).
 *   what   0 or NUFFT_RESERVE_STEP_HOST: also the device copies, copy stream and events of
 *          nufft2_step_host (1D plans only).
 * Allocates device memory and synchronises `stream`; call it outside any stream capture.
 * Errors: NUFFT_EINVAL (B_max < 0, unknown bits in what), NUFFT_EUNSUPPORTED
 * (NUFFT_RESERVE_STEP_HOST on a 2D plan), NUFFT_ENOMEM, NUFFT_ECUDA. */
#define NUFFT_RESERVE_STEP_HOST 1u
int nufft2_plan_reserve(nufft_plan p, int64_t B_max, unsigned what, void *stream);

/* What is reserved: *B_max = the largest batch the batch calls accept (INT64_MAX for plans
 * that run members in turn), *step_host = 1 when nufft2_step_host's buffers exist.  Either
 * output may be NULL.  No GPU call. */
int nufft2_plan_reserved(nufft_plan p, int64_t *B_max, int *step_host);

/* B coefficient vectors on one plan (the same samples): f_b = A c_b, b = 0..B-1, with
 * c_b at c_dev + b*ldc elements and f_b at f_dev + b*ldf elements (ldc >= N, or m n for
 * a 2D plan; ldf >= M).  FP32 plans on grids of up to 2^18 points run all members in one
 * launch per pass, in the workspace nufft2_plan_reserve made: B beyond the reserved B_max
 * returns NUFFT_ESTATE; other plans run the members in turn.  No allocation, no host
 * synchronisation.  Results are bit-identical to B nufft2_exec calls. */
int nufft2_exec_batch(nufft_plan p, int64_t B, const void *c_dev, int64_t ldc,
                      void *f_dev, int64_t ldf, void *stream);

/* The adjoint of B members: c_b = A^H g_b (g_b at g_dev + b*ldg, ldg >= M; c_b at
 * c_dev + b*ldc, ldc >= N).  Batched launches as nufft2_exec_batch; bit-identical to B
 * nufft1_exec calls. */
int nufft1_exec_batch(nufft_plan p, int64_t B, const void *g_dev, int64_t ldg, void *c_dev, int64_t ldc,
                      void *stream);

/* nufft2_exec_deriv for B members: f_b and fprime_b = df_b/dx at f_dev, fprime_dev +
 * b*ldf (ldf >= M); c_b at c_dev + b*ldc.  Batched launches as nufft2_exec_batch. */
int nufft2_exec_deriv_batch(nufft_plan p, int64_t B, const void *c_dev, int64_t ldc, void *f_dev,
                            void *fprime_dev, int64_t ldf, void *stream);

/* gx_j (+)= sum_b Re(conj(g_bj) fprime_bj) over B members (g_b, fprime_b at + b*ld,
 * ld >= M): the x-gradient of a loss summed over a batch sharing x, in one launch. */
int nufft2_grad_x_batch(nufft_plan p, int64_t B, const void *g_dev, const void *fprime_dev, int64_t ld,
                        void *gx_dev, int accumulate, void *stream);

/* One training step with HOST buffers: f = A c and f' = df/dx (nufft2_exec_deriv),
 * A^H g (nufft1_exec) and gx_j = Re(conj(g_j) f'_j) (nufft2_grad_x), with c and g
 * copied in and f, A^H g and gx copied out.  c is copied in first and the forward runs
 * while g arrives; f and gx are copied out while the adjoint runs.  The copies run on a
 * stream of the plan's own, each as soon as its data is ready; `stream` waits for
 * the last one, and the host buffers hold the results once `stream` has completed (the
 * call does not synchronise).  Pinned host memory makes the copies asynchronous.
 * c_host, gc_host N complex; g_host, f_host M complex; gx_host M reals of the plan's
 * precision.  Uses the device copies of g, f', A^H g and gx that
 * nufft2_plan_reserve(p, ., NUFFT_RESERVE_STEP_HOST, .) made: NUFFT_ESTATE without them.
 * Allocates nothing. */
int nufft2_step_host(nufft_plan p, const void *c_host, const void *g_host, void *f_host, void *gc_host,
                     void *gx_host, void *stream);

/* The same as nufft2_exec with HOST buffers: copies c host->device into a
 * plan-owned staging buffer, runs the transform, copies f device->host and
 * synchronises `stream`. */
int nufft2_exec_host(nufft_plan p, const void *c_host, void *f_host, void *stream);

/* The unfused form of the same method, the section 2.3 one-liner run step by
 * step: W = D_v c for all ranks, K plain FFTs of length L, row gather X(t,:),
 * then f = (U .* X) 1 with the materialised factors.  Needs a plan made with
 * NUFFT_PLAN_UNFUSED (else NUFFT_ESTATE).  A comparator, not the fast path. */
int nufft2_exec_unfused(nufft_plan p, const void *c_dev, void *f_dev, void *stream);

/* Device time of each kernel launched by the plan's most recent exec call, in
 * launch order (forward and dx: pass 1, pass 2; adjoint: pass A, pass B), from
 * CUDA events recorded on the exec's stream.  Needs NUFFT_PLAN_TIMING (else
 * NUFFT_ESTATE).  Writes min(cap, count) values to ms_out and the count to
 * *count.  Waits for the last event. */
int nufft_kernel_times(nufft_plan p, float *ms_out, int cap, int *count);

/* The forward transform without a plan and without any device allocation, for
 * callers that cannot call cudaMalloc (code running inside another allocator's
 * callbacks, plug-ins whose host forbids device allocation, latency-critical
 * paths).  The paper has no counterpart.  It computes what nufft2_plan (FP32) +
 * nufft2_exec compute, with the same rank rule and factors, and keeps every
 * intermediate in one fixed device array compiled into the library (about 17 MiB,
 * held by each GPU that loads the library until exit).
 *   N, M   1 <= N <= 65536, 0 <= M <= 65536; larger sizes return
 *          NUFFT_EUNSUPPORTED (they do not fit the fixed array).
 *   x_dev  M doubles (device), finite, as for nufft2_plan.
 *   eps    working accuracy, 0 < eps < 1.
 *   c_dev  N complex64 (device).   f_dev  M complex64 (device, written).
 * The first call on a device looks up that array's device address.  Every call uses
 * the same array, so calls whose GPU work overlaps (other streams, other threads)
 * race; serialise them.  Synchronises `stream` twice (to read gamma, and at the end to
 * read the device error word), so it cannot be called inside a stream capture or
 * recorded into a CUDA graph.  Errors: NUFFT_EINVAL, NUFFT_EUNSUPPORTED, NUFFT_ECUDA;
 * NUFFT_ETIMEOUT when a bounded device-side wait gave up and NUFFT_ECHECK when an index
 * check failed (libnufft_check.so), as nufft2_check reports them for a plan: f is then
 * invalid. */
int nufft2_exec_noalloc(int64_t N, int64_t M, const double *x_dev, double eps, const void *c_dev,
                        void *f_dev, void *stream);

/* Inverse NUFFT-II (section 3.3): solve A c = f for c (N values) from f (M values),
 * A the NUDFT-II matrix of the plan's samples, by conjugate gradients on the normal
 * equations A^H A c = A^H f.  A^H A is Toeplitz (entries sum_p exp(2 pi i x_p (j - k)));
 * its first column is A^H applied to the all-ones vector, and each iteration applies it
 * with one FFT and one inverse FFT of P >= 2N points through its circulant embedding.
 * The paper takes perturbed equispaced samples with gamma < 1/2 (M = N) so that A is
 * invertible; with M > N this is the least-squares solution when A has full column rank.
 *
 *   f_dev, c_dev   M and N complex values of the plan's precision (device).
 *   tol            stop when ||A^H f - A^H A c||_2 <= tol ||A^H f||_2 (reachable tol: ~1e-13
 *                  in FP64 plans, ~1e-6 in FP32 plans); the accuracy of c is further limited
 *                  by the plan's eps and by the conditioning of A.
 *   maxit          at most this many iterations (0: c = 0).
 *   iterations, relres   if not NULL: iterations taken and the final relative residual.
 *
 * The first call on a plan builds the solver state (an FFT plan of P points, the
 * circulant's eigenvalues, four work vectors: allocates device memory); later calls
 * reuse it.  Synchronises `stream` once per iteration (the convergence test reads the
 * residual).  Errors: NUFFT_EINVAL, NUFFT_EUNSUPPORTED (2D plans; 2N beyond 2^22),
 * NUFFT_ENOMEM, NUFFT_ECUDA, NUFFT_ETIMEOUT (see nufft2_check). */
int nufft2_inverse(nufft_plan p, const void *f_dev, void *c_dev, double tol, int maxit, int *iterations,
                   double *relres, void *stream);

/* ---- The two-dimensional NUFFT-II (section 4) ---------------------------------
 *
 *     f_j = sum_{k1<m} sum_{k2<n} C[k1][k2] exp(-2 pi i (k1 x_j + k2 y_j))   (eq. (4.1))
 *
 * computed as eq. (4.4): each direction is the 1D method at accuracy eps / 2 (x
 * rounded on an m-point grid, y on an n-point grid; the tensor product of the two
 * rank-K approximations is then within eps (1 + eps / 4) of the 2D matrix entrywise),
 * and f is a sum over K_x K_y diagonally scaled 2D FFTs, read at each sample's grid
 * point.  The transforms along k1 (one per x rank) are shared by every y rank.
 * Grids are powers of two of at least 32 points per direction (oversampled when m or n
 * is not one).
 *
 * Reading of section 4's indices, which the text mixes up between m and n: C is m x n,
 * k1 < m pairs with x and k2 < n with y.
 *
 *   m, n    1 <= m, n <= 2048.
 *   M       number of samples, 0 <= M < 2^31.
 *   x_dev, y_dev   M doubles each on the device; read during the call only.
 *   prec    NUFFT_F32 (C and f complex64) or NUFFT_F64 (complex128).  When the
 *           transformed rows of all K_y ranks do not fit in shared memory (FP64 rows
 *           of 1024 or more points, FP32 rows of 2048), the row pass transforms and
 *           gathers the y ranks in groups.
 *   flags   0 or NUFFT_PLAN_TIMING.
 *
 * The plan is a nufft_plan: nufft2_exec(p, C_dev, f_dev, stream) computes f from the
 * row-major m x n matrix C (of the plan's precision), and nufft1_exec(p, g_dev, C_dev,
 * stream) the adjoint, C[k1][k2] = sum_j g_j exp(+2 pi i (k1 x_j + k2 y_j)) (C written
 * row-major m x n): every step of eq. (4.4) conjugated and reversed -- each sample's
 * conj(u^x_r1 u^y_r2) g_j scattered onto its grid row (a segmented sum over the samples
 * sorted by grid point, no atomics, so repeated calls give the same bits), inverse row
 * FFTs over y scaled by the y-factors and summed over r2, then inverse column FFTs over
 * x scaled by the x-factors and summed over r1.  nufft2_exec_batch, nufft1_exec_batch
 * (members in turn; ldc >= m n), nufft2_check and nufft_destroy apply; the x-derivative
 * calls return NUFFT_EUNSUPPORTED on a 2D plan.  nufft2_plan_info reports K_x, gamma_x and
 * L = L_x L_y.  Synchronises `stream`. */
int nufft2d_plan(nufft_plan *out, int64_t m, int64_t n, int64_t M, const double *x_dev, const double *y_dev,
                 double eps, int prec, unsigned flags, void *stream);

/* Ranks, gammas and grid sizes of a 2D plan, per direction.  Any output may be NULL.
 * NUFFT_EINVAL for a 1D plan. */
int nufft2d_plan_info(nufft_plan p, int *Kx, int *Ky, double *gamma_x, double *gamma_y, int64_t *Lx,
                      int64_t *Ly);

/* ---- Batches: many independent problems of uneven sizes ----------------------
 *
 * No counterpart in the paper, which plans and runs one transform at a time.  A
 * batch is `count` independent NUFFT-II problems (its own N_i, M_i, x_i, eps_i
 * each), each planned exactly as by nufft2_plan and run together: problems whose
 * grids have the same length L and four-step split and whose ranks share a rank
 * bound (4, 8, 12, 16) form a class, and one kernel launch per pass covers a whole class, so a batch
 * of 512 problems runs in a few dozen launches instead of 1024.  Batched launches
 * cover NUFFT_F32 problems on grids of up to 2^18 points; other problems run their
 * own plan's launches inside the batch calls.  Forward results are bit-identical to
 * each problem's own plan (the same arithmetic in the same order); the batched
 * adjoint splits a class's rank sum over its own number of CTAs, so it agrees with
 * the single plans to rounding.
 *
 * Packed layout: problem i's coefficients are c[offN_i .. offN_i + N_i) with
 * offN_i = sum_{j<i} N_j; its samples (x, f, g) are [offM_i .. offM_i + M_i) with
 * offM_i = sum_{j<i} M_j.  Precision, stream and ownership rules are those of the
 * single-plan calls. */
typedef struct nufft_batch_s *nufft_batch;

#define NUFFT_BATCH_GRAPH 8u   /* nufft2_plan_many: a second exec call with the same
                                  pointers captures the batch's launches as one CUDA
                                  graph (each class a parallel branch); later calls
                                  with those pointers replay it.  Other pointers run
                                  the launches directly. */
#define NUFFT_BATCH_PERSISTENT 128u /* nufft2_plan_many: run every batched class of a
                                  direction in ONE launch of a persistent kernel: about as
                                  many 256-thread CTAs as fit on the GPU take the classes'
                                  blocks (first passes of every problem, then second passes)
                                  from one queue by an atomic ticket; a second-pass block
                                  waits (bounded by time; a timeout is reported by
                                  nufft_batch_check) until its problem's first pass is done.
                                  Results equal the class launches' bit for bit.  Combines
                                  with NUFFT_BATCH_GRAPH (the graph then holds that one
                                  launch).  Calls on one batch must not overlap. */
#define NUFFT_BATCH_PER_PROBLEM 32u /* nufft2_plan_many: run every problem with its
                                  own plan's launches (with NUFFT_BATCH_GRAPH, one
                                  parallel graph branch per problem) instead of
                                  batched launches.  Always the case for NUFFT_F64
                                  batches and for grids longer than 2^18 points. */

/* Plan a batch.
 *
 *   out       receives the handle (NULL on failure).
 *   count     number of problems, 1 <= count <= 65535.
 *   N_host, M_host, eps_host   count entries each (host): as nufft2_plan's N, M, eps.
 *   L_host    count grid sizes as nufft2_plan's L, or NULL (all 0: the default grid).
 *   x_dev     sum M_i doubles on the device, packed; read during the call only.
 *   prec      NUFFT_F32 or NUFFT_F64 for every problem.
 *   flags     NUFFT_BATCH_GRAPH, NUFFT_BATCH_PER_PROBLEM, NUFFT_BATCH_PERSISTENT,
 *             NUFFT_PLAN_AUTOTUNE (applied to each problem's plan).
 *
 * Synchronises `stream` once per problem (each plan reads its gamma).  Errors: those
 * of nufft2_plan for any problem (the batch is then not created), NUFFT_EINVAL. */
int nufft2_plan_many(nufft_batch *out, int64_t count, const int64_t *N_host, const int64_t *M_host,
                     const int64_t *L_host, const double *x_dev, const double *eps_host, int prec,
                     unsigned flags, void *stream);

/* Number of classes (= launches per pass), the packed lengths sum N_i and sum M_i,
 * and per problem its rank K_i and grid size L_i (K_host, L_host: count entries or
 * NULL).  Any output pointer may be NULL. */
int nufft_batch_info(nufft_batch b, int64_t *classes, int64_t *total_N, int64_t *total_M, int *K_host,
                     int64_t *L_host);

/* Kernel launches per direction of nufft2_exec_many / nufft1_exec_many: two per class, or
 * with NUFFT_BATCH_PERSISTENT one for all batched classes (plus two per problem that runs
 * its own plan's launches).  No GPU call.  NUFFT_EINVAL for NULL arguments. */
int nufft_batch_launches(nufft_batch b, int64_t *per_direction);

/* Forward transform of every problem: f_i = A_i c_i (packed c: sum N_i, f: sum M_i
 * complex values on the device).  Two launches per class (one for all of them with
 * NUFFT_BATCH_PERSISTENT). */
int nufft2_exec_many(nufft_batch b, const void *c_dev, void *f_dev, void *stream);

/* Adjoint of every problem: c_i = A_i^H g_i (packed g: sum M_i, c: sum N_i). */
int nufft1_exec_many(nufft_batch b, const void *g_dev, void *c_dev, void *stream);

/* The same transforms with one single-plan exec call per problem, in order (two
 * launches per problem): the per-problem comparator of nufft2_exec_many /
 * nufft1_exec_many.  adjoint = 0: c_dev -> f_dev (forward); 1: f_dev holds g and
 * c_dev receives A^H g. */
int nufft2_exec_each(nufft_batch b, const void *c_dev, void *f_dev, int adjoint, void *stream);

/* nufft2_check over every problem of the batch (synchronises `stream`). */
int nufft_batch_check(nufft_batch b, void *stream);

/* Free the batch and its plans.  NULL is accepted.  Must not race with work in
 * flight on the batch. */
int nufft_batch_destroy(nufft_batch b);

/* ---- Test hooks: failure detection without a GPU fault ------------------------
 * No counterpart in the paper.  Failures are made on the host, or by a bounded
 * device-side wait; nothing here faults, traps or hangs a GPU. */

/* Make a device allocation of the library fail as if out of memory: the one after the
 * next `after` allocations (after >= 0; after < 0 turns the injection off).  The call
 * that meets it returns NUFFT_ENOMEM and releases what it had allocated (plans,
 * batches, the inverse's solver state).  Process-wide; for tests. */
int nufft_test_fail_alloc(int after);

/* Launch one CTA that waits on an mbarrier which nothing completes.  Its bounded wait
 * gives up after the library's time limit (2 s), records the timeout in an error word
 * and returns, so the context stays usable.  Returns NUFFT_ETIMEOUT (the expected
 * outcome), NUFFT_OK (the wait completed: a bug) or NUFFT_ECUDA.  Synchronises
 * `stream`. */
int nufft_test_wait_timeout(void *stream);

/* Synchronise `stream` and report whether any exec call on this plan since the
 * last check had a device-side wait give up (a bulk copy that did not complete
 * within its time limit): NUFFT_ETIMEOUT, and the results of those calls are
 * invalid; or, in a library built with NUFFT_CHECK (libnufft_check.so: every
 * data-dependent shared and global index is checked, and an out-of-range access is
 * recorded and skipped instead of made), whether an index check failed:
 * NUFFT_ECHECK; else NUFFT_OK.  Clears the condition. */
int nufft2_check(nufft_plan p, void *stream);

/* ---- Measurement ----------------------------------------------------------------
 * No counterpart in the paper.  The exec kernels are bound by the plain FP32 pipes (FFT
 * butterflies, factor recurrences), so their roofline is reported against the FP32 FMA
 * rate of the device, measured by this kernel: blocks_per_sm (1 or 2) CTAs of 1024
 * threads per SM, each thread running 16 independent FMA chains for 8 * iters steps.
 * Writes the kernel's device time (CUDA events on `stream`) to *ms_out and the flops it
 * did (2 per FMA) to *flop_out; synchronises `stream`.  iters >= 1.  Errors:
 * NUFFT_EINVAL, NUFFT_ECUDA. */
int nufft_fp32_fma_peak(int64_t iters, int blocks_per_sm, void *stream, float *ms_out, double *flop_out);

/* Human-readable name of a status code. */
const char *nufft_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* NUFFT_H */
