/*
 * rsvd.h -- C ABI of the GB300 randomized SVD library.
 *
 * The library computes the rank-k randomized SVD of Algorithm 4 of
 * X. Li, "Randomized Algorithms for Solving Singular Value Decomposition
 * Problems with MATLAB Toolbox" (2021), Section 3.3 ("Accuracy Enhanced
 * Randomized SVD with Orthonormalization"), truncated to rank k as in
 * Section 3.1; with q = 0 it is Algorithm 2 (Section 3.1):
 *
 *   1. Omega: n x (k+p) standard Gaussian test matrix
 *   2. Y = A Omega
 *   3. Q = orth(Y)
 *   4-5. for j = 1..q:  W = orth(A^T Q);  Q = orth(A W)
 *   6. B = Q^T A              (computed as B^T = A^T Q)
 *   7. B = U~ Sigma V^T       (small SVD)
 *   8. U = Q U~, keep the leading k triplets
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Matrices are column-major (the thesis' MATLAB/LAPACK setting).  A
 *   matrix "r x c with leading dimension ld" holds element (i, j) at
 *   ptr[i + j*ld], ld >= r.
 * - Every matrix pointer passed to a compute entry point is a DEVICE pointer
 *   owned by the caller; the library never frees it.  Host pointers are
 *   named as such.
 * - The library allocates nothing on the device after rsvd_plan_create():
 *   all scratch lives in one caller-provided workspace
 *   (rsvd_workspace_size / rsvd_set_workspace).
 * - Compute entry points only enqueue work on the plan's CUDA stream and
 *   return.  Their return value reports argument and launch errors; the
 *   numerical status of the enqueued work (Cholesky breakdown, Jacobi not
 *   converged, non-finite input) is read by rsvd_plan_status(), which waits
 *   for the stream.
 * - Return values: RSVD_OK (0); -i when the i-th argument (1-based) of the
 *   call is invalid; a positive RSVD_ERR_* code otherwise.
 * - Random numbers: Omega is drawn from Philox4x32-10 (Salmon et al., SC'11)
 *   with Box-Muller, element (i, j) using counter (lo32(t), hi32(t),
 *   stream, 0) with t = j*n + i and key (lo32(seed), hi32(seed)); words 0,1
 *   give u1 and words 2,3 give u2 as (x + 1/2) 2^-52 with
 *   x = (w_a >> 6) 2^26 + (w_b >> 6); z = sqrt(-2 ln u1) cos(2 pi u2).
 *   The thesis does not fix a generator (Algorithm 1 step 1 only asks for
 *   a Gaussian matrix); this one makes results reproducible from the seed.
 */
#ifndef RSVD_GB300_H
#define RSVD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rsvd_plan_s* rsvd_plan_t;

/* Element types.  A plan's A is RSVD_F64 (plain mode), RSVD_BF16 or
 * RSVD_FP8E4M3 (mixed mode); RSVD_F32 is an output type of rsvd_gaussian and
 * the type of the mixed mode's FP32 buffers. */
typedef enum {
  RSVD_F64 = 0,     /* FP64 A; plain mode computes every step in FP64        */
  RSVD_F32 = 1,
  RSVD_BF16 = 2,    /* BF16 A; mixed mode (tensor cores, FP32 accumulation)  */
  RSVD_FP8E4M3 = 3  /* FP8 E4M3 A (OCP 8-bit format: sign, 4-bit exponent of
                       bias 7, 3-bit mantissa, no infinities, S.1111.111 NaN)
                       with one FP32 scale per 128 x 128 tile; mixed mode.
                       The thesis stores A in full precision; this compressed
                       storage halves the bytes each pass over A streams. */
} rsvd_dtype_t;

typedef enum {
  RSVD_MODE_PLAIN = 0, /* FP64 arithmetic throughout (A must be RSVD_F64)   */
  RSVD_MODE_MIXED = 1, /* BF16 operands on tcgen05 tensor cores, FP32
                          accumulation, FP32 for the other steps            */
  RSVD_MODE_F64_TENSOR = 2
                       /* FP64 A, FP64 results, every step as in plain mode
                          except the passes over A: those run on the tcgen05
                          tensor cores as exact products of BF16 digit
                          slices.  Each row of A gets a power-of-two scale
                          and six balanced base-256 digits (A = scale * sum
                          of digits * 2^(-7-8s) + a remainder below 2^-48 of
                          the scale); the operand is split the same way per
                          column; the 21 digit products of weight >= 2^-40
                          are accumulated exactly (integer sums in FP32
                          drained to 64-bit integers every 256 terms) or, for
                          the two smallest weights, in FP32.  A pass with
                          contraction length K is then within about
                          2^-45 K max|a_i.| max|x_.c| of the exact product
                          (worst case; near 2^-45 sqrt(K) of that scale in
                          practice).  Every call that reads A first builds
                          its digit slices (12 bytes per element of A, in the
                          workspace).  Entry points and outputs as in plain
                          mode; A must be RSVD_F64.                        */
} rsvd_mode_t;

/* Status codes (positive). */
#define RSVD_OK 0
#define RSVD_ERR_CHOLESKY 1    /* Gram Cholesky failed even after a shift   */
#define RSVD_ERR_JACOBI 2      /* Jacobi SVD did not converge (30 sweeps)   */
#define RSVD_ERR_TIMEOUT 3     /* a device-side wait hit its iteration cap  */
#define RSVD_ERR_WORKSPACE 4   /* no workspace set, or it is too small      */
#define RSVD_ERR_CUDA 5        /* a CUDA runtime call or launch failed      */
#define RSVD_ERR_NONFINITE 6   /* NaN or Inf met in A (through Y = A Omega) */
#define RSVD_ERR_UNSUPPORTED 7 /* dtype/mode/size not built into this library */
#define RSVD_ERR_NOT_REACHED 8 /* adaptive range finder: the tolerance was not
                                  met within l_cap columns (the result holds
                                  l_cap columns and is otherwise valid)      */

/* Largest k+p the library accepts (the l x l steps keep l x l FP64 tiles). */
#define RSVD_L_MAX 288

/* ---------------------------------------------------------------------- */
/* Plans                                                                   */
/* ---------------------------------------------------------------------- */

/*
 * rsvd_plan_create: a plan for problems up to m_max x n_max with
 * k + p <= l_max, A stored as a_dtype, computed in `mode`, enqueued on
 * `cuda_stream` (a cudaStream_t; NULL = the legacy default stream).
 * Allocates a small pinned host status buffer and nothing on the device.
 * Errors: -1 plan NULL; -2/-3 sizes < 1; -4 l_max < 1 or > RSVD_L_MAX (256 in
 * mixed mode); -5 unknown dtype; -6 unknown mode or mode/dtype mismatch;
 * RSVD_ERR_CUDA if the host allocation fails.  RSVD_MODE_F64_TENSOR plans
 * need 12 m_max n_max bytes more workspace than plain ones (A's digit
 * slices).
 */
int rsvd_plan_create(rsvd_plan_t* plan, int64_t m_max, int64_t n_max, int l_max,
                     int a_dtype, int mode, void* cuda_stream);

/* Bytes of device workspace the plan needs (256-byte aligned pointer). */
int rsvd_workspace_size(rsvd_plan_t plan, size_t* bytes);

/*
 * rsvd_set_workspace: hands the plan `bytes` bytes of device memory at
 * `dev_ptr` (caller-owned, must outlive the plan's use, 256-byte aligned).
 * Errors: -2 NULL pointer or misaligned; RSVD_ERR_WORKSPACE if too small.
 */
int rsvd_set_workspace(rsvd_plan_t plan, void* dev_ptr, size_t bytes);

/*
 * rsvd_plan_status: waits for the plan's stream, then returns the status of
 * the work enqueued since the previous call (RSVD_OK or a positive code) and
 * clears it.  RSVD_ERR_CUDA if the stream reported an error.  For a batch
 * plan this is the plan-wide word of the tensor engine (RSVD_ERR_TIMEOUT
 * when a grouped launch's bounded wait expired); per-problem codes come from
 * rsvd_batch_status.
 */
int rsvd_plan_status(rsvd_plan_t plan);

/*
 * rsvd_plan_diagnostics: waits for the plan's stream and reports, for the
 * work enqueued so far, the sweeps the last Jacobi SVD took and the number of
 * columns CholeskyQR dropped as numerically dependent (cumulative).  Either
 * pointer (host) may be NULL.
 */
int rsvd_plan_diagnostics(rsvd_plan_t plan, int* jacobi_sweeps, int* dropped_columns);

/* Sets the stream later calls enqueue on. */
int rsvd_plan_set_stream(rsvd_plan_t plan, void* cuda_stream);

/*
 * rsvd_plan_set_wait_limit: the bound, in SM clock cycles (clock64), of every
 * wait inside the tensor-core passes of a mixed plan (a pipeline stage's
 * data, a free stage, the accumulator).  0 (the default) means about one
 * second (2e9 cycles).  A wait that runs past its bound does not hang the
 * GPU: the pass stops issuing, waits (up to one second) for its own copies and
 * products in flight, frees its tensor memory, and rsvd_plan_status() then
 * returns RSVD_ERR_TIMEOUT; the outputs of that call are undefined.  A limit
 * below about 1e6 cycles polls without blocking and reads the clock on every
 * poll, so a limit of a few cycles makes the first incomplete wait expire:
 * that is how the tests exercise this failure path without a GPU fault.
 * Takes effect for calls enqueued afterwards.  Errors: -1 plan; -2 cycles < 0.
 * The thesis has no counterpart: this is the failure-detection bound of the
 * GPU pipeline.
 */
int rsvd_plan_set_wait_limit(rsvd_plan_t plan, int64_t cycles);

/*
 * rsvd_plan_prepare_a / rsvd_plan_release_a: RSVD_MODE_F64_TENSOR plans build
 * the digit slices of A at the start of every call that reads A.
 * rsvd_plan_prepare_a builds them now (enqueued on the plan's stream) and
 * keeps them: later calls that name the same (A, m, n, lda) skip that step,
 * until rsvd_plan_release_a or a call on another matrix (whose slices then
 * replace them).  The caller must not change A's contents while it is
 * prepared: the kept slices would no longer match it.  On plans of other
 * modes both calls return RSVD_OK and do nothing.  Errors: -1 plan; -2 A
 * NULL; -3 m; -4 n; -5 lda < m; RSVD_ERR_WORKSPACE if the plan has no
 * workspace or m, n exceed it.  The thesis has no counterpart: this is a
 * cache of the tensor passes' operand format.
 */
int rsvd_plan_prepare_a(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda);
int rsvd_plan_release_a(rsvd_plan_t plan);

/*
 * rsvd_set_tile_scales (RSVD_FP8E4M3 plans): the scales of A.  Element (i, j)
 * of A is the E4M3 value of code A[i + j*lda] times scales[I + J*lds] with
 * I = i / 128, J = j / 128; `scales` is a DEVICE array of rows x cols FP32
 * values (rows >= ceil(m / 128), cols >= ceil(n / 128) of every later call),
 * caller-owned, read by every later solve or pass of the plan.  Each scale
 * must be a positive power of two (then code * scale is exact in BF16, the
 * tensor cores' operand type); the call copies the scales to the host once to
 * check that (synchronous).  FP8 calls also need lda a multiple of 16.
 * Errors: -1 plan; -2 scales NULL or a scale that is not a positive power of
 * two; -3 rows < 1; -4 cols < 1; -5 lds < rows; RSVD_ERR_UNSUPPORTED if the
 * plan's A is not FP8; RSVD_ERR_CUDA if the copy fails.  A solve or pass of an
 * FP8 plan without covering scales returns RSVD_ERR_UNSUPPORTED.
 */
int rsvd_set_tile_scales(rsvd_plan_t plan, const float* scales, int64_t rows, int64_t cols,
                         int64_t lds);

int rsvd_plan_destroy(rsvd_plan_t plan);

const char* rsvd_status_string(int status);

/*
 * rsvd_kernel_launches: number of CUDA kernels this library has launched in
 * this process (all plans, all streams), counted on the host at each launch.
 * A diagnostic for callers that account GPU work; it never blocks.
 */
uint64_t rsvd_kernel_launches(void);

/* ---------------------------------------------------------------------- */
/* Full solve: Algorithm 4 (Section 3.3), truncated to rank k (Section 3.1) */
/* ---------------------------------------------------------------------- */

/*
 * rsvd_solve: rank-k randomized SVD  A ~= U diag(S) VT.
 *   A    m x n, leading dimension lda >= m, stored as the plan's dtype.
 *   k >= 1 target rank, p >= 0 oversampling, k + p <= min(m, n) and
 *   <= the plan's l_max (Theorem 2's premise k + p <= min{m, n}), q >= 0
 *   power steps, seed selects Omega (stream 0).
 *   U    m x k, ldu >= m: FP64 in plain mode, FP32 in mixed mode.
 *   S    k FP64 values, descending.
 *   VT   k x n, ldvt >= k: FP64 in plain mode, FP32 in mixed mode.
 * Signs: each pair (u_i, v_i) is flipped so the entry of u_i with the
 * largest magnitude is positive (lowest row index on ties).
 * Argument errors: -1 plan; -2 A NULL; -3 m; -4 n; -5 lda; -6 k; -7 p;
 * -8 q; -10 U NULL; -11 ldu; -12 S NULL; -13 VT NULL; -14 ldvt.
 * m, n above the plan's maxima or k+p above l_max: RSVD_ERR_WORKSPACE.
 * Mixed mode reads A with TMA: lda must be a multiple of 8 (16 for FP8 A)
 * and A 16-byte aligned, else RSVD_ERR_UNSUPPORTED.  Mixed mode runs q power steps with a
 * BF16 copy of the operand, then one more power step with the operand split
 * in two BF16 slices, then B^T = A^T Q with Q split in three BF16 slices.
 */
int rsvd_solve(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda,
               int k, int p, int q, uint64_t seed,
               void* U, int64_t ldu, double* S, void* VT, int64_t ldvt);

/*
 * rsvd_solve_algorithm: the rank-k randomized SVD by one of the thesis'
 * algorithms, all truncated to rank k (Section 3.1) with outputs and signs as
 * rsvd_solve:
 *   2  Algorithm 2 (Section 3.1): Algorithm 4 with q = 0 (q is ignored);
 *   3  Algorithm 3 (Section 3.2, "Accuracy Enhanced Randomized SVD"): q power
 *      steps Z = A^T Y, Y = A Z with no orthonormalisation in between, then
 *      one orth(Y).  The sample's condition number grows like
 *      (sigma_1/sigma_l)^(2q+1), so orth is shifted CholeskyQR3 (a Cholesky
 *      QR with the Gram shifted by 11 (m l + l (l+1)) u ||Y||_F^2, then
 *      CholeskyQR2), defined up to condition numbers near 1/u; the thesis
 *      notes that round-off limits this algorithm's accuracy.  Plain plans.
 *   4  Algorithm 4 (Section 3.3): rsvd_solve.
 *   6  Algorithm 6 (Section 3.4.2): rsvd_solve_singlepass (q is ignored).
 * Argument errors: -1 plan; -2 algorithm; -3 A NULL; -4 m; -5 n; -6 lda;
 * -7 k; -8 p (or k+p > min(m, n)); -9 q; -11 U NULL; -12 ldu; -13 S NULL;
 * -14 VT NULL; -15 ldvt.  RSVD_ERR_WORKSPACE as rsvd_solve;
 * RSVD_ERR_UNSUPPORTED for batch plans, and for 3 or 6 on a mixed plan.
 */
int rsvd_solve_algorithm(rsvd_plan_t plan, int algorithm, const void* A, int64_t m, int64_t n,
                         int64_t lda, int k, int p, int q, uint64_t seed, void* U, int64_t ldu,
                         double* S, void* VT, int64_t ldvt);

/*
 * rsvd_solve_singlepass: rank-k randomized SVD by Algorithm 6 ("Single-Pass
 * Randomized SVD for a General Matrix", Section 3.4.2): A is read by exactly
 * two sketching products, Y_c = A Omega_c and Y_r = A^T Omega_r (Omega_c
 * n x (k+p) from Philox stream 0 of `seed`, Omega_r m x (k+p) from stream 1),
 * and never again.  Q_c, Q_r are the k dominant left singular vectors of Y_c
 * and Y_r; C (k x k) is the least-squares solution of the joint system
 * (Omega_r^T Q_c) C = Y_r^T Q_r, C (Q_r^T Omega_c) = Q_c^T Y_c, both
 * equations weighted equally; C = U^ Sigma V^^T; U = Q_c U^, V = Q_r V^.
 * Less accurate than Algorithm 4 (the thesis notes it), but A is streamed
 * only in Stage 1.  Plain (FP64) plans; outputs and signs as rsvd_solve.
 * Argument errors: -1 plan; -2 A NULL; -3 m; -4 n; -5 lda; -6 k; -7 p (or
 * k+p > min(m, n)); -9 U NULL; -10 ldu; -11 S NULL; -12 VT NULL; -13 ldvt.
 * RSVD_ERR_WORKSPACE as rsvd_solve; RSVD_ERR_UNSUPPORTED for mixed or batch
 * plans.
 */
int rsvd_solve_singlepass(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda,
                          int k, int p, uint64_t seed, void* U, int64_t ldu, double* S,
                          void* VT, int64_t ldvt);

/*
 * rsvd_solve_hermitian: rank-k randomized eigendecomposition A ~ U diag(D) U^T
 * of a real symmetric (Hermitian) n x n matrix by Algorithm 5 ("Single-Pass
 * Randomized SVD for a Hermitian Matrix", Section 3.4.1; Eqs. 3.6-3.13).  A
 * is read by exactly one product, Y = A Omega (Omega n x (k+p) from Philox
 * stream 0 of `seed`, as in rsvd_solve), and never again.  Q is the k
 * dominant left singular vectors of Y; C (k x k) is the least-squares
 * solution of C (Q^T Omega) = Q^T Y (Eq. 3.13; an overdetermined system of
 * k+p equations per row of C); its symmetric part (C + C^T)/2 is decomposed
 * as U^ diag(D) U^^T and U = Q U^.  Only the upper and lower triangles' sum
 * of A enters through Y, so A must be symmetric: the library does not check.
 * Outputs (device, caller-owned): U n x k column-major (ldu), each column's
 * largest-magnitude entry positive; D[k] the eigenvalues, FP64, ordered by
 * decreasing magnitude (A may be indefinite).  Eigenvalues of equal
 * magnitude and opposite sign make the eigenvectors of that pair arbitrary
 * within their 2-D space.  Plain (FP64) plans with m_max, n_max >= n.
 * Argument errors: -1 plan; -2 A NULL; -3 n; -4 lda < n; -5 k; -6 p (or
 * k+p > n); -8 U NULL; -9 ldu; -10 D NULL.  RSVD_ERR_WORKSPACE as rsvd_solve;
 * RSVD_ERR_UNSUPPORTED for mixed or batch plans.
 */
int rsvd_solve_hermitian(rsvd_plan_t plan, const void* A, int64_t n, int64_t lda, int k, int p,
                         uint64_t seed, void* U, int64_t ldu, double* D);

/*
 * rsvd_range_adaptive: the adaptive randomized range finder ("Adaptive_randRF"
 * in Section 4's function list, which names Algorithm 4.2 of Halko,
 * Martinsson and Tropp, SIAM Review 53 (2011) as its source).  Given A, a
 * tolerance eps and an integer r, it builds Q with orthonormal columns such
 * that ||(I - Q Q^T) A||_2 <= eps with probability at least
 * 1 - min(m, n) 10^-r.  Samples A omega_1, A omega_2, ... (omega_i = column
 * i-1 of the Gaussian of rsvd_gaussian, stream 0 of `seed`) are
 * orthonormalised in order (Gram-Schmidt order, so q_j is fixed by the first
 * j samples); the search stops at the first j where the next r samples'
 * residuals against Q_j are all at most eps / (10 sqrt(2/pi)).  The rank j is
 * then written to *rank (host int) and Q's first j columns are valid.
 * Work is done in blocks of up to 64 samples (one pass over A each); the
 * call WAITS on the plan's stream once per block to read the stopping test,
 * and returns with the last column copy still enqueued.  Plain (FP64) plans.
 *   eps    > 0, absolute (the norm of A is not applied).  Below about 1e-12
 *          of ||A|| the residuals are rounding noise: the search then stops
 *          where CholeskyQR finds the sample numerically dependent.
 *   r      1 <= r < min(64, plan l_max); r = 10 is the usual choice.
 *   l_cap  1 <= l_cap <= min(m, n, plan l_max): the most columns accepted.
 *   Q      m x l_cap, ldq >= m (device, FP64).
 * Returns RSVD_OK when the test passed, RSVD_ERR_NOT_REACHED when l_cap
 * columns were accepted first (Q then holds l_cap valid columns), or the
 * status (RSVD_ERR_NONFINITE, ...) that the device work of this call set.
 * Argument errors: -1 plan; -2 A NULL; -3 m; -4 n; -5 lda; -6 eps; -7 r;
 * -8 l_cap; -10 Q NULL; -11 ldq; -12 rank NULL.  RSVD_ERR_WORKSPACE if the
 * plan's sizes do not cover m, n, l_cap; RSVD_ERR_UNSUPPORTED for mixed or
 * batch plans.
 */
int rsvd_range_adaptive(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda,
                        double eps, int r, int l_cap, uint64_t seed, void* Q, int64_t ldq,
                        int* rank);

/*
 * rsvd_solve_adaptive: rsvd_range_adaptive, then Stage B of the prototype
 * (Algorithm 1 / Section 2.2) with every column of Q kept: B = Q^T A (as
 * B^T = A^T Q), B = U~ Sigma V^T, U = Q U~.  The tolerance, not k, fixes the
 * rank j = *rank; U (m x j, ldu >= m), S (j, descending) and VT (j x n,
 * ldvt >= l_cap) are FP64 with the signs of rsvd_solve.  Returns as
 * rsvd_range_adaptive (the outputs are valid for RSVD_OK and
 * RSVD_ERR_NOT_REACHED; nothing is written when j = 0).
 * Argument errors: -1 .. -8 as rsvd_range_adaptive; -10 U NULL; -11 ldu;
 * -12 S NULL; -13 VT NULL; -14 ldvt; -15 rank NULL.
 */
int rsvd_solve_adaptive(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda,
                        double eps, int r, int l_cap, uint64_t seed, void* U, int64_t ldu,
                        double* S, void* VT, int64_t ldvt, int* rank);

/*
 * rsvd_range_srft: the fast randomized range finder ("FastRandRF" in Section
 * 4's function list, Algorithm 4.5 of Halko, Martinsson and Tropp 2011) with
 * the subsampled random Fourier transform the thesis defines ("SRFT"):
 *   Omega = sqrt(n/l) D F R  (n x l, complex), Y = A Omega, Q = orth(Y),
 *   D  diagonal, d_j = exp(2 pi i u_j), u_j the 52-bit Philox uniform of
 *      counter j on stream 2 of `seed` (uniform on the unit circle);
 *   F  the unitary DFT, f_pq = n^-1/2 exp(-2 pi i p q / n) (0-based p, q);
 *   R  l distinct coordinates of [0, n) drawn by Floyd's algorithm (step s,
 *      j = n-l+s: t = min(floor(u_s (j+1)), j) with u_s the Philox uniform of
 *      counter s on stream 3; add t, or j if t is taken), used in ascending
 *      order.
 * Q (m x l, complex, orthonormal columns; column c is the Gram-Schmidt vector
 * of Y's column c, normalised so that q_c^H y_c > 0) is written PLANAR: the
 * real m x 2l matrix [Re Q | Im Q] with leading dimension ldq >= m.
 * Plain (FP64) plans whose l_max is at least 2l (the complex sample is held
 * as 2l real columns); 2l <= RSVD_L_MAX.  Enqueued on the plan's stream.
 * Argument errors: -1 plan; -2 A NULL; -3 m; -4 n (also n > INT32_MAX);
 * -5 lda; -6 l (1 <= l <= min(m, n), 2l <= RSVD_L_MAX); -8 Q NULL; -9 ldq.
 * RSVD_ERR_WORKSPACE if the plan does not cover m, n or 2l;
 * RSVD_ERR_UNSUPPORTED for mixed or batch plans.
 */
int rsvd_range_srft(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda, int l,
                    uint64_t seed, void* Q, int64_t ldq);

/*
 * rsvd_solve_srft: FastRandRF with l = k + p (as rsvd_range_srft), then
 * Stage B of the prototype (Section 2.2) on the complex basis, truncated to
 * rank k (Section 3.1): B = Q^H A (computed as B^H = A^T Q), B = U~ S V^H,
 * U = Q U~.  Complex outputs are planar:
 *   U    m x 2k real (ldu >= m): [Re U | Im U];
 *   S    k FP64 values, descending;
 *   VT   k x 2n real (ldvt >= k): [Re V^H | Im V^H].
 * Each (u_i, v_i) is multiplied by the unit factor that makes the entry of
 * u_i with the largest modulus real and positive (lowest row on ties).
 * Plain plans with l_max >= 2(k+p); 2(k+p) <= RSVD_L_MAX.
 * Argument errors: -1 plan; -2 A NULL; -3 m; -4 n; -5 lda; -6 k; -7 p (or
 * k+p > min(m, n)); -9 U NULL; -10 ldu; -11 S NULL; -12 VT NULL; -13 ldvt.
 * RSVD_ERR_WORKSPACE / RSVD_ERR_UNSUPPORTED as rsvd_range_srft.
 */
int rsvd_solve_srft(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda, int k,
                    int p, uint64_t seed, void* U, int64_t ldu, double* S, void* VT,
                    int64_t ldvt);

/*
 * rsvd_srft_sketch: the sketch alone, Y = A Omega with the SRFT Omega of
 * rsvd_range_srft (same seed, same D and R), written planar to Y (real
 * m x 2l, ldy >= m).  Arguments and errors as rsvd_range_srft (Y for Q).
 */
int rsvd_srft_sketch(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda, int l,
                     uint64_t seed, void* Y, int64_t ldy);

/* ---------------------------------------------------------------------- */
/* Step-level entry points (the rows of the hot path, one call per step).   */
/* In plain mode every buffer is FP64; the mixed-mode types are noted.     */
/* ---------------------------------------------------------------------- */

/*
 * rsvd_gaussian: Algorithm 4 step 1 (Section 3.3; "Gaussian test matrix",
 * Algorithm 1 step 1, Section 2.2).  Writes the n x l matrix Omega for
 * (seed, stream) to `out` (ldo >= n) as FP64 (out_dtype RSVD_F64), FP32
 * (RSVD_F32) or BF16 (RSVD_BF16), rounded to nearest even from the FP64 value.
 * Errors: -2 n < 1; -3 l < 1; -6 out_dtype; -7 out NULL; -8 ldo < n.
 */
int rsvd_gaussian(rsvd_plan_t plan, int64_t n, int l, uint64_t seed, uint32_t stream,
                  int out_dtype, void* out, int64_t ldo);

/*
 * rsvd_apply_a: Y = A X  (Algorithm 4 steps 2 and 5, "Form Y = A Omega",
 * "Q = orth(A W)").  A m x n (lda), X n x l (ldx), Y m x l (ldy).
 * Plain: A, X, Y FP64.  Mixed: A BF16, X BF16, Y FP32; mixed mode also needs
 * lda and ldx multiples of 8 and A, X 16-byte aligned (TMA), else
 * RSVD_ERR_UNSUPPORTED.
 * Errors: -2 A; -3 m; -4 n; -5 lda; -6 X; -7 ldx; -8 l; -9 Y; -10 ldy.
 */
int rsvd_apply_a(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda,
                 const void* X, int64_t ldx, int l, void* Y, int64_t ldy);

/*
 * rsvd_apply_at: Z = A^T X  (Algorithm 4 step 5 "W = orth(A* Q)" and step 6
 * "B = Q* A", computed as B^T = A^T Q).  A m x n (lda), X m x l (ldx),
 * Z n x l (ldz).  Plain: FP64.  Mixed: A BF16, X BF16, Z FP32.
 * Errors as rsvd_apply_a, with ldx >= m and ldz >= n.
 */
int rsvd_apply_at(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda,
                  const void* X, int64_t ldx, int l, void* Z, int64_t ldz);

/*
 * rsvd_apply_split: one pass over A as the mixed solve runs it (Algorithm 4
 * steps 2, 5 and 6, Section 3.3): out = A X (trans = 0; X n x l, out m x l)
 * or out = A^T X (trans = 1; X m x l, out n x l), with X FP32 (ldx) split on
 * the device into slices whose sum carries its leading bits: BF16 plans use
 * `slices` BF16 slices (about 8 significant bits each); FP8 plans use
 * 2 x `slices` E4M3 slices (4 bits each, one power-of-two weight per slice
 * and 64-row chunk) on block-scaled MMAs (kind::mxf8f6f4) with A's tile
 * scales as the tensor core's block scales.  out is FP32 (ldo), FP32
 * accumulation; A as for rsvd_apply_a (FP8: rsvd_set_tile_scales first).
 * Mixed plans only (else RSVD_ERR_UNSUPPORTED).  X and out are caller-owned
 * device buffers; nothing is allocated.
 * Errors: -2 A; -3 m; -4 n; -5 lda; -6 trans; -7 X; -8 ldx; -9 l;
 * -10 slices not in 1..3; -11 out; -12 ldo.
 */
int rsvd_apply_split(rsvd_plan_t plan, const void* A, int64_t m, int64_t n, int64_t lda,
                     int trans, const float* X, int64_t ldx, int l, int slices, float* out,
                     int64_t ldo);

/*
 * rsvd_orth: Q = orth(Y) by CholeskyQR2 (Algorithm 4 step 3; the thesis
 * leaves the orthonormalisation method open).  Y rows x l (ldy), Q rows x l
 * (ldq) and, if non-NULL, R (l x l, ldr) are FP64 in plain mode and FP32 in
 * mixed mode; Y is left unchanged; R receives the upper triangular factor
 * with Y = Q R.  Columns of Y that are numerically in the span of earlier
 * columns (Gram pivot <= l * eps * max diag) come out as zero columns of Q
 * and zero rows of R.
 * Errors: -2 Y; -3 rows; -4 l; -5 ldy; -6 Q; -7 ldq; -9 ldr.
 */
int rsvd_orth(rsvd_plan_t plan, const void* Y, int64_t rows, int l, int64_t ldy,
              void* Q, int64_t ldq, void* R, int64_t ldr);

/*
 * rsvd_small_svd: SVD of an l x l matrix M (ldm) by one-sided Jacobi
 * (Algorithm 4 step 7, applied to the triangular factor of B^T):
 * M = Um diag(sig) Vm^T with sig descending (l values), Um and Vm l x l
 * (ldu, ldv) with orthonormal columns (a column of Um is zero where sig is
 * zero).  All pointers device; FP64 in plain mode, FP32 in mixed mode.  M is
 * left unchanged.
 * Errors: -2 M; -3 l; -4 ldm; -5 sig; -6 Um; -7 ldu; -8 Vm; -9 ldv.
 */
int rsvd_small_svd(rsvd_plan_t plan, const void* M, int l, int64_t ldm,
                   void* sig, void* Um, int64_t ldu, void* Vm, int64_t ldv);

/* ---------------------------------------------------------------------- */
/* Batches: many independent problems of uneven size in grouped launches    */
/* (the thesis' method applied per problem; every step of Algorithm 4 runs  */
/* once for the whole batch).                                               */
/* ---------------------------------------------------------------------- */

/* One problem of a batch: the arguments of rsvd_solve (device pointers). */
typedef struct rsvd_problem_s {
  const void* A;          /* m x n, lda >= m, the batch plan's dtype */
  int64_t m, n, lda;
  int k, p, q;            /* 1 <= k, 0 <= p, k + p <= min(m, n), q >= 0 */
  uint64_t seed;
  void* U;                /* m x k, ldu >= m, the plan's dtype */
  int64_t ldu;
  double* S;              /* k, descending */
  void* VT;               /* k x n, ldvt >= k, the plan's dtype */
  int64_t ldvt;
} rsvd_problem_t;

/*
 * rsvd_batch_plan_create: a plan for batches of up to max_count problems
 * whose m's sum to at most rows_total and whose n's sum to at most
 * cols_total, each with k + p <= l_max.  a_dtype RSVD_F64 (every step in
 * FP64 on the CUDA cores) or RSVD_F32 (every step in FP32: the grouped
 * products on the tensor cores by default, see rsvd_batch_set_engine).
 * Workspace is queried and set as for other plans.  Allocates pinned host
 * memory for the per-batch problem table and an event, nothing on the
 * device.
 * Errors: -1 plan; -2 max_count < 1; -3 rows_total < 1; -4 cols_total < 1;
 * -5 l_max outside 1..RSVD_L_MAX; -6 dtype; RSVD_ERR_CUDA.
 */
int rsvd_batch_plan_create(rsvd_plan_t* plan, int max_count, int64_t rows_total,
                           int64_t cols_total, int l_max, int a_dtype, void* cuda_stream);

/*
 * rsvd_solve_batched: enqueues the rank-k randomized SVD (Algorithm 4) of every
 * problem in `problems` (host array of `count` entries) on the plan's stream.
 * Each problem's result depends only on its own inputs (no work is split
 * across problems), so it is the same in any batch.  Waits on the host only
 * until the previous batched solve's problem table has left the pinned
 * staging buffer.
 * Errors: -1 plan is not a batch plan; -2 count outside 1..max_count;
 * -3 problems NULL; RSVD_ERR_WORKSPACE when sizes exceed the plan or no
 * workspace is set; -(100 + i) when problem i has an invalid argument.
 */
int rsvd_solve_batched(rsvd_plan_t plan, int count, const rsvd_problem_t* problems);

/*
 * rsvd_batch_status: waits for the plan's stream and writes each problem's
 * status (RSVD_OK or a positive RSVD_ERR_* code) of the last batched solve to
 * the host array codes[0..count-1].
 */
int rsvd_batch_status(rsvd_plan_t plan, int count, int* codes);

/*
 * Engines of an FP32 batch plan's grouped products (the passes over each A,
 * the Gram and R^-1 products of CholeskyQR2 and the products with the small
 * SVD's factors, Algorithm 4 steps 2-8):
 *   RSVD_BATCH_ENGINE_TENSOR (default for FP32): one persistent tcgen05
 *     launch per step over all problems.  Each FP32 value is split exactly
 *     into three BF16 values and the six slice products with i + j <= 4 are
 *     accumulated in FP32 (the accuracy of an FP32 product).  Work units
 *     (128-row x column-tile output tiles, optionally split along the
 *     contraction) are dealt to the SMs longest first.
 *   RSVD_BATCH_ENGINE_SIMT: grouped CUDA-core launches (the only engine of
 *     FP64 batch plans).
 * rsvd_batch_set_engine errors: -1 plan is not a batch plan; -2 engine;
 * RSVD_ERR_UNSUPPORTED for the tensor engine on an FP64 plan.
 */
#define RSVD_BATCH_ENGINE_SIMT 0
#define RSVD_BATCH_ENGINE_TENSOR 1
int rsvd_batch_set_engine(rsvd_plan_t plan, int engine);

/*
 * rsvd_batch_set_graphs: on != 0 makes each rsvd_solve_batched of an FP32
 * plan on the tensor engine one CUDA graph launch.  The graph (table copy,
 * status resets and every grouped step of Algorithm 4) is captured on the
 * plan's stream when the batch's launch signature -- each problem's m, n,
 * k, p, q, the tuning table and the wait limit -- differs from the last
 * capture, and replayed otherwise; operands and seeds may change between
 * replays.  A capture costs about as much as a solve, so this pays for
 * batches that repeat their shapes.  Needs a stream other than the legacy
 * default stream.
 * Errors: -1 not a batch plan; -2 the plan's stream is the default stream;
 * RSVD_ERR_UNSUPPORTED unless the plan is FP32 on the tensor engine.
 */
int rsvd_batch_set_graphs(rsvd_plan_t plan, int on);

/*
 * rsvd_batch_set_sm_limit: the tensor engine's persistent launches of this
 * plan use at most `sms` SMs (0: all of them), leaving the rest to work on
 * other streams -- for instance FP64 solves of the problems an FP32 batch
 * could not resolve.  The work split into units, and so every result, does
 * not depend on the limit.  Errors: -1 not a batch plan; -2 sms < 0.
 */
int rsvd_batch_set_sm_limit(rsvd_plan_t plan, int sms);

/*
 * rsvd_batch_autotune: times the tensor engine's schedule candidates on the
 * products of this batch (same arguments as rsvd_solve_batched) and keeps
 * the fastest per shape bucket in a process-wide table:
 *   - the contraction chunk (split-K: 4, 8, 16, 32, 64, 128 or 256 blocks
 *     of 64) for each form, contraction-length bucket (64 2^(b-1), 64 2^b]
 *     and output-row class (one 128-row tile, as in the Gram products, or
 *     more);
 *   - the column-tile limit (48, 64 or 80) for each l bucket above 80.
 * The first value recorded for a bucket stays for the life of the process,
 * so every later solve gives a problem the same schedule -- and the same
 * bits -- alone or in any batch.  Untuned buckets use 64 blocks and 80
 * columns.  Enqueues trial runs on the plan's stream and waits for them;
 * overwrites the plan's workspace (not the problems' outputs).
 * Errors: as rsvd_solve_batched; RSVD_ERR_UNSUPPORTED unless the plan is an
 * FP32 batch plan on the tensor engine.
 */
int rsvd_batch_autotune(rsvd_plan_t plan, int count, const rsvd_problem_t* problems);

/*
 * rsvd_grouped_gemm_f32: the tensor engine's grouped product on its own:
 * for every entry, C (M x N, ldc >= M) = A X (trans = 0; A M x K, lda >= M)
 * or A^T X (trans = 1; A stored K x M, lda >= K), X K x N (ldx >= K); all
 * FP32 device memory, FP32-accurate (three BF16 slices of each operand).
 * x_upper != 0: X is upper triangular (entries below its diagonal are read
 * as zero).  M = 0 skips an entry.  Uses an FP32 batch plan's workspace and
 * stream (up to max_count entries; the operand slices of all entries must
 * fit the plan's slice space, 6 (rows_total + cols_total + 64 max_count)
 * (l_max rounded up to 16, + 80) bytes); a timeout (an expired bounded
 * wait, RSVD_ERR_TIMEOUT) shows in rsvd_plan_status of the batch plan.
 * Errors: -1 not an FP32 batch plan on the tensor engine; -2 count outside
 * 1..max_count; -3 gemms NULL; -(100 + i) entry i invalid;
 * RSVD_ERR_WORKSPACE; RSVD_ERR_CUDA.
 */
typedef struct rsvd_gemm_s {
  const float* A;
  int64_t lda;
  const float* X;
  int64_t ldx;
  float* C;
  int64_t ldc;
  int64_t M, K;
  int N;
  int x_upper;
} rsvd_gemm_t;
int rsvd_grouped_gemm_f32(rsvd_plan_t plan, int count, const rsvd_gemm_t* gemms, int trans);

/*
 * rsvd_grouped_schedule: the tensor engine's work schedule for `count`
 * products of shapes shapes[3i .. 3i+2] = (M, K, N) (M = 0: skipped) in the
 * given form (trans as in rsvd_grouped_gemm_f32) on `num_sms` SMs, with the
 * process's current tuning table.  Host computation only (no device work):
 * a planning query, also usable without a GPU.
 *   units: NULL, or room for max_units entries of 7 ints each:
 *     (product, row0, col0, kb0, kb1, slot, t) -- output rows row0 ..
 *     row0 + 127 and columns col0 .. col0 + t - 1 over contraction blocks
 *     kb0 .. kb1 - 1 of 64; slot >= 0 marks a split tile's partial slot.
 *   cta_off: NULL, or room for num_sms + 1 ints: CTA c takes units
 *     cta_off[c] .. cta_off[c+1] - 1 (in the order listed).
 *   info: 4 ints: unit count, grid (CTAs), partial slots, largest t.
 * Errors: -1 count < 1; -2 shapes or info NULL; -3 num_sms < 1;
 * -(100 + i) shape i invalid; RSVD_ERR_WORKSPACE when units or cta_off
 * are too small (info is still written).
 */
int rsvd_grouped_schedule(int count, const int64_t* shapes, int trans, int num_sms,
                          int* units, int max_units, int* cta_off, int* info);

/* ---------------------------------------------------------------------- */
/* Allocation-free entry point                                             */
/* ---------------------------------------------------------------------- */

/*
 * rsvd_apply_a_f64_static: Y = A X in FP64 (the product of
 * rsvd_apply_a on a plain plan) for callers that may not allocate device
 * memory -- for instance code running inside a host framework that owns all
 * device memory and forbids allocation during the call, or a section that
 * was handed only its inputs and outputs -- and so cannot own a plan
 * workspace.  The thesis has no counterpart; this is a deployment aid.
 *   A  m x n (lda >= m), X n x l (ldx >= n), Y m x l (ldy >= m): device FP64.
 *   cuda_stream: the cudaStream_t the work is enqueued on (NULL = default).
 * The split-K partial sums live in one fixed device array built into the
 * library (32 MiB, 4 Mi doubles), held by every GPU that loads the library
 * until the process exits.  Limit: m * l <= 4 Mi (4194304); larger sizes
 * return RSVD_ERR_WORKSPACE without touching Y.  The call allocates nothing
 * (no cudaMalloc, no library allocator).  All calls share the array, so
 * calls that overlap on the GPU (other streams, other host threads) race;
 * the array needs no clearing (each call writes every element it reads).
 * The first call on a device looks up the array's device address for that
 * device, so make it before any stream capture.
 * Errors: -1 A NULL; -2 m; -3 n; -4 lda; -5 X NULL; -6 ldx; -7 l; -8 Y NULL;
 * -9 ldy; RSVD_ERR_CUDA if a CUDA call fails.
 */
int rsvd_apply_a_f64_static(const double* A, int64_t m, int64_t n, int64_t lda,
                            const double* X, int64_t ldx, int l, double* Y, int64_t ldy,
                            void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* RSVD_GB300_H */
