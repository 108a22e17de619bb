/*
 * mpjsvd.h -- C ABI of libmpjsvd, a GB300 (sm_103a) implementation of the mixed-precision
 * one-sided Jacobi SVD of Gao, Ma and Shao ("A mixed precision Jacobi SVD algorithm",
 * arXiv 2209.04626).
 *
 * What is computed: the thin SVD A = U diag(S) V^T of a dense real m x n matrix
 * (m >= n), to high relative accuracy, by Algorithm 4 of the paper:
 *   1. QR preconditioning (Section 3.1): Householder QR with column pivoting of A
 *      (optionally preceded by a plain QR when m > n), A P = Q R; by default the
 *      mixed-precision RRQR of Alg. 5 (pivot order from a binary32 search, then the
 *      binary64 QR of A P);
 *   2. the special-case tests of Section 3.5 (cond_R, small trailing columns, orth);
 *   3. a binary32 one-sided Jacobi SVD (Alg. 1, Section 3.2) of the triangular factor,
 *      left singular vectors only;
 *   4. the precision switch of Section 3.3: B = X^T U_low, B = Q R2, Y = X Q;
 *   5. binary64 one-sided Jacobi refinement of Y (Alg. 1, Section 3.4) accumulating V
 *      (both Jacobi stages stop as params.stop says: by default also after a sweep whose
 *      rotations were all negligible, as the paper's experiments run Alg. 1);
 *   6. Sigma = column norms, U_X = normalized columns, sorted descending; U and V are
 *      assembled from the factors (Alg. 4, last line).
 * Every stage runs as hand-written CUDA kernels on the handle's stream. For large n the
 * binary64 sweeps split each visit of a block pair by rows over a thread-block cluster
 * (params.work_kernel), and the blocked QRs apply their reflectors in 256-column blocks
 * whose binary64 products run on the bf16 tensor cores by error-free splitting
 * (params.qr_update); both compute the same method.
 *
 * Departures from the plain statement of the method, each with the same limit:
 *   - the binary64 stage evaluates each rotation's tangent in binary32 from the binary64
 *     alpha, beta, gamma (scaled by a power of two) and its cosine in binary64 for that
 *     tangent: every rotation is orthogonal to binary64 precision and only how completely a
 *     pair is annihilated (to about 2^-23 of gamma) depends on the binary32 tangent; the
 *     dot products, the rotation test and the convergence test are binary64;
 *   - the binary32 stage at large n (params.low_kernel) runs in blocked form on the tensor
 *     cores: each visit's rotations are computed from the block pair's Gram matrix (TF32 with a
 *     3-term split, binary32 accumulation) instead of from the columns.
 *
 * Conventions for every entry point:
 *   - Matrices are column-major FP64 (element (i, j) at ptr[j * ld + i]).
 *   - Matrix pointers are DEVICE pointers owned by the caller; the library never frees
 *     them and never modifies the input A. Outputs are fully overwritten.
 *   - Calls are asynchronous and stream-ordered on the handle's stream: a return value of
 *     0 means "arguments valid, work enqueued". Numeric status (non-convergence,
 *     non-finite input, a device wait that timed out) is read with mpjsvd_get_stats(),
 *     which synchronizes the stream.
 *   - Return values: 0 = success; -i = argument i (1-based, the handle counts as 1) is
 *     invalid; MPJSVD_ERR_CUDA (-100) = a CUDA call failed (see mpjsvd_last_error());
 *     MPJSVD_ERR_NOMEM (-101) = the workspace could not be allocated.
 *   - The handle owns a device workspace that grows on demand (cudaMalloc) and is freed
 *     by mpjsvd_destroy(). A handle must not be used from two host threads at once.
 */
#ifndef MPJSVD_H
#define MPJSVD_H

#ifdef __cplusplus
extern "C" {
#endif

#define MPJSVD_ERR_CUDA (-100)
#define MPJSVD_ERR_NOMEM (-101)

/* Numeric status bits (mpjsvd_stats.status, batched info[]). */
#define MPJSVD_STATUS_OK 0
#define MPJSVD_STATUS_NOT_CONVERGED 1  /* a Jacobi stage hit maxsweep sweeps */
#define MPJSVD_STATUS_NONFINITE 2      /* A contains Inf or NaN; outputs are not meaningful */
#define MPJSVD_STATUS_TIMEOUT 4        /* a bounded device wait gave up (or a kernel found its launch
                                          geometry not the one it was launched for); outputs not
                                          meaningful */
#define MPJSVD_STATUS_ZERO_SIGMA 8     /* some singular value is exactly zero (rank deficient) */

/* Algorithm choices. */
#define MPJSVD_MODE_AUTO 0   /* Alg. 4 special-case tests decide whether stage 3 runs */
#define MPJSVD_MODE_MIXED 1  /* always run the binary32 stage (force the mixed path) */
#define MPJSVD_MODE_PLAIN 2  /* never run it: plain FP64 preconditioned Jacobi (Alg. 2) */

#define MPJSVD_PRECOND_RT 0  /* Jacobi on X = R^T (lower triangular); default */
#define MPJSVD_PRECOND_R 1   /* Jacobi on X = R (Alg. 4 with Q2 = I) */
#define MPJSVD_PRECOND_L 2   /* Jacobi on X = L from the second preconditioning R = L Q2^T
                                (the LQ of R as the QR of R^T; Alg. 2, Section 2.2) */
#define MPJSVD_PRECOND_AUTO 3 /* Alg. 2's choice: X = R when R is "almost diagonal" (every
                                column diagonally dominant, |r_jj| >= sum_{i<j} |r_ij|), else
                                X = L; decided on the device (single-matrix path only) */

/* params.qrcp: the rank-revealing QR of the preconditioning (Section 3.1). */
#define MPJSVD_QRCP_MIXED 0  /* Alg. 5: binary32 pivot search on lower(A), binary64 QR of A P;
                                default */
#define MPJSVD_QRCP_F64 1    /* Businger-Golub QR with column pivoting in binary64 */

/* params.low_kernel: the kernel of the binary32 stage (Section 3.2). */
#define MPJSVD_LOWK_AUTO 0   /* the tensor-core form where it is faster (chosen by size) */
#define MPJSVD_LOWK_TC 1     /* blocked form on the tensor cores: 64-column blocks, pair Gram
                                matrices and rotation application by TF32x3 tcgen05 MMAs */
#define MPJSVD_LOWK_REG 2    /* register-resident level-1 visits (no tensor cores) */

/* params.gemm_kernel: the n x n x n binary64 products (the switch of Section 3.3, the safeguard
 * and the V from QR of Section 3.4). */
#define MPJSVD_GEMMK_AUTO 0  /* tensor cores for 1024 <= n <= 4096 (where measured faster) */
#define MPJSVD_GEMMK_TC 1    /* bf16 tensor cores by error-free operand splitting (see
                                mpjsvd_dgemm_tc) */
#define MPJSVD_GEMMK_F64 2   /* the FP64 pipe (register-blocked SIMT kernel) */

/* params.work_kernel: the visits of the binary64 sweeps (Section 3.4, Alg. 1). */
#define MPJSVD_WORKK_AUTO 0    /* cluster-split visits when a block pair of width 4 does not fit
                                  one CTA's registers (more than 2048 rows), else one CTA per visit */
#define MPJSVD_WORKK_CLUSTER 1 /* every visit split by rows over a thread-block cluster of 2, 4 or
                                  8 CTAs (block width 4; up to 16384 rows) */
#define MPJSVD_WORKK_CTA 2     /* one CTA per visit, the block pair in its registers */

/* params.qr_update: the trailing updates of the blocked Householder QRs and the applications of
 * their Q (the preconditioning of Section 3.1, the QR of B and its Q in Section 3.3, U of Alg. 4). */
#define MPJSVD_QRU_AUTO 0  /* tensor cores for the preconditioner's QR from n = 6144 and for
                              U = Q [U_R; 0] (and mpjsvd_geqrf / mpjsvd_apply_q) from n = 4096
                              on; the switch's QR of B and its Q stay on the FP64 pipe (B is
                              graded by rows, which the split products' per-column scaling does
                              not follow: the refinement then rotates more) */
#define MPJSVD_QRU_TC 1    /* two-level everywhere (n > 256): 256-column outer blocks applied in
                              the compact UT form with the binary64 products on the bf16 tensor
                              cores (error-free operand splitting, see mpjsvd_dgemm_tc) */
#define MPJSVD_QRU_F64 2   /* one-level compact-WY updates on the FP64 pipe */

/* params.switch_method: the precision switch of Section 3.3. */
#define MPJSVD_SWITCH_U 0    /* B = X^T U_low, B = Q R2, Y = X Q (the method the paper prefers;
                                default) */
#define MPJSVD_SWITCH_V 1    /* the alternative: the binary32 stage also accumulates V_low
                                (its rotations applied in binary64), V_low = Q R2, Y = X Q;
                                runs the register-resident binary32 stage */

/* params.stop: when Alg. 1 (both precisions) stops. */
#define MPJSVD_STOP_XGESVJ 0 /* default: after a sweep without rotations, or after a sweep other
                                than the first whose rotations were all negligible (largest
                                cosine among the rotated pairs below sqrt(n) tol and n times it
                                times the largest |tan| below tol): the rule of LAPACK's xGESVJ,
                                with which the paper's experiments run Alg. 1 (Section 7.1) */
#define MPJSVD_STOP_ALG1 1   /* only after a sweep without rotations (Alg. 1 as printed) */

typedef struct mpjsvd_ctx* mpjsvd_handle;

/* Tunables. Defaults (mpjsvd_default_params) are the paper's values of Section 7.1. */
typedef struct {
    double tol_alg;       /* 1e-2: recorded only (the binary32 stage always uses Jacobi) */
    double tol_orth;      /* 1e-5: skip stage 3 when |Xt^T Xt - I|_max <= tol_orth (Sec. 3.5) */
    double tol_cond_coef; /* 1.5: skip stage 3 when |R11|/|Rnn| <= coef * n^(1/4) (Sec. 3.5) */
    double trailing_frac; /* 0.25: skip stage 3 when the last ceil(frac*n) columns of X all
                             have norm <= 2^-12 * max column norm (Sec. 3.5 footnote) */
    int maxsweep;         /* 30: Alg. 1 maxiter, both precisions */
    int block_w;          /* column-block width of the sweeps; 0 = pick from the size */
    int mode;             /* MPJSVD_MODE_* */
    int precond;          /* MPJSVD_PRECOND_* */
    int qr_first;         /* 1: plain QR of A before the QRCP when m > n (Alg. 4 lines 1-3);
                             0 (default): QRCP applied to A directly (same R and P) */
    int timing;           /* 1: record per-phase CUDA-event times in mpjsvd_stats */
    int qrcp;             /* MPJSVD_QRCP_*; Alg. 5 falls back to binary64 when the binary32
                             matrix does not fit the resident kernel (stats.qrcp tells) */
    int stop;             /* MPJSVD_STOP_* */
    int wait_limit_ms;    /* 4000: every bounded device wait of a call (a grid barrier, a block
                             hand-off between CTAs) gives up after this many milliseconds and
                             records MPJSVD_STATUS_TIMEOUT; 1 .. 600000 */
    int low_kernel;       /* MPJSVD_LOWK_* */
    int v_by_qr;          /* 1: the refinement runs without V, then V comes from the QR of
                             X^T U_X and one more Alg. 1 with V accumulated from that Q
                             (Section 3.4); 0 (default): V accumulated through the refinement */
    int switch_method;    /* MPJSVD_SWITCH_* */
    int gemm_kernel;      /* MPJSVD_GEMMK_* */
    double y_tol;         /* > 0: the Y1/Y2 safeguard of Section 3.4 with this cosine
                             threshold (Y2 = the columns of Y from the first one whose largest
                             cosine with an earlier column exceeds y_tol: Alg. 1 on Y2, one pass
                             over the Y1 x Y2 pairs, then the refinement); 0 (default): off */
    int work_kernel;      /* MPJSVD_WORKK_* */
    int work_cluster;     /* CTAs per visit of the cluster form: 0 (default) the fewest that hold
                             the rows (2048 per CTA), or 2, 4, 8 (at least that many) */
    int qr_update;        /* MPJSVD_QRU_* */
} mpjsvd_params;

/* Per-call record of what ran (read after the call with mpjsvd_get_stats). */
typedef struct {
    int status;           /* MPJSVD_STATUS_* bits */
    int branch;           /* 0 stage 3 ran; 1 skipped: cond_R; 2 skipped: trailing columns;
                             3 skipped: orth; 4 skipped: MPJSVD_MODE_PLAIN */
    int sweeps_low;       /* binary32 sweeps (0 if skipped) */
    int sweeps_work;      /* binary64 sweeps */
    long long rot_low;    /* rotations applied in binary32 */
    long long rot_work;   /* rotations applied in binary64 */
    double cond_r;        /* |R(0,0)| / |R(n-1,n-1)| */
    double orth;          /* |Xt^T Xt - I|_max (computed in MPJSVD_MODE_AUTO only, else -1) */
    int block_w_low;      /* block widths used */
    int block_w_work;
    float ms_qr;          /* per-phase times (ms) when params.timing = 1, else 0 */
    float ms_branch;
    float ms_low;
    float ms_switch;
    float ms_work;
    float ms_final;
    int launches;         /* CUDA kernels the call launched (gated-off stages included) */
    int qrcp;             /* the RRQR that ran: MPJSVD_QRCP_MIXED or MPJSVD_QRCP_F64 */
    int precond;          /* the Jacobi input that ran: MPJSVD_PRECOND_RT, _R or _L */
    int sweeps_v;         /* binary64 sweeps outside the refinement proper: the safeguard's
                             Alg. 1 on Y2 and its pass over Y1 x Y2, the final Alg. 1 with V of
                             params.v_by_qr */
    long long rot_v;      /* rotations of those sweeps */
    int y2_cols;          /* columns the safeguard put in Y2 (0: inactive or off) */
    int n_flagged;        /* near-degenerate count of the handle's last mpjsvd_svd_backward
                             (pairs with |s_i - s_j| <= gap_tol max(s_i, s_j) plus s_i <= 2^-53 s_0);
                             -1 if the handle has run none */
    int work_cluster;     /* CTAs per visit of the binary64 sweeps (1: one CTA per visit) */
    /* per sweep (the first 16 of each stage): rotations, and the largest cosine |gamma| /
       (|x_a| |x_b|) among the rotated pairs (0 when none rotated) */
    long long rot_sweep_low[16];
    long long rot_sweep_work[16];
    float cos_sweep_low[16];
    float cos_sweep_work[16];
} mpjsvd_stats;

/* Fill *p with the defaults. Returns 0, or -1 if p is NULL. */
int mpjsvd_default_params(mpjsvd_params* p);

/* Create a handle on the current CUDA device. p may be NULL (defaults). cuda_stream is a
 * cudaStream_t (NULL = legacy default stream); it can be changed with
 * mpjsvd_set_stream(). */
int mpjsvd_create(mpjsvd_handle* h, const mpjsvd_params* p, void* cuda_stream);

/* Switch the handle's stream. The new stream is made to wait (on the device, through an
 * event; the host does not block) for the work already queued on the previous one, since the
 * workspace is shared by all calls of the handle. Passing the current stream is a no-op.
 * Returns 0, -1 if h is NULL, MPJSVD_ERR_CUDA if the ordering could not be set up. */
int mpjsvd_set_stream(mpjsvd_handle h, void* cuda_stream);
int mpjsvd_set_params(mpjsvd_handle h, const mpjsvd_params* p);

/* Thin SVD of one matrix (Algorithm 4).
 *   m, n : 1 <= n <= m <= 24576, n <= 8192 (a visit of the sweeps keeps its columns' n rows
 *          in one CTA's registers)
 *   A    : device, m x n, leading dimension lda >= m; not modified. Entries must be finite
 *          (else MPJSVD_STATUS_NONFINITE) and their squares summed over a column must not
 *          overflow binary64 (|a_ij| well below 1e154; column norms are not pre-scaled)
 *   U    : device, m x n output, leading dimension m
 *   S    : device, n output, descending
 *   V    : device, n x n output, leading dimension n
 *   tol  : Alg. 1 threshold of the binary64 stage; <= 0 selects sqrt(n) * 2^-53
 * A = U diag(S) V^T with U^T U = I, V^T V = I. Sign convention: each pair (u_k, v_k) is
 * flipped so that the entry of v_k with the largest magnitude is positive (ties: lowest
 * row index). */
int mpjsvd_svd(mpjsvd_handle h, int m, int n, const double* A, int lda, double* U, double* S,
               double* V, double tol);

/* Thin SVDs of `batch` independent matrices of uneven sizes in one persistent launch
 * (one CTA per matrix, largest first). With params.block_w = 0 the first call that contains
 * a size class of n tunes it (host-synchronizing: each kernel variant runs on a sample of the
 * class; see mpjsvd_get_batched_tuning); params.qrcp selects Alg. 5 (default) or binary64
 * Businger-Golub for the RRQR; params.precond must be RT or R.
 *   m, n, lda : HOST arrays of length batch (1 <= n_i <= m_i <= 1024, n_i <= 512,
 *               lda_i >= m_i)
 *   A, U, S, V: DEVICE arrays of length batch holding device pointers laid out as in
 *               mpjsvd_svd (U_i leading dimension m_i, V_i leading dimension n_i)
 *   info      : DEVICE int array of length batch, written with the MPJSVD_STATUS_* bits
 *               of each matrix
 * Same algorithm, parameters and sign convention as mpjsvd_svd. */
int mpjsvd_svd_batched(mpjsvd_handle h, int batch, const int* m, const int* n, const int* lda,
                       const double* const* A, double* const* U, double* const* S,
                       double* const* V, double tol, int* info);

/* mpjsvd_svd_batched with the sizes in DEVICE memory (the layout of the hot-path table's
 * boundary): nothing is read or copied on the host, so once a call of the same batch, max_m and
 * max_n has run (its workspace then exists) the call can be captured in a CUDA graph and
 * replayed. The order of the work queue (largest n^2 m first) is computed on the device.
 *   max_m, max_n : HOST bounds of the sizes, 1 <= max_n <= max_m <= 1024, max_n <= 512
 *   m, n, lda : DEVICE int arrays of length batch; a matrix whose sizes fall outside the
 *               bounds (or n < 1, m < n, lda < m) is not computed and gets info = -1
 *   A, U, S, V, tol, info : as in mpjsvd_svd_batched
 * Uses the kernel variants the handle's autotuner picked in an earlier mpjsvd_svd_batched call
 * (the defaults otherwise). */
int mpjsvd_svd_batched_dev(mpjsvd_handle h, int batch, int max_m, int max_n, const int* m, const int* n,
                           const int* lda, const double* const* A, double* const* U, double* const* S,
                           double* const* V, double tol, int* info);

/* The batched autotuner's picks (params.block_w = 0): per size class of n (<= 32, <= 64,
 * <= 128, <= 256, <= 512), the block widths of the binary32 and binary64 stages that ran
 * fastest on a sample of the class's matrices in the first mpjsvd_svd_batched call that
 * contained the class, and that sample's time (ms). 0 for a class not tuned yet. Any pointer
 * may be NULL; each array has 5 entries. */
int mpjsvd_get_batched_tuning(mpjsvd_handle h, int* w_low, int* w_work, float* ms);

/* Adjoint of the thin SVD (not part of the paper). Given U (m x n), S (n, descending,
 * positive), V (n x n) from mpjsvd_svd and the cotangents gU (m x n), gS (n), gV (n x n)
 * (device; each may be NULL = zero), writes
 *   gA = U [(F o (U^T gU - gU^T U)) S + diag(gS) + S (F o (V^T gV - gV^T V))] V^T
 *        + (I - U U^T) gU S^-1 V^T,     F_ij = 1/(s_j^2 - s_i^2) (i != j), F_ii = 0,
 * (device, m x n, leading dimension m). Near-degenerate inputs are counted, never
 * clamped: *n_flagged (host, may be NULL; the call then synchronizes the stream) receives
 * the number of pairs with |s_i - s_j| <= gap_tol * max(s_i, s_j) plus the number of
 * s_i <= 2^-53 * s_0. */
int mpjsvd_svd_backward(mpjsvd_handle h, int m, int n, const double* U, const double* S,
                        const double* V, const double* gU, const double* gS, const double* gV,
                        double* gA, double gap_tol, int* n_flagged);

/* Adjoints of a batch of thin SVDs (the differentiation workload's many small matrices) in
 * one launch, one CTA per matrix; the formula and the flags of mpjsvd_svd_backward.
 *   m, n      : HOST arrays of length batch, 1 <= n_i <= m_i <= 4096, n_i <= 512
 *   U, S, V, gA : DEVICE arrays of length batch holding device pointers (U_i m_i x n_i, leading
 *               dimension m_i; V_i n_i x n_i; gA_i m_i x n_i, leading dimension m_i)
 *   gU, gS, gV : DEVICE arrays of device pointers or NULL (all zero); a NULL entry is a zero
 *               cotangent for that matrix
 *   n_flagged : DEVICE int array of length batch: per matrix, the near-degenerate count
 * Asynchronous on the handle's stream; uses the handle's adjoint workspace. */
int mpjsvd_svd_backward_batched(mpjsvd_handle h, int batch, const int* m, const int* n,
                                const double* const* U, const double* const* S,
                                const double* const* V, const double* const* gU,
                                const double* const* gS, const double* const* gV,
                                double* const* gA, double gap_tol, int* n_flagged);

/* Allocation-free thin SVD of one small matrix (the paper has no counterpart: this is a
 * deployment variant of mpjsvd_svd). It takes no handle and calls no cudaMalloc, cudaFree or
 * allocating library routine, for callers that cannot allocate device memory: code whose
 * allocator owns the GPU's memory up front, latency-critical loops where an allocation's
 * implicit device synchronization is not acceptable, or code that must not grow its memory
 * footprint after start-up. Its scratch is one static device array of 6 MiB that every GPU
 * loading this library holds until the process exits.
 *   m, n : 1 <= n <= m, m <= 512, n <= 256 (larger sizes return -1 / -2 with a message in
 *          mpjsvd_last_error())
 *   A, U, S, V, lda, tol : as in mpjsvd_svd (device pointers, default parameters,
 *          MPJSVD_MODE_AUTO)
 *   status : DEVICE int, may be NULL; written on the stream after the last stage with the
 *          call's MPJSVD_STATUS_* bits (read it after synchronizing the stream). A call whose
 *          status has MPJSVD_STATUS_NONFINITE or MPJSVD_STATUS_TIMEOUT set produced no
 *          meaningful U, S, V (they are filled with NaN)
 *   cuda_stream : the stream the work is enqueued on (cudaStream_t; NULL = legacy stream)
 * The call does not block: 0 means "arguments valid, work enqueued". The first call on a
 * device looks up the scratch array's device address (once per device, with that device
 * current); make that first call before any stream capture. Every call shares the scratch
 * array: calls that overlap on the GPU (other streams, other host threads) race and must be
 * ordered by the caller. */
int mpjsvd_svd_noalloc(int m, int n, const double* A, int lda, double* U, double* S, double* V,
                       double tol, int* status, void* cuda_stream);

/* Householder QR of one matrix, in place (the QR preconditioning of Section 3.1 and the QR
 * of the precision switch of Section 3.3 as a standalone call; blocked, compact-WY form).
 *   m, n : 1 <= n <= m <= 12480, n <= 12288
 *   A    : device, m x n, leading dimension lda >= m; on return R on and above the
 *          diagonal and the tails of the reflectors below it (LAPACK geqrf layout)
 *   tau  : device, n output; H_j = I - tau_j v_j v_j^T with v_j(j) = 1, Q = H_0 ... H_{n-1}
 * Reflector convention: beta = -sign(alpha) |x| (alpha = the diagonal entry, sign(0) = +),
 * tail = x(j+1:) / (alpha - beta), tau = (beta - alpha) / beta; tau = 0 and v = e_j when
 * the tail is zero. Stream-ordered on the handle's stream; uses the handle's workspace. */
int mpjsvd_geqrf(mpjsvd_handle h, int m, int n, double* A, int lda, double* tau);

/* The rank-revealing QR of the preconditioning (Section 3.1; Alg. 5 by default, see
 * params.qrcp) as a standalone call: A P = Q R.
 *   m, n : 1 <= n <= m <= 24576, n <= 12288
 *   A    : device, m x n, lda >= m; on return the Householder QR of A P in pivot order
 *          (mpjsvd_geqrf layout: R on and above the diagonal, reflector tails below)
 *   jpvt : device, n output: column j of A P is column jpvt[j] of A
 *   tau  : device, n output
 * Alg. 5: jpvt from a Businger-Golub pivot search in binary32 on A scaled by a power of two,
 * then the binary64 QR of A P; MPJSVD_QRCP_F64: Businger-Golub in binary64 throughout (the
 * first maximum of the downdated norms wins in both). stats.qrcp records which ran. */
int mpjsvd_geqp3(mpjsvd_handle h, int m, int n, double* A, int lda, int* jpvt, double* tau);

/* C <- Q C with Q = H_0 ... H_{k-1} from mpjsvd_geqrf (A: m x k reflectors, lda >= m; tau: k).
 *   C : device, m x ncols, leading dimension ldc >= m, overwritten
 * 1 <= k <= m <= 12480, 1 <= ncols <= 12288. Forming the thin Q is this call applied to the
 * first ncols columns of the identity. */
int mpjsvd_apply_q(mpjsvd_handle h, int m, int ncols, int k, const double* A, int lda,
                   const double* tau, double* C, int ldc);

/* The two tensor-core steps of a visit of the blocked binary32 stage (Section 3.2 in blocked
 * form) as a standalone call, for one block pair Z = [X_I X_J] of 128 columns:
 *   G = Z^T Z     (if G is not NULL; G: device, 128 x 128 binary32, column-major)
 *   Z <- Z W      (if W is not NULL, after G; W: device, 128 x 128 binary32, column-major)
 * both by TF32 tcgen05 MMAs with a 3-term split (hi = tf32(z), lo = tf32(z - hi);
 * hi hi' + hi lo' + lo hi'), accumulated in binary32.
 *   m : rows of Z, 1 <= m; Z: device, m x 128 binary32, leading dimension ldz >= m
 * Stream-ordered on the handle's stream; one CTA. */
int mpjsvd_tc_block_f32(mpjsvd_handle h, int m, float* Z, int ldz, float* G, const float* W);

/* C = op(A) B in binary64 on the bf16 tensor cores (the products of the precision switch of
 * Section 3.3 as a standalone call): each row of op(A) and each column of B is scaled by a
 * power of two and split into 8 slices of 7 bits (bf16 values); the slice products of the
 * weight classes that matter are accumulated exactly in binary32 on the tensor cores
 * (tcgen05.mma) over chunks of 512 k and added in binary64 (the Ozaki scheme); products of
 * integers that are exact in binary64 come out exact. Error per
 * entry: about 2^-52 K max_k |op(A)_ik| max_k |B_kj|, the bound of a binary64 GEMM with the
 * row and column maxima in place of the entries.
 *   op(A) = A (transA = 0; A: M x K, lda >= M) or A^T (transA = 1; A: K x M, lda >= K)
 *   B : K x N, ldb >= K;  C : M x N, ldc >= M (overwritten). Device pointers, column-major.
 * Stream-ordered on the handle's stream; uses the handle's workspace (about 4 K (M + N) bytes
 * for the split operands). */
int mpjsvd_dgemm_tc(mpjsvd_handle h, int M, int N, int K, const double* A, int lda, int transA,
                    const double* B, int ldb, double* C, int ldc);

/* Measurement utility (not part of the paper): the FP64 FMA throughput of the current GPU in
 * TFLOP/s (2 flops per FMA), from a kernel of independent FMA chains on every SM, timed with
 * CUDA events on cuda_stream (best of three launches after a warm-up; about 0.4 s). This is
 * the denominator of the FP64 roofline fractions. Returns 0, -2 for a NULL tflops,
 * MPJSVD_ERR_CUDA. Synchronizes cuda_stream. */
int mpjsvd_measure_fp64_peak(void* cuda_stream, double* tflops);

/* Failure-detection check (not part of the paper): enqueue on the handle's stream a kernel
 * whose cross-CTA waits can never be satisfied (a block hand-off on a counter that nothing
 * releases, and a grid barrier that one CTA never reaches). Both waits are the library's
 * own bounded waits: after params.wait_limit_ms they give up, record MPJSVD_STATUS_TIMEOUT
 * and return, so the kernel exits and the handle stays usable. The status is then read with
 * mpjsvd_get_stats(). Uses the handle's workspace. Returns 0 (enqueued), -1 for a NULL
 * handle, MPJSVD_ERR_CUDA. */
int mpjsvd_selftest_timeout(mpjsvd_handle h);

/* Synchronize the handle's stream and copy the stats of the last mpjsvd_svd call. */
int mpjsvd_get_stats(mpjsvd_handle h, mpjsvd_stats* st);

/* Free the workspace and the handle. */
int mpjsvd_destroy(mpjsvd_handle h);

/* Text of the last CUDA error seen by any call on this thread (static storage). */
const char* mpjsvd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
