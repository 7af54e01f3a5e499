/*
 * oz2 — Ozaki-II emulation of FP64 / FP32 matrix multiplication on one B300.
 *
 * C ABI of liboz2.so.  Method: Uchino, Ozaki, Imamura, "Error Analysis of
 * Matrix Multiplication Emulation Using Ozaki-II Scheme", arXiv 2602.02549.
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major: X[i*ldx + j].  A is m x k (lda >= k), B is k x n
 *     (ldb >= n), C is m x n (ldc >= n).  With OZ2_TRANS_A the array passed as
 *     A holds A^T (k x m, lda >= m); with OZ2_TRANS_B it holds B^T (n x k,
 *     ldb >= k).  These are the only transposes; there is no alpha/beta.
 *   - A, B, C, the workspace and every optional output are DEVICE pointers
 *     owned by the caller (oz2_gemm_host / oz2_sgemm_host: A, B and C in host
 *     memory).  Nothing is freed by the library.
 *   - All work is enqueued on opts->stream (NULL: the legacy default stream)
 *     and the call returns without synchronising.  Argument errors are
 *     returned before anything is enqueued, and C is then left untouched.
 *   - Return value: OZ2_OK (0) or one of the negative OZ2_E* codes.
 *   - NaN or Inf inputs violate the paper's preconditions (A, B finite); the
 *     result for them is unspecified but no out-of-bounds access occurs.
 */
#ifndef OZ2_H
#define OZ2_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define OZ2_API __attribute__((visibility("default")))
#else
#define OZ2_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define OZ2_OK          0
#define OZ2_EINVAL     -1   /* bad dimension, leading dimension, N, mode or null pointer */
#define OZ2_ERANGE     -2   /* k > 2^17 in a batched problem (Section 3: k <= 2^17 keeps
                                the INT32 sums exact; single calls split K instead)      */
#define OZ2_ENOMEM     -3   /* workspace smaller than oz2_workspace_size()               */
#define OZ2_ECUDA      -4   /* a CUDA runtime or driver call failed                      */
#define OZ2_ETIMEOUT   -5   /* a bounded device-side wait gave up (see oz2_sync)         */
#define OZ2_ENOTSUP    -6   /* combination not supported                                 */

/* mode bits */
#define OZ2_ACCURATE    0   /* Algorithm 2 as printed: Cbar = Abar*Bbar on the tensor cores */
#define OZ2_FAST        1   /* Cbar replaced by a Cauchy-Schwarz majorant (no extra GEMM)    */
#define OZ2_TRANS_A     2
#define OZ2_TRANS_B     4
#define OZ2_CONJ_A      8   /* complex calls only: op(A) conjugated (with OZ2_TRANS_A: A^H) */
#define OZ2_CONJ_B     16   /* complex calls only: op(B) conjugated                        */
#define OZ2_COMPONENTWISE 32 /* bound rule (nmoduli == 0) per entry: see below              */

/* Limits stated by the paper (Section 3, Algorithm 1).  Single calls with a
 * larger k split K into ranges of at most OZ2_K_MAX (oz2_k_ranges). */
#define OZ2_K_MAX   131072  /* k <= 2^17 */
#define OZ2_N_MIN   2
#define OZ2_N_MAX   49      /* p_l <= 256 pairwise coprime, eq. (p_list) */

/* Phases of one call, in launch order (for oz2_opts.phase_events). */
#define OZ2_PHASE_STATS     0   /* max |x| per row/column, sums for the N rule   */
#define OZ2_PHASE_QUANT     1   /* Abar, Bbar (Algorithm 2)                       */
#define OZ2_PHASE_SCALEGEMM 2   /* Cbar = Abar Bbar, row/column maxima            */
#define OZ2_PHASE_EXPONENTS 3   /* N rule, mu, nu                                 */
#define OZ2_PHASE_RESIDUES  4   /* A'_l, B'_l (Algorithm 3)                       */
#define OZ2_PHASE_GEMM      5   /* C'_l = A'_l B'_l, W_l = mod(C'_l, p_l)         */
#define OZ2_PHASE_CRT       6   /* C'(1), C'(2), Q, C'', inverse scaling          */
#define OZ2_NPHASES         7

typedef struct oz2_opts {
    void   *stream;          /* cudaStream_t; NULL = legacy default stream                 */
    void   *workspace;       /* device scratch of >= oz2_workspace_size(...) bytes,
                                256-byte aligned.  NULL: the library uses one cached
                                buffer per device, shared by every call without a
                                workspace and grown with cudaMalloc (a buffer it replaces
                                stays allocated until exit); such calls must not overlap
                                on the GPU (serialise them per device: calls on two
                                streams or from two host threads race on that buffer).   */
    size_t  workspace_bytes;
    double  target;          /* nmoduli == 0: target normwise relative error tau           */
    int     nmax;            /* nmoduli == 0: largest N tried (0 = 20 DGEMM, 14 SGEMM)     */
    int    *n_out;           /* optional device int: the N used                            */
    int32_t *mu_out;         /* optional device int32[m]: the exponents mu of Algorithm 2  */
    int32_t *nu_out;         /* optional device int32[n]: the exponents nu                  */
    const int32_t *mu_in;    /* optional device int32[m] and int32[n]: use these exponents  */
    const int32_t *nu_in;    /*   instead of Algorithm 2's (both or neither; needs N > 0)  */
                             /* k > 2^17 (S K ranges, oz2_k_ranges): n_out int[S], and the
                                four exponent vectors S of them back to back (range s at
                                mu_out + s*m, nu_out + s*n, likewise mu_in, nu_in)         */
    int8_t *w_out;           /* optional device int8[N*m*n]: the residue products W_l of
                                Algorithm 3, plane l at w_out + l*m*n, row-major m x n     */
    void  **phase_events;    /* optional cudaEvent_t[OZ2_NPHASES + 1], created by the
                                caller: event i is recorded on the stream before phase i,
                                event OZ2_NPHASES after the last one (for timing).
                                w_out and phase_events: k <= 2^17 only (OZ2_ENOTSUP)       */
} oz2_opts;

/*
 * C = OS_II(A, B): Algorithm 1 of the paper (Scaling, Algorithm 2; CRT,
 * Algorithm 3; inverse scaling) for FP64 A, B, C (DGEMM emulation, b = 64).
 *   nmoduli  N in [2, 49] uses the first N moduli of eq. (p_list);
 *            0 picks the smallest N in [2, opts->nmax] whose N-dependent part
 *            of the Theorem 2 bound (eq. thm:err-2) is <= opts->target times a
 *            lower bound of max_ij (|A||B|)_ij (requires opts with target > 0).
 *            With mode | OZ2_COMPONENTWISE (nmoduli == 0 only) the N-dependent
 *            part must be <= target * L_ij on every entry, L_ij =
 *            2^-(mu'_i + nu'_j) (floor(2^mu' |A|) floor(|B| 2^nu'))_ij <=
 *            (|A||B|)_ij, one more integer product on the tensor cores; an
 *            entry whose L_ij is 0 while its bound terms are not gets nmax.
 *   k        up to 2^17 as in the paper (Section 3).  A larger k is split
 *            into S consecutive K ranges of at most 2^17 (oz2_k_ranges); each
 *            range is a full OS_II of A[:, range] B[range, :] with its own
 *            exponents and its own N (the bound rule then targets target / S,
 *            so the N-dependent parts of the ranges' Theorem 2 bounds add up
 *            to at most target times the same lower bound of max (|A||B|)),
 *            and the S results are added into C in range order, one rounding
 *            in the output precision per addition.
 *   m, n, k  >= 1.
 * oz2_gemm uses the library-managed workspace (see oz2_opts.workspace: calls
 * without a workspace share one buffer per device and must be serialised per
 * device) and the legacy default stream.
 */
OZ2_API int oz2_gemm(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                     double *C, int ldc, int nmoduli, int mode);
OZ2_API int oz2_gemm_ex(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                        double *C, int ldc, int nmoduli, int mode, const oz2_opts *opts);

/* FP32 A, B, C (SGEMM emulation, b = 32): Section 3.1 constants for b = 32
 * (P2 = 0, s_l1 = double(P/p_l q_l), s_l2 = 0).  C'' is rounded to FP32 after
 * the inverse scaling (identical to Algorithm 3's order unless single(C'')
 * would overflow, which happens once P > 2^128, N >= 17). */
OZ2_API int oz2_sgemm(int m, int n, int k, const float *A, int lda, const float *B, int ldb,
                      float *C, int ldc, int nmoduli, int mode);
OZ2_API int oz2_sgemm_ex(int m, int n, int k, const float *A, int lda, const float *B, int ldb,
                         float *C, int ldc, int nmoduli, int mode, const oz2_opts *opts);

/*
 * Complex products (ZGEMM: FP64 parts, CGEMM: FP32 parts), C = op(A) op(B) for
 * interleaved complex matrices (real, imaginary; each pointer aligned to one
 * complex element, lda/ldb/ldc counted in complex elements).  The paper treats
 * real products only (complex emulation is left to other work); here a complex
 * product is two real emulated products over 2k with the same Algorithms 1-3:
 *   Re C = [Re op(A), Im op(A)] [Re op(B); -Im op(B)],
 *   Im C = [Re op(A), Im op(A)] [Im op(B);  Re op(B)],
 * so each part carries the Theorem 2 bound of its real product (k -> 2k, and
 * 2k > 2^17 runs split-K).  mode: OZ2_FAST, OZ2_TRANS_A/B, OZ2_CONJ_A/B.
 * opts as for the real calls, applied to both parts (the bound rule targets
 * opts->target for each part); the exports are per part: n_out int[2S],
 * mu_out int32[2Sm], nu_out int32[2Sn] (part 0 = Re, then part 1 = Im; S = the
 * K ranges of 2k), likewise mu_in, nu_in; w_out and phase_events: OZ2_ENOTSUP.
 * The workspace is oz2_zworkspace_size(...) bytes.  Returns as oz2_gemm_ex.
 */
OZ2_API int oz2_zgemm(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C,
                      int ldc, int nmoduli, int mode, const oz2_opts *opts);
OZ2_API int oz2_cgemm(int m, int n, int k, const float *A, int lda, const float *B, int ldb, float *C,
                      int ldc, int nmoduli, int mode, const oz2_opts *opts);
/* Workspace bytes of oz2_zgemm (fp32 = 0) or oz2_cgemm (fp32 = 1); 0 for invalid
 * sizes.  Host-only. */
OZ2_API size_t oz2_zworkspace_size(int m, int n, int k, int nmax, int mode, int fp32);

/*
 * Row-sharded emulated DGEMM (the paper treats one product on one device):
 * the ranks of a job each hold a block of rows of A and all of B and compute
 * the same rows of C = OS_II(A, B), bit for bit as one unsharded call would.
 * Algorithm 2's mu_i needs only row i, but nu_j needs max_h cbar_hj over ALL
 * rows of A, and the bound rule (nmoduli == 0) needs the maxima over all rows
 * of |A| v and 2^alpha' and the per-k maxima of |A|: one exchange, an
 * element-wise MAX over the ranks of three arrays that live in the workspace.
 *   1. oz2_gemm_rows_begin on every rank (its rows: m, A): scaling up to the
 *      bound rule's reductions; *ex receives the three device arrays:
 *        cmax_col  int32[n]   column maxima of Cbar over this rank's rows
 *        kmax      int64[k]   per-k maxima of |A| (bits of nonnegative doubles,
 *                             which order like the values)
 *        red       int64[8]   the bound rule's maxima (bits, likewise)
 *   2. the caller replaces each array by the element-wise maximum over the
 *      ranks, in place (e.g. an NCCL all-reduce with ncclMax on opts->stream);
 *   3. oz2_gemm_rows_end on every rank with the same arguments plus C: the
 *      rest of Algorithms 2 and 3 and the inverse scaling for its rows.
 * Both calls take the same m, n, k, A, lda, B, ldb, nmoduli, mode and opts;
 * opts->workspace (oz2_workspace_size(m, n, k, nmax, mode, 0) bytes) is
 * required and carries the state from one call to the other.  k <= 2^17;
 * mode: OZ2_TRANS_A, OZ2_TRANS_B (OZ2_FAST, OZ2_COMPONENTWISE, mu_in/nu_in,
 * w_out and phase_events: OZ2_ENOTSUP).  Returns as oz2_gemm_ex.
 */
typedef struct oz2_exchange {
    int32_t *cmax_col;
    size_t n;
    int64_t *kmax;
    size_t k;
    int64_t *red;
    size_t nred;
} oz2_exchange;

OZ2_API int oz2_gemm_rows_begin(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                                int nmoduli, int mode, const oz2_opts *opts, oz2_exchange *ex);
OZ2_API int oz2_gemm_rows_end(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                              double *C, int ldc, int nmoduli, int mode, const oz2_opts *opts);

/*
 * Batched emulated DGEMM: many independent problems of uneven shapes, each
 * with its own exponents and its own N (fixed, or the bound rule for its own
 * target).  The scaling GEMMs of all problems run as one persistent tcgen05
 * launch and the N residue GEMMs of all problems as another (64 problems per
 * launch; heaviest first), and every other phase is one launch over the work
 * of all problems, each on opts->stream (there are no library-owned streams).
 * With a caller workspace the call allocates nothing and enqueues only kernel
 * launches (and, with phase_events, event records) on that stream, so it can be
 * captured into a CUDA graph and replayed as one launch.  Each result is bit-identical to oz2_gemm_ex on the
 * same problem.  opts: stream, workspace, phase_events are used; the other
 * fields are ignored (per-problem settings live in oz2_problem).
 */
typedef struct oz2_problem {
    int m, n, k;
    const double *A;
    int lda;
    const double *B;
    int ldb;
    double *C;
    int ldc;
    int nmoduli;       /* N in [2, 49], or 0 for the bound rule with `target`  */
    double target;     /* nmoduli == 0: target normwise relative error         */
    int nmax;          /* nmoduli == 0: largest N tried (0 = 20)               */
    int mode;          /* OZ2_FAST | OZ2_TRANS_A | OZ2_TRANS_B | OZ2_COMPONENTWISE */
    int *n_out;        /* optional device int: the N used                      */
} oz2_problem;

OZ2_API int oz2_gemm_batched(int count, const oz2_problem *problems, const oz2_opts *opts);

/*
 * Tile autotuning for oz2_gemm_batched (the paper has no counterpart).  Each
 * problem's residue GEMMs run with 128 x 256 or 128 x 128 output tiles; the
 * results are identical either way (the products are exact), only the time
 * differs.  oz2_batched_autotune runs this batch (the inputs as given, on
 * opts->stream, with opts->workspace or the library's own) under each policy
 *   0  every problem 128 x 256
 *   1  every problem 128 x 128
 *   2  128 x 128 where n mod 256 is in [1, 128] (less padding), else 128 x 256
 *   3  per problem, the width that ran faster for that problem alone
 * with one warm-up and three timed calls each, and keeps the fastest for later
 * oz2_gemm_batched calls on problems with the same shapes and settings (C is
 * overwritten by the runs).  It synchronises the stream and must not be
 * captured into a graph.  *policy (optional): the policy kept; ms (optional,
 * float[4]): milliseconds per batched call under each policy.  Without a kept
 * policy a batch runs with policy 0.  Returns OZ2_OK, OZ2_EINVAL, OZ2_ENOMEM,
 * OZ2_ECUDA or a status of the runs.
 */
OZ2_API int oz2_batched_autotune(int count, const oz2_problem *problems, const oz2_opts *opts, int *policy,
                                 float *ms);

/* Keep policy 0, 1 or 2 (above) for batches with these shapes and settings,
 * without timing.  Returns OZ2_OK or OZ2_EINVAL. */
OZ2_API int oz2_batched_set_policy(int count, const oz2_problem *problems, int policy);

/*
 * C = OS_II(A, B) as oz2_gemm_ex / oz2_sgemm_ex, with A, B and C in host
 * memory (the problem as Section 3 states it: A in F_b^{m x k}, B in
 * F_b^{k x n}, the product in the same format).  On opts->stream, in this order: A and B are
 * copied into device memory (packed in their stored layout: A as (TRANS_A ?
 * k x m : m x k), B as (TRANS_B ? n x k : k x n)), the emulation runs, and C
 * is copied back into the host array (rows of n at stride ldc).  The device
 * memory is carved from opts->workspace, which must hold
 * oz2_host_workspace_size(...) bytes (NULL: the library-managed buffer, with
 * the serialisation rule of oz2_opts.workspace).  With pinned (page-locked)
 * host memory the call returns once everything is enqueued and C is valid when
 * the stream has completed (oz2_sync): calls on two streams with two
 * workspaces overlap one call's copies with the other's kernels.  With
 * pageable host memory the copies are staged by the CUDA runtime and the call
 * returns with C in place.  Any memory the CUDA runtime can address works as
 * the source and destination (device pointers too).  The other options
 * (n_out, mu/nu in/out, w_out, phase_events) are device pointers as in
 * oz2_gemm_ex.  Returns as oz2_gemm_ex, plus OZ2_ENOMEM for a workspace below
 * oz2_host_workspace_size.
 */
OZ2_API int oz2_gemm_host(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                          double *C, int ldc, int nmoduli, int mode, const oz2_opts *opts);
OZ2_API int oz2_sgemm_host(int m, int n, int k, const float *A, int lda, const float *B, int ldb,
                           float *C, int ldc, int nmoduli, int mode, const oz2_opts *opts);

/* Bytes of device workspace oz2_gemm_host (fp32 = 0) or oz2_sgemm_host
 * (fp32 = 1) needs: the packed device copies of A, B and C (each rounded up to
 * 256 bytes) followed by oz2_workspace_size(m, n, k, nmax, mode, fp32).
 * Returns 0 for invalid sizes.  Host-only. */
OZ2_API size_t oz2_host_workspace_size(int m, int n, int k, int nmax, int mode, int fp32);

/* Workspace bytes of oz2_gemm_batched for these problems (0 if any is invalid). */
OZ2_API size_t oz2_batched_workspace_size(int count, const oz2_problem *problems);

/* Bytes of device workspace a call with these sizes needs; nmax is the largest
 * N the call may use (its nmoduli, or opts->nmax when nmoduli == 0).  For
 * k > 2^17 the ranges run one after another in the same workspace (sized for
 * the longest range).  Returns 0 for invalid sizes.  Host-only; touches no GPU. */
OZ2_API size_t oz2_workspace_size(int m, int n, int k, int nmax, int mode, int fp32);

/* The split of K that oz2_gemm[_ex] and oz2_sgemm[_ex] use: *count ranges of
 * *kc consecutive k each (the last one k - (*count - 1) *kc), where S =
 * ceil(k / 2^17), *kc = 64 ceil(ceil(k / S) / 64) and *count = ceil(k / *kc)
 * <= S; k <= 2^17 gives one range of k.  Returns OZ2_OK or OZ2_EINVAL (k < 1
 * or a null pointer).  Host-only. */
OZ2_API int oz2_k_ranges(int k, int *count, int *kc);

/* Waits for `stream` and reports device-side status collected since the last
 * call: OZ2_ETIMEOUT if a kernel's bounded wait expired (the kernel then
 * stopped early and C is invalid), OZ2_ECUDA on a CUDA error, else OZ2_OK.
 * The status word is cleared. */
OZ2_API int oz2_sync(void *stream);

/* Host-only: the library's own constant tables for N moduli (Section 3.1,
 * Algorithm 2 first line, Algorithm 3), for tests.  fp32 = 0: DGEMM tables,
 * 1: SGEMM tables.  Fills s1[N], s2[N] (doubles), scal[6] = {P1, P2, Pinv, g,
 * t, gN} (g = grid of s_l1, 0 for SGEMM; t = 1/sqrt(32(P-1)) rounded up; gN =
 * the P-proportional part of R_b in Lemma 4, rounded up) and *pprime = P'.
 * Returns OZ2_OK or OZ2_EINVAL.  Touches no GPU. */
OZ2_API int oz2_tables(int N, int fp32, double *s1, double *s2, double *scal, float *pprime);

/* The constants of the two CRT sums of Algorithm 3 as integers on the grid
 * the device sums them on: s_l2 (fp32 == 0) or s_l1 (fp32 != 0) =
 * (k[2l+1] 2^31 + k[2l]) 2^(*esum), with 0 <= k[2l], k[2l+1] < 2^31, for
 * l = 0..N-1 (k: host int[2N]); the device holds the same integers as four
 * 16-bit pieces each.
 * Returns OZ2_OK, OZ2_EINVAL (N out of range or a null pointer) or
 * OZ2_ENOTSUP (some constant does not fit that form).  Touches no GPU. */
OZ2_API int oz2_sum_tables(int N, int fp32, int *k, int *esum);

/* Diagnostic for assumption (1) of Section 1.2 (|log2f(x) - log2 x| <=
 * 4 u32 log2 x, which Lemmas 0 and 1 rely on), for the __log2f used by the
 * exponent kernel: enqueues a check of every FP32 value that is an integer in
 * [1, 2^29] (the values Dbar can take).  dev_out: device uint64[2]; on
 * completion dev_out[0] = number of violations, dev_out[1] = bits of the
 * largest |__log2f(x) - log2 x| / (u32 log2 x) seen (a double). */
OZ2_API int oz2_check_log2f(void *stream, unsigned long long *dev_out);

/* Diagnostic for the device-side failure path: enqueues on `stream` one kernel
 * whose thread waits, with the loop and status reporting of the GEMM's
 * bounded waits, on an mbarrier that nothing arrives on, giving up after
 * limit_us microseconds (1 .. 10^6).  The kernel then returns normally and the
 * next oz2_sync on that stream reports OZ2_ETIMEOUT (and clears the status).
 * Returns OZ2_OK, OZ2_EINVAL or OZ2_ECUDA.  No GPU fault is involved. */
OZ2_API int oz2_wait_selftest(void *stream, unsigned int limit_us);

/* Diagnostic for the failure path of the residue GEMM (the paper has no
 * counterpart): the same call as oz2_gemm_ex (mode 0, 64 < k <= 2^17),
 * except that in the residue GEMM every CTA arms the mbarrier of the operand
 * stage of k-block 1 of its first tile but issues no copy for it.  The MMA
 * warp's wait on that stage gives up after limit_us microseconds (1 .. 10^6;
 * every wait of that launch uses this limit), the CTA stops its loops, waits
 * (again at most limit_us) for the copies and MMAs it had already issued, frees
 * its TMEM and returns.  The next oz2_sync on that stream reports OZ2_ETIMEOUT
 * and clears the status; C is invalid.  No GPU fault is involved, and later
 * calls run normally.  Returns as oz2_gemm_ex, or OZ2_EINVAL for a limit or k
 * out of range. */
OZ2_API int oz2_gemm_timeout_selftest(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                                      double *C, int ldc, int nmoduli, unsigned int limit_us,
                                      const oz2_opts *opts);

/* Size of the fixed device scratch used by oz2_gemm_noalloc (32 MiB). */
#define OZ2_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * oz2_gemm_noalloc: the same emulated DGEMM as oz2_gemm_ex, for callers that
 * cannot have any device memory allocated for them, e.g. an application that
 * owns all device memory through its own pool under a hard budget, or a
 * latency-critical loop that cannot afford cudaMalloc's implicit device-wide
 * synchronisation, and that cannot hand over a workspace either.  (The paper
 * has no counterpart; this is an interface convenience.)
 *   - Works in a fixed OZ2_NOALLOC_SCRATCH_BYTES array that this library
 *     places in the device memory of every GPU it is loaded on, held until the
 *     process exits.  Nothing is allocated or freed per call.
 *   - Problems whose workspace (oz2_workspace_size with nmax = nmoduli, or 20
 *     when nmoduli == 0) exceeds that size are rejected with OZ2_ENOMEM before
 *     anything is enqueued.  For 512^3 at N = 20 the workspace is 25 MiB.
 *   - nmoduli: N in [2, 49], or 0 for the bound rule with `target` and N <= 20.
 *   - The first call on a device looks up the array's device address; make that
 *     first call before any stream capture.
 *   - All calls share the one array, which keeps the previous call's contents
 *     (each call clears what must start at zero).  Calls whose work overlaps
 *     on the GPU (different streams, or different host threads) race on it:
 *     serialise them.
 * Other conventions as for oz2_gemm_ex (device pointers, row-major, `stream`
 * is a cudaStream_t or NULL for the legacy default stream).
 */
OZ2_API int oz2_gemm_noalloc(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                             double *C, int ldc, int nmoduli, int mode, double target, void *stream);

/* The last CUDA failure behind an OZ2_ECUDA: returns the cudaError_t value
 * (or 10000 + a CUresult of a driver call), 0 if none; *line (optional) gets
 * the library source line that caught it.  For diagnostics. */
OZ2_API int oz2_last_error(int *line);

/* The number of kernels this library has launched in this process so far (all
 * host threads, all devices; diagnostic kernels included).  For accounting:
 * the difference over a span of calls is the number of kernels they enqueued
 * (a call's count depends on its sizes: small problems merge some phases into
 * one launch).  Not part of the paper's method. */
OZ2_API long long oz2_launch_count(void);

/* Human-readable name of a status code (static string). */
OZ2_API const char *oz2_status_str(int status);

/* Library version, major*10000 + minor*100 + patch. */
OZ2_API int oz2_version(void);

#ifdef __cplusplus
}
#endif

#endif /* OZ2_H */
