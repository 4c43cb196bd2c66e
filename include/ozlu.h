/*
 * ozlu.h -- C ABI of the GB300 Ozaki-scheme-II multiple-precision GEMM and LU.
 *
 * The operations follow T. Kouya, "Accelerating Multiple-Precision LU
 * Decomposition with Ozaki Scheme II":
 *   ozlu_gemm   the Ozaki-II GEMM, steps (S1)-(S6) of Sec. 3.1, with the
 *               slice splitting and per-digit-group CRT of Sec. 3.2 (Eqs. (2),
 *               (3), (8), (11)) and the direct expansion conversion of
 *               Sec. 3.3 (Eq. (12));
 *   ozlu_getrf  the blocked right-looking LU with partial pivoting of
 *               Sec. 3.4, (P1)-(P4), whose trailing update Eq. (13),
 *               A22 <- A22 - L21 U12, is an ozlu_gemm;
 *   ozlu_getrs  the forward and backward substitution used in Sec. 4.4.
 *
 * Number format.  A multiple-precision element is a non-overlapping
 * expansion of nc = 2, 3 or 4 binary64 components (DD, TD, QD; Sec. 2.1),
 * stored as nc contiguous doubles, largest first.  Matrices are column-major:
 * element (i, j) of a matrix with leading dimension ld starts at
 * base + (i + j * ld) * nc doubles.  p is the target precision in bits
 * (0 means 53 * nc).
 *
 * Memory.  Matrix, pivot and info pointers may be device pointers or host
 * pointers (pageable or pinned).  Host arguments are copied to a device
 * workspace and back inside the call, on the handle's stream, and the call
 * then waits for the stream; device arguments are used in place and the call
 * returns without waiting (stream ordered).  The caller owns every argument
 * buffer.  The handle owns its workspace (residue planes, CRT inputs, plan
 * tables), grown on demand and released by ozlu_destroy.
 *
 * Errors.  0 on success.  -i: argument i (1-based, handle = 1) is invalid.
 * Positive: one of the OZLU_ERR_* codes.  A handle is not thread safe; use one
 * handle per host thread.
 */
#ifndef OZLU_H
#define OZLU_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ozlu_handle ozlu_handle;

enum {
    OZLU_OK = 0,
    OZLU_ERR_CUDA = 1001,      /* a CUDA runtime call failed                     */
    OZLU_ERR_NOMEM = 1002,     /* device workspace could not be allocated        */
    OZLU_ERR_CAPACITY = 1003,  /* p, K or the format is beyond what a plan holds */
    OZLU_ERR_TIMEOUT = 1004,   /* a bounded device wait gave up                  */
    OZLU_ERR_UNSUPPORTED = 1005 /* back-end not available in this build/device   */
};

/* Residue back-ends of (S4) (Sec. 3.5, Table backend_origin). */
enum {
    OZLU_BE_AUTO = 0, /* measured choice per shape: each feasible back-end is timed on
                         the first call of a shape (the call then waits for the
                         stream) and the fastest is cached in the handle          */
    OZLU_BE_INT8 = 1, /* centered residues in int8, exact int32 accumulation          */
    OZLU_BE_FP8 = 2,  /* balanced base-17 digits in E4M3, Eq. (15), fp32 accumulation */
    OZLU_BE_FP64 = 3, /* residues of ~23-bit primes in binary64, Eq. (17)             */
    OZLU_BE_FP16 = 4  /* centered residues in binary16, fp32 accumulation, Eq. (14)   */
};

/* Options; an all-zero struct (or NULL) selects the defaults. */
typedef struct {
    int backend;      /* OZLU_BE_*                                                 */
    int nslice;       /* S override (Sec. 3.2); 0 = smallest feasible S            */
    int extra_groups; /* digit groups kept below S-1 (Sec. 3.2, cancellation)      */
    int g_ex;         /* extra guard bits in the slack of Sec. 3.2                 */
    int native;       /* ozlu_getrf only: 1 = trailing update (P4) by per-element
                         multiply-adds in expansion arithmetic, the "blocked naive"
                         comparison of Sec. 3.4 (panels unchanged); 2 = the
                         "unblocked naive" LU of Sec. 3.4 (b = 1: pivot, scale
                         and a rank-1 update of the whole trailing matrix in
                         expansion arithmetic for every column; nb is ignored) */
    int graph;        /* ozlu_getrf/ozlu_getrs (device pointers) and the batched
                         calls: 1 = capture the call's work in a CUDA graph on the
                         second call with the same sizes and pointers and replay it
                         from then on (no host synchronisation inside the call; a
                         bounded-wait timeout shows in info, see the batched LU) */
    int panel_width;  /* ozlu_getrf: widest base block of the cooperative panel kernel
                         (32, 64 or 128; 0 = chosen from the rows per thread block) */
    int modset;       /* p-bit calls (ozlu_mp_set_opts): OZLU_MODSET_INT8 = the 54
                         moduli <= 255 with slice splitting (Sec. 3.2),
                         OZLU_MODSET_EXT = the extended table of 1882 moduli
                         <= 16191 (Sec. 4.2.4), three int8 planes per modulus */
    int reserved[8];
} ozlu_opts;

/* Modulus tables of the p-bit Ozaki-II GEMM (ozlu_opts.modset). */
enum { OZLU_MODSET_INT8 = 0, OZLU_MODSET_EXT = 1 };

/* Plan of one Ozaki-II GEMM (Sec. 3.2 "Determining w and N"). */
typedef struct {
    int p, K, backend, S, w, Q, n_mod, g0, n_groups, pair_terms;
    int moduli[64];   /* m_1 > m_2 > ... (descending), n_mod entries */
} ozlu_plan_info;

/* Create a handle bound to a CUDA stream (cudaStream_t passed as void*; NULL =
 * the default stream).  The current device at creation is the handle's
 * device.  Calls may fork independent kernels onto a second stream the handle
 * owns (made on the first call outside a graph capture) and join it back into
 * the handle's stream before they return, so the work stays ordered on the
 * handle's stream.  Returns OZLU_ERR_CUDA when no device is usable. */
int ozlu_create(ozlu_handle** handle, void* stream);
/* Release the workspace and the handle.  NULL is accepted. */
int ozlu_destroy(ozlu_handle* handle);
int ozlu_set_stream(ozlu_handle* handle, void* stream);

/* The plan ozlu_gemm uses for precision p, inner dimension k and options. */
int ozlu_plan(int p, int k, const ozlu_opts* opts, ozlu_plan_info* out);

/*
 * C = beta * C + alpha * A * B  (Sec. 3.1, (S1)-(S6)).
 *   nc      2, 3 or 4;  p in [1, 53*nc] (0 = 53*nc)
 *   m, n, k >= 0 (k = 0 or m = 0 or n = 0: C is scaled by beta only)
 *   alpha   +1 or -1;  beta 0 or 1
 *   A       m x k expansions, lda >= max(1, m)
 *   B       k x n expansions, ldb >= max(1, k)
 *   C       m x n expansions, ldc >= max(1, m); not aliased with A or B
 * Result: one rounding per element (S6): the exact integer of the retained
 * digit groups, scaled by 2^-(mu_i + nu_j), plus beta * C brought to the same
 * grid, rounded component by component to nc doubles.
 */
int ozlu_gemm(ozlu_handle* handle, int nc, int p, int m, int n, int k, int alpha,
              const double* A, long long lda, const double* B, long long ldb,
              int beta, double* C, long long ldc, const ozlu_opts* opts);

/*
 * Blocked LU with partial pivoting, P A = L U (Sec. 3.4, (P1)-(P4)).
 *   A      n x n expansions, overwritten by L (unit, strictly below) and U
 *   ipiv   n ints: row i was interchanged with row ipiv[i] (1-based, LAPACK)
 *   nb     panel width b; 0 = measured choice among 64, 128, 256 and 512 (not
 *          above n) on the first call for a size class (nc, p, log2 n,
 *          back-end): the candidates factor a scratch copy of A and the
 *          fastest is cached in the handle (ozlu_stats.tuned_nb)
 *   info   one int: 0, or the 1-based column of the first exactly zero pivot
 *          (the factorisation continues, as in LAPACK)
 * Panels (P1)-(P3) run in error-free expansion arithmetic; the trailing
 * update (P4) is ozlu_gemm with alpha = -1, beta = 1.
 */
int ozlu_getrf(ozlu_handle* handle, int nc, int p, int n, double* A, long long lda,
               int* ipiv, int nb, int* info, const ozlu_opts* opts);

/*
 * Solve A X = B from ozlu_getrf's factors (P b, forward L, backward U).
 *   LU, ipiv  as returned by ozlu_getrf;  B n x nrhs, overwritten by X.
 */
int ozlu_getrs(ozlu_handle* handle, int nc, int p, int n, int nrhs,
               const double* LU, long long lda, const int* ipiv,
               double* B, long long ldb, const ozlu_opts* opts);

/*
 * Batched LU of `count` independent instances of different sizes (the
 * batched, uneven workload; each instance is the LU of Sec. 3.4).
 *   n, A, lda, ipiv   host arrays of length count; A[i] (n[i] x n[i] expansions,
 *                     column-major, lda[i]) and ipiv[i] (n[i] ints) are device
 *                     pointers, factored in place as by ozlu_getrf
 *   info              device array of count ints: LAPACK info per instance (0, or
 *                     the 1-based column of the first exactly zero pivot), or
 *                     -OZLU_ERR_TIMEOUT when a bounded device wait gave up
 *   nb                panel width (0 = the measured choice of ozlu_getrf for
 *                     each instance's size class, made on the first call)
 * Instances run on up to 32 streams owned by the handle (joined back into the
 * handle's stream before return; the call does not wait for the GPU).  With
 * opts->graph the batch is captured into a CUDA graph on the second call with
 * the same sizes and pointers and replayed afterwards; the first call warms the
 * workspaces and the back-end autotuner.
 */
int ozlu_getrf_batched(ozlu_handle* handle, int nc, int p, int count, const int* n,
                       double* const* A, const long long* lda, int* const* ipiv, int* info,
                       int nb, const ozlu_opts* opts);

/*
 * Batched solve A_i X_i = B_i from ozlu_getrf_batched's factors; B[i] is
 * n[i] x nrhs (device, ldb[i]), overwritten by X_i.  Streams and graphs as
 * for ozlu_getrf_batched.
 */
int ozlu_getrs_batched(ozlu_handle* handle, int nc, int p, int count, const int* n, int nrhs,
                       const double* const* LU, const long long* lda, const int* const* ipiv,
                       double* const* B, const long long* ldb, const ozlu_opts* opts);

/*
 * Intermediates of the last ozlu_gemm on this handle, copied to host memory
 * for parity checks against a reference (the workspace keeps them until the
 * next call).  what:
 *   1 mu  (m int32)        2 nu (n int32)
 *   3 residues of A  int8 [l][t][i][h], h < k, planes (l, t) in order
 *   4 residues of B  int8 [l][t][j][h]
 *   5 t values      uint8 [gi][l][j][i] (column-major m x n per plane);
 *                   uint32 for the binary64 back-end
 *   6 device error word (int32): 0, or OZLU_ERR_TIMEOUT when a bounded
 *     wait inside a tensor-core GEMM gave up since the start of the last
 *     ozlu_gemm, ozlu_getrf or ozlu_getrs call on this handle
 * Residues (3, 4) are available for the INT8 back-end only.
 * bytes must be at least the size of the requested array.
 */
int ozlu_debug_fetch(ozlu_handle* handle, int what, void* dst, size_t bytes);

/* Counters since the last ozlu_set_timing call.  With timing enabled the
 * library records CUDA events around each phase on the handle's stream
 * (no host synchronisation until ozlu_get_stats resolves them):
 *   convert_ms  (S1)-(S3) exponents, conversion and residues
 *   gemm_ms     (S4) residue GEMMs with the modular epilogue
 *   crt_ms      (S5)-(S6) CRT, recombination and rounding
 *   panel_ms    (P1) base-block panel kernels of the LU
 *   trsm_ms     (P3) and getrs base triangular-solve kernels
 *   other_ms    row interchanges (P2)
 * launches counts every kernel the library launched; gemm_ops, crt_bytes and
 * convert_bytes are the algorithmic work of those phases (tensor operations
 * 2 M N K per residue product, and the bytes each phase must move). */
typedef struct {
    double convert_ms, gemm_ms, crt_ms, panel_ms, other_ms;
    long long gemm_launches, crt_launches, panel_launches, launches;
    double gemm_ops, crt_bytes, convert_bytes;
    int last_backend;  /* back-end of the last residue GEMM (after autotuning) */
    int graph_status;  /* last batched call with opts->graph: 0 ran eagerly (first
                          call), 1 captured and launched a graph, 2 replayed one,
                          -e capture or instantiation failed with cudaError_t e
                          (the batch then runs eagerly on every call)        */
    double trsm_ms;
    int last_nslice;   /* slice count S of the last residue GEMM (after autotuning) */
    int tuned_nb;      /* panel width the last ozlu_getrf with nb = 0 used     */
} ozlu_stats;
int ozlu_set_timing(ozlu_handle* handle, int enable);
int ozlu_get_stats(ozlu_handle* handle, ozlu_stats* out);

/*
 * C = beta * C + alpha * A * B like ozlu_gemm with backend OZLU_BE_INT8, for
 * callers that must not allocate (the paper has no counterpart: this is an
 * interface of this library).  A host that has given nearly all device memory
 * to its own pool allocator, or a latency-critical caller that cannot afford
 * the synchronisation a cudaMalloc may imply, can call it: it takes no
 * handle and allocates neither device nor host memory.
 *   Arguments as ozlu_gemm (without handle and options), plus the stream
 *   (cudaStream_t as void*, NULL = default stream); A, B, C must be device
 *   pointers of the current device (a host pointer, or one into another
 *   GPU's memory, is rejected as an invalid argument), k >= 1.
 *   Scratch: one fixed 16 MiB device array inside the library, held by every
 *   GPU that loads it until the process exits.  Problems whose intermediates
 *   do not fit (for QD, m = n = k = 256 fits; 384 does not) return
 *   OZLU_ERR_CAPACITY.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and caches it; make that
 *   first call before any stream capture.
 *   All calls share the array: calls that overlap on the GPU (other streams,
 *   other host threads) race and must be serialised by the caller.  Nothing
 *   needs clearing between calls: each call writes the exponents, the residue
 *   rows of A and B with their zero K padding, and the t values before it
 *   reads them; the padding rows of the residue planes (beyond m and n, up to
 *   the next multiple of 128) may keep bytes of an earlier call, and those
 *   only reach output tiles outside m x n, which are discarded.
 * Returns 0, -i for invalid argument i (nc = 1), or an OZLU_ERR_* code; the
 * work is stream ordered (the call does not wait for it).
 */
int ozlu_gemm_noalloc(int nc, int p, int m, int n, int k, int alpha, const double* A,
                      long long lda, const double* B, long long ldb, int beta, double* C,
                      long long ldc, void* stream);

/*
 * p-bit multi-limb matrices (the arbitrary-precision LU of Sec. 3.4 / 4.4,
 * where the paper uses MPFR numbers).  Element (i, j) has a sign, an
 * exponent and L 32-bit limbs of a magnitude normalised to its top bit:
 *   value = (-1)^signs[x] * (sum_k limbs[k * plane + x] 2^(32 k)) * 2^(exps[x] - 32 L),
 *   x = i + j * ld,
 * so 2^(exps - 1) <= |value| < 2^exps; zero has all limbs 0 (exponent and
 * sign 0).  Limb-major planes keep one limb of consecutive elements
 * contiguous.  All three arrays are device memory owned by the caller; a
 * submatrix is the same struct with the three pointers advanced by x.
 * Results are rounded to p bits (round to nearest even), p <= 32 L.
 */
typedef struct {
    unsigned int* limbs;
    int* exps;
    int* signs;
    long long ld;     /* elements between columns, >= rows          */
    long long plane;  /* elements between limb planes, >= ld * cols */
    int L;            /* limbs per element                          */
    int pad_;
} ozlu_mp_matrix;

/*
 * C = beta * C + alpha * A * B on p-bit matrices by the Ozaki-II GEMM with
 * INT8 residues (Sec. 3.1 (S1)-(S6) with p-bit significands in place of the
 * expansions: S1 shared exponents, S2 trunc(a 2^mu) and S balanced digits,
 * S3-S5 as for ozlu_gemm, S6 one rounding to p bits of beta C + alpha P_int
 * with the old C truncated onto the product grid).
 *   p >= 1; m, n >= 0; k >= 1; alpha +1 or -1; beta 0 or 1; C not aliased
 *   with A or B; every matrix's L with 32 L >= p.
 * The output is split into column chunks so that the t values of one chunk
 * stay below 4 GiB.  Returns 0, -i for invalid argument i, or an OZLU_ERR_*
 * code (OZLU_ERR_CAPACITY when no plan exists for p and k).
 */
int ozlu_mp_gemm(ozlu_handle* handle, int p, int m, int n, int k, int alpha, const ozlu_mp_matrix* A,
                 const ozlu_mp_matrix* B, int beta, const ozlu_mp_matrix* C);

/*
 * LU with partial pivoting of an n x n p-bit matrix in place (Sec. 3.4): the
 * recursive panel and triangular solves reduce to Ozaki-II GEMMs; a column
 * of the panel takes a pivot search (largest |a|, lowest row on ties), a
 * row interchange, and its scaling by the reciprocal of the pivot (Newton's
 * iteration in fixed point by one thread block).  ipiv (device, n ints,
 * 1-based) and info (device int: 0, or the first exactly zero pivot) as in
 * ozlu_getrf; nb = 0 picks 128.
 */
int ozlu_mp_getrf(ozlu_handle* handle, int p, int n, const ozlu_mp_matrix* A, int* ipiv, int nb,
                  int* info);

/*
 * The plan ozlu_mp_gemm uses for precision p and inner dimension k (Sec. 3.2
 * "Determining w and N" with the 54 INT8 moduli: the smallest S whose width
 * w = ceil((p + slack) / S) the moduli cover, within the INT32 accumulator
 * bound).  Host only, no device work.  Returns 0, -i for invalid argument i,
 * or OZLU_ERR_CAPACITY when no S satisfies both.
 */
int ozlu_mp_plan(int p, int k, ozlu_plan_info* out);

/*
 * Options of the handle's p-bit calls (ozlu_mp_gemm, ozlu_mp_getrf,
 * ozlu_mp_getrs); NULL restores the defaults.  Used fields:
 *   modset  OZLU_MODSET_INT8 (default): the 54 moduli <= 255, the smallest S
 *           with enough capacity; OZLU_MODSET_EXT: the extended table of
 *           Sec. 4.2.4 (moduli up to 16191, residues split into base-128
 *           digits r = 128 q + r0 and multiplied as the three int8 planes
 *           r0, q, r0 + q by Karatsuba), which needs far fewer GEMMs per
 *           product (about 2x per doubling of p instead of 3x) at the cost of
 *           O(p^2) conversion and CRT work per element
 *   nslice  the slice count S for OZLU_MODSET_EXT (0 = the smallest feasible)
 *   backend residue GEMMs of the 54-modulus table for products with more than
 *           16 columns and 8 inner indices: OZLU_BE_AUTO (default; measured
 *           per shape class on the first call, the call then waits for the
 *           stream), OZLU_BE_INT8 (mma.sync) or OZLU_BE_FP8 (balanced base-17
 *           digits on tcgen05, Eq. (15), when K_pad S 15^2 < 2^24); both run the
 *           same plan, so the results are identical; narrower products use the
 *           integer pipe (K <= 8) or INT8
 * Returns 0, -1 for a NULL handle, -2 for an unknown modset or backend or
 * nslice < 0.
 */
int ozlu_mp_set_opts(ozlu_handle* handle, const ozlu_opts* opts);

/*
 * The plan ozlu_mp_gemm uses with the given options (modset, nslice) for
 * precision p and inner dimension k; host only.  moduli[] lists the first 64.
 */
int ozlu_mp_plan_opts(int p, int k, const ozlu_opts* opts, ozlu_plan_info* out);

/* Solve A X = B from ozlu_mp_getrf's factors; B is n x nrhs (p-bit), overwritten. */
int ozlu_mp_getrs(ozlu_handle* handle, int p, int n, int nrhs, const ozlu_mp_matrix* LU, const int* ipiv,
                  const ozlu_mp_matrix* B);

/*
 * Test hooks for failure handling (no counterpart in the paper).  Neither
 * faults the GPU: the failures are made on the host or by a wait that runs
 * out on a flag nothing sets.
 *
 * ozlu_debug_fail_alloc: the next `count` device allocations the library
 * makes (handle workspaces and scratch) fail as if cudaMalloc had failed, so
 * the calls that needed them return OZLU_ERR_NOMEM; 0 turns it off.  The
 * counter is process-wide.  Returns 0, or -1 for count < 0.
 *
 * ozlu_debug_wait_expiry: runs one of the library's bounded device waits on
 * the handle's stream with a short limit, on a flag or barrier that nothing
 * sets, and then the LU's finish step that turns the error word into info:
 *   which 1  the panel kernel's stamp wait (limit in ns of the global timer);
 *            its error word is the panel scratch of the handle
 *   which 2  the tensor-core GEMM's mbarrier wait (limit in polls of ~0.1 us);
 *            its error word is the handle's (ozlu_debug_fetch what = 6)
 * out (host, 3 ints): 1 if the wait gave up, the error word after it
 * (OZLU_ERR_TIMEOUT), and the info the finish step wrote (-OZLU_ERR_TIMEOUT).
 * Waits for the stream.  Returns OZLU_ERR_TIMEOUT when the wait gave up (as
 * ozlu_getrf does with host arguments), 0 if it did not, -i for an invalid
 * argument i, or OZLU_ERR_CUDA / OZLU_ERR_NOMEM.  The next ozlu_gemm,
 * ozlu_getrf or ozlu_getrs call clears both error words.
 */
int ozlu_debug_fail_alloc(int count);
int ozlu_debug_wait_expiry(ozlu_handle* handle, int which, long long limit, int* out);

/* Version string of the library. */
const char* ozlu_version(void);

#ifdef __cplusplus
}
#endif
#endif /* OZLU_H */
