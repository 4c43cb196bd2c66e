// Blocked right-looking LU with partial pivoting and the solve (Sec. 3.4).
//
//   for each panel of width nb:
//     (P1) factor the n - r0 by nb panel: recursive halving down to base
//          blocks of BASE columns; a base block is factored column by column
//          in expansion arithmetic (pivot search, interchange across the
//          panel, scaling, rank-1 update of the base block); between halves
//          U12 = L11^-1 A12 by a recursive triangular solve and
//          A22 -= L21 U12 by the Ozaki-II GEMM;
//     (P2) apply the interchanges to the columns left and right of the panel;
//     (P3) U12 = L11^-1 A12, recursive triangular solve;
//     (P4) A22 <- A22 - L21 U12 (Eq. (13)) by the Ozaki-II GEMM.
// Only (P4) is the update the paper moves to Ozaki scheme II; the recursion
// puts the larger part of (P1) and (P3) on the same GEMM as well, leaving
// O(n^2 BASE) operations in FP64 expansion arithmetic (the GB300 FP64 rate is
// about 1 TFLOP/s).  getrs: interchanges, then blocked forward (unit L) and
// backward (U) substitution with base triangles in expansion arithmetic and
// the off-diagonal updates by the Ozaki-II GEMM.
#include <string.h>

#include <tuple>

#include "expansion.cuh"
#include "mpf.cuh"
#include "ozlu_handle.h"

namespace ozlu {
namespace {

constexpr int BASE = 32;        // triangular-solve leaves and the fallback panel path
constexpr int PBASE = 128;      // widest base block of the cooperative panel kernel
constexpr int PIV_THREADS = 256;
constexpr int PIV_BLOCKS = 152;
constexpr int MAXPART = 1024;   // block partials of a column step
constexpr int STEP_ROWS = 16;   // rows per block of a column step
constexpr int LCT = 4;          // laswp: columns per block
constexpr int LHASH = 2048;     // laswp: hash slots (>= 2 x affected rows)
constexpr int LMAXB = 512;      // laswp: interchanges per call
constexpr int TRI_SLOTS = 8;    // triangles of base solves converted ahead (256 / BASE)

// limbs of the panel arithmetic: 32 L >= 53 nc + 12 (DD 4, TD 6, QD 7)
template <int N>
struct Limbs { static constexpr int L = N == 2 ? 4 : (N == 3 ? 6 : 7); };

struct LuScratch {
    uint32_t rm[8];             // reciprocal of the current pivot (MPF words)
    int re, rneg;
    int piv;
    int zero;
    unsigned int counter;
    int info;
    int result;                 // info as reported by ozlu_getrf (finish_kernel)
    double pval[MAXPART][4];    // block candidates (expansion values)
    int pidx[MAXPART];
    int plist[1 + 4 * LMAXB];   // interchange permutation: count, (dst, src) pairs
    // triangles of base triangular solves as L-limb floats: [k][i], then the
    // reciprocal diagonal (upper case); slot q holds the q-th diagonal block of
    // a unit lower triangle converted ahead of its recursion
    unsigned char tri[TRI_SLOTS][(BASE * BASE + BASE) * sizeof(MPF<8>)];
};

template <int L>
__device__ __forceinline__ void put_recip(LuScratch* sc, const MPF<L>& r) {
#pragma unroll
    for (int i = 0; i < L; ++i) sc->rm[i] = r.m[i];
    sc->re = r.e;
    sc->rneg = r.neg;
}

template <int L>
__device__ __forceinline__ MPF<L> get_recip(const LuScratch* sc) {
    MPF<L> r;
#pragma unroll
    for (int i = 0; i < L; ++i) r.m[i] = sc->rm[i];
    r.e = sc->re;
    r.neg = sc->rneg;
    return r;
}

__device__ __forceinline__ double* elem(double* A, long long lda, int nc, long long i, long long j) {
    return A + (i + j * lda) * nc;
}

// better(a, ia, b, ib): |a| > |b|, or equal and ia < ib (first index on ties)
template <int N>
__device__ __forceinline__ bool better(const Exp<N>& a, int ia, const Exp<N>& b, int ib) {
    if (ib < 0) return ia >= 0;
    if (ia < 0) return false;
    const int c = abs_cmp<N>(a, b);
    return c > 0 || (c == 0 && ia < ib);
}

// Last-block reduction of the block candidates: each thread scans a strided
// share of the partials, then a shared-memory tree keeps the best (largest
// magnitude, first index on ties).  All threads of the block must call it;
// the result is valid in thread 0.
template <int N, int THREADS>
__device__ __forceinline__ void reduce_partials(const LuScratch* sc, int nparts, Exp<N>& b, int& ib) {
    __shared__ double rv[THREADS][N];
    __shared__ int ri[THREADS];
    Exp<N> best;
    int bi = -1;
#pragma unroll
    for (int q = 0; q < N; ++q) best.x[q] = 0.0;
    for (int k = threadIdx.x; k < nparts; k += THREADS) {
        Exp<N> v;
#pragma unroll
        for (int q = 0; q < N; ++q) v.x[q] = ((volatile const double*)sc->pval[k])[q];
        const int iv = ((volatile const int*)sc->pidx)[k];
        if (better<N>(v, iv, best, bi)) { best = v; bi = iv; }
    }
#pragma unroll
    for (int q = 0; q < N; ++q) rv[threadIdx.x][q] = best.x[q];
    ri[threadIdx.x] = bi;
    __syncthreads();
    for (int s = THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            Exp<N> u, v;
#pragma unroll
            for (int q = 0; q < N; ++q) { u.x[q] = rv[threadIdx.x][q]; v.x[q] = rv[threadIdx.x + s][q]; }
            if (better<N>(v, ri[threadIdx.x + s], u, ri[threadIdx.x])) {
#pragma unroll
                for (int q = 0; q < N; ++q) rv[threadIdx.x][q] = v.x[q];
                ri[threadIdx.x] = ri[threadIdx.x + s];
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < N; ++q) b.x[q] = rv[0][q];
    ib = ri[0];
}

// Pivot search of column c over rows [c, n); the last block to finish reduces
// the block results, interchanges rows c and piv over columns [p0, p1),
// records ipiv[c] (1-based) and the reciprocal of the pivot.
template <int N>
__global__ void __launch_bounds__(PIV_THREADS) pivot_kernel(double* A, long long lda, int n, int c,
                                                            int p0, int p1, int* ipiv,
                                                            LuScratch* sc) {
    __shared__ double sv[PIV_THREADS][N];
    __shared__ int si[PIV_THREADS];
    __shared__ bool last;
    Exp<N> best;
    int bi = -1;
#pragma unroll
    for (int q = 0; q < N; ++q) best.x[q] = 0.0;
    for (int i = c + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        Exp<N> v = load<N>(elem(A, lda, N, i, c));
        if (better<N>(v, i, best, bi)) { best = v; bi = i; }
    }
#pragma unroll
    for (int q = 0; q < N; ++q) sv[threadIdx.x][q] = best.x[q];
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int s = PIV_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            Exp<N> a, b;
#pragma unroll
            for (int q = 0; q < N; ++q) { a.x[q] = sv[threadIdx.x][q]; b.x[q] = sv[threadIdx.x + s][q]; }
            if (better<N>(b, si[threadIdx.x + s], a, si[threadIdx.x])) {
#pragma unroll
                for (int q = 0; q < N; ++q) sv[threadIdx.x][q] = b.x[q];
                si[threadIdx.x] = si[threadIdx.x + s];
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) sc->pval[blockIdx.x][q] = sv[0][q];
        sc->pidx[blockIdx.x] = si[0];
        __threadfence();
        const unsigned int done = atomicAdd(&sc->counter, 1u);
        last = done == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ int piv;
    Exp<N> b;
    int ib;
    reduce_partials<N, PIV_THREADS>(sc, gridDim.x, b, ib);
    if (threadIdx.x == 0) {
        if (ib < 0) ib = c;
        piv = ib;
        sc->piv = ib;
        ipiv[c] = ib + 1;
        sc->counter = 0;
        const bool zero = b.x[0] == 0.0;
        sc->zero = zero ? 1 : 0;
        if (zero && sc->info == 0) sc->info = c + 1;
        if (!zero) {
            constexpr int L = Limbs<N>::L;
            put_recip<L>(sc, mpf_recip<L>(mpf_from_exp<L, N>(b.x)));
        }
    }
    __syncthreads();
    const int pv = piv;
    if (pv != c) {
        for (int j = p0 + threadIdx.x; j < p1; j += blockDim.x) {
            double* a = elem(A, lda, N, c, j);
            double* b = elem(A, lda, N, pv, j);
#pragma unroll
            for (int q = 0; q < N; ++q) { const double t = a[q]; a[q] = b[q]; b[q] = t; }
        }
    }
}

// One column step of a base block, fused with the next pivot search.
// Rows i in (c, n): l_i = a_ic * (1 / pivot), a_ik -= l_i a_ck for k in (c, c1),
// all in L-limb integer floating point; each block then offers its best
// candidate for column c + 1 and the last block to finish reduces them,
// interchanges rows c + 1 and piv over the outer panel columns [p0, p1),
// records ipiv and the reciprocal of the new pivot.
template <int N>
__global__ void __launch_bounds__(128) column_step_kernel(double* A, long long lda, int n, int c,
                                                          int c1, int p0, int p1, int* ipiv,
                                                          LuScratch* sc) {
    constexpr int L = Limbs<N>::L;
    __shared__ MPF<L> urow[BASE];
    __shared__ MPF<L> lrow[STEP_ROWS];
    __shared__ double cand[STEP_ROWS][N];
    __shared__ int candi[STEP_ROWS];
    __shared__ bool last;
    __shared__ int piv;
    const int cols = c1 - c - 1;
    const bool zero = sc->zero != 0;
    for (int k = threadIdx.x; k < cols; k += blockDim.x)
        urow[k] = mpf_from_exp<L, N>(elem(A, lda, N, c, c + 1 + k));
    // candidate of this thread (threads < STEP_ROWS) over its rows of all chunks
    Exp<N> best;
    int bi = -1;
#pragma unroll
    for (int q = 0; q < N; ++q) best.x[q] = 0.0;
    const int nchunks = (n - c - 1 + STEP_ROWS - 1) / STEP_ROWS;
    for (int chunk = blockIdx.x; chunk < nchunks; chunk += gridDim.x) {
        const int i0 = c + 1 + chunk * STEP_ROWS;
        __syncthreads();
        if (threadIdx.x < STEP_ROWS) {
            const int i = i0 + threadIdx.x;
            if (i < n && !zero) {
                double* ai = elem(A, lda, N, i, c);
                MPF<L> l = mpf_mul<L>(mpf_from_exp<L, N>(ai), get_recip<L>(sc));
                mpf_to_exp<L, N>(l, ai);
                lrow[threadIdx.x] = l;
            }
        }
        __syncthreads();
        if (!zero) {
            for (int pidx = threadIdx.x; pidx < STEP_ROWS * cols; pidx += blockDim.x) {
                const int k = pidx / STEP_ROWS, rr = pidx - k * STEP_ROWS;
                const int i = i0 + rr;
                if (i >= n) continue;
                double* a = elem(A, lda, N, i, c + 1 + k);
                mpf_to_exp<L, N>(mpf_fms<L>(mpf_from_exp<L, N>(a), lrow[rr], urow[k]), a);
            }
        }
        if (cols > 0) {
            __syncthreads();
            if (threadIdx.x < STEP_ROWS) {
                const int i = i0 + threadIdx.x;
                if (i < n) {
                    const Exp<N> v = load<N>(elem(A, lda, N, i, c + 1));
                    if (better<N>(v, i, best, bi)) { best = v; bi = i; }
                }
            }
        }
    }
    if (cols == 0) return;  // last column of the base block: no next pivot here
    if (threadIdx.x < STEP_ROWS) {
#pragma unroll
        for (int q = 0; q < N; ++q) cand[threadIdx.x][q] = best.x[q];
        candi[threadIdx.x] = bi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Exp<N> b;
        int ib = -1;
#pragma unroll
        for (int q = 0; q < N; ++q) b.x[q] = 0.0;
        for (int r = 0; r < STEP_ROWS; ++r) {
            Exp<N> v;
#pragma unroll
            for (int q = 0; q < N; ++q) v.x[q] = cand[r][q];
            if (better<N>(v, candi[r], b, ib)) { b = v; ib = candi[r]; }
        }
#pragma unroll
        for (int q = 0; q < N; ++q) sc->pval[blockIdx.x][q] = b.x[q];
        sc->pidx[blockIdx.x] = ib;
        __threadfence();
        const unsigned int done = atomicAdd(&sc->counter, 1u);
        last = done == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int cn = c + 1;
    Exp<N> b;
    int ib;
    reduce_partials<N, 128>(sc, gridDim.x, b, ib);
    if (threadIdx.x == 0) {
        if (ib < 0) ib = cn;
        piv = ib;
        ipiv[cn] = ib + 1;
        sc->counter = 0;
        const bool z = b.x[0] == 0.0;
        sc->zero = z ? 1 : 0;
        if (z && sc->info == 0) sc->info = cn + 1;
        if (!z) put_recip<L>(sc, mpf_recip<L>(mpf_from_exp<L, N>(b.x)));
    }
    __syncthreads();
    const int pv = piv;
    if (pv != cn) {
        for (int j = p0 + threadIdx.x; j < p1; j += blockDim.x) {
            double* a = elem(A, lda, N, cn, j);
            double* b = elem(A, lda, N, pv, j);
#pragma unroll
            for (int q = 0; q < N; ++q) { const double t = a[q]; a[q] = b[q]; b[q] = t; }
        }
    }
}

// ---------------------------------------------------------------------------
// Cooperative factorisation of one base block: columns [c0, c0 + b) over rows
// [c0, n).  One block per SM owns a contiguous slice of rows and keeps its
// b-column slice in shared memory as L-limb floats for the whole block.  A
// column step needs one exchange: each block publishes its best candidate row
// for the column (its index and the whole row) in its slot, then one 64-bit
// word holding the column number and an ordering key of the candidate; every
// block waits for all G stamp words (one load each when they are there),
// reduces the same keys to the same pivot, takes the pivot row from the
// winner's slot, swaps it into place among its rows, scales and updates.
// The exchange overlaps the trailing update: a block first updates only the
// rows the next step needs from it (its next candidate and the row that the
// pivot will replace), publishes them, and only then updates the rest of its
// rows; meanwhile one thread forms the reciprocal of its candidate and
// publishes it under a second stamp, which the other blocks wait for (from
// the winner only) when they need the multipliers.  Waiting on the stamps
// replaces a grid barrier, and the slots are double-buffered by column
// parity: a block can only stamp column kc + 2 after every block has stamped
// kc + 1, i.e. after every block has finished reading the slots of column kc.
// The interchanges of the columns outside the base block are applied once,
// after the last column.
// Every wait is bounded (2 s of the global timer); on expiry the kernel
// records OZLU_ERR_TIMEOUT in the scratch and every block returns.
constexpr int COOP_MAXG = 304;           // blocks (up to 2 per SM)
constexpr int COOP_THREADS = 512;
static_assert(2 * PBASE + 2 <= COOP_THREADS, "one pivot-row element per thread");
constexpr unsigned long long COOP_WAIT_NS = 2000000000ull;

// stamp word of a slot: bits 63..44 the column (c0 + kc + 1, modulo 2^20),
// bits 43..0 the candidate's key (mpf_key; 0: no candidate).  One 64-bit
// store publishes both, after the rest of the slot.
constexpr int STAMP_SHIFT = 44;
constexpr unsigned long long KEY_MASK = (1ull << STAMP_SHIFT) - 1;

template <int L>
struct CoopSlot {
    unsigned long long stamp;      // column tag and key: idx and row are published
    unsigned long long stamp_rec;  // column tag: rec is published
    int idx;                 // the candidate's global row index, -1 if none
    int pad;
    MPF<L> rec;              // 1 / the candidate (0 for a zero candidate)
    MPF<L> row[PBASE];       // the candidate row (all b columns)
};

template <int L>
struct CoopScratch {
    int error;
    int pad[3];
    CoopSlot<L> part[2][COOP_MAXG];  // double-buffered by column parity
    MPF<L> orow[2][PBASE];           // old row c, for the owner of the pivot row
};

// the error word and every slot stamp start at zero for each factorisation
// (one thread per slot; the scratch was laid out for L limbs)
template <int L>
__global__ void coop_reset_kernel(CoopScratch<L>* sc) {
    const int t = threadIdx.x;
    if (t == 0) sc->error = 0;
    if (t < 2 * COOP_MAXG) {
        sc->part[t / COOP_MAXG][t % COOP_MAXG].stamp = 0ull;
        sc->part[t / COOP_MAXG][t % COOP_MAXG].stamp_rec = 0ull;
    }
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// load with acquire semantics at GPU scope: this thread's later loads see
// everything the writer of the value made visible before it
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// store with release semantics at GPU scope
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// wait until the stamp word carries column `want`; returns it, or 0 on
// expiry after limit_ns of the global timer (the error word is then set) or
// when another block has given up
__device__ __forceinline__ unsigned long long wait_stamp(const unsigned long long* p, unsigned want,
                                                         int* err,
                                                         unsigned long long limit_ns = COOP_WAIT_NS) {
    const unsigned long long t0 = global_ns();
    for (int it = 1;; ++it) {
        const unsigned long long v = ld_acquire(p);
        if ((unsigned)(v >> STAMP_SHIFT) == want) return v;
        if ((it & 63) == 0) {
            if (*(volatile int*)err) return 0;
            if (global_ns() - t0 > limit_ns) {
                atomicExch(err, OZLU_ERR_TIMEOUT);
                return 0;
            }
        }
    }
}

// load an L-limb float written by another block (bypassing L1)
template <int L>
__device__ __forceinline__ MPF<L> ld_cg(const MPF<L>* p) {
    MPF<L> v;
    const unsigned int* w = reinterpret_cast<const unsigned int*>(p);
#pragma unroll
    for (int i = 0; i < L; ++i) v.m[i] = __ldcg(w + i);
    v.e = __ldcg(reinterpret_cast<const int*>(w + L));
    v.neg = __ldcg(reinterpret_cast<const int*>(w + L + 1));
    return v;
}

// 44-bit order key of |v|: exponent (12 bits), then the top limb (values are
// normalised); a larger key means a larger |v|, equal keys need the full
// comparison.  An exact zero gets 1 (below every nonzero value, above "no
// candidate" = 0).  Exponents outside [-2047, 2047] share the lowest or the
// highest nonzero key, so that they always go through the full comparison.
template <int L>
__device__ __forceinline__ unsigned long long mpf_key(const MPF<L>& v) {
    if (mpf_zero<L>(v)) return 1ull;
    if (v.e < -2047) return 1ull << 32;
    if (v.e > 2047) return KEY_MASK;
    return ((unsigned long long)(unsigned)(v.e + 2048) << 32) | v.m[L - 1];
}

// |a| > |b|, or equal and ia < ib (first index on ties); ib < 0: b is empty
template <int L>
__device__ __forceinline__ bool mpf_better(const MPF<L>& a, int ia, const MPF<L>& b, int ib) {
    if (ia < 0) return false;
    if (ib < 0) return true;
    const int c = mpf_abs_cmp<L>(a, b);
    return c > 0 || (c == 0 && ia < ib);
}

// warp-wide argmax of (|v|, first index): every lane ends with the winner
template <int L>
__device__ __forceinline__ void warp_best(MPF<L>& v, int& idx, int& aux) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        MPF<L> w;
#pragma unroll
        for (int q = 0; q < L; ++q) w.m[q] = __shfl_xor_sync(0xffffffffu, v.m[q], o);
        w.e = __shfl_xor_sync(0xffffffffu, v.e, o);
        w.neg = __shfl_xor_sync(0xffffffffu, v.neg, o);
        const int wi = __shfl_xor_sync(0xffffffffu, idx, o);
        const int wa = __shfl_xor_sync(0xffffffffu, aux, o);
        if (mpf_better<L>(w, wi, v, idx)) { v = w; idx = wi; aux = wa; }
    }
}

// warp-wide max of (key, then lowest index); idx < 0: none
__device__ __forceinline__ void warp_best_key(unsigned long long& k, int& idx, int& aux) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, k, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        const int a2 = __shfl_xor_sync(0xffffffffu, aux, o);
        if (i2 >= 0 && (idx < 0 || k2 > k || (k2 == k && i2 < idx))) { k = k2; idx = i2; aux = a2; }
    }
}

// named barrier of warps 1 .. COOP_THREADS / 32 - 1 (warp 0 takes no part)
__device__ __forceinline__ void bar_rest() {
    asm volatile("bar.sync 1, %0;" ::"r"(COOP_THREADS - 32) : "memory");
}

template <int N>
__global__ void __launch_bounds__(COOP_THREADS, 1) base_block_coop_kernel(
    double* A, long long lda, int n, int c0, int b, int p0, int p1, int rows_per_block,
    int* ipiv, int* info, CoopScratch<Limbs<N>::L>* sc) {
    constexpr int L = Limbs<N>::L;
    constexpr int T = COOP_THREADS;
    extern __shared__ __align__(16) unsigned char smraw[];
    MPF<L>* a = reinterpret_cast<MPF<L>*>(smraw);  // [r][k], r < rows_per_block, k < b
    // rows padded to b + 1 entries: threads on consecutive rows of one column
    // then fall on different shared-memory banks
    const int bs = b + 1;
    __shared__ MPF<L> prow[2][PBASE];  // the pivot row, double-buffered by column parity
    __shared__ MPF<L> otmp[PBASE];     // old row c (for the owner of the pivot row)
    __shared__ MPF<L> rec;         // 1 / pivot
    __shared__ MPF<L> cv;          // this block's next candidate
    __shared__ int ci, s_piv, s_fail;
    __shared__ int s_pivs[PBASE];
    const int g = blockIdx.x, G = gridDim.x, tid = threadIdx.x;
    const int r0 = c0 + g * rows_per_block;
    const int r1 = min(n, r0 + rows_per_block);
    const int nr = max(0, r1 - r0);
    auto owner = [&](int row) { return (row - c0) / rows_per_block; };

    for (int p = tid; p < nr * b; p += T) {
        const int r = p / b, k = p - r * b;
        a[r * bs + k] = mpf_from_exp<L, N>(elem(A, lda, N, r0 + r, c0 + k));
    }
    __syncthreads();

    // warp 0: this block's best candidate in local column kc among rows >=
    // row_lo (cv, ci)
    auto candidate = [&](int kc, int row_lo) {
        unsigned long long bk = 0;
        int bi = -1, aux = 0;
        for (int r = tid; r < nr; r += 32) {
            const int i = r0 + r;
            if (i < row_lo) continue;
            const unsigned long long k = mpf_key<L>(a[r * bs + kc]);
            if (bi < 0 || k > bk ||
                (k == bk && mpf_abs_cmp<L>(a[r * bs + kc], a[(bi - r0) * bs + kc]) > 0)) {
                bk = k;
                bi = i;
            }
        }
        unsigned long long K = bk;
        int I = bi;
        warp_best_key(K, I, aux);
        if (__any_sync(0xffffffffu, bi >= 0 && bk == K && bi != I)) {  // equal keys: compare exactly
            MPF<L> v = (bi >= 0 && bk == K) ? a[(bi - r0) * bs + kc] : mpf_make_zero<L>();
            int vi = (bi >= 0 && bk == K) ? bi : -1;
            warp_best<L>(v, vi, aux);
            I = vi;
        }
        if (tid == 0) {
            ci = I;
            cv = I >= 0 ? a[(I - r0) * bs + kc] : mpf_make_zero<L>();
        }
    };
    // all threads: publish the candidate of column kc (every column of its row
    // final) and, from the owner of row c0 + kc, that row's old contents;
    // stamp A carries the key
    auto publish = [&](int kc) {
        CoopSlot<L>& slot = sc->part[kc & 1][g];
        const int wi = ci;
        const int c = c0 + kc;
        if (wi >= 0)
            for (int k = tid; k < b; k += T) slot.row[k] = a[(wi - r0) * bs + k];
        if (owner(c) == g)
            for (int k = tid; k < b; k += T) sc->orow[kc & 1][k] = a[(c - r0) * bs + k];
        if (tid == 0) slot.idx = wi;
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const unsigned long long key = wi >= 0 ? mpf_key<L>(cv) : 0ull;
            *reinterpret_cast<volatile unsigned long long*>(&slot.stamp) =
                ((unsigned long long)((c + 1) & 0xfffff) << STAMP_SHIFT) | key;
        }
    };
    // thread 0: the reciprocal of the candidate of column kc, then stamp B
    auto publish_rec = [&](int kc) {
        CoopSlot<L>& slot = sc->part[kc & 1][g];
        const MPF<L> r = (ci >= 0 && !mpf_zero<L>(cv)) ? mpf_recip<L, true>(cv) : mpf_make_zero<L>();
        slot.rec = r;
        st_release(&slot.stamp_rec, (unsigned long long)((c0 + kc + 1) & 0xfffff) << STAMP_SHIFT);
    };

    if (tid < 32) candidate(0, c0);
    __syncthreads();
    publish(0);
    if (tid == 0) publish_rec(0);
    // warps that share a scheduler with warp 0 (warp ids 4, 8, ...) leave the
    // priority rows to the others, so that the reciprocal on thread 0 issues
    // alone there
    constexpr int NPRIO_T = 32 * (T / 32 - (T / 32 + 3) / 4);
    const int warp = tid >> 5;
    // the update of the rows outside the priority pair by column bulk_kc is
    // deferred to the next column's exchange (bulk_kc < 0: none pending)
    int bulk_kc = -1, bulk_lo = 0, bulk_pa = -1, bulk_pb = -1;
    for (int kc = 0; kc < b; ++kc) {
        const int c = c0 + kc;
        MPF<L>* pr = prow[kc & 1];
        if (tid < 32) {
            // warp 0: wait for every stamp A of column kc, reduce the keys to
            // the pivot, wait for the winner's stamp B (its reciprocal), then
            // load the pivot row, its reciprocal and index and old row c
            constexpr int PER = (COOP_MAXG + 31) / 32;
            const unsigned want = (unsigned)((c + 1) & 0xfffff);
            unsigned long long key[PER];
            bool ok = true;
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int q = tid + 32 * u;
                key[u] = 0;
                if (q < G) key[u] = ld_acquire(&sc->part[kc & 1][q].stamp);
            }
#pragma unroll
            for (int u = 0; u < PER; ++u) {
                const int q = tid + 32 * u;
                if (q < G && ok && (unsigned)(key[u] >> STAMP_SHIFT) != want) {
                    key[u] = wait_stamp(&sc->part[kc & 1][q].stamp, want, &sc->error);
                    ok = key[u] != 0;
                }
                key[u] &= KEY_MASK;
            }
            bool fail = __any_sync(0xffffffffu, !ok);
            __syncwarp();
            if (!fail) {
                // the slots' contents are visible after their stamps (acquire loads)
                unsigned long long K = 0;
                int W = -1, dummy = 0;
#pragma unroll
                for (int u = 0; u < PER; ++u) {
                    const int q = tid + 32 * u;
                    if (q < G && key[u] > 0 && (W < 0 || key[u] > K)) { K = key[u]; W = q; }
                }
                warp_best_key(K, W, dummy);  // lowest slot among equal keys
                int same = 0;
#pragma unroll
                for (int u = 0; u < PER; ++u) same += (tid + 32 * u < G && key[u] == K) ? 1 : 0;
                same = __reduce_add_sync(0xffffffffu, same);
                if (same > 1) {
                    // equal keys: compare the candidates exactly (lowest row on ties)
                    MPF<L> v = mpf_make_zero<L>();
                    int vi = -1, vw = -1;
#pragma unroll
                    for (int u = 0; u < PER; ++u) {
                        const int q = tid + 32 * u;
                        if (q >= G || key[u] != K) continue;
                        const CoopSlot<L>& slot = sc->part[kc & 1][q];
                        const int iv = __ldcg(&slot.idx);
                        const MPF<L> x = ld_cg<L>(&slot.row[kc]);
                        if (mpf_better<L>(x, iv, v, vi)) { v = x; vi = iv; vw = q; }
                    }
                    warp_best<L>(v, vi, vw);
                    W = vw;
                }
                if (W < 0) W = 0;  // W >= 0: the owner of row c has a candidate
                // the pivot row (under stamp A) with all loads in flight before
                // the first shared-memory store, then the reciprocal (stamp B)
                const CoopSlot<L>& ws = sc->part[kc & 1][W];
                const int piv = __ldcg(&ws.idx);
                constexpr int PL = PBASE / 32;
                MPF<L> v[PL];
#pragma unroll
                for (int q = 0; q < PL; ++q) {
                    const int k = tid + 32 * q;
                    if (k < b) v[q] = ld_cg<L>(&ws.row[k]);
                }
#pragma unroll
                for (int q = 0; q < PL; ++q) {
                    const int k = tid + 32 * q;
                    if (k < b) pr[k] = v[q];
                }
                if (piv != c && owner(piv) == g) {
#pragma unroll
                    for (int q = 0; q < PL; ++q) {
                        const int k = tid + 32 * q;
                        if (k < b) v[q] = ld_cg<L>(&sc->orow[kc & 1][k]);
                    }
#pragma unroll
                    for (int q = 0; q < PL; ++q) {
                        const int k = tid + 32 * q;
                        if (k < b) otmp[k] = v[q];
                    }
                }
                int sb_ok = 1;
                if (tid == 0) sb_ok = wait_stamp(&ws.stamp_rec, want, &sc->error) != 0;
                fail = __shfl_sync(0xffffffffu, sb_ok, 0) == 0;
                if (!fail && tid == 0) {
                    rec = ld_cg<L>(&ws.rec);
                    s_piv = piv;
                }
            }
            if (tid == 0) s_fail = fail ? 1 : 0;
        } else if (bulk_kc >= 0) {
            // warps 1 ..: the deferred update of the other rows by column bulk_kc
            const int kb = bulk_kc, rest = b - kb - 2;
            const MPF<L>* pk = prow[kb & 1];
            const int total = (nr - bulk_lo) * rest;
            for (int p = tid - 32; p < total; p += T - 32) {
                const int r = bulk_lo + p / rest, k = kb + 2 + (p - (p / rest) * rest);
                if (r == bulk_pa || r == bulk_pb) continue;
                a[r * bs + k] = mpf_fms_oolv<L>(a[r * bs + k], a[r * bs + kb], pk[k]);
            }
        }
        __syncthreads();
        if (s_fail) return;
        const int piv = s_piv;
        if (tid == 0) s_pivs[kc] = piv;
        const bool zero = mpf_zero<L>(pr[kc]);
        if (g == 0 && tid == 0) {
            ipiv[c] = piv + 1;
            if (zero && *info == 0) *info = c + 1;
        }
        if (!zero && piv != c) {
            if (owner(c) == g)
                for (int k = tid; k < b; k += T) a[(c - r0) * bs + k] = pr[k];
            if (owner(piv) == g)
                for (int k = tid; k < b; k += T) a[(piv - r0) * bs + k] = otmp[k];
        }
        __syncthreads();
        const int lo = max(r0, c + 1) - r0;
        const int cols = b - kc - 1;
        if (!zero) {
            // multipliers, then the next column first (its candidate is needed next)
            for (int r = lo + tid; r < nr; r += T) {
                mpf_mul_ool<L>(&a[r * bs + kc], &a[r * bs + kc], &rec);
                if (cols > 0) a[r * bs + kc + 1] = mpf_fms_oolv<L>(a[r * bs + kc + 1], a[r * bs + kc], pr[kc + 1]);
            }
        }
        __syncthreads();
        if (cols == 0) break;
        // warp 0: the next candidate
        if (tid < 32) candidate(kc + 1, c + 1);
        __syncthreads();
        // the rows the next step reads from this block: the candidate and (from
        // its owner) row c + 1, which the pivot will replace
        const int pa = ci >= 0 ? ci - r0 : -1;
        const int pb = owner(c + 1) == g ? c + 1 - r0 : -1;
        const int rest = cols - 1;
        if (tid == 0) {
            // the candidate's reciprocal and stamp B, beside the priority rows
            publish_rec(kc + 1);
        } else if (tid >= 32) {
            if (!zero && rest > 0 && (warp & 3) != 0) {
                const int nprio = (pa >= 0 ? 1 : 0) + (pb >= 0 && pb != pa ? 1 : 0);
                const int pt = (warp - 1 - (warp >> 2)) * 32 + (tid & 31);
                for (int p = pt; p < nprio * rest; p += NPRIO_T) {
                    const int which = p / rest, k = kc + 2 + (p - which * rest);
                    const int r = (which == 0 && pa >= 0) ? pa : pb;
                    a[r * bs + k] = mpf_fms_oolv<L>(a[r * bs + k], a[r * bs + kc], pr[k]);
                }
            }
            bar_rest();
            // publish the candidate row of column kc + 1 and, from its owner,
            // row c + 1; then stamp A with the key
            CoopSlot<L>& slot = sc->part[(kc + 1) & 1][g];
            const int wi = ci;
            if (wi >= 0)
                for (int k = tid - 32; k < b; k += T - 32) slot.row[k] = a[(wi - r0) * bs + k];
            if (pb >= 0)
                for (int k = tid - 32; k < b; k += T - 32) sc->orow[(kc + 1) & 1][k] = a[pb * bs + k];
            if (tid == 32) slot.idx = wi;
            bar_rest();
            if (tid == 32) {
                __threadfence();
                const unsigned long long key = wi >= 0 ? mpf_key<L>(cv) : 0ull;
                *reinterpret_cast<volatile unsigned long long*>(&slot.stamp) =
                    ((unsigned long long)((c + 2) & 0xfffff) << STAMP_SHIFT) | key;
            }
        }
        bulk_kc = (!zero && rest > 0) ? kc : -1;
        bulk_lo = lo;
        bulk_pa = pa;
        bulk_pb = pb;
    }
    for (int p = tid; p < nr * b; p += T) {
        const int r = p / b, k = p - r * b;
        mpf_to_exp<L, N>(a[r * bs + k], elem(A, lda, N, r0 + r, c0 + k));
    }
    // the interchanges of this base block on the rest of the outer panel
    // (columns [p0, c0) and [c0 + b, p1)), one column per thread
    const int left = c0 - p0, span = left + (p1 - c0 - b);
    for (int t = g * T + tid; t < span; t += G * T) {
        const int j = t < left ? p0 + t : c0 + b + (t - left);
        for (int kc = 0; kc < b; ++kc) {
            const int pv = s_pivs[kc], c = c0 + kc;
            if (pv == c) continue;
            double* x = elem(A, lda, N, c, j);
            double* y = elem(A, lda, N, pv, j);
#pragma unroll
            for (int q = 0; q < N; ++q) { const double tt = x[q]; x[q] = y[q]; y[q] = tt; }
        }
    }
}

// Apply interchanges k in [k0, k1) (ipiv 1-based) to columns [j0, j1).
template <int N>
__global__ void laswp_kernel(double* A, long long lda, int j0, int j1, int k0, int k1,
                             const int* ipiv) {
    const int j = j0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= j1) return;
    for (int k = k0; k < k1; ++k) {
        const int p = ipiv[k] - 1;
        if (p != k) {
            double* a = elem(A, lda, N, k, j);
            double* b = elem(A, lda, N, p, j);
#pragma unroll
            for (int q = 0; q < N; ++q) { const double t = a[q]; a[q] = b[q]; b[q] = t; }
        }
    }
}

// Interchanges k in [k0, k1) (ipiv 1-based) applied to columns [j0, j1) as one
// permutation: every block replays the swaps on the few affected rows (a
// shared-memory hash map: position -> row whose contents end up there), then
// gathers those rows of its LCT columns into shared memory and writes them
// back permuted.  Replaces the column-serial swap chain.

// one block: the (destination, source) row pairs of the interchanges
__global__ void __launch_bounds__(256) laswp_list_kernel(int k0, int k1, const int* ipiv, int* list) {
    __shared__ int hkey[LHASH], hval[LHASH];
    __shared__ int cnt;
    for (int i = threadIdx.x; i < LHASH; i += blockDim.x) hkey[i] = -1;
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        auto slot = [&](int row) {
            int h = (int)(((unsigned)row * 2654435761u) & (LHASH - 1));
            while (hkey[h] != -1 && hkey[h] != row) h = (h + 1) & (LHASH - 1);
            return h;
        };
        for (int k = k0; k < k1; ++k) {
            const int p = ipiv[k] - 1;
            if (p == k) continue;
            const int sk = slot(k);
            if (hkey[sk] == -1) { hkey[sk] = k; hval[sk] = k; }
            const int sp = slot(p);
            if (hkey[sp] == -1) { hkey[sp] = p; hval[sp] = p; }
            const int t = hval[sk];
            hval[sk] = hval[sp];
            hval[sp] = t;
        }
    }
    __syncthreads();
    for (int h = threadIdx.x; h < LHASH; h += blockDim.x)
        if (hkey[h] != -1 && hval[h] != hkey[h]) {
            const int c = atomicAdd(&cnt, 1);
            list[1 + 2 * c] = hkey[h];
            list[2 + 2 * c] = hval[h];
        }
    __syncthreads();
    if (threadIdx.x == 0) list[0] = cnt;
}

template <int N>
__global__ void __launch_bounds__(256) laswp_apply_kernel(double* A, long long lda, int j0, int j1,
                                                          const int* list) {
    extern __shared__ __align__(16) double buf[];  // [entry][col][N]
    const int ne = list[0];
    const int jb = j0 + blockIdx.x * LCT;
    for (int t = threadIdx.x; t < ne * LCT; t += blockDim.x) {
        const int e = t / LCT, cc = t - e * LCT, j = jb + cc;
        if (j < j1) {
            const double* x = elem(A, lda, N, list[2 + 2 * e], j);
#pragma unroll
            for (int q = 0; q < N; ++q) buf[(e * LCT + cc) * N + q] = x[q];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ne * LCT; t += blockDim.x) {
        const int e = t / LCT, cc = t - e * LCT, j = jb + cc;
        if (j < j1) {
            double* x = elem(A, lda, N, list[1 + 2 * e], j);
#pragma unroll
            for (int q = 0; q < N; ++q) x[q] = buf[(e * LCT + cc) * N + q];
        }
    }
}

// the permutation of interchanges [k0, k1) applied to column ranges
template <int N>
void laswp2(double* A, long long lda, int ja0, int ja1, int jb0, int jb1, int k0, int k1, const int* ipiv,
            int* list, cudaStream_t s) {
    if (k1 <= k0 || (ja1 <= ja0 && jb1 <= jb0)) return;
    if (k1 - k0 > LMAXB) {
        if (ja1 > ja0) laswp_kernel<N><<<(ja1 - ja0 + 127) / 128, 128, 0, s>>>(A, lda, ja0, ja1, k0, k1, ipiv);
        if (jb1 > jb0) laswp_kernel<N><<<(jb1 - jb0 + 127) / 128, 128, 0, s>>>(A, lda, jb0, jb1, k0, k1, ipiv);
        return;
    }
    laswp_list_kernel<<<1, 256, 0, s>>>(k0, k1, ipiv, list);
    const size_t smem = sizeof(double) * 2 * (k1 - k0) * LCT * N;
    raise_smem_limit((const void*)laswp_apply_kernel<N>, (int)(sizeof(double) * 2 * LMAXB * LCT * N));
    if (ja1 > ja0) laswp_apply_kernel<N><<<(ja1 - ja0 + LCT - 1) / LCT, 256, smem, s>>>(A, lda, ja0, ja1, list);
    if (jb1 > jb0) laswp_apply_kernel<N><<<(jb1 - jb0 + LCT - 1) / LCT, 256, smem, s>>>(A, lda, jb0, jb1, list);
}

// Native trailing update for the blocked-naive comparison (Sec. 3.4):
// C -= A B with every multiply-add rounded in expansion arithmetic (binary64
// TwoSum / TwoProd), 16 x 16 outputs per block, A and B tiles in shared memory.
template <int N>
__global__ void __launch_bounds__(256) naive_update_kernel(const double* A, long long lda, const double* B,
                                                           long long ldb, double* C, long long ldc, int m,
                                                           int n, int k) {
    __shared__ double sa[16][16][N];
    __shared__ double sb[16][16][N];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int i = blockIdx.x * 16 + tx, j = blockIdx.y * 16 + ty;
    Exp<N> acc;
    if (i < m && j < n) acc = load<N>(C + ((long long)i + (long long)j * ldc) * N);
    for (int h0 = 0; h0 < k; h0 += 16) {
        {
            const int ii = blockIdx.x * 16 + tx, hh = h0 + ty;
#pragma unroll
            for (int q = 0; q < N; ++q)
                sa[ty][tx][q] = (ii < m && hh < k) ? A[((long long)ii + (long long)hh * lda) * N + q] : 0.0;
            const int hb = h0 + tx, jj = blockIdx.y * 16 + ty;
#pragma unroll
            for (int q = 0; q < N; ++q)
                sb[ty][tx][q] = (hb < k && jj < n) ? B[((long long)hb + (long long)jj * ldb) * N + q] : 0.0;
        }
        __syncthreads();
        if (i < m && j < n) {
            const int hmax = min(16, k - h0);
            for (int h = 0; h < hmax; ++h) {
                Exp<N> a, b;
#pragma unroll
                for (int q = 0; q < N; ++q) { a.x[q] = sa[h][tx][q]; b.x[q] = sb[ty][h][q]; }
                acc = fms<N>(acc, a, b);
            }
        }
        __syncthreads();
    }
    if (i < m && j < n) store<N>(C + ((long long)i + (long long)j * ldc) * N, acc);
}

// The b x b triangle of a base triangular solve, converted once to L-limb
// floats (and the reciprocal diagonal for the upper case) in the scratch:
// blockIdx.y = q converts the q-th b x b diagonal block from T into slot q.
template <int N>
__global__ void __launch_bounds__(256) tri_convert_kernel(const double* T, long long ldt, int b, int lower,
                                                          LuScratch* sc) {
    constexpr int L = Limbs<N>::L;
    const int q = blockIdx.y;
    T += ((long long)q * b + (long long)q * b * ldt) * N;
    MPF<L>* tl = reinterpret_cast<MPF<L>*>(sc->tri[q]);
    MPF<L>* rd = tl + BASE * BASE;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < b * b; idx += gridDim.x * blockDim.x) {
        const int i = idx / b, k = idx - i * b;
        const bool need = lower ? (k < i) : (k >= i);
        const MPF<L> v = need ? mpf_from_exp<L, N>(T + ((long long)i + (long long)k * ldt) * N) : mpf_make_zero<L>();
        tl[k * BASE + i] = v;  // column-major: a step reads one column across the rows
        if (!lower && i == k) rd[k] = mpf_zero<L>(v) ? mpf_make_zero<L>() : mpf_recip<L>(v);
    }
}

// X <- L^-1 X for a unit lower (lower = 1) or U^-1 X for an upper (lower = 0,
// non-unit) b x b triangle, b <= BASE; X is b x ncols.  L-limb integer
// floating point.  One warp per column, lane i holding x_i in registers: step
// k broadcasts the final x_k by warp shuffles and every lane below (lower) or
// above (upper) row k subtracts l_ik x_k, so the b steps need no block-wide
// barrier and the warps of a block progress independently.  The triangle is
// read from shared memory column by column ([k][i], conflict-free).
template <int N>
__global__ void __launch_bounds__(256) trsm_base_kernel(const LuScratch* sc, double* X, long long ldx, int b,
                                                        int ncols, int lower, int slot) {
    constexpr int L = Limbs<N>::L;
    extern __shared__ __align__(16) unsigned char smraw[];
    MPF<L>* sl = reinterpret_cast<MPF<L>*>(smraw);   // [k][i]
    MPF<L>* rd = sl + BASE * BASE;                   // reciprocal diagonal (upper)
    const int row = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int col = blockIdx.x * (blockDim.x >> 5) + w;
    const MPF<L>* tl = reinterpret_cast<const MPF<L>*>(sc->tri[slot]);
    for (int idx = threadIdx.x; idx < BASE * BASE; idx += blockDim.x) sl[idx] = tl[idx];
    if (!lower)
        for (int k = threadIdx.x; k < b; k += blockDim.x) rd[k] = tl[BASE * BASE + k];
    __syncthreads();
    if (col >= ncols) return;  // whole warps: col is uniform in a warp
    double* xp = X + ((long long)row + (long long)col * ldx) * N;
    MPF<L> x = row < b ? mpf_from_exp<L, N>(xp) : mpf_make_zero<L>();
    for (int s = 0; s < b; ++s) {
        const int k = lower ? s : b - 1 - s;
        if (!lower && row == k) x = mpf_mul<L>(x, rd[k]);
        MPF<L> xk;
#pragma unroll
        for (int q = 0; q < L; ++q) xk.m[q] = __shfl_sync(0xffffffffu, x.m[q], k);
        xk.e = __shfl_sync(0xffffffffu, x.e, k);
        xk.neg = __shfl_sync(0xffffffffu, x.neg, k);
        if (row < b && (lower ? row > k : row < k)) x = mpf_fms<L>(x, sl[k * BASE + row], xk);
    }
    if (row < b) mpf_to_exp<L, N>(x, xp);
}

// slot < 0: convert the triangle into slot 0 first; else it is in `slot`
template <int N>
void trsm_base(const double* T, long long ldt, double* X, long long ldx, int b, int ncols, int lower,
               LuScratch* sc, cudaStream_t s, int slot = -1) {
    if (ncols <= 0 || b <= 0) return;
    constexpr int L = Limbs<N>::L;
    if (slot < 0) {
        tri_convert_kernel<N><<<(b * b + 255) / 256, 256, 0, s>>>(T, ldt, b, lower, sc);
        slot = 0;
    }
    // 8 columns (warps) per block, fewer when that leaves SMs idle
    const int wpb = ncols >= 8 * 152 ? 8 : (ncols >= 4 * 152 ? 4 : 2);
    const size_t smem = sizeof(MPF<L>) * (BASE * BASE + BASE);
    raise_smem_limit((const void*)trsm_base_kernel<N>, (int)smem);
    trsm_base_kernel<N><<<(ncols + wpb - 1) / wpb, 32 * wpb, smem, s>>>(sc, X, ldx, b, ncols, lower, slot);
}

// Launch the cooperative base-block kernel; returns false when the slice of
// rows does not fit in shared memory (the caller then uses column kernels).
template <int N>
bool base_block_coop(double* A, long long lda, int n, int c0, int b, int p0, int p1, int* ipiv,
                     int* info, void* scratch, int min_rows, cudaStream_t s) {
    constexpr int L = Limbs<N>::L;
    const int sms = device_sms();
    // at least min_rows rows per block: a small panel takes a few SMs and
    // leaves the rest to concurrent work (the batched driver runs instances
    // side by side and asks for 32, single factorisations for 16)
    const int g_rows = (n - c0 + min_rows - 1) / min_rows;
    for (int per_sm = 1; per_sm <= 2; ++per_sm) {
        int G = sms * per_sm;
        if (G > COOP_MAXG) G = COOP_MAXG;
        if (G > g_rows) G = g_rows < 1 ? 1 : g_rows;
        const int rows = (n - c0 + G - 1) / G;
        const size_t smem = sizeof(MPF<L>) * (size_t)rows * (b + 1);
        if (smem > 200 * 1024 / per_sm) continue;
        raise_smem_limit((const void*)base_block_coop_kernel<N>, (int)(smem < 1024 ? 1024 : smem));
        int active = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&active, base_block_coop_kernel<N>, COOP_THREADS,
                                                      smem);
        if (active * sms < G) continue;
        auto* sc = reinterpret_cast<CoopScratch<L>*>(scratch);
        // cooperative launch (all blocks co-resident), also valid under stream capture
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(G);
        cfg.blockDim = dim3(COOP_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, base_block_coop_kernel<N>, A, lda, n, c0, b, p0, p1, rows, ipiv, info, sc) !=
            cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return true;
    }
    return false;
}

struct Ctx {
    ozlu_handle* h;
    int nc, p;
    const ozlu_opts* opts;
    double* A;
    long long lda;
    int n;
    int* ipiv;
    LuScratch* sc;
    int rc = 0;
};

double* at(const Ctx& c, long long i, long long j) { return c.A + (i + j * c.lda) * c.nc; }

// widest base block for the cooperative panel kernel: the caller's choice,
// else PBASE (measured fastest on GB300 for n from 512 to 4096; a block
// whose rows do not fit in shared memory is split by the recursion)
int coop_width(const Ctx& c, int) {
    if (c.opts && c.opts->panel_width) return c.opts->panel_width < PBASE ? c.opts->panel_width : PBASE;
    return PBASE;
}

// r_top >= 0: the unit lower triangle's BASE x BASE diagonal blocks from row
// r_top on are already converted, block q in slot q
template <int N>
void trsm_rec(Ctx& c, long long r, int b, long long j0, int ncols, bool lower, long long r_top = -1) {
    if (c.rc || ncols <= 0) return;
    // (a power of two: the halving recursion then ends on the BASE blocks)
    if (lower && r_top < 0 && b > BASE && (b & (b - 1)) == 0 && b / BASE <= TRI_SLOTS) {
        // every leaf's triangle in one launch, ahead of the recursion
        c.h->phase(PH_TRSM);
        tri_convert_kernel<N><<<dim3((BASE * BASE + 255) / 256, b / BASE), 256, 0, c.h->stream>>>(
            at(c, r, r), c.lda, BASE, 1, c.sc);
        c.h->count(1);
        r_top = r;
    }
    if (b <= BASE) {
        c.h->phase(PH_TRSM);
        const int slot = (lower && r_top >= 0) ? (int)((r - r_top) / BASE) : -1;
        trsm_base<N>(at(c, r, r), c.lda, at(c, r, j0), c.lda, b, ncols, lower ? 1 : 0, c.sc, c.h->stream, slot);
        c.h->count(slot < 0 ? 2 : 1);
        return;
    }
    const int b1 = b / 2;
    if (lower) {
        trsm_rec<N>(c, r, b1, j0, ncols, true, r_top);
        c.rc = c.rc ? c.rc : gemm_device(c.h, N, c.p, b - b1, ncols, b1, -1, at(c, r + b1, r), c.lda,
                                         at(c, r, j0), c.lda, 1, at(c, r + b1, j0), c.lda, c.opts);
        trsm_rec<N>(c, r + b1, b - b1, j0, ncols, true, r_top);
    } else {
        trsm_rec<N>(c, r + b1, b - b1, j0, ncols, false);
        c.rc = c.rc ? c.rc : gemm_device(c.h, N, c.p, b1, ncols, b - b1, -1, at(c, r, r + b1), c.lda,
                                         at(c, r + b1, j0), c.lda, 1, at(c, r, j0), c.lda, c.opts);
        trsm_rec<N>(c, r, b1, j0, ncols, false);
    }
}

// factor the panel block with top-left (r, r), width b, rows [r, n); row
// interchanges are applied across the outer panel columns [p0, p1)
template <int N>
void panel_rec(Ctx& c, int r, int b, int p0, int p1) {
    if (c.rc) return;
    cudaStream_t s = c.h->stream;
    // up to coop_width columns in one cooperative kernel when its rows fit
    // in shared memory (else the block is split further)
    if (b <= coop_width(c, r)) {
        c.h->phase(PH_PANEL);
        if (base_block_coop<N>(c.A, c.lda, c.n, r, b, p0, p1, c.ipiv, &c.sc->info, c.h->coop_scratch,
                               c.h->coop_min_rows, s)) {
            c.h->count(1);
            c.h->stats.panel_launches += 1;
            return;
        }
    }
    if (b <= BASE) {
        c.h->count(1 + b);
        c.h->stats.panel_launches += 1 + b;
        {
            const int rows = c.n - r;
            const int blocks = rows > PIV_THREADS * PIV_BLOCKS ? PIV_BLOCKS
                                                               : (rows + PIV_THREADS - 1) / PIV_THREADS;
            pivot_kernel<N><<<blocks, PIV_THREADS, 0, s>>>(c.A, c.lda, c.n, r, p0, p1, c.ipiv, c.sc);
        }
        for (int col = r; col < r + b; ++col) {
            const int rows = c.n - col - 1;
            if (rows <= 0) break;
            int blocks = (rows + STEP_ROWS - 1) / STEP_ROWS;
            if (blocks > MAXPART) blocks = MAXPART;
            column_step_kernel<N><<<blocks, 128, 0, s>>>(c.A, c.lda, c.n, col, r + b, p0, p1, c.ipiv,
                                                          c.sc);
        }
        return;
    }
    const int b1 = b / 2;
    panel_rec<N>(c, r, b1, p0, p1);
    trsm_rec<N>(c, r, b1, r + b1, b - b1, true);
    if (!c.rc && c.n - r - b1 > 0)
        c.rc = gemm_device(c.h, N, c.p, c.n - r - b1, b - b1, b1, -1, at(c, r + b1, r), c.lda,
                           at(c, r, r + b1), c.lda, 1, at(c, r + b1, r + b1), c.lda, c.opts);
    panel_rec<N>(c, r + b1, b - b1, p0, p1);
}

}  // namespace

template <int N>
int getrf_device(ozlu_handle* h, int p, int n, double* A, long long lda, int* ipiv, int nb,
                 LuScratch* sc, const ozlu_opts* opts) {
    Ctx c{h, N, p, opts, A, lda, n, ipiv, sc};
    cudaStream_t s = h->stream;
    for (int r0 = 0; r0 < n && !c.rc; r0 += nb) {
        const int b = nb < n - r0 ? nb : n - r0;
        panel_rec<N>(c, r0, b, r0, r0 + b);
        // (P2) interchanges on the columns left and right of the panel
        h->phase(PH_OTHER);
        h->count((r0 > 0) + (r0 + b < n));
        laswp2<N>(A, lda, 0, r0, r0 + b, n, r0, r0 + b, ipiv, sc->plist, s);
        if (r0 + b < n) {
            // (P3) U12 = L11^-1 A12
            trsm_rec<N>(c, r0, b, r0 + b, n - r0 - b, true);
            // (P4) A22 <- A22 - L21 U12
            if (!c.rc && opts && opts->native) {
                h->phase(PH_GEMM);
                const int mm = n - r0 - b;
                dim3 grid((mm + 15) / 16, (mm + 15) / 16);
                naive_update_kernel<N><<<grid, 256, 0, s>>>(at(c, r0 + b, r0), lda, at(c, r0, r0 + b), lda,
                                                            at(c, r0 + b, r0 + b), lda, mm, mm, b);
                h->count(1);
            } else if (!c.rc) {
                c.rc = gemm_device(h, N, p, n - r0 - b, n - r0 - b, b, -1, at(c, r0 + b, r0), lda,
                                   at(c, r0, r0 + b), lda, 1, at(c, r0 + b, r0 + b), lda, opts);
            }
        }
    }
    h->phase(-1);
    if (!c.rc && cudaGetLastError() != cudaSuccess) c.rc = OZLU_ERR_CUDA;
    return c.rc;
}

template <int N>
int getrs_device(ozlu_handle* h, int p, int n, int nrhs, double* LU, long long lda, const int* ipiv,
                 double* B, long long ldb, const ozlu_opts* opts, LuScratch* sc) {
    cudaStream_t s = h->stream;
    laswp_kernel<N><<<(nrhs + 127) / 128, 128, 0, s>>>(B, ldb, 0, nrhs, 0, n, ipiv);
    int rc = 0;
    auto L = [&](long long i, long long j) { return LU + (i + j * lda) * N; };
    auto X = [&](long long i) { return B + i * N; };
    h->phase(PH_TRSM);
    h->count(1 + 3 * ((n + BASE - 1) / BASE));
    for (int r = 0; r < n && !rc; r += BASE) {
        const int b = BASE < n - r ? BASE : n - r;
        trsm_base<N>(L(r, r), lda, X(r), ldb, b, nrhs, 1, sc, s);
        if (r + b < n)
            rc = gemm_device(h, N, p, n - r - b, nrhs, b, -1, L(r + b, r), lda, X(r), ldb, 1,
                             X(r + b), ldb, opts);
    }
    const int last = ((n - 1) / BASE) * BASE;
    for (int r = last; r >= 0 && !rc; r -= BASE) {
        const int b = BASE < n - r ? BASE : n - r;
        trsm_base<N>(L(r, r), lda, X(r), ldb, b, nrhs, 0, sc, s);
        if (r > 0)
            rc = gemm_device(h, N, p, r, nrhs, b, -1, L(0, r), lda, X(r), ldb, 1, X(0), ldb, opts);
    }
    h->phase(-1);
    if (!rc && cudaGetLastError() != cudaSuccess) rc = OZLU_ERR_CUDA;
    return rc;
}

namespace {
size_t align256(size_t v) { return (v + 255) / 256 * 256; }
}  // namespace

int lu_scratch(ozlu_handle* h, LuScratch** out);
int coop_reset(ozlu_handle* h, int nc, cudaStream_t s);

namespace {
// info of one factorisation: the first zero pivot (1-based), or
// -OZLU_ERR_TIMEOUT when a bounded wait of the panel kernel (its error word)
// or of a tensor-core GEMM (the handle's error word) gave up
__global__ void finish_kernel(int* info_out, const LuScratch* sc, const int* coop, const int* gerr) {
    int v = sc->info;
    if (coop[0]) v = -coop[0];
    else if (*gerr) v = -*gerr;
    *info_out = v;
}

// Self-test of the panel kernel's bounded wait: one thread waits with
// wait_stamp for a stamp that nothing writes (a zeroed word, column 1), with a
// short limit, into the panel's own error word; out[0] = 1 if it gave up.
__global__ void stamp_expiry_selftest_kernel(const unsigned long long* word, unsigned long long limit_ns,
                                             int* err, int* out) {
    if (threadIdx.x != 0) return;
    out[0] = wait_stamp(word, 1u, err, limit_ns) == 0 ? 1 : 0;
}
}  // namespace

int launch_mbar_expiry_selftest(long long limit, int* err, int* out, cudaStream_t s);

// which = 1: the panel's stamp wait, then the factorisation's finish step
// (info); which = 2: the tensor-core GEMM's mbarrier wait.  out (host, 3
// ints): whether the wait gave up, the error word, info (which = 1).
int wait_expiry_selftest(ozlu_handle* h, int which, long long limit, int* out) {
    LuScratch* sc;
    int rc = lu_scratch(h, &sc);
    if (rc) return rc;
    cudaStream_t s = h->stream;
    int* gerr = err_word(h);
    if (!gerr) return OZLU_ERR_NOMEM;
    if (cudaMemsetAsync(sc, 0, sizeof(LuScratch), s)) return OZLU_ERR_CUDA;
    if ((rc = coop_reset(h, 4, s))) return rc;
    if ((rc = clear_err_word(h))) return rc;
    // the candidate area of the scratch (zeroed above) holds a stamp word that
    // nothing writes and the kernel's flag
    unsigned long long* word = reinterpret_cast<unsigned long long*>(&sc->pval[0][0]);
    int* flag = &sc->pidx[0];
    if (which == 1) {
        stamp_expiry_selftest_kernel<<<1, 32, 0, s>>>(word, (unsigned long long)limit,
                                                       (int*)h->coop_scratch, flag);
        finish_kernel<<<1, 1, 0, s>>>(&sc->result, sc, (const int*)h->coop_scratch, gerr);
    } else if (which == 2) {
        if ((rc = launch_mbar_expiry_selftest(limit, gerr, flag, s))) return rc;
        finish_kernel<<<1, 1, 0, s>>>(&sc->result, sc, (const int*)h->coop_scratch, gerr);
    } else {
        return -2;
    }
    if (cudaGetLastError() != cudaSuccess) return OZLU_ERR_CUDA;
    int host[3] = {0, 0, 0};
    if (cudaMemcpyAsync(&host[0], flag, sizeof(int), cudaMemcpyDeviceToHost, s) ||
        cudaMemcpyAsync(&host[1], which == 1 ? (const int*)h->coop_scratch : gerr, sizeof(int),
                        cudaMemcpyDeviceToHost, s) ||
        cudaMemcpyAsync(&host[2], &sc->result, sizeof(int), cudaMemcpyDeviceToHost, s) ||
        cudaStreamSynchronize(s))
        return OZLU_ERR_CUDA;
    for (int i = 0; i < 3; ++i) out[i] = host[i];
    return host[2] < 0 ? -host[2] : OZLU_OK;
}

// one factorisation on device pointers (the batched driver calls it per
// instance on its own streams); info of the instance goes to *info_out
int getrf_one(ozlu_handle* h, int nc, int p, int n, double* A, long long lda, int* ipiv, int nb, int* info_out,
              const ozlu_opts* opts) {
    LuScratch* sc;
    int rc = lu_scratch(h, &sc);
    if (rc) return rc;
    cudaStream_t s = h->stream;
    // the unblocked naive comparison of Sec. 3.4: b = 1, every column's
    // rank-1 update of the whole trailing matrix in expansion arithmetic
    if (opts && opts->native == 2) nb = 1;
    if (cudaMemsetAsync(sc, 0, sizeof(LuScratch), s)) return OZLU_ERR_CUDA;
    if ((rc = coop_reset(h, nc, s))) return rc;
    if ((rc = clear_err_word(h))) return rc;
    if (n > 0) {
        switch (nc) {
            case 2: rc = getrf_device<2>(h, p, n, A, lda, ipiv, nb, sc, opts); break;
            case 3: rc = getrf_device<3>(h, p, n, A, lda, ipiv, nb, sc, opts); break;
            default: rc = getrf_device<4>(h, p, n, A, lda, ipiv, nb, sc, opts); break;
        }
    }
    if (rc) return rc;
    finish_kernel<<<1, 1, 0, s>>>(info_out, sc, (const int*)h->coop_scratch, h->dev_err);
    h->count(1);
    return cudaGetLastError() == cudaSuccess ? OZLU_OK : OZLU_ERR_CUDA;
}

int getrs_one(ozlu_handle* h, int nc, int p, int n, int nrhs, const double* LU, long long lda, const int* ipiv,
              double* B, long long ldb, const ozlu_opts* opts) {
    LuScratch* sc;
    int rc = lu_scratch(h, &sc);
    if (rc) return rc;
    if ((rc = clear_err_word(h))) return rc;
    switch (nc) {
        case 2: return getrs_device<2>(h, p, n, nrhs, (double*)LU, lda, ipiv, B, ldb, opts, sc);
        case 3: return getrs_device<3>(h, p, n, nrhs, (double*)LU, lda, ipiv, B, ldb, opts, sc);
        default: return getrs_device<4>(h, p, n, nrhs, (double*)LU, lda, ipiv, B, ldb, opts, sc);
    }
}

int lu_scratch(ozlu_handle* h, LuScratch** out) {
    if (!h->lu_scratch) {
        if (!dev_alloc(&h->lu_scratch, sizeof(LuScratch))) return OZLU_ERR_NOMEM;
    }
    if (!h->coop_scratch) {
        h->coop_bytes = std::max(std::max(sizeof(CoopScratch<Limbs<2>::L>), sizeof(CoopScratch<Limbs<3>::L>)),
                                 sizeof(CoopScratch<Limbs<4>::L>));
        if (!dev_alloc(&h->coop_scratch, h->coop_bytes)) {
            h->coop_scratch = nullptr;
            return OZLU_ERR_NOMEM;
        }
    }
    *out = (LuScratch*)h->lu_scratch;
    return OZLU_OK;
}

// the error word and the slot stamps start at zero for every factorisation
int coop_reset(ozlu_handle* h, int nc, cudaStream_t s) {
    // the slot layout is that of the panel kernel's limb count for nc
    constexpr int L2 = Limbs<2>::L, L3 = Limbs<3>::L, L4 = Limbs<4>::L;
    switch (nc) {
        case 2: coop_reset_kernel<L2><<<1, 2 * COOP_MAXG, 0, s>>>((CoopScratch<L2>*)h->coop_scratch); break;
        case 3: coop_reset_kernel<L3><<<1, 2 * COOP_MAXG, 0, s>>>((CoopScratch<L3>*)h->coop_scratch); break;
        default: coop_reset_kernel<L4><<<1, 2 * COOP_MAXG, 0, s>>>((CoopScratch<L4>*)h->coop_scratch); break;
    }
    h->count(1);
    return cudaGetLastError() == cudaSuccess ? OZLU_OK : OZLU_ERR_CUDA;
}

// Panel width by measurement (nb = 0 in ozlu_getrf and the batched LU): the
// candidates 64, 128, 256 and 512 (not above n) each factor a scratch copy of
// A twice on the handle's stream, the second run timed with events (the first
// grows workspaces and lets the back-end autotuner see the new shapes); the
// fastest is cached per (nc, p, log2 n, back-end).  Never inside a capture.
int tune_nb(ozlu_handle* h, int nc, int p, int n, const double* A, long long lda, const ozlu_opts* opts,
            int* nb_out) {
    int lgn = 0;
    while ((1 << lgn) < n) ++lgn;
    const int be = opts ? opts->backend : 0;
    const auto key = std::make_tuple(nc, p, lgn, be);
    auto it = h->tuned_nb.find(key);
    if (it != h->tuned_nb.end()) {
        *nb_out = it->second;
        h->stats.tuned_nb = it->second;
        return OZLU_OK;
    }
    if (n <= 64 || h->capturing) {
        *nb_out = n <= 64 ? (n > 0 ? n : 1) : 256;
        return OZLU_OK;
    }
    ozlu_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    o.graph = 0;
    const size_t abytes = align256(sizeof(double) * nc * (size_t)n * n);
    int rc = h->nb_ws.ensure(abytes + align256(sizeof(int) * (size_t)n) + 256);
    if (rc) return rc;
    double* Ac = (double*)h->nb_ws.base;
    int* ipv = (int*)((char*)h->nb_ws.base + abytes);
    int* inf = (int*)((char*)ipv + align256(sizeof(int) * (size_t)n));
    cudaStream_t s = h->stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool timing = h->timing;
    h->timing = false;
    float best = 1e30f;
    int choice = 256 < n ? 256 : n;
    const int cands[4] = {64, 128, 256, 512};
    for (int c = 0; c < 4 && !rc; ++c) {
        const int nb = cands[c];
        if (nb > n && c > 0) break;
        for (int rep = 0; rep < 2 && !rc; ++rep) {
            if (cudaMemcpy2DAsync(Ac, sizeof(double) * nc * n, A, sizeof(double) * nc * lda, sizeof(double) * nc * n,
                                  n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
                rc = OZLU_ERR_CUDA;
                break;
            }
            cudaEventRecord(e0, s);
            rc = getrf_one(h, nc, p, n, Ac, n, ipv, nb, inf, &o);
            cudaEventRecord(e1, s);
            if (rc) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = OZLU_ERR_CUDA; break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 1 && ms < best) { best = ms; choice = nb; }
        }
    }
    h->timing = timing;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    h->tuned_nb[key] = choice;
    h->stats.tuned_nb = choice;
    *nb_out = choice;
    return OZLU_OK;
}

// waits for the stream; OZLU_ERR_TIMEOUT if a bounded device wait gave up
int lu_result(ozlu_handle* h, cudaStream_t s, int* result) {
    LuScratch* sc = (LuScratch*)h->lu_scratch;
    if (cudaMemcpyAsync(result, &sc->result, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return OZLU_ERR_CUDA;
    return *result < 0 ? -*result : OZLU_OK;
}

}  // namespace ozlu

using namespace ozlu;

extern "C" int ozlu_getrf(ozlu_handle* h, int nc, int p, int n, double* A, long long lda, int* ipiv,
                          int nb, int* info, const ozlu_opts* opts) {
    if (!h) return -1;
    if (nc < 2 || nc > 4) return -2;
    if (p == 0) p = 53 * nc;
    if (p < 1 || p > 53 * nc) return -3;
    if (n < 0) return -4;
    if (!A && n) return -5;
    if (lda < (n > 1 ? n : 1)) return -6;
    if (!ipiv && n) return -7;
    if (nb < 0) return -8;
    if (!info) return -9;
    if (cudaSetDevice(h->device) != cudaSuccess) return OZLU_ERR_CUDA;
    cudaStream_t s = h->stream;
    LuScratch* sc;
    int rc = lu_scratch(h, &sc);
    if (rc) return rc;
    const bool dA = is_device_ptr(A), dP = is_device_ptr(ipiv), dI = is_device_ptr(info);
    if (opts && opts->graph && n > 0 && dA && dP && dI) {  // graph capture and replay
        if (nb == 0 && (rc = tune_nb(h, nc, p, n, A, lda, opts, &nb))) return rc;
        return ozlu_getrf_batched(h, nc, p, 1, &n, &A, &lda, &ipiv, info, nb, opts);
    }
    const size_t abytes = sizeof(double) * nc * (size_t)lda * (n ? n : 1);
    double* gA = A;
    int* gP = ipiv;
    if (!dA || !dP) {
        rc = h->stage.ensure(abytes + sizeof(int) * (size_t)(n + 1) + 512);
        if (rc) return rc;
        if (!dA) {
            gA = (double*)h->stage.base;
            if (cudaMemcpyAsync(gA, A, abytes, cudaMemcpyHostToDevice, s)) return OZLU_ERR_CUDA;
        }
        if (!dP) gP = (int*)((char*)h->stage.base + align256(abytes));
    }
    if (nb == 0 && n > 0 && (rc = tune_nb(h, nc, p, n, gA, lda, opts, &nb))) return rc;
    if (nb == 0) nb = 1;
    if ((rc = getrf_one(h, nc, p, n, gA, lda, gP, nb, &sc->result, opts))) return rc;
    int result = 0;
    if ((rc = lu_result(h, s, &result))) return rc;
    if (!dA && cudaMemcpyAsync(A, gA, abytes, cudaMemcpyDeviceToHost, s)) return OZLU_ERR_CUDA;
    if (n && gP != ipiv &&
        cudaMemcpyAsync(ipiv, gP, sizeof(int) * n, dP ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s))
        return OZLU_ERR_CUDA;
    if (cudaMemcpyAsync(info, &sc->info, sizeof(int), dI ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s))
        return OZLU_ERR_CUDA;
    if (!dA || !dP || !dI) return cuda_rc(cudaStreamSynchronize(s));
    return OZLU_OK;
}

extern "C" int ozlu_debug_wait_expiry(ozlu_handle* h, int which, long long limit, int* out) {
    if (!h) return -1;
    if (which != 1 && which != 2) return -2;
    if (limit < 1) return -3;
    if (!out) return -4;
    if (cudaSetDevice(h->device) != cudaSuccess) return OZLU_ERR_CUDA;
    return wait_expiry_selftest(h, which, limit, out);
}

extern "C" int ozlu_getrs(ozlu_handle* h, int nc, int p, int n, int nrhs, const double* LU,
                          long long lda, const int* ipiv, double* B, long long ldb,
                          const ozlu_opts* opts) {
    if (!h) return -1;
    if (nc < 2 || nc > 4) return -2;
    if (p == 0) p = 53 * nc;
    if (p < 1 || p > 53 * nc) return -3;
    if (n < 0) return -4;
    if (nrhs < 0) return -5;
    if (!LU && n) return -6;
    if (lda < (n > 1 ? n : 1)) return -7;
    if (!ipiv && n) return -8;
    if (!B && n && nrhs) return -9;
    if (ldb < (n > 1 ? n : 1)) return -10;
    if (n == 0 || nrhs == 0) return OZLU_OK;
    if (cudaSetDevice(h->device) != cudaSuccess) return OZLU_ERR_CUDA;
    cudaStream_t s = h->stream;
    LuScratch* sc;
    int rc0 = lu_scratch(h, &sc);
    if (rc0) return rc0;
    if ((rc0 = clear_err_word(h))) return rc0;
    const bool dL = is_device_ptr(LU), dP = is_device_ptr(ipiv), dB = is_device_ptr(B);
    if (opts && opts->graph && dL && dP && dB)  // graph capture and replay
        return ozlu_getrs_batched(h, nc, p, 1, &n, nrhs, &LU, &lda, &ipiv, &B, &ldb, opts);
    const size_t lbytes = sizeof(double) * nc * (size_t)lda * n;
    const size_t bbytes = sizeof(double) * nc * (size_t)ldb * nrhs;
    const double* gL = LU;
    const int* gP = ipiv;
    double* gB = B;
    int rc = 0;
    if (!dL || !dP || !dB) {
        rc = h->stage.ensure(align256(lbytes) + align256(bbytes) + sizeof(int) * (size_t)n + 256);
        if (rc) return rc;
        char* base = (char*)h->stage.base;
        if (!dL) { gL = (double*)base; if (cudaMemcpyAsync((void*)gL, LU, lbytes, cudaMemcpyHostToDevice, s)) return OZLU_ERR_CUDA; }
        if (!dB) { gB = (double*)(base + align256(lbytes)); if (cudaMemcpyAsync(gB, B, bbytes, cudaMemcpyHostToDevice, s)) return OZLU_ERR_CUDA; }
        if (!dP) {
            int* t = (int*)(base + align256(lbytes) + align256(bbytes));
            if (cudaMemcpyAsync(t, ipiv, sizeof(int) * n, cudaMemcpyHostToDevice, s)) return OZLU_ERR_CUDA;
            gP = t;
        }
    }
    switch (nc) {
        case 2: rc = getrs_device<2>(h, p, n, nrhs, (double*)gL, lda, gP, gB, ldb, opts, sc); break;
        case 3: rc = getrs_device<3>(h, p, n, nrhs, (double*)gL, lda, gP, gB, ldb, opts, sc); break;
        default: rc = getrs_device<4>(h, p, n, nrhs, (double*)gL, lda, gP, gB, ldb, opts, sc); break;
    }
    if (rc) return rc;
    if (!dB && cudaMemcpyAsync(B, gB, bbytes, cudaMemcpyDeviceToHost, s)) return OZLU_ERR_CUDA;
    if (!dL || !dP || !dB) return cuda_rc(cudaStreamSynchronize(s));
    return OZLU_OK;
}
