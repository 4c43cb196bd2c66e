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

#include "expansion.cuh"
#include "ozlu_handle.h"

namespace ozlu {
namespace {

constexpr int BASE = 32;        // base-block width of the recursion
constexpr int PIV_THREADS = 256;
constexpr int PIV_BLOCKS = 152;

struct LuScratch {
    double recip[4];
    double pivot[4];
    int piv;
    int zero;
    unsigned int counter;
    int info;
    double pval[PIV_BLOCKS][4];
    int pidx[PIV_BLOCKS];
};

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
    if (threadIdx.x == 0) {
        Exp<N> b;
        int ib = -1;
#pragma unroll
        for (int q = 0; q < N; ++q) b.x[q] = 0.0;
        for (int k = 0; k < (int)gridDim.x; ++k) {
            Exp<N> v;
#pragma unroll
            for (int q = 0; q < N; ++q) v.x[q] = ((volatile double*)sc->pval[k])[q];
            const int iv = ((volatile int*)sc->pidx)[k];
            if (better<N>(v, iv, b, ib)) { b = v; ib = iv; }
        }
        if (ib < 0) ib = c;
        piv = ib;
        sc->piv = ib;
        ipiv[c] = ib + 1;
        sc->counter = 0;
        const bool zero = b.x[0] == 0.0;
        sc->zero = zero ? 1 : 0;
        if (zero && sc->info == 0) sc->info = c + 1;
        if (!zero) {
            Exp<N> one;
            one.x[0] = 1.0;
#pragma unroll
            for (int q = 1; q < N; ++q) one.x[q] = 0.0;
            Exp<N> r = div<N>(one, b);
            store<N>(sc->recip, r);
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

// Rows i in (c, n): l_i = a_ic / pivot (times the reciprocal), then
// a_ik -= l_i a_ck for k in (c, c1).
template <int N>
__global__ void __launch_bounds__(128) scale_update_kernel(double* A, long long lda, int n, int c,
                                                           int c1, const LuScratch* sc) {
    __shared__ double urow[BASE][N];
    const int cols = c1 - c - 1;
    for (int k = threadIdx.x; k < cols; k += blockDim.x)
#pragma unroll
        for (int q = 0; q < N; ++q) urow[k][q] = elem(A, lda, N, c, c + 1 + k)[q];
    __syncthreads();
    if (sc->zero) return;
    const int i = c + 1 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Exp<N> r = load<N>(sc->recip);
    double* ai = elem(A, lda, N, i, c);
    const Exp<N> l = mul<N>(load<N>(ai), r);
    store<N>(ai, l);
    for (int k = 0; k < cols; ++k) {
        Exp<N> u;
#pragma unroll
        for (int q = 0; q < N; ++q) u.x[q] = urow[k][q];
        double* a = elem(A, lda, N, i, c + 1 + k);
        store<N>(a, fms<N>(load<N>(a), l, u));
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

// X <- L^-1 X for a unit lower (lower = 1) or U^-1 X for an upper (lower = 0,
// non-unit) b x b triangle, b <= BASE; X is b x ncols.  A block holds 32
// columns; thread (tx, ty) owns column tx and rows ty, ty + 8, ...
template <int N>
__global__ void __launch_bounds__(256) trsm_base_kernel(const double* T, long long ldt, double* X,
                                                        long long ldx, int b, int ncols, int lower) {
    extern __shared__ double sm[];
    double* sl = sm;                       // b x b triangle, [i][k][q]
    double* sx = sm + BASE * BASE * N;     // b x 32 block of X, [i][col][q]
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + tx;
    for (int idx = threadIdx.x; idx < b * b; idx += blockDim.x) {
        const int i = idx / b, k = idx % b;
#pragma unroll
        for (int q = 0; q < N; ++q) sl[(i * BASE + k) * N + q] = T[((long long)i + (long long)k * ldt) * N + q];
    }
    for (int i = ty; i < b; i += 8)
#pragma unroll
        for (int q = 0; q < N; ++q)
            sx[(i * 32 + tx) * N + q] = col < ncols ? X[((long long)i + (long long)col * ldx) * N + q] : 0.0;
    __syncthreads();
    for (int s = 0; s < b; ++s) {
        const int k = lower ? s : b - 1 - s;
        if (!lower && ty == 0) {
            // x_k /= u_kk
            Exp<N> d, x;
#pragma unroll
            for (int q = 0; q < N; ++q) { d.x[q] = sl[(k * BASE + k) * N + q]; x.x[q] = sx[(k * 32 + tx) * N + q]; }
            if (d.x[0] != 0.0) x = div<N>(x, d);
#pragma unroll
            for (int q = 0; q < N; ++q) sx[(k * 32 + tx) * N + q] = x.x[q];
        }
        __syncthreads();
        Exp<N> xk;
#pragma unroll
        for (int q = 0; q < N; ++q) xk.x[q] = sx[(k * 32 + tx) * N + q];
        for (int i = ty; i < b; i += 8) {
            if ((lower && i > k) || (!lower && i < k)) {
                Exp<N> lik, xi;
#pragma unroll
                for (int q = 0; q < N; ++q) { lik.x[q] = sl[(i * BASE + k) * N + q]; xi.x[q] = sx[(i * 32 + tx) * N + q]; }
                xi = fms<N>(xi, lik, xk);
#pragma unroll
                for (int q = 0; q < N; ++q) sx[(i * 32 + tx) * N + q] = xi.x[q];
            }
        }
        __syncthreads();
    }
    if (col < ncols)
        for (int i = ty; i < b; i += 8)
#pragma unroll
            for (int q = 0; q < N; ++q) X[((long long)i + (long long)col * ldx) * N + q] = sx[(i * 32 + tx) * N + q];
}

template <int N>
void trsm_base(const double* T, long long ldt, double* X, long long ldx, int b, int ncols, int lower,
               cudaStream_t s) {
    if (ncols <= 0 || b <= 0) return;
    const size_t smem = sizeof(double) * N * (BASE * BASE + BASE * 32);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(trsm_base_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    trsm_base_kernel<N><<<(ncols + 31) / 32, 256, smem, s>>>(T, ldt, X, ldx, b, ncols, lower);
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

template <int N>
void trsm_rec(Ctx& c, long long r, int b, long long j0, int ncols, bool lower) {
    if (c.rc || ncols <= 0) return;
    if (b <= BASE) {
        c.h->phase(PH_PANEL);
        trsm_base<N>(at(c, r, r), c.lda, at(c, r, j0), c.lda, b, ncols, lower ? 1 : 0, c.h->stream);
        c.h->count(1);
        return;
    }
    const int b1 = b / 2;
    if (lower) {
        trsm_rec<N>(c, r, b1, j0, ncols, true);
        c.rc = c.rc ? c.rc : gemm_device(c.h, N, c.p, b - b1, ncols, b1, -1, at(c, r + b1, r), c.lda,
                                         at(c, r, j0), c.lda, 1, at(c, r + b1, j0), c.lda, c.opts);
        trsm_rec<N>(c, r + b1, b - b1, j0, ncols, true);
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
    if (b <= BASE) {
        c.h->phase(PH_PANEL);
        c.h->count(2 * b);
        c.h->stats.panel_launches += 2 * b;
        for (int col = r; col < r + b; ++col) {
            const int rows = c.n - col;
            const int blocks = rows > PIV_THREADS * PIV_BLOCKS ? PIV_BLOCKS
                                                               : (rows + PIV_THREADS - 1) / PIV_THREADS;
            pivot_kernel<N><<<blocks, PIV_THREADS, 0, s>>>(c.A, c.lda, c.n, col, p0, p1, c.ipiv, c.sc);
            if (rows > 1)
                scale_update_kernel<N><<<(rows - 1 + 127) / 128, 128, 0, s>>>(c.A, c.lda, c.n, col,
                                                                              r + b, c.sc);
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
        if (r0 > 0) laswp_kernel<N><<<(r0 + 127) / 128, 128, 0, s>>>(A, lda, 0, r0, r0, r0 + b, ipiv);
        if (r0 + b < n)
            laswp_kernel<N><<<(n - r0 - b + 127) / 128, 128, 0, s>>>(A, lda, r0 + b, n, r0, r0 + b, ipiv);
        if (r0 + b < n) {
            // (P3) U12 = L11^-1 A12
            trsm_rec<N>(c, r0, b, r0 + b, n - r0 - b, true);
            // (P4) A22 <- A22 - L21 U12
            if (!c.rc)
                c.rc = gemm_device(h, N, p, n - r0 - b, n - r0 - b, b, -1, at(c, r0 + b, r0), lda,
                                   at(c, r0, r0 + b), lda, 1, at(c, r0 + b, r0 + b), lda, opts);
        }
    }
    h->phase(-1);
    if (!c.rc && cudaGetLastError() != cudaSuccess) c.rc = OZLU_ERR_CUDA;
    return c.rc;
}

template <int N>
int getrs_device(ozlu_handle* h, int p, int n, int nrhs, double* LU, long long lda, const int* ipiv,
                 double* B, long long ldb, const ozlu_opts* opts) {
    cudaStream_t s = h->stream;
    laswp_kernel<N><<<(nrhs + 127) / 128, 128, 0, s>>>(B, ldb, 0, nrhs, 0, n, ipiv);
    int rc = 0;
    auto L = [&](long long i, long long j) { return LU + (i + j * lda) * N; };
    auto X = [&](long long i) { return B + i * N; };
    h->phase(PH_PANEL);
    h->count(1 + 2 * ((n + BASE - 1) / BASE));
    for (int r = 0; r < n && !rc; r += BASE) {
        const int b = BASE < n - r ? BASE : n - r;
        trsm_base<N>(L(r, r), lda, X(r), ldb, b, nrhs, 1, s);
        if (r + b < n)
            rc = gemm_device(h, N, p, n - r - b, nrhs, b, -1, L(r + b, r), lda, X(r), ldb, 1,
                             X(r + b), ldb, opts);
    }
    const int last = ((n - 1) / BASE) * BASE;
    for (int r = last; r >= 0 && !rc; r -= BASE) {
        const int b = BASE < n - r ? BASE : n - r;
        trsm_base<N>(L(r, r), lda, X(r), ldb, b, nrhs, 0, s);
        if (r > 0)
            rc = gemm_device(h, N, p, r, nrhs, b, -1, L(0, r), lda, X(r), ldb, 1, X(0), ldb, opts);
    }
    h->phase(-1);
    if (!rc && cudaGetLastError() != cudaSuccess) rc = OZLU_ERR_CUDA;
    return rc;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

int lu_scratch(ozlu_handle* h, LuScratch** out) {
    if (!h->lu_scratch) {
        if (cudaMalloc(&h->lu_scratch, sizeof(LuScratch)) != cudaSuccess) {
            cudaGetLastError();
            return OZLU_ERR_NOMEM;
        }
    }
    *out = (LuScratch*)h->lu_scratch;
    return OZLU_OK;
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
    if (nb == 0) nb = 256;
    if (nb < 1) return -8;
    if (!info) return -9;
    if (cudaSetDevice(h->device) != cudaSuccess) return OZLU_ERR_CUDA;
    cudaStream_t s = h->stream;
    LuScratch* sc;
    int rc = lu_scratch(h, &sc);
    if (rc) return rc;
    if (cudaMemsetAsync(sc, 0, sizeof(LuScratch), s)) return OZLU_ERR_CUDA;
    const bool dA = is_device_ptr(A), dP = is_device_ptr(ipiv), dI = is_device_ptr(info);
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
    if (n > 0) {
        switch (nc) {
            case 2: rc = getrf_device<2>(h, p, n, gA, lda, gP, nb, sc, opts); break;
            case 3: rc = getrf_device<3>(h, p, n, gA, lda, gP, nb, sc, opts); break;
            default: rc = getrf_device<4>(h, p, n, gA, lda, gP, nb, sc, opts); break;
        }
    }
    if (rc) return rc;
    if (!dA && cudaMemcpyAsync(A, gA, abytes, cudaMemcpyDeviceToHost, s)) return OZLU_ERR_CUDA;
    if (n && gP != ipiv &&
        cudaMemcpyAsync(ipiv, gP, sizeof(int) * n, dP ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s))
        return OZLU_ERR_CUDA;
    if (cudaMemcpyAsync(info, &sc->info, sizeof(int), dI ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s))
        return OZLU_ERR_CUDA;
    if (!dA || !dP || !dI) return cuda_rc(cudaStreamSynchronize(s));
    return OZLU_OK;
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
    const bool dL = is_device_ptr(LU), dP = is_device_ptr(ipiv), dB = is_device_ptr(B);
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
        case 2: rc = getrs_device<2>(h, p, n, nrhs, (double*)gL, lda, gP, gB, ldb, opts); break;
        case 3: rc = getrs_device<3>(h, p, n, nrhs, (double*)gL, lda, gP, gB, ldb, opts); break;
        default: rc = getrs_device<4>(h, p, n, nrhs, (double*)gL, lda, gP, gB, ldb, opts); break;
    }
    if (rc) return rc;
    if (!dB && cudaMemcpyAsync(B, gB, bbytes, cudaMemcpyDeviceToHost, s)) return OZLU_ERR_CUDA;
    if (!dL || !dP || !dB) return cuda_rc(cudaStreamSynchronize(s));
    return OZLU_OK;
}
