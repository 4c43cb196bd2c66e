// LU with partial pivoting and the solve for p-bit multi-limb matrices
// (ozlu_mp_getrf / ozlu_mp_getrs, Sec. 3.4 at arbitrary precision).
//
// The factorisation is recursive down to single columns, so that all of its
// arithmetic except the pivot search is Ozaki-II GEMMs (ozlu_mp_gemm):
//   panel(r, b):  b = 1: pivot search (largest |a|, lowest row on ties), row
//                 interchange across the outer panel, reciprocal of the pivot
//                 (one block: Newton's iteration in fixed point from a
//                 binary64 start), and the scaling of the column below it
//                 (an m x 1 x 1 product);
//                 else: panel(r, b/2), L11^-1 A12 on the right half, the
//                 Schur update, panel(r + b/2, b - b/2)
//   blocked over nb columns: panel, interchanges on the other columns,
//   U12 = L11^-1 A12 (recursive, unit diagonal: no work at single rows),
//   A22 -= L21 U12.
// The solve applies P, then L^-1 and U^-1 recursively (division by a
// diagonal entry = reciprocal and scaling, as in the panel).
#include <math.h>
#include <string.h>

#include <utility>

#include "mp_device.cuh"
#include "ozlu_handle.h"

namespace ozlu {
namespace {

struct MPV {
    uint32_t* limbs;
    int* exps;
    int* signs;
    long long ld, plane;
    int L;
};

MPV dv(const ozlu_mp_matrix& M) { return MPV{M.limbs, M.exps, M.signs, M.ld, M.plane, M.L}; }

ozlu_mp_matrix sub(const ozlu_mp_matrix& M, long long i, long long j) {
    ozlu_mp_matrix r = M;
    const long long off = i + j * M.ld;
    r.limbs += off;
    r.exps += off;
    r.signs += off;
    return r;
}

// |x| vs |y| of two elements (maybe of different matrices with the same L)
__device__ int mp_abs_cmp(const MPV& A, long long x, const MPV& B, long long y) {
    const bool za = A.limbs[(long long)(A.L - 1) * A.plane + x] == 0;
    const bool zb = B.limbs[(long long)(B.L - 1) * B.plane + y] == 0;
    if (za || zb) return za && zb ? 0 : (za ? -1 : 1);
    if (A.exps[x] != B.exps[y]) return A.exps[x] > B.exps[y] ? 1 : -1;
    for (int k = A.L - 1; k >= 0; --k) {
        const uint32_t a = A.limbs[(long long)k * A.plane + x], b = B.limbs[(long long)k * B.plane + y];
        if (a != b) return a > b ? 1 : -1;
    }
    return 0;
}

// pivot of column c over rows [c, n): one block; ipiv[c] = piv + 1, info
constexpr int PT = 512;
__global__ void __launch_bounds__(PT) mp_pivot_kernel(MPV A, int n, int c, int* piv_out, int* ipiv, int* info) {
    __shared__ int best[PT];
    int bi = -1;
    for (int i = c + threadIdx.x; i < n; i += PT) {
        const long long x = (long long)i + (long long)c * A.ld;
        if (bi < 0 || mp_abs_cmp(A, x, A, (long long)bi + (long long)c * A.ld) > 0) bi = i;
    }
    best[threadIdx.x] = bi;
    __syncthreads();
    for (int s = PT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const int o = best[threadIdx.x + s], me = best[threadIdx.x];
            if (o >= 0) {
                int cmp = me < 0 ? 1 : mp_abs_cmp(A, (long long)o + (long long)c * A.ld, A, (long long)me + (long long)c * A.ld);
                if (cmp > 0 || (cmp == 0 && o < me)) best[threadIdx.x] = o;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int p = best[0] < 0 ? c : best[0];
        *piv_out = p;
        ipiv[c] = p + 1;
        const long long x = (long long)p + (long long)c * A.ld;
        if (A.limbs[(long long)(A.L - 1) * A.plane + x] == 0 && *info == 0) *info = c + 1;
        piv_out[1] = A.limbs[(long long)(A.L - 1) * A.plane + x] == 0 ? 1 : 0;  // zero pivot flag
    }
}

__device__ void swap_elem(const MPV& A, long long x, long long y) {
    for (int k = 0; k < A.L; ++k) {
        uint32_t* a = A.limbs + (long long)k * A.plane;
        const uint32_t t = a[x];
        a[x] = a[y];
        a[y] = t;
    }
    int t = A.exps[x];
    A.exps[x] = A.exps[y];
    A.exps[y] = t;
    t = A.signs[x];
    A.signs[x] = A.signs[y];
    A.signs[y] = t;
}

// rows r and *piv exchanged over columns [j0, j1)
__global__ void mp_swap_kernel(MPV A, int r, const int* piv, int j0, int j1) {
    const int j = j0 + blockIdx.x * blockDim.x + threadIdx.x;
    const int p = *piv;
    if (j >= j1 || p == r) return;
    swap_elem(A, (long long)r + (long long)j * A.ld, (long long)p + (long long)j * A.ld);
}

// interchanges k in [k0, k1) (ipiv 1-based) on columns [j0, j1), one column per thread
__global__ void mp_laswp_kernel(MPV A, int k0, int k1, const int* ipiv, int j0, int j1) {
    const int j = j0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= j1) return;
    for (int k = k0; k < k1; ++k) {
        const int p = ipiv[k] - 1;
        if (p != k) swap_elem(A, (long long)k + (long long)j * A.ld, (long long)p + (long long)j * A.ld);
    }
}

// Block-cooperative fixed-point arithmetic for the reciprocal of one p-bit
// number (one block of RT threads, words in shared memory).
constexpr int RT = 256;

// out[0, olen) = (X[0, nx) * Y[0, ny)) >> (32 shift), truncated: column sums
// of the 32-bit halves of the limb products by all threads (64-bit, below
// 2^(33 + log2 n)), then one thread propagates the carries
__device__ void blk_mul(const uint32_t* X, int nx, const uint32_t* Y, int ny, uint32_t* out, int shift, int olen,
                        unsigned long long* S) {
    const int ncol = nx + ny;
    for (int k = threadIdx.x; k < ncol; k += RT) {
        unsigned long long acc = 0;
        const int i0 = max(0, k - ny + 1), i1 = min(nx - 1, k);
        for (int i = i0; i <= i1; ++i) acc += (uint32_t)((uint64_t)X[i] * Y[k - i]);
        const int j0 = max(0, k - 1 - ny + 1), j1 = min(nx - 1, k - 1);
        for (int i = j0; i <= j1; ++i) acc += (uint64_t)X[i] * Y[k - 1 - i] >> 32;
        S[k] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long c = 0;
        for (int k = 0; k < ncol; ++k) {
            const unsigned long long v = S[k] + c;
            if (k >= shift && k - shift < olen) out[k - shift] = (uint32_t)v;
            c = v >> 32;
        }
        for (int k = ncol; k - shift < olen; ++k) {
            if (k >= shift) out[k - shift] = (uint32_t)c;
            c = 0;
        }
    }
    __syncthreads();
}

// 1 / (element x of A) into element 0 of R (R.L limbs; truncated) by
// Newton's iteration on the mantissa in fixed point: with f = |a| 2^-e in
// [1/2, 1) (F = its L limbs) and y ~ 1/f (Y = y 2^(32 W), W = R.L):
//   T = F Y 2^-(32 L) ~ f y 2^(32 W),  E = 2^(32 W) - T,  Y += Y E 2^-(32 W)
// from a binary64 start; `iters` steps double the 53 correct bits each.
__global__ void __launch_bounds__(RT) mp_recip_kernel(MPV A, long long x, MPV R, int iters) {
    extern __shared__ unsigned long long rsm[];
    const int La = A.L, W = R.L;
    unsigned long long* S = rsm;                          // La + 2 W + 4 column sums
    uint32_t* F = (uint32_t*)(S + La + 2 * W + 4);        // La
    uint32_t* Y = F + La;                                 // W + 1
    uint32_t* T = Y + W + 1;                              // W + 1
    uint32_t* U = T + W + 1;                              // W + 1
    for (int k = threadIdx.x; k < La; k += RT) F[k] = A.limbs[(long long)k * A.plane + x];
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t top = ((uint64_t)F[La - 1] << 32) | (La > 1 ? F[La - 2] : 0u);
        const double f = (double)(top >> 11) * 0x1p-53;
        int ey;
        const double fr = frexp(1.0 / f, &ey);         // 1/f = fr 2^ey, ey in {1, 2}
        const uint64_t m53 = (uint64_t)ldexp(fr, 53);  // 1/f = m53 2^(ey - 53)
        for (int k = 0; k <= W; ++k) Y[k] = 0;
        const int pos = 32 * W + ey - 53;             // bit of Y holding m53's bit 0
        const int q = pos >> 5, r = pos & 31;
        Y[q] = (uint32_t)(m53 << r);
        if (q + 1 <= W) Y[q + 1] = (uint32_t)(r ? (m53 >> (32 - r)) : (m53 >> 32));
        if (q + 2 <= W && r) Y[q + 2] = (uint32_t)(m53 >> (64 - r));
    }
    __syncthreads();
    for (int it = 0; it < iters; ++it) {
        blk_mul(F, La, Y, W + 1, T, La, W + 1, S);      // T = F Y >> 32 La
        if (threadIdx.x == 0) {
            // E = 2^(32 W) - T (two's complement in W + 1 words), sign, |E| into T
            uint64_t c = 1;
            for (int k = 0; k <= W; ++k) {
                const uint32_t o = k == W ? 1u : 0u;
                const uint64_t v = (uint64_t)o + (uint32_t)~T[k] + c;
                T[k] = (uint32_t)v;
                c = v >> 32;
            }
            const bool eneg = (T[W] >> 31) != 0;
            if (eneg) {
                uint64_t c2 = 1;
                for (int k = 0; k <= W; ++k) {
                    const uint64_t v = (uint64_t)(uint32_t)~T[k] + c2;
                    T[k] = (uint32_t)v;
                    c2 = v >> 32;
                }
            }
            U[0] = eneg ? 1u : 0u;  // sign, read below
        }
        __syncthreads();
        const bool eneg = U[0] != 0;
        __syncthreads();
        blk_mul(Y, W + 1, T, W + 1, U, W, W + 1, S);     // U = Y |E| >> 32 W
        if (threadIdx.x == 0) {
            uint64_t c = eneg ? 1u : 0u;
            for (int k = 0; k <= W; ++k) {
                const uint32_t u = eneg ? ~U[k] : U[k];
                const uint64_t v = (uint64_t)Y[k] + u + c;
                Y[k] = (uint32_t)v;
                c = v >> 32;
            }
        }
        __syncthreads();
    }
    // normalise Y (value y 2^(32 W), y in (1, 2]) into R's W limbs, truncating
    if (threadIdx.x == 0) {
        int b = 0;
        for (int k = W; k >= 0; --k)
            if (Y[k]) {
                b = 32 * k + 32 - __clz(Y[k]);
                break;
            }
        const int first = b - 32 * W;  // Y bit at R's limb 0, bit 0
        for (int k = 0; k < W; ++k) {
            const int pos = first + 32 * k;
            const int q = pos >> 5, r = pos & 31;
            const uint32_t lo = (q >= 0 && q <= W) ? Y[q] : 0u, hi = (q + 1 >= 0 && q + 1 <= W) ? Y[q + 1] : 0u;
            R.limbs[(long long)k * R.plane] = r ? (lo >> r) | (hi << (32 - r)) : lo;
        }
        R.exps[0] = b - 32 * W - A.exps[x];
        R.signs[0] = A.signs[x];
    }
}

// copy an m x n block (D, S with the same L)
__global__ void mp_copy_kernel(MPV S, MPV D, int m, int n) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)m * n) return;
    const long long i = e % m, j = e / m;
    const long long xs = i + j * S.ld, xd = i + j * D.ld;
    for (int k = 0; k < D.L; ++k) D.limbs[(long long)k * D.plane + xd] = S.limbs[(long long)k * S.plane + xs];
    D.exps[xd] = S.exps[xs];
    D.signs[xd] = S.signs[xs];
}

// scratch p-bit elements of one factorisation or solve: x, y, z, two (one
// element each, L + 1 limbs) and a block of up to `cnt` elements (L limbs)
struct Scratch {
    ozlu_mp_matrix x, y, z, two, blk;
    int* piv = nullptr;  // device: pivot row, zero-pivot flag
    void* mem = nullptr;
    int alloc(int L, long long cnt) {
        const int L1 = L + 1;
        const size_t words = 4 * ((size_t)L1 + 2) + ((size_t)L + 2) * (size_t)cnt + 16;
        if (!dev_alloc(&mem, words * 4)) {
            mem = nullptr;
            return OZLU_ERR_NOMEM;
        }
        uint32_t* w = (uint32_t*)mem;
        auto one = [&](ozlu_mp_matrix& M, int LL, long long c) {
            M.limbs = w;
            w += (size_t)LL * c;
            M.exps = (int*)w;
            w += c;
            M.signs = (int*)w;
            w += c;
            M.ld = c;
            M.plane = c;
            M.L = LL;
            M.pad_ = 0;
        };
        one(x, L1, 1);
        one(y, L1, 1);
        one(z, L1, 1);
        one(two, L1, 1);
        one(blk, L, cnt);
        piv = (int*)w;
        return OZLU_OK;
    }
    ~Scratch() {
        if (mem) cudaFree(mem);
    }
};

struct Ctx {
    ozlu_handle* h;
    int p;
    ozlu_mp_matrix A;
    int n;
    int* ipiv;
    int* info;
    Scratch* sc;
    int rc = 0;
};

// 1 / M(i, j) into sc->x (L + 1 limbs, correct to about p + 32 bits)
int mp_reciprocal(Ctx& c, const ozlu_mp_matrix& M, long long i, long long j) {
    const int W = c.sc->x.L, La = M.L;
    int iters = 0;
    for (int prec = 53; prec < c.p + 40; prec *= 2) ++iters;
    const size_t smem = sizeof(unsigned long long) * (La + 2 * W + 4) + sizeof(uint32_t) * (La + 3 * (W + 1));
    cudaFuncSetAttribute(mp_recip_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    mp_recip_kernel<<<1, RT, smem, c.h->stream>>>(dv(M), i + j * M.ld, dv(c.sc->x), iters);
    c.h->count(1);
    return cudaGetLastError() == cudaSuccess ? OZLU_OK : OZLU_ERR_CUDA;
}

// rows [r0, r0 + m) x columns [j0, j0 + nc) of A scaled by sc->x (through
// the scratch block): A <- A * x
int mp_scale(Ctx& c, const ozlu_mp_matrix& M, long long r0, long long j0, int m, int nc, bool row_vector) {
    if (m <= 0 || nc <= 0) return OZLU_OK;
    cudaStream_t s = c.h->stream;
    Scratch& sc = *c.sc;
    ozlu_mp_matrix blk = sc.blk;
    blk.ld = m;
    int rc;
    if (!row_vector) {
        // column (m x 1) times x (1 x 1)
        rc = mp_gemm_device(c.h, c.p, m, 1, 1, 1, sub(M, r0, j0), sc.x, 0, blk);
    } else {
        // x (1 x 1) times a row (1 x nc)
        blk.ld = 1;
        rc = mp_gemm_device(c.h, c.p, 1, nc, 1, 1, sc.x, sub(M, r0, j0), 0, blk);
    }
    if (rc) return rc;
    const long long cnt = (long long)m * nc;
    mp_copy_kernel<<<(unsigned)((cnt + 127) / 128), 128, 0, s>>>(dv(blk), dv(sub(M, r0, j0)), m, nc);
    c.h->count(1);
    return cudaGetLastError() == cudaSuccess ? OZLU_OK : OZLU_ERR_CUDA;
}

// X <- L11^-1 X, L11 the unit lower b x b block at (r, r) of M, X = M rows
// [r, r + b) x columns [j0, j0 + ncols) (or of another matrix X)
void mp_trsm_lower(Ctx& c, const ozlu_mp_matrix& M, long long r, int b, const ozlu_mp_matrix& X, long long xr,
                   long long j0, int ncols) {
    if (c.rc || b <= 1 || ncols <= 0) return;
    const int b1 = b / 2;
    mp_trsm_lower(c, M, r, b1, X, xr, j0, ncols);
    if (!c.rc)
        c.rc = mp_gemm_device(c.h, c.p, b - b1, ncols, b1, -1, sub(M, r + b1, r), sub(X, xr, j0), 1,
                              sub(X, xr + b1, j0));
    mp_trsm_lower(c, M, r + b1, b - b1, X, xr + b1, j0, ncols);
}

// X <- U11^-1 X, U11 the upper b x b block at (r, r) of M
void mp_trsm_upper(Ctx& c, const ozlu_mp_matrix& M, long long r, int b, const ozlu_mp_matrix& X, long long xr,
                   long long j0, int ncols) {
    if (c.rc || b <= 0 || ncols <= 0) return;
    if (b == 1) {
        c.rc = mp_reciprocal(c, M, r, r);
        if (!c.rc) c.rc = mp_scale(c, X, xr, j0, 1, ncols, true);
        return;
    }
    const int b1 = b / 2;
    mp_trsm_upper(c, M, r + b1, b - b1, X, xr + b1, j0, ncols);
    if (!c.rc)
        c.rc = mp_gemm_device(c.h, c.p, b1, ncols, b - b1, -1, sub(M, r, r + b1), sub(X, xr + b1, j0), 1,
                              sub(X, xr, j0));
    mp_trsm_upper(c, M, r, b1, X, xr, j0, ncols);
}

// factor columns [r, r + b), rows [r, n); interchanges across [p0, p1)
void mp_panel(Ctx& c, int r, int b, int p0, int p1) {
    if (c.rc) return;
    cudaStream_t s = c.h->stream;
    if (b == 1) {
        mp_pivot_kernel<<<1, PT, 0, s>>>(dv(c.A), c.n, r, c.sc->piv, c.ipiv, c.info);
        mp_swap_kernel<<<(p1 - p0 + 127) / 128, 128, 0, s>>>(dv(c.A), r, c.sc->piv, p0, p1);
        c.h->count(2);
        // the zero-pivot flag is on the device: skip the scaling only when the
        // pivot is exactly zero (the host cannot see it without a sync), so
        // the reciprocal of a zero pivot is avoided by checking on the host
        // once per column (a short copy; factorisations of singular matrices
        // keep going as in LAPACK)
        int flag = 0;
        if (cudaMemcpyAsync(&flag, c.sc->piv + 1, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            c.rc = OZLU_ERR_CUDA;
            return;
        }
        if (flag) return;
        c.rc = mp_reciprocal(c, c.A, r, r);
        if (!c.rc) c.rc = mp_scale(c, c.A, r + 1, r, c.n - r - 1, 1, false);
        return;
    }
    const int b1 = b / 2;
    mp_panel(c, r, b1, p0, p1);
    mp_trsm_lower(c, c.A, r, b1, c.A, r, r + b1, b - b1);
    if (!c.rc && c.n - r - b1 > 0)
        c.rc = mp_gemm_device(c.h, c.p, c.n - r - b1, b - b1, b1, -1, sub(c.A, r + b1, r), sub(c.A, r, r + b1), 1,
                              sub(c.A, r + b1, r + b1));
    mp_panel(c, r + b1, b - b1, p0, p1);
}

bool mp_ok(const ozlu_mp_matrix* M, int p, int rows, int cols) {
    if (!M || M->L < 1 || 32LL * M->L < p) return false;
    if (rows == 0 || cols == 0) return true;
    if (!M->limbs || !M->exps || !M->signs) return false;
    if (M->ld < (rows > 1 ? rows : 1) || M->plane < M->ld * (long long)cols) return false;
    return is_device_ptr(M->limbs) && is_device_ptr(M->exps) && is_device_ptr(M->signs);
}

}  // namespace
}  // namespace ozlu

using namespace ozlu;

extern "C" int ozlu_mp_getrf(ozlu_handle* h, int p, int n, const ozlu_mp_matrix* A, int* ipiv, int nb,
                             int* info) {
    if (!h) return -1;
    if (p < 1) return -2;
    if (n < 0) return -3;
    if (!mp_ok(A, p, n, n)) return -4;
    if (n && (!ipiv || !is_device_ptr(ipiv))) return -5;
    if (nb == 0) nb = 128;
    if (nb < 1) return -6;
    if (!info || !is_device_ptr(info)) return -7;
    if (cudaSetDevice(h->device) != cudaSuccess) return OZLU_ERR_CUDA;
    cudaStream_t s = h->stream;
    if (cudaMemsetAsync(info, 0, sizeof(int), s) != cudaSuccess) return OZLU_ERR_CUDA;
    if (n == 0) return OZLU_OK;
    Scratch sc;
    int rc = sc.alloc(A->L, n);
    if (rc) return rc;
    Ctx c{h, p, *A, n, ipiv, info, &sc};
    for (int r0 = 0; r0 < n && !c.rc; r0 += nb) {
        const int b = nb < n - r0 ? nb : n - r0;
        mp_panel(c, r0, b, r0, r0 + b);
        if (c.rc) break;
        // interchanges of this panel on the columns left and right of it
        if (r0 > 0) mp_laswp_kernel<<<(r0 + 127) / 128, 128, 0, s>>>(dv(c.A), r0, r0 + b, ipiv, 0, r0);
        if (r0 + b < n)
            mp_laswp_kernel<<<(n - r0 - b + 127) / 128, 128, 0, s>>>(dv(c.A), r0, r0 + b, ipiv, r0 + b, n);
        h->count(2);
        if (r0 + b < n) {
            mp_trsm_lower(c, c.A, r0, b, c.A, r0, r0 + b, n - r0 - b);
            if (!c.rc)
                c.rc = mp_gemm_device(h, p, n - r0 - b, n - r0 - b, b, -1, sub(c.A, r0 + b, r0), sub(c.A, r0, r0 + b),
                                      1, sub(c.A, r0 + b, r0 + b));
        }
    }
    if (!c.rc && cudaStreamSynchronize(s) != cudaSuccess) c.rc = OZLU_ERR_CUDA;
    return c.rc;
}

extern "C" int ozlu_mp_getrs(ozlu_handle* h, int p, int n, int nrhs, const ozlu_mp_matrix* LU, const int* ipiv,
                             const ozlu_mp_matrix* B) {
    if (!h) return -1;
    if (p < 1) return -2;
    if (n < 0) return -3;
    if (nrhs < 0) return -4;
    if (!mp_ok(LU, p, n, n)) return -5;
    if (n && (!ipiv || !is_device_ptr(ipiv))) return -6;
    if (!mp_ok(B, p, n, nrhs)) return -7;
    if (n == 0 || nrhs == 0) return OZLU_OK;
    if (cudaSetDevice(h->device) != cudaSuccess) return OZLU_ERR_CUDA;
    cudaStream_t s = h->stream;
    Scratch sc;
    int rc = sc.alloc(B->L, nrhs > n ? nrhs : n);
    if (rc) return rc;
    Ctx c{h, p, *LU, n, const_cast<int*>(ipiv), nullptr, &sc};
    mp_laswp_kernel<<<(nrhs + 127) / 128, 128, 0, s>>>(dv(*B), 0, n, ipiv, 0, nrhs);
    h->count(1);
    mp_trsm_lower(c, *LU, 0, n, *B, 0, 0, nrhs);
    mp_trsm_upper(c, *LU, 0, n, *B, 0, 0, nrhs);
    if (!c.rc && cudaStreamSynchronize(s) != cudaSuccess) c.rc = OZLU_ERR_CUDA;
    return c.rc;
}
