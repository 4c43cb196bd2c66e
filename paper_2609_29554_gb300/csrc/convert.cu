// (S1) shared exponents and (S2)+(S3) fused conversion of expansions to
// centered residue planes (Sec. 3.1, Sec. 3.2 Eq. (2), Sec. 3.3 Eq. (12)).
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <limits.h>

#include "mp_device.cuh"
#include "ozlu_internal.h"

namespace ozlu {
namespace {

constexpr int NO_EXP = INT_MIN;

// mu_i = (Q-1) - max_h frexp_exp(a_ih[0]); 0 for an all-zero row.
// Block of 32 rows x 8 lanes along h (consecutive rows are adjacent in memory).
__global__ void __launch_bounds__(256) row_shift_kernel(const double* __restrict__ A, long long lda,
                                                        int nc, int m, int k, int Q,
                                                        int* __restrict__ mu) {
    __shared__ int red[8][32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + tx;
    int E = NO_EXP;
    if (i < m)
        for (int h = ty; h < k; h += 8) {
            const double x = A[((long long)i + (long long)h * lda) * nc];
            if (x != 0.0) E = max(E, frexp_exp(x));
        }
    red[ty][tx] = E;
    __syncthreads();
    if (ty == 0 && i < m) {
#pragma unroll
        for (int r = 1; r < 8; ++r) E = max(E, red[r][tx]);
        mu[i] = E == NO_EXP ? 0 : (Q - 1) - E;
    }
}

// nu_j over column j of B (k x n): one warp per column.
__global__ void col_shift_kernel(const double* __restrict__ B, long long ldb, int nc, int k,
                                 int n, int Q, int* __restrict__ nu) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    int E = NO_EXP;
    const double* col = B + (long long)warp * ldb * nc;
    for (int h = lane; h < k; h += 32) {
        const double x = col[(long long)h * nc];
        if (x != 0.0) E = max(E, frexp_exp(x));
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) E = max(E, __shfl_xor_sync(0xffffffffu, E, o));
    if (lane == 0) nu[warp] = E == NO_EXP ? 0 : (Q - 1) - E;
}

constexpr int MAXD = 9;  // words of one balanced digit (w + 2 bits)

// Residue of sign * mag (mag < 2^(16 H)) modulo m, centered (S3):
// r in [-floor(m/2), ceil(m/2) - 1].  H (16-bit halves) is a template
// parameter so the sum unrolls exactly.
template <int H>
__device__ __forceinline__ int centered_residue(const uint32_t (&mag)[MAXD], bool neg,
                                                const DevTable& tab, int l) {
    const uint32_t m = (uint32_t)tab.mod[l];
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const uint32_t half = (mag[j >> 1] >> (16 * (j & 1))) & 0xffffu;
        acc += half * tab.pow16[l][j];
    }
    uint32_t r = mod_small(acc, m, tab.magic[l]);
    if (neg && r) r = m - r;
    int c = (int)r;
    if (c > (int)(m - 1) / 2) c -= (int)m;
    return c;
}

// One element per thread: x -> X = Eq. (12) -> S balanced digits (Eq. (2)) ->
// centered residues for every modulus, written to the int8 planes.
//   A side (is_b = 0): element (r, h) of an R x K matrix, plane [l][t][r][h]
//   B side (is_b = 1): element (h, r) of a K x R matrix, plane [l][t][r][h]
// Threads cover [0, R) x [0, Kpad) and write zeros in the K padding; the
// padded rows are left as they are (they only reach discarded outputs).
// store residue r of plane (l, t) at element offset off, in the back-end's encoding
// Residue modulo a binary64-back-end prime (m < 2^27): 64-bit sum of the
// half products, then one 64-bit remainder.
template <int H>
__device__ __forceinline__ int centered_residue64(const uint32_t (&mag)[MAXD], bool neg,
                                                  const DevTable& tab, int l) {
    const uint64_t m = (uint64_t)tab.mod[l];
    uint64_t acc = 0;
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const uint64_t half = (mag[j >> 1] >> (16 * (j & 1))) & 0xffffu;
        acc += half * tab.pow16[l][j];
    }
    uint64_t r = acc % m;
    if (neg && r) r = m - r;
    long long c = (long long)r;
    if (c > (long long)(m - 1) / 2) c -= (long long)m;
    return (int)c;
}

template <int MODE>
__device__ __forceinline__ void put_residue(void* planes, size_t plane, int l, int S, int t,
                                            size_t off, int r) {
    if (MODE == 3) {
        ((double*)planes)[(size_t)(l * S + t) * plane + off] = (double)r;
    } else if (MODE == 0) {
        ((int8_t*)planes)[(size_t)(l * S + t) * plane + off] = (int8_t)r;
    } else if (MODE == 1) {
        // Eq. (15): r = 17 d1 + d0, d1 = round(r / 17) (no ties: 17 is odd)
        const int d1 = (2 * r + 17 + 238) / 34 - 7;
        const int d0 = r - 17 * d1;
        uint8_t* p8 = (uint8_t*)planes + (size_t)((l * S + t) * 3) * plane + off;
        p8[0] = (uint8_t)__nv_cvt_float_to_fp8((float)d0, __NV_SATFINITE, __NV_E4M3);
        p8[plane] = (uint8_t)__nv_cvt_float_to_fp8((float)d1, __NV_SATFINITE, __NV_E4M3);
        p8[2 * plane] = (uint8_t)__nv_cvt_float_to_fp8((float)(d0 + d1), __NV_SATFINITE, __NV_E4M3);
    } else {
        ((__half*)planes)[(size_t)(l * S + t) * plane + off] = __int2half_rn(r);
    }
}

template <int MODE, int H>
__global__ void __launch_bounds__(256) convert_kernel(
    const double* __restrict__ X, long long ld, int nc, int R, int K, int is_b,
    const int* __restrict__ shifts, const __grid_constant__ DevTable tab, int Kpad, int Rpad,
    void* __restrict__ planes) {
    const int h = blockIdx.x * 32 + (threadIdx.x & 31);
    const int r = blockIdx.y * 8 + (threadIdx.x >> 5);
    if (h >= Kpad || r >= R) return;
    const size_t plane = (size_t)Rpad * Kpad;
    const size_t off = (size_t)r * Kpad + h;
    if (h >= K) {
        for (int l = 0; l < tab.N; ++l)
            for (int t = 0; t < tab.S; ++t) put_residue<MODE>(planes, plane, l, tab.S, t, off, 0);
        return;
    }
    const double* x = is_b ? X + ((long long)h + (long long)r * ld) * nc
                           : X + ((long long)r + (long long)h * ld) * nc;
    const int shift = shifts[r];
    uint32_t V[MAXWX];
#pragma unroll
    for (int wd = 0; wd < MAXWX; ++wd) V[wd] = 0;
    for (int c = 0; c < nc; ++c) add_component<MAXWX>(V, x[c], shift);

    const int w = tab.w, S = tab.S;
    const int nw = (w + 2 + 31) >> 5;  // words of a digit with its carry
    uint32_t carry = 0;
    for (int t = 0; t < S; ++t) {
        uint32_t D[MAXD];
#pragma unroll
        for (int k2 = 0; k2 < MAXD; ++k2) D[k2] = 0;
        bool neg = false;
        if (t < S - 1) {
            // unsigned field [t w, t w + w) plus the incoming carry
#pragma unroll
            for (int k2 = 0; k2 < MAXD; ++k2)
                if (k2 < nw) D[k2] = field32<MAXWX>(V, t * w + 32 * k2);
            mask_below<MAXD>(D, w);
            uint64_t c = carry;
#pragma unroll
            for (int k2 = 0; k2 < MAXD; ++k2) {
                const uint64_t s = (uint64_t)D[k2] + c;
                D[k2] = (uint32_t)s;
                c = s >> 32;
            }
            // balanced: D >= 2^(w-1) -> digit D - 2^w (negative), carry out 1
            const bool big = bit_at<MAXD>(D, w - 1) || bit_at<MAXD>(D, w);
            if (big) {
                complement_below<MAXD>(D, w);  // |digit| = 2^w - D (0 when D = 2^w)
                neg = true;
                carry = 1;
            } else {
                carry = 0;
            }
            // D = 2^w exactly (field all ones plus carry) gives digit 0
        } else {
            // top digit: signed field from bit t w upward, plus the carry
            uint32_t T[MAXD + 1];
#pragma unroll
            for (int k2 = 0; k2 <= MAXD; ++k2) T[k2] = field32<MAXWX>(V, t * w + 32 * k2);
            uint64_t c = carry;
#pragma unroll
            for (int k2 = 0; k2 <= MAXD; ++k2) {
                const uint64_t s = (uint64_t)T[k2] + c;
                T[k2] = (uint32_t)s;
                c = s >> 32;
            }
            neg = (T[MAXD] >> 31) != 0;
            if (neg) negate<MAXD + 1>(T);
#pragma unroll
            for (int k2 = 0; k2 < MAXD; ++k2) D[k2] = T[k2];
        }
        for (int l = 0; l < tab.N; ++l) {
            const int res = MODE == 3 ? centered_residue64<H>(D, neg, tab, l) : centered_residue<H>(D, neg, tab, l);
            put_residue<MODE>(planes, plane, l, S, t, off, res);
        }
    }
}

}  // namespace

void launch_row_shifts(const double* A, long long lda, int nc, int m, int k, int Q, int* mu,
                       cudaStream_t s) {
    if (m <= 0) return;
    row_shift_kernel<<<(m + 31) / 32, 256, 0, s>>>(A, lda, nc, m, k, Q, mu);
}

void launch_col_shifts(const double* B, long long ldb, int nc, int k, int n, int Q, int* nu,
                       cudaStream_t s) {
    if (n <= 0) return;
    const int warps_per_block = 8;
    col_shift_kernel<<<(n + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(
        B, ldb, nc, k, n, Q, nu);
}

void launch_convert(const double* X, long long ld, int nc, int rows, int cols, bool is_b,
                    const int* shifts, const DevTable& tab, int Kpad, int Rpad, void* planes,
                    int mode, cudaStream_t s) {
    // A side: rows = R, cols = K; B side: rows = K, cols = R
    const int R = is_b ? cols : rows;
    const int K = is_b ? rows : cols;
    // rows [0, R) only: padded rows only feed padded output rows and columns,
    // which the epilogue discards; the padded K columns must be zero
    dim3 grid((Kpad + 31) / 32, (R + 7) / 8);
    if (R == 0) return;
    switch (mode * 32 + tab.H) {
#define OZLU_CONV(M, HH) \
    case M * 32 + HH: \
        convert_kernel<M, HH><<<grid, 256, 0, s>>>(X, ld, nc, R, K, is_b ? 1 : 0, shifts, tab, Kpad, Rpad, planes); \
        break;
#define OZLU_CONV_M(M) OZLU_CONV(M, 2) OZLU_CONV(M, 3) OZLU_CONV(M, 4) OZLU_CONV(M, 5) OZLU_CONV(M, 6) \
    OZLU_CONV(M, 7) OZLU_CONV(M, 8) OZLU_CONV(M, 9) OZLU_CONV(M, 10) OZLU_CONV(M, 11) OZLU_CONV(M, 12) \
    OZLU_CONV(M, 13) OZLU_CONV(M, 14) OZLU_CONV(M, 15) OZLU_CONV(M, 16)
        OZLU_CONV_M(0)
        OZLU_CONV_M(1)
        OZLU_CONV_M(2)
        OZLU_CONV_M(3)
#undef OZLU_CONV_M
#undef OZLU_CONV
        default:
            convert_kernel<0, 16><<<grid, 256, 0, s>>>(X, ld, nc, R, K, is_b ? 1 : 0, shifts, tab, Kpad, Rpad,
                                                      planes);
    }
}

}  // namespace ozlu
