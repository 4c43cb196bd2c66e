// (S4) binary64 residue GEMMs with the (S5) modular epilogue (Sec. 4.2.6).
//
// Moduli are primes m < sqrt(2^55 / K) (Eq. (17)), about 23 bits at K = 512,
// so a residue product summed over K stays below 2^53 and every DFMA is exact.
// Each pair term of a digit group is its own exact accumulation; it is reduced
// modulo m before the pair terms are added (the bound of Eq. (17) covers one
// accumulation of length K), then t_l = (C mod m) y_l mod m is stored as a
// 32-bit word.  The tile loop is a plain shared-memory DFMA GEMM: on GB300
// the binary64 rate (about 1 TFLOP/s) makes this back-end a reference point
// for the autotuner rather than a contender.
#include "mp_device.cuh"
#include "ozlu_internal.h"

namespace ozlu {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, THREADS = 256;

__device__ __forceinline__ long long mod_signed(long long v, long long m) {
    long long r = v % m;
    return r < 0 ? r + m : r;
}

__global__ void __launch_bounds__(THREADS) gemm_f64_kernel(const double* __restrict__ RA,
                                                           const double* __restrict__ RB, int m, int n,
                                                           int Mpad, int Npad, int Kpad,
                                                           const __grid_constant__ DevTable tab,
                                                           uint32_t* __restrict__ T) {
    __shared__ double sa[BK][BM + 1];
    __shared__ double sb[BK][BN + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int tm = blockIdx.x, tn = blockIdx.y;
    const int l = blockIdx.z % tab.N, gi = blockIdx.z / tab.N;
    const int S = tab.S, g = tab.g0 + gi;
    const int ta0 = max(0, g - (S - 1)), ta1 = min(g, S - 1);
    const long long md = tab.mod[l];
    const size_t aplane = (size_t)Mpad * Kpad, bplane = (size_t)Npad * Kpad;
    long long tsum[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) tsum[i][j] = 0;
    for (int ta = ta0; ta <= ta1; ++ta) {
        const int tb = g - ta;
        const double* A = RA + (size_t)(l * S + ta) * aplane + (size_t)tm * BM * Kpad;
        const double* B = RB + (size_t)(l * S + tb) * bplane + (size_t)tn * BN * Kpad;
        double acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
        for (int k0 = 0; k0 < Kpad; k0 += BK) {
            for (int idx = tid; idx < BM * BK; idx += THREADS) {
                const int r = idx / BK, kk = idx - r * BK;
                sa[kk][r] = A[(size_t)r * Kpad + k0 + kk];
                sb[kk][r] = B[(size_t)r * Kpad + k0 + kk];
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                double av[4], bv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) av[i] = sa[kk][ty * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bv[j] = sb[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) tsum[i][j] += mod_signed((long long)acc[i][j], md);
    }
    const long long yd = tab.y[l];
    uint32_t* out = T + ((size_t)gi * tab.N + l) * (size_t)m * n;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int row = tm * BM + ty * 4 + i, col = tn * BN + tx * 4 + j;
            if (row < m && col < n) out[(size_t)col * m + row] = (uint32_t)((tsum[i][j] % md) * yd % md);
        }
}

}  // namespace

void launch_gemm_f64(const double* RA, const double* RB, int m, int n, int Mpad, int Npad, int Kpad,
                     const DevTable& tab, uint32_t* T, cudaStream_t s) {
    dim3 grid(Mpad / BM, Npad / BN, tab.N * tab.G);
    gemm_f64_kernel<<<grid, THREADS, 0, s>>>(RA, RB, m, n, Mpad, Npad, Kpad, tab, T);
}

}  // namespace ozlu
