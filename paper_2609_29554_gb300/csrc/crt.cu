// (S5) CRT per digit group and (S6) recombination, scaling, fused update and
// the single rounding (Sec. 3.1, Sec. 3.2 Eq. (11), Sec. 3.3).
//
// One thread per output element.  For every retained digit group g:
//   S_g = sum_l t_l M_l - round(F) P,   F = sum_l t_l / m_l       (Eq. (11))
// evaluated modulo 2^(32 WG): |S_g| < 2^(32 WG - 1) by the plan, so the low
// words of M_l and P suffice and the wrap-around is the two's-complement
// representation of the centered value.  F is summed in binary32: the plan's
// need leaves |S_g| / P < 2^-7, so frac(F) lies within 2^-7 of an integer and
// the binary32 error (below 2^-12 for up to 64 moduli) cannot change round(F).
// Then P_int = sum_g S_g 2^(w (g - g0)) on the grid 2^E0, E0 = w g0 - mu_i - nu_j,
// and C <- fl(beta C + alpha P_int 2^E0): the old C is brought to the grid
// component by component as Eq. (12) does for the inputs, the exact sum is
// rounded into nc binary64 components by successive round-to-nearest-even.
#include "mp_device.cuh"
#include "ozlu_internal.h"

namespace ozlu {
namespace {

// X (two's complement, WACC words) += v * 2^pos for v a WG-word two's-complement
// value (sign-extended), pos >= 0
__device__ __forceinline__ void add_group(uint32_t (&X)[WACC], const uint32_t (&v)[MAXWG], int WG,
                                          int pos) {
    const uint32_t sext = (v[WG - 1] >> 31) ? 0xffffffffu : 0u;
    const int q = pos >> 5, r = pos & 31;
    uint64_t c = 0;
#pragma unroll
    for (int wd = 0; wd < WACC; ++wd) {
        // word wd of (v << pos): bits from v at word offsets (wd - q) and (wd - q - 1)
        const int a = wd - q, b = wd - q - 1;
        uint32_t va = 0, vb = 0;
#pragma unroll
        for (int k = 0; k < MAXWG; ++k) {
            if (k < WG && k == a) va = v[k];
            if (k < WG && k == b) vb = v[k];
        }
        if (a >= WG) va = sext;
        if (b >= WG) vb = sext;
        if (a < 0) va = 0;
        if (b < 0) vb = 0;
        const uint32_t word = r ? (va << r) | (vb >> (32 - r)) : va;
        const uint64_t s = (uint64_t)X[wd] + word + c;
        X[wd] = (uint32_t)s;
        c = s >> 32;
    }
}

// |X| >> s (X non-negative), s >= 0
__device__ __forceinline__ void shr_mag(uint32_t (&X)[WACC], int s) {
    const int q = s >> 5, r = s & 31;
    uint32_t out[WACC];
#pragma unroll
    for (int wd = 0; wd < WACC; ++wd) {
        uint32_t lo = 0, hi = 0;
#pragma unroll
        for (int k = 0; k < WACC; ++k) {
            if (k == wd + q) lo = X[k];
            if (k == wd + q + 1) hi = X[k];
        }
        out[wd] = r ? (lo >> r) | (hi << (32 - r)) : lo;
    }
#pragma unroll
    for (int wd = 0; wd < WACC; ++wd) X[wd] = out[wd];
}

// 53-bit field of a non-negative value starting at bit pos
__device__ __forceinline__ uint64_t field53(const uint32_t (&X)[WACC], int pos) {
    const uint64_t lo = field32<WACC>(X, pos);
    const uint64_t hi = field32<WACC>(X, pos + 32);
    return (lo | (hi << 32)) & ((1ull << 53) - 1);
}

// Successive round-to-nearest-even of sign * mag * 2^E into nc doubles.
__device__ __forceinline__ void round_out(uint32_t (&mag)[WACC], bool neg, int E, int nc,
                                          double* out) {
    for (int c = 0; c < nc; ++c) {
        const int L = bit_length<WACC>(mag);
        double x = 0.0;
        if (L > 0) {
            if (L <= 53) {
                const uint64_t q = field53(mag, 0);
                x = scalbn((double)q, E);
#pragma unroll
                for (int wd = 0; wd < WACC; ++wd) mag[wd] = 0;
            } else {
                const int sh = L - 53;
                uint64_t q = field53(mag, sh);
                const bool rb = bit_at<WACC>(mag, sh - 1) != 0;
                const bool sticky = any_below<WACC>(mag, sh - 1);
                mask_below<WACC>(mag, sh);
                if (rb && (sticky || (q & 1))) {
                    q += 1;                           // rounded up: residual changes sign
                    complement_below<WACC>(mag, sh);  // 2^sh - low
                    x = scalbn((double)q, E + sh);
                    if (neg) x = -x;
                    neg = !neg;
                    out[c] = x;
                    continue;
                }
                x = scalbn((double)q, E + sh);
            }
            if (neg) x = -x;
        }
        out[c] = x;
    }
}

__global__ void __launch_bounds__(128) crt_kernel(const uint8_t* __restrict__ T, int m, int n,
                                                  const int* __restrict__ mu,
                                                  const int* __restrict__ nu,
                                                  const __grid_constant__ DevTable tab, int nc,
                                                  int alpha, int beta, double* __restrict__ C,
                                                  long long ldc) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long mn = (long long)m * n;
    if (e >= mn) return;
    const int i = (int)(e % m), j = (int)(e / m);
    const int WG = tab.WG;

    uint32_t X[WACC];
#pragma unroll
    for (int wd = 0; wd < WACC; ++wd) X[wd] = 0;

    for (int gi = 0; gi < tab.G; ++gi) {
        uint64_t acc[MAXWG];
#pragma unroll
        for (int wd = 0; wd < MAXWG; ++wd) acc[wd] = 0;
        float F = 0.0f;
        const uint8_t* tp = T + (size_t)gi * tab.N * mn + e;
        for (int l = 0; l < tab.N; ++l) {
            const uint32_t t = tp[(size_t)l * mn];
#pragma unroll
            for (int wd = 0; wd < MAXWG; ++wd)
                if (wd < WG) acc[wd] += (uint64_t)t * tab.Mlow[l][wd];
            F = fmaf((float)t, tab.invm[l], F);
        }
        const uint32_t R = (uint32_t)rintf(F);
        uint32_t sg[MAXWG];
        long long carry = 0;
#pragma unroll
        for (int wd = 0; wd < MAXWG; ++wd) {
            if (wd < WG) {
                const long long cur = (long long)acc[wd] + carry - (long long)((uint64_t)R * tab.Plow[wd]);
                sg[wd] = (uint32_t)cur;
                carry = cur >> 32;  // arithmetic shift (floor)
            } else {
                sg[wd] = 0;
            }
        }
        add_group(X, sg, WG, tab.w * gi);
    }
    // X = P_int (two's complement) on the grid 2^E0
    int E = tab.w * tab.g0 - mu[i] - nu[j];
    bool neg = is_negative<WACC>(X);
    if (neg) negate<WACC>(X);
    if (alpha < 0) neg = !neg;
    double* cp = C + ((long long)i + (long long)j * ldc) * nc;
    double out[4];
    const double c0 = beta ? cp[0] : 0.0;
    if (c0 != 0.0) {
        // window: e_top = max(E0 + bitlen|P_int|, frexp_exp(C[0])) + 1
        const int L = bit_length<WACC>(X);
        int etop = max(E + L, frexp_exp(c0)) + 1;
        const int E0 = E;
        if (etop - E0 > WINDOW_BITS) {
            E = etop - WINDOW_BITS;
            shr_mag(X, E - E0);  // truncation toward zero of the product
        }
        if (neg) negate<WACC>(X);  // back to two's complement, with alpha applied
        for (int c = 0; c < nc; ++c) add_component<WACC>(X, cp[c], -E);
        neg = is_negative<WACC>(X);
        if (neg) negate<WACC>(X);
    }
    round_out(X, neg, E, nc, out);
    for (int c = 0; c < nc; ++c) cp[c] = out[c];
}

}  // namespace

void launch_crt(const uint8_t* T, int m, int n, const int* mu, const int* nu,
                const DevTable& tab, int nc, int alpha, int beta, double* C, long long ldc,
                cudaStream_t s) {
    const long long mn = (long long)m * n;
    if (mn == 0) return;
    const int threads = 128;
    crt_kernel<<<(unsigned)((mn + threads - 1) / threads), threads, 0, s>>>(
        T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc);
}

}  // namespace ozlu
