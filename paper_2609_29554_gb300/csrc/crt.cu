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
//
// The group accumulators live in registers (WG is a template parameter, so
// the word loops unroll); the wide integers that need shifts by run-time
// amounts live in shared memory, one column per thread ([word][thread]).
#include "mp_device.cuh"
#include "ozlu_internal.h"

namespace ozlu {
namespace {

constexpr int CT = 128;  // threads per block

struct Wide {
    uint32_t* w;  // word k at w[k * CT]
    __device__ __forceinline__ uint32_t& operator[](int k) const { return w[k * CT]; }
};

__device__ __forceinline__ void wide_clear(const Wide& X, int words) {
    for (int k = 0; k < words; ++k) X[k] = 0;
}

// X += v * 2^pos, v a WGw-word two's-complement value (sign-extended to WACC)
__device__ __forceinline__ void wide_add_shifted(const Wide& X, const Wide& v, int WGw, int pos) {
    const uint32_t sext = (v[WGw - 1] >> 31) ? 0xffffffffu : 0u;
    const int q = pos >> 5, r = pos & 31;
    uint64_t c = 0;
    for (int k = q; k < WACC; ++k) {
        const int a = k - q, b = a - 1;
        const uint32_t va = a < WGw ? v[a] : sext;
        const uint32_t vb = b < 0 ? 0u : (b < WGw ? v[b] : sext);
        const uint32_t word = r ? (va << r) | (vb >> (32 - r)) : va;
        const uint64_t s = (uint64_t)X[k] + word + c;
        X[k] = (uint32_t)s;
        c = s >> 32;
    }
}

__device__ __forceinline__ bool wide_negative(const Wide& X) { return (X[WACC - 1] >> 31) != 0; }

__device__ __forceinline__ void wide_negate(const Wide& X) {
    uint64_t c = 1;
    for (int k = 0; k < WACC; ++k) {
        const uint64_t s = (uint64_t)(~X[k]) + c;
        X[k] = (uint32_t)s;
        c = s >> 32;
    }
}

// index of the top nonzero word, -1 for zero
__device__ __forceinline__ int wide_top(const Wide& X) {
    int t = WACC - 1;
    while (t >= 0 && X[t] == 0) --t;
    return t;
}

__device__ __forceinline__ uint32_t wide_word(const Wide& X, int k) { return (k >= 0 && k < WACC) ? X[k] : 0u; }

// bits [pos, pos + 64) of a non-negative value
__device__ __forceinline__ uint64_t wide_field64(const Wide& X, int pos) {
    const int q = pos >> 5, r = pos & 31;
    const uint64_t w0 = wide_word(X, q), w1 = wide_word(X, q + 1), w2 = wide_word(X, q + 2);
    if (r == 0) return w0 | (w1 << 32);
    return (w0 >> r) | (w1 << (32 - r)) | (w2 << (64 - r));
}

// X >>= s (non-negative value), truncation
__device__ __forceinline__ void wide_shr(const Wide& X, int s) {
    const int q = s >> 5, r = s & 31;
    for (int k = 0; k < WACC; ++k) {
        const uint32_t lo = wide_word(X, k + q), hi = wide_word(X, k + q + 1);
        X[k] = r ? (lo >> r) | (hi << (32 - r)) : lo;
    }
}

// X += mant * 2^s, s >= 0
__device__ __forceinline__ void wide_add_u64(const Wide& X, uint64_t mant, int s) {
    const int q = s >> 5, r = s & 31;
    const uint32_t p0 = (uint32_t)(mant << r);
    const uint32_t p1 = r ? (uint32_t)(mant >> (32 - r)) : (uint32_t)(mant >> 32);
    const uint32_t p2 = r ? (uint32_t)(mant >> (64 - r)) : 0u;
    uint64_t c = 0;
    for (int k = q; k < WACC; ++k) {
        const uint32_t a = k == q ? p0 : k == q + 1 ? p1 : k == q + 2 ? p2 : 0u;
        const uint64_t t = (uint64_t)X[k] + a + c;
        X[k] = (uint32_t)t;
        c = t >> 32;
        if (k > q + 2 && c == 0) break;
    }
}

// X += sign * mant * 2^s, s may be negative (truncate the magnitude, Eq. (12))
__device__ __forceinline__ void wide_add_component(const Wide& X, double x, int shift) {
    uint64_t mant;
    int e;
    bool neg;
    if (!decompose(x, mant, e, neg)) return;
    int s = e - 53 + shift;
    if (s < 0) {
        if (s <= -64) return;
        mant >>= -s;
        s = 0;
        if (!mant) return;
    }
    if (s >= 32 * WACC) return;
    if (!neg) {
        wide_add_u64(X, mant, s);
    } else {
        // subtract: X - mant 2^s = X + ~(mant 2^s) + 1 over the words from q
        // up (below word q, ~0 + 1 leaves every word and the carry of 1)
        const int q = s >> 5, r = s & 31;
        const uint32_t p0 = (uint32_t)(mant << r);
        const uint32_t p1 = r ? (uint32_t)(mant >> (32 - r)) : (uint32_t)(mant >> 32);
        const uint32_t p2 = r ? (uint32_t)(mant >> (64 - r)) : 0u;
        uint64_t c = 1;
        for (int k = q; k < WACC; ++k) {
            const uint32_t a = k == q ? p0 : k == q + 1 ? p1 : k == q + 2 ? p2 : 0u;
            const uint64_t t = (uint64_t)X[k] + (uint32_t)~a + c;
            X[k] = (uint32_t)t;
            c = t >> 32;
        }
    }
}

// successive round-to-nearest-even of sign * X * 2^E into nc components
__device__ __forceinline__ void wide_round_out(const Wide& X, bool neg, int E, int nc, double* out) {
    int top = wide_top(X);
    for (int c = 0; c < nc; ++c) {
        if (top < 0) {
            out[c] = 0.0;
            continue;
        }
        const int L = 32 * top + 32 - __clz(X[top]);
        double x;
        if (L <= 53) {
            const uint64_t q = wide_field64(X, 0);
            x = scalbn((double)q, E);
            for (int k = 0; k <= top; ++k) X[k] = 0;
            top = -1;
            out[c] = neg ? -x : x;
            continue;
        }
        const int sh = L - 53;
        uint64_t q = wide_field64(X, sh) & ((1ull << 53) - 1);
        const int rp = sh - 1;  // round bit position
        const bool rb = (wide_word(X, rp >> 5) >> (rp & 31)) & 1u;
        bool sticky = false;
        {
            const int wq = rp >> 5;
            for (int k = 0; k < wq; ++k) sticky |= X[k] != 0;
            if (rp & 31) sticky |= (X[wq] & ((1u << (rp & 31)) - 1u)) != 0;
        }
        // keep only the bits below sh (the residual)
        const int wq = sh >> 5, wr = sh & 31;
        for (int k = wq + (wr ? 1 : 0); k <= top; ++k) X[k] = 0;
        if (wr) X[wq] &= (1u << wr) - 1u;
        const bool up = rb && (sticky || (q & 1));
        if (up) {
            q += 1;
            // residual becomes 2^sh - low (opposite sign)
            uint64_t cc = 1;
            for (int k = 0; k <= wq; ++k) {
                const uint64_t t = (uint64_t)(~X[k]) + cc;
                X[k] = (uint32_t)t;
                cc = t >> 32;
            }
            if (wr) X[wq] &= (1u << wr) - 1u;
            else X[wq] = 0;
        }
        x = scalbn((double)q, E + sh);
        out[c] = neg ? -x : x;
        if (up) neg = !neg;
        top = wq;
        while (top >= 0 && X[top] == 0) --top;
    }
}

template <int WG, typename TT>
__global__ void __launch_bounds__(CT) crt_kernel(const TT* __restrict__ T, int m, int n,
                                                 const int* __restrict__ mu, const int* __restrict__ nu,
                                                 const __grid_constant__ DevTable tab, int nc, int alpha,
                                                 int beta, double* __restrict__ C, long long ldc) {
    __shared__ uint32_t sx[WACC * CT];
    __shared__ uint32_t ss[MAXWG * CT];
    const long long e = (long long)blockIdx.x * CT + threadIdx.x;
    const long long mn = (long long)m * n;
    if (e >= mn) return;
    const int i = (int)(e % m), j = (int)(e / m);
    const Wide X{sx + threadIdx.x}, Sg{ss + threadIdx.x};
    if (tab.G == 0) wide_clear(X, WACC);

    for (int gi = 0; gi < tab.G; ++gi) {
        uint64_t acc[WG];
#pragma unroll
        for (int w = 0; w < WG; ++w) acc[w] = 0;
        float F = 0.0f;
        const TT* tp = T + (size_t)gi * tab.N * mn + e;
        for (int l = 0; l < tab.N; ++l) {
            const uint32_t t = tp[(size_t)l * mn];
#pragma unroll
            for (int w = 0; w < WG; ++w) acc[w] += (uint64_t)t * tab.Mlow[l][w];
            F = fmaf((float)t, tab.invm[l], F);
        }
        const uint32_t R = (uint32_t)rintf(F);
        // the first group sits at bit 0 of the window: it is written there
        // (sign-extended) instead of added to a cleared window
        const Wide& D = gi == 0 ? X : Sg;
        long long carry = 0;
#pragma unroll
        for (int w = 0; w < WG; ++w) {
            const long long cur = (long long)acc[w] + carry - (long long)((uint64_t)R * tab.Plow[w]);
            D[w] = (uint32_t)cur;
            carry = cur >> 32;  // arithmetic shift (floor)
        }
        if (gi == 0) {
            const uint32_t sext = (X[WG - 1] >> 31) ? 0xffffffffu : 0u;
            for (int k = WG; k < WACC; ++k) X[k] = sext;
        } else {
            wide_add_shifted(X, Sg, WG, tab.w * gi);
        }
    }
    // X = P_int (two's complement) on the grid 2^E0
    int E = tab.w * tab.g0 - mu[i] - nu[j];
    bool neg = wide_negative(X);
    if (neg) wide_negate(X);
    if (alpha < 0) neg = !neg;
    double* cp = C + ((long long)i + (long long)j * ldc) * nc;
    const double c0 = beta ? cp[0] : 0.0;
    if (c0 != 0.0) {
        // window: e_top = max(E0 + bitlen|P_int|, frexp_exp(C[0])) + 1
        const int top = wide_top(X);
        const int L = top < 0 ? 0 : 32 * top + 32 - __clz(X[top]);
        const int etop = max(E + L, frexp_exp(c0)) + 1;
        const int E0 = E;
        if (etop - E0 > WINDOW_BITS) {
            E = etop - WINDOW_BITS;
            wide_shr(X, E - E0);  // truncation toward zero of the product
        }
        if (neg) wide_negate(X);  // back to two's complement, alpha applied
        double cl[4];
        for (int c = 0; c < nc; ++c) cl[c] = cp[c];
        for (int c = 0; c < nc; ++c) wide_add_component(X, cl[c], -E);
        neg = wide_negative(X);
        if (neg) wide_negate(X);
    }
    double out[4];
    wide_round_out(X, neg, E, nc, out);
    for (int c = 0; c < nc; ++c) cp[c] = out[c];
}

template <int WG, typename TT>
void launch_wg(const TT* T, int m, int n, const int* mu, const int* nu, const DevTable& tab, int nc,
               int alpha, int beta, double* C, long long ldc, cudaStream_t s) {
    const long long mn = (long long)m * n;
    crt_kernel<WG, TT><<<(unsigned)((mn + CT - 1) / CT), CT, 0, s>>>(T, m, n, mu, nu, tab, nc, alpha, beta, C,
                                                                     ldc);
}

template <typename TT>
void launch_tt(const TT* T, int m, int n, const int* mu, const int* nu, const DevTable& tab, int nc, int alpha,
               int beta, double* C, long long ldc, cudaStream_t s) {
    switch (tab.WG) {
        case 1: case 2: case 3: case 4: launch_wg<4>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
        case 5: launch_wg<5>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
        case 6: launch_wg<6>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
        case 7: launch_wg<7>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
        case 8: launch_wg<8>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
        case 9: launch_wg<9>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
        case 10: launch_wg<10>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
        case 11: launch_wg<11>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
        case 12: launch_wg<12>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
        case 13: launch_wg<13>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
        case 14: launch_wg<14>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
        case 15: launch_wg<15>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
        default: launch_wg<16>(T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s); break;
    }
}

}  // namespace

void launch_crt(const void* T, bool t32, int m, int n, const int* mu, const int* nu, const DevTable& tab, int nc,
                int alpha, int beta, double* C, long long ldc, cudaStream_t s) {
    const long long mn = (long long)m * n;
    if (mn == 0) return;
    if (t32)
        launch_tt<uint32_t>((const uint32_t*)T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s);
    else
        launch_tt<uint8_t>((const uint8_t*)T, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s);
}

}  // namespace ozlu
