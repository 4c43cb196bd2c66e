// Device helpers: binary64 decomposition and small fixed-width two's-complement
// integers held in per-thread arrays of 32-bit words (little-endian).
#pragma once

#include <stdint.h>

namespace ozlu {

// x = sign * mant * 2^(e - 53) with mant < 2^53 (Sec. 3.3: x[c] = +-m_c 2^(e_c - 53)).
// Returns false for zero.
__device__ __forceinline__ bool decompose(double x, uint64_t& mant, int& e, bool& neg) {
    const uint64_t bits = (uint64_t)__double_as_longlong(x);
    const int biased = (int)((bits >> 52) & 0x7ff);
    const uint64_t frac = bits & ((1ull << 52) - 1);
    neg = (bits >> 63) != 0;
    if (biased == 0) {
        if (frac == 0) return false;
        mant = frac;       // subnormal: x = frac 2^-1074
        e = -1021;
    } else {
        mant = frac | (1ull << 52);
        e = biased - 1022;  // frexp exponent
    }
    return true;
}

// frexp exponent of a nonzero finite double: 2^(e-1) <= |x| < 2^e
__device__ __forceinline__ int frexp_exp(double x) { return ilogb(x) + 1; }

// X += (neg ? -1 : 1) * mag * 2^pos  (mod 2^(32 W)), pos >= 0
template <int W>
__device__ __forceinline__ void add_shifted(uint32_t (&X)[W], uint64_t mag, int pos, bool neg) {
    const int q = pos >> 5, r = pos & 31;
    const uint32_t lo = (uint32_t)(mag << r);
    const uint32_t mid = r ? (uint32_t)(mag >> (32 - r)) : (uint32_t)(mag >> 32);
    const uint32_t hi = r ? (uint32_t)(mag >> (64 - r)) : 0u;
    uint64_t c = neg ? 1u : 0u;
#pragma unroll
    for (int wd = 0; wd < W; ++wd) {
        uint32_t a = wd == q ? lo : wd == q + 1 ? mid : wd == q + 2 ? hi : 0u;
        if (neg) a = ~a;
        const uint64_t s = (uint64_t)X[wd] + a + c;
        X[wd] = (uint32_t)s;
        c = s >> 32;
    }
}

// Eq. (12): X += sum_c +-(m_c << (e_c + shift - 53)), a negative count being a
// right shift of the magnitude (truncation toward zero of that component).
template <int W>
__device__ __forceinline__ void add_component(uint32_t (&X)[W], double x, int shift) {
    uint64_t mant;
    int e;
    bool neg;
    if (!decompose(x, mant, e, neg)) return;
    int s = e - 53 + shift;
    if (s < 0) {
        if (s <= -64) return;
        mant >>= -s;
        s = 0;
        if (mant == 0) return;
    }
    if (s >= 32 * W) return;  // beyond the window: cannot happen for valid plans
    add_shifted<W>(X, mant, s, neg);
}

template <int W>
__device__ __forceinline__ bool is_negative(const uint32_t (&X)[W]) {
    return (X[W - 1] >> 31) != 0;
}

template <int W>
__device__ __forceinline__ void negate(uint32_t (&X)[W]) {
    uint64_t c = 1;
#pragma unroll
    for (int wd = 0; wd < W; ++wd) {
        const uint64_t s = (uint64_t)(~X[wd]) + c;
        X[wd] = (uint32_t)s;
        c = s >> 32;
    }
}

// bit length of a non-negative value (0 for zero)
template <int W>
__device__ __forceinline__ int bit_length(const uint32_t (&X)[W]) {
    int L = 0;
#pragma unroll
    for (int wd = 0; wd < W; ++wd)
        if (X[wd]) L = 32 * wd + 32 - __clz(X[wd]);
    return L;
}

// 32-bit field starting at bit pos of a two's-complement value (sign-extended)
template <int W>
__device__ __forceinline__ uint32_t field32(const uint32_t (&X)[W], int pos) {
    const uint32_t sext = (X[W - 1] >> 31) ? 0xffffffffu : 0u;
    const int q = pos >> 5, r = pos & 31;
    uint32_t lo = sext, hi = sext;
#pragma unroll
    for (int wd = 0; wd < W; ++wd) {
        if (wd == q) lo = X[wd];
        if (wd == q + 1) hi = X[wd];
    }
    return r ? (lo >> r) | (hi << (32 - r)) : lo;
}

// bit at position pos (pos < 32 W)
template <int W>
__device__ __forceinline__ uint32_t bit_at(const uint32_t (&X)[W], int pos) {
    uint32_t v = 0;
#pragma unroll
    for (int wd = 0; wd < W; ++wd)
        if (wd == (pos >> 5)) v = (X[wd] >> (pos & 31)) & 1u;
    return v;
}

// any bit set below position pos
template <int W>
__device__ __forceinline__ bool any_below(const uint32_t (&X)[W], int pos) {
    bool any = false;
#pragma unroll
    for (int wd = 0; wd < W; ++wd) {
        const int lo = 32 * wd;
        if (pos >= lo + 32) any |= X[wd] != 0;
        else if (pos > lo) any |= (X[wd] & ((1u << (pos - lo)) - 1u)) != 0;
    }
    return any;
}

// keep only the bits below position pos
template <int W>
__device__ __forceinline__ void mask_below(uint32_t (&X)[W], int pos) {
#pragma unroll
    for (int wd = 0; wd < W; ++wd) {
        const int lo = 32 * wd;
        if (pos <= lo) X[wd] = 0;
        else if (pos < lo + 32) X[wd] &= (1u << (pos - lo)) - 1u;
    }
}

// X = 2^pos - X for 0 <= X < 2^pos (pos < 32 W)
template <int W>
__device__ __forceinline__ void complement_below(uint32_t (&X)[W], int pos) {
    negate<W>(X);
    mask_below<W>(X, pos);
}

// x mod m for x < 2^32 with magic = ceil(2^32/m)
__device__ __forceinline__ uint32_t mod_small(uint32_t x, uint32_t m, uint32_t magic) {
    const uint32_t q = __umulhi(x, magic);
    int32_t r = (int32_t)(x - q * m);
    if (r < 0) r += (int32_t)m;
    return (uint32_t)r;
}

}  // namespace ozlu
