// Multi-limb binary floating point on 32-bit integer limbs (device).
//
// value = (-1)^neg * m * 2^(e - 32 L), with m an L-word magnitude whose top
// bit is set (normalised), or zero (m = 0).  Every operation rounds its
// exact (or sticky-truncated) result to L words, round to nearest even.
// The arithmetic runs on the integer pipes (IMAD), which on GB300 issue
// about 40 times the binary64 FMA rate; the LU panel uses it for DD/TD/QD
// elements at 32 L >= 53 nc + 22 bits and converts to and from the
// expansion format (successive round-to-nearest on the way out).
#pragma once

#include <stdint.h>

#include "mp_device.cuh"

namespace ozlu {

template <int L>
struct MPF {
    uint32_t m[L];
    int e;
    int neg;
};

template <int L>
__device__ __forceinline__ bool mpf_zero(const MPF<L>& a) {
    return a.m[L - 1] == 0;
}

template <int L>
__device__ __forceinline__ MPF<L> mpf_make_zero() {
    MPF<L> r;
#pragma unroll
    for (int i = 0; i < L; ++i) r.m[i] = 0;
    r.e = 0;
    r.neg = 0;
    return r;
}

// Round the W-word magnitude X (top word nonzero or all zero) to L words:
// normalise, keep the top 32 L bits, round to nearest even with a sticky.
// `ex` is the exponent such that value = X * 2^(ex - 32 W).
template <int L, int W>
__device__ __forceinline__ MPF<L> mpf_round(uint32_t (&X)[W], int ex, int neg, bool sticky_in) {
    MPF<L> r;
    r.neg = neg;
    const int bl = bit_length<W>(X);
    if (bl == 0) {
        r = mpf_make_zero<L>();
        return r;
    }
    // shift left so that the top bit is bit 32W-1
    const int sh = 32 * W - bl;
    if (sh > 0 && sh < 32) {
        // common case: the top word is nonzero, a funnel shift of every word
#pragma unroll
        for (int i = W - 1; i > 0; --i) X[i] = __funnelshift_l(X[i - 1], X[i], sh);
        X[0] <<= sh;
    } else if (sh >= 32) {
        // whole words by a logarithmic shifter (selects, no dynamic indexing), then bits
        const int q = sh >> 5, rr = sh & 31;
#pragma unroll
        for (int s = 8; s >= 1; s >>= 1) {
            if (s < W) {
                const bool on = (q & s) != 0;
#pragma unroll
                for (int i = W - 1; i >= 0; --i) X[i] = on ? (i >= s ? X[i - s] : 0u) : X[i];
            }
        }
#pragma unroll
        for (int i = W - 1; i > 0; --i) X[i] = __funnelshift_l(X[i - 1], X[i], rr);
        X[0] <<= rr;
    }
    ex -= sh;
    // top L words; round bit = top bit of word W-L-1; sticky = the rest
    bool rbit = false, sticky = sticky_in;
    if (W > L) {
        rbit = (X[W - L - 1] >> 31) != 0;
        sticky |= (X[W - L - 1] & 0x7fffffffu) != 0;
#pragma unroll
        for (int i = 0; i < W - L - 1; ++i) sticky |= X[i] != 0;
    }
#pragma unroll
    for (int i = 0; i < L; ++i) r.m[i] = X[W - L + i];
    // X * 2^(ex - 32 W) with the top L words kept: m * 2^(ex - 32 L)
    r.e = ex;
    if (rbit && (sticky || (r.m[0] & 1u))) {
        uint64_t c = 1;
#pragma unroll
        for (int i = 0; i < L; ++i) {
            const uint64_t s = (uint64_t)r.m[i] + c;
            r.m[i] = (uint32_t)s;
            c = s >> 32;
        }
        if (c) {  // carried out: 1000...0
            r.m[L - 1] = 0x80000000u;
            r.e += 1;
        }
    }
    return r;
}

// from an expansion of N binary64 components (sticky-truncated to 32(L+2) bits,
// then rounded to L words)
template <int L, int N>
__device__ __forceinline__ MPF<L> mpf_from_exp(const double* x) {
    constexpr int W = L + 2;
    if (x[0] == 0.0) return mpf_make_zero<L>();
    const int top = frexp_exp(x[0]) + 1;  // |value| < 2^top
    const int base = top - 32 * W;        // bit 0 of the window
    uint32_t X[W];
#pragma unroll
    for (int i = 0; i < W; ++i) X[i] = 0;
    bool sticky = false;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        uint64_t mant;
        int e;
        bool ng;
        if (!decompose(x[c], mant, e, ng)) continue;
        int s = e - 53 - base;
        if (s < 0) {
            if (s <= -64) { sticky = true; continue; }
            if (mant & ((1ull << (-s)) - 1)) sticky = true;
            mant >>= -s;
            s = 0;
        }
        add_shifted<W>(X, mant, s, ng);
    }
    int neg = 0;
    if (is_negative<W>(X)) {
        negate<W>(X);
        neg = 1;
        // a dropped positive remainder of a negative sum rounds the magnitude up
    }
    return mpf_round<L, W>(X, top, neg, sticky);
}

// successive round-to-nearest-even into N binary64 components
template <int L, int N>
__device__ __forceinline__ void mpf_to_exp(const MPF<L>& a, double* out) {
    uint32_t mag[L];
#pragma unroll
    for (int i = 0; i < L; ++i) mag[i] = a.m[i];
    bool neg = a.neg != 0;
    const int E = a.e - 32 * L;
#pragma unroll
    for (int c = 0; c < N; ++c) {
        const int Lb = bit_length<L>(mag);
        double x = 0.0;
        if (Lb > 0) {
            if (Lb <= 53) {
                const uint64_t q = (uint64_t)field32<L>(mag, 0) | ((uint64_t)field32<L>(mag, 32) << 32);
                x = scalbn((double)(q & ((1ull << 53) - 1)), E);
#pragma unroll
                for (int i = 0; i < L; ++i) mag[i] = 0;
                if (neg) x = -x;
            } else {
                const int sh = Lb - 53;
                uint64_t q = ((uint64_t)field32<L>(mag, sh) | ((uint64_t)field32<L>(mag, sh + 32) << 32)) &
                             ((1ull << 53) - 1);
                const bool rb = bit_at<L>(mag, sh - 1) != 0;
                const bool st = any_below<L>(mag, sh - 1);
                mask_below<L>(mag, sh);
                if (rb && (st || (q & 1))) {
                    q += 1;
                    complement_below<L>(mag, sh);
                    x = scalbn((double)q, E + sh);
                    if (neg) x = -x;
                    neg = !neg;
                } else {
                    x = scalbn((double)q, E + sh);
                    if (neg) x = -x;
                }
            }
        }
        out[c] = x;
    }
}

template <int L>
__device__ __forceinline__ MPF<L> mpf_neg(MPF<L> a) {
    a.neg ^= 1;
    return a;
}

// |a| vs |b|
template <int L>
__device__ __forceinline__ int mpf_abs_cmp(const MPF<L>& a, const MPF<L>& b) {
    const bool za = mpf_zero<L>(a), zb = mpf_zero<L>(b);
    if (za || zb) return za && zb ? 0 : (za ? -1 : 1);
    if (a.e != b.e) return a.e > b.e ? 1 : -1;
#pragma unroll
    for (int i = L - 1; i >= 0; --i)
        if (a.m[i] != b.m[i]) return a.m[i] > b.m[i] ? 1 : -1;
    return 0;
}

// Exact product of two L-word magnitudes (2 L words): column sums of the
// 32-bit halves of the limb products (independent, each below
// 2^(33 + log2 L)), then one carry pass.  (Carry-flag chains of 32-bit
// multiply-adds measured slower on GB300: they serialise on the flag.)
template <int L>
__device__ __forceinline__ void mul_words(const uint32_t (&a)[L], const uint32_t (&b)[L], uint32_t (&P)[2 * L]) {
    uint64_t S[2 * L];
#pragma unroll
    for (int k = 0; k < 2 * L; ++k) S[k] = 0;
#pragma unroll
    for (int i = 0; i < L; ++i)
#pragma unroll
        for (int j = 0; j < L; ++j) {
            const uint64_t t = (uint64_t)a[i] * b[j];
            S[i + j] += (uint32_t)t;
            S[i + j + 1] += t >> 32;
        }
    uint64_t c = 0;
#pragma unroll
    for (int k = 0; k < 2 * L; ++k) {
        const uint64_t v = S[k] + c;
        P[k] = (uint32_t)v;
        c = v >> 32;
    }
}

// a * b, rounded to L words
template <int L>
__device__ __forceinline__ MPF<L> mpf_mul(const MPF<L>& a, const MPF<L>& b) {
    if (mpf_zero<L>(a) || mpf_zero<L>(b)) return mpf_make_zero<L>();
    uint32_t P[2 * L];
    mul_words<L>(a.m, b.m, P);
    // value = P * 2^(a.e + b.e - 64 L) = P * 2^((a.e + b.e) - 32 * 2L)
    return mpf_round<L, 2 * L>(P, a.e + b.e, a.neg ^ b.neg, false);
}

// a + b, rounded to L words (guard words and a sticky keep it correctly rounded)
template <int L>
__device__ __forceinline__ MPF<L> mpf_add(const MPF<L>& a, const MPF<L>& b) {
    if (mpf_zero<L>(b)) return a;
    if (mpf_zero<L>(a)) return b;
    const bool swap = mpf_abs_cmp<L>(a, b) < 0;
    const MPF<L>& x = swap ? b : a;  // |x| >= |y|
    const MPF<L>& y = swap ? a : b;
    constexpr int W = L + 2;
    uint32_t X[W], Y[W];
    X[0] = 0;
    X[1] = 0;
    Y[0] = 0;
    Y[1] = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) {
        X[i + 2] = x.m[i];
        Y[i + 2] = y.m[i];
    }
    // y shifted right by d = x.e - y.e bits (whole words by a logarithmic
    // shifter, then bits); sticky collects the bits shifted out
    const int d = x.e - y.e;
    bool sticky = false;
    if (d >= 32 * W) {
#pragma unroll
        for (int i = 0; i < W; ++i) Y[i] = 0;
        sticky = true;
    } else {
        const int q = d >> 5, r = d & 31;
#pragma unroll
        for (int s = 8; s >= 1; s >>= 1) {
            if (s < W) {
                const bool on = (q & s) != 0;
                uint32_t lost = 0;
#pragma unroll
                for (int i = 0; i < s; ++i) lost |= Y[i];
                sticky |= on && lost != 0;
#pragma unroll
                for (int i = 0; i < W; ++i) Y[i] = on ? (i + s < W ? Y[i + s] : 0u) : Y[i];
            }
        }
        sticky |= r != 0 && (Y[0] & ((1u << r) - 1u)) != 0;
#pragma unroll
        for (int i = 0; i < W - 1; ++i) Y[i] = __funnelshift_r(Y[i], Y[i + 1], r);
        Y[W - 1] >>= r;
    }
    if (x.neg == y.neg) {
        uint64_t c = 0;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const uint64_t s = (uint64_t)X[i] + Y[i] + c;
            X[i] = (uint32_t)s;
            c = s >> 32;
        }
        // carry out of the window: shift right one bit, keep the lost bit
        if (c) {
            sticky |= (X[0] & 1u) != 0;
#pragma unroll
            for (int i = 0; i < W - 1; ++i) X[i] = (X[i] >> 1) | (X[i + 1] << 31);
            X[W - 1] = (X[W - 1] >> 1) | 0x80000000u;
            return mpf_round<L, W>(X, x.e + 1, x.neg, sticky);
        }
        return mpf_round<L, W>(X, x.e, x.neg, sticky);
    }
    // |x| >= |y|: the exact difference is X - Y - delta with 0 <= delta < 1
    // unit of the window (the bits of y below it); X - Y - 1 plus a set sticky
    // stands for it whenever delta > 0
    uint64_t brw = sticky ? 1u : 0u;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint64_t s = (uint64_t)X[i] - Y[i] - brw;
        X[i] = (uint32_t)s;
        brw = (s >> 63) & 1u;
    }
    return mpf_round<L, W>(X, x.e, x.neg, sticky);
}

template <int L>
__device__ __forceinline__ MPF<L> mpf_sub(const MPF<L>& a, const MPF<L>& b) {
    return mpf_add<L>(a, mpf_neg<L>(b));
}

// Y >>= d bits (d >= 0) by a logarithmic word shifter and a funnel shift;
// sticky collects the bits shifted out
template <int W>
__device__ __forceinline__ void shr_sticky(uint32_t (&Y)[W], int d, bool& sticky) {
    if (d >= 32 * W) {
        bool any = false;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            any |= Y[i] != 0;
            Y[i] = 0;
        }
        sticky |= any;
        return;
    }
    const int q = d >> 5, r = d & 31;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        if (s < W) {
            const bool on = (q & s) != 0;
            uint32_t lost = 0;
#pragma unroll
            for (int i = 0; i < s; ++i) lost |= Y[i];
            sticky |= on && lost != 0;
#pragma unroll
            for (int i = 0; i < W; ++i) Y[i] = on ? (i + s < W ? Y[i + s] : 0u) : Y[i];
        }
    }
    sticky |= r != 0 && (Y[0] & ((1u << r) - 1u)) != 0;
#pragma unroll
    for (int i = 0; i < W - 1; ++i) Y[i] = __funnelshift_r(Y[i], Y[i + 1], r);
    Y[W - 1] >>= r;
}

// (-1)^xn X 2^(ex - 32 W) + (-1)^yn Y 2^(ey - 32 W), both W-word magnitudes
// normalised (top bit set) or zero (xz, yz), rounded to L words; ysticky:
// Y stands for a value with more nonzero bits below its last word
template <int L, int W>
__device__ __forceinline__ MPF<L> add_windows(uint32_t (&X)[W], int ex, int xn, bool xz, uint32_t (&Y)[W], int ey,
                                              int yn, bool yz, bool ysticky) {
    if (yz) return mpf_round<L, W>(X, ex, xn, false);
    if (xz) return mpf_round<L, W>(Y, ey, yn, ysticky);
    bool swap = ey > ex;  // |Y| > |X|
    if (ey == ex) {
        int cmp = 0;
#pragma unroll
        for (int i = W - 1; i >= 0; --i)
            if (cmp == 0 && X[i] != Y[i]) cmp = X[i] > Y[i] ? 1 : -1;
        swap = cmp < 0;
    }
    uint32_t A[W], B[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
        A[i] = swap ? Y[i] : X[i];
        B[i] = swap ? X[i] : Y[i];
    }
    const int ea = swap ? ey : ex, eb = swap ? ex : ey;
    const int an = swap ? yn : xn, bn = swap ? xn : yn;
    bool sticky = swap ? false : ysticky;
    shr_sticky<W>(B, ea - eb, sticky);
    if (an == bn) {
        uint64_t c = 0;
#pragma unroll
        for (int i = 0; i < W; ++i) {
            const uint64_t s = (uint64_t)A[i] + B[i] + c;
            A[i] = (uint32_t)s;
            c = s >> 32;
        }
        if (c) {
            sticky |= (A[0] & 1u) != 0;
#pragma unroll
            for (int i = 0; i < W - 1; ++i) A[i] = (A[i] >> 1) | (A[i + 1] << 31);
            A[W - 1] = (A[W - 1] >> 1) | 0x80000000u;
            return mpf_round<L, W>(A, ea + 1, an, sticky);
        }
        return mpf_round<L, W>(A, ea, an, sticky);
    }
    // the exact difference is A - B - delta with 0 <= delta < 1 unit of the
    // window: A - B - 1 plus a set sticky stands for it whenever delta > 0
    uint64_t brw = sticky ? 1u : 0u;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const uint64_t s = (uint64_t)A[i] - B[i] - brw;
        A[i] = (uint32_t)s;
        brw = (s >> 63) & 1u;
    }
    // a borrow out means A == B with the sticky set: the exact difference is
    // below one unit of the window's last word (zero for an exact
    // cancellation such as c = a b) and is returned as zero
    if (brw) return mpf_make_zero<L>();
    return mpf_round<L, W>(A, ea, an, sticky);
}

// c - a b with one rounding: the product's top L + 2 words (words L - 2 ..
// 2L - 1 of the 2L-word product, from the limb products that reach them; the
// carry lost from the words below is under 2^5 units of the lowest window
// word) are added to c in an (L + 2)-word window, the lower words counting as
// a set sticky.  The result is the correctly rounded c - a b unless the exact
// value lies within about 2^-58 of a unit of its last word from a rounding
// boundary.
template <int L>
__device__ __forceinline__ MPF<L> mpf_fms(const MPF<L>& c, const MPF<L>& a, const MPF<L>& b) {
    static_assert(L >= 4, "two guard words below the product window");
    constexpr int W = L + 2;
    if (mpf_zero<L>(a) || mpf_zero<L>(b)) return c;
    // window word k = product word k + L - 2: lo(a_i b_j) for i + j >= L - 2,
    // hi(a_i b_j) for i + j >= L - 3
    uint64_t S[W + 1];
#pragma unroll
    for (int k = 0; k <= W; ++k) S[k] = 0;
#pragma unroll
    for (int i = 0; i < L; ++i)
#pragma unroll
        for (int j = 0; j < L; ++j) {
            const int k = i + j - (L - 2);
            if (k >= 0) {
                const uint64_t t = (uint64_t)a.m[i] * b.m[j];
                S[k] += (uint32_t)t;
                S[k + 1] += t >> 32;
            } else if (k == -1) {
                S[0] += __umulhi(a.m[i], b.m[j]);
            }
        }
    uint32_t P[W];
    uint64_t cy = 0;
#pragma unroll
    for (int k = 0; k < W; ++k) {
        const uint64_t v = S[k] + cy;
        P[k] = (uint32_t)v;
        cy = v >> 32;
    }
    // a b ~ P 2^(ep - 32 W); normalise (the top bit may be clear)
    int ep = a.e + b.e;
    if (!(P[W - 1] >> 31)) {
#pragma unroll
        for (int i = W - 1; i > 0; --i) P[i] = __funnelshift_l(P[i - 1], P[i], 1);
        P[0] <<= 1;
        ep -= 1;
    }
    const bool sticky = true;
    uint32_t C[W];
    C[0] = 0;
    C[1] = 0;
#pragma unroll
    for (int i = 0; i < L; ++i) C[i + 2] = c.m[i];
    return add_windows<L, W>(C, c.e, c.neg, mpf_zero<L>(c), P, ep, a.neg ^ b.neg ^ 1, false, sticky);
}

// Out-of-line copies of the fused multiply-subtract and the product.  A kernel
// whose warps run several of them at once on different code paths (the LU
// panel) then keeps one copy of each in the instruction cache instead of one
// per call site.  The fused multiply-subtract takes its operands and returns
// its result by value (in registers); the product works on operands in
// memory (shared memory in the panel), by address.
template <int L>
__device__ __noinline__ MPF<L> mpf_fms_oolv(MPF<L> c, MPF<L> a, MPF<L> b) {
    return mpf_fms<L>(c, a, b);
}

template <int L>
__device__ __noinline__ void mpf_mul_ool(MPF<L>* out, const MPF<L>* a, const MPF<L>* b) {
    *out = mpf_mul<L>(*a, *b);
}

// c - a b by the inline (OOL = false) or the out-of-line copy
template <int L, bool OOL>
__device__ __forceinline__ MPF<L> mpf_fms_sel(const MPF<L>& c, const MPF<L>& a, const MPF<L>& b) {
    if constexpr (OOL) {
        return mpf_fms_oolv<L>(c, a, b);
    } else {
        return mpf_fms<L>(c, a, b);
    }
}

template <int L>
__device__ __forceinline__ MPF<L> mpf_from_double(double v) {
    return mpf_from_exp<L, 1>(&v);
}

template <int L>
__device__ __forceinline__ MPF<L> mpf_one() {
    MPF<L> r = mpf_make_zero<L>();
    r.m[L - 1] = 0x80000000u;
    r.e = 1;
    return r;
}

// (top word of |a|)^2: a^2 to about 30 bits, positive (integer pipes only)
template <int L>
__device__ __forceinline__ MPF<L> mpf_top_square(const MPF<L>& a) {
    MPF<L> r = mpf_make_zero<L>();
    if (mpf_zero<L>(a)) return r;
    // |a| ~ m_top 2^(a.e - 32), a^2 ~ q 2^(2 a.e - 64) with q = m_top^2 >= 2^62
    uint64_t q = (uint64_t)a.m[L - 1] * a.m[L - 1];
    int e = 2 * a.e;
    if (!(q >> 63)) {
        q <<= 1;
        e -= 1;
    }
    r.m[L - 1] = (uint32_t)(q >> 32);
    r.m[L - 2] = (uint32_t)q;
    r.e = e;
    return r;
}

// the same value with K < L words (low words zero)
template <int L, int K>
__device__ __forceinline__ MPF<L> mpf_widen(const MPF<K>& a) {
    MPF<L> r;
#pragma unroll
    for (int i = 0; i < L - K; ++i) r.m[i] = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) r.m[L - K + i] = a.m[i];
    r.e = a.e;
    r.neg = a.neg;
    return r;
}

// 1 / f to about 60 bits for f = T 2^-64 + (lower bits) in [1/2, 1),
// T in [2^63, 2^64): a binary32 reciprocal of the top 24 bits (relative error
// below 2^-22), then two Newton steps r <- r + r e, e = 1 - T r 2^-64, in
// 62-bit fixed point R = r 2^62 with 64 x 64-bit integer products (error
// about 2^-44, then about 2^-61, the limit of R and of T).  No binary64.
__device__ __forceinline__ MPF<4> mpf_recip_seed(uint64_t T) {
    const float tf = (float)(uint32_t)(T >> 40);  // [2^23, 2^24), exact
    const uint32_t bits = __float_as_uint(__frcp_rn(tf));
    const int ex = (int)((bits >> 23) & 0xffu) - 127;  // 1 / tf in (2^-24, 2^-23]: -24 or -23
    uint64_t R = (uint64_t)((bits & 0x7fffffu) | 0x800000u) << (ex + 63);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        // E = 2^126 - T R (signed 128-bit), e = E 2^-126; |E| < 2^104, then < 2^82,
        // so E >> sh fits in 63 bits
        const uint64_t lo = T * R, hi = __umul64hi(T, R);
        const uint64_t elo = 0ull - lo;
        const uint64_t ehi = (1ull << 62) - hi - (lo != 0ull ? 1ull : 0ull);
        const int sh = s == 0 ? 41 : 20;
        const int64_t es = (int64_t)((ehi << (64 - sh)) | (elo >> sh));
        // R e = R es 2^(sh - 126) = umulhi(R, |es|) 2^(sh - 62)
        const uint64_t d = __umul64hi(R, es < 0 ? (uint64_t)(-es) : (uint64_t)es) >> (62 - sh);
        R = es < 0 ? R - d : R + d;
    }
    // r = R 2^-62 as a 4-word float: R normalised into the top two words
    const int z = __clzll((long long)R);
    const uint64_t M = R << z;
    MPF<4> r;
    r.m[3] = (uint32_t)(M >> 32);
    r.m[2] = (uint32_t)M;
    r.m[1] = 0;
    r.m[0] = 0;
    r.e = 2 - z;
    r.neg = 0;
    return r;
}

// 1 / b on the mantissa f = |b| 2^-e in [1/2, 1), the exponent applied last.
// From the seed r (above), the residual e = 1 - f r of one fused multiply-
// subtract (a single rounding) gives r = (1 - e) / f exactly, so
//   r (1 + e)       = (1 - e^2) / f   (second order),
//   r (1 + e + e^2) = (1 - e^3) / f   (third order, e^2 from the top word of e),
// each formed as r + r t by one more fused multiply-subtract.  A 4-word step
// on the top 128 bits of f goes first (third order, about 180 bits, for
// L = 4; second order, about 120 bits, otherwise), then one L-word step:
// second order (about 240 bits) for L <= 7, third order (about 360 bits) for
// L <= 11; longer formats continue with second-order steps.  Everything runs
// on the integer pipes apart from one binary32 reciprocal.  OOL: the fused
// multiply-subtracts through their out-of-line copies.
template <int L, bool OOL = false>
__device__ __forceinline__ MPF<L> mpf_recip(const MPF<L>& b) {
    static_assert(L >= 4, "a 4-word first step");
    MPF<4> r4 = mpf_recip_seed(((uint64_t)b.m[L - 1] << 32) | b.m[L - 2]);
    MPF<4> f4;
#pragma unroll
    for (int i = 0; i < 4; ++i) f4.m[i] = b.m[L - 4 + i];
    f4.e = 0;
    f4.neg = 0;
    {
        MPF<4> t4 = mpf_fms_sel<4, OOL>(mpf_one<4>(), f4, r4);
        if (L == 4) t4 = mpf_add<4>(t4, mpf_top_square<4>(t4));
        r4 = mpf_fms_sel<4, OOL>(r4, r4, mpf_neg<4>(t4));
    }
    MPF<L> r = mpf_widen<L, 4>(r4);
    if (L > 4) {
        MPF<L> f = b;
        f.neg = 0;
        f.e = 0;
        MPF<L> t = mpf_fms_sel<L, OOL>(mpf_one<L>(), f, r);
        if (L > 7) t = mpf_add<L>(t, mpf_top_square<L>(t));
        r = mpf_fms_sel<L, OOL>(r, r, mpf_neg<L>(t));
        for (int prec = L > 7 ? 360 : 240; prec < 32 * L + 8; prec *= 2) {
            t = mpf_fms_sel<L, OOL>(mpf_one<L>(), f, r);
            r = mpf_fms_sel<L, OOL>(r, r, mpf_neg<L>(t));
        }
    }
    r.e -= b.e;
    r.neg = b.neg;
    return r;
}

}  // namespace ozlu
