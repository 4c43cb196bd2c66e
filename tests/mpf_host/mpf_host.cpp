// Host build of the device multi-limb float arithmetic (paper_2609_29554_gb300/csrc/mpf.cuh)
// for CPU tests: the CUDA intrinsics it uses are given portable definitions
// with the same results, the header is compiled as plain C++, and seeded
// cases are printed for an exact check in Python.
//
// Output, one case per line: an op name, then each operand and the result as
// "neg e m[L-1] ... m[0]" (words in hex), value = (-1)^neg m 2^(e - 32 L).
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>

#define __device__
#define __forceinline__ inline
#define __noinline__
static inline int __clz(uint32_t x) { return x ? __builtin_clz(x) : 32; }
static inline int __clzll(long long x) { return x ? __builtin_clzll((unsigned long long)x) : 64; }
static inline long long __double_as_longlong(double d) { long long r; memcpy(&r, &d, 8); return r; }
static inline double __longlong_as_double(long long x) { double r; memcpy(&r, &x, 8); return r; }
static inline uint32_t __float_as_uint(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static inline float __frcp_rn(float x) { volatile float one = 1.0f; return one / x; }
static inline uint32_t __umulhi(uint32_t a, uint32_t b) { return (uint32_t)(((uint64_t)a * b) >> 32); }
static inline uint64_t __umul64hi(uint64_t a, uint64_t b) { return (uint64_t)(((unsigned __int128)a * b) >> 64); }
static inline uint32_t __funnelshift_l(uint32_t lo, uint32_t hi, uint32_t s) {
    s &= 31;
    return s ? (hi << s) | (lo >> (32 - s)) : hi;
}
static inline uint32_t __funnelshift_r(uint32_t lo, uint32_t hi, uint32_t s) {
    s &= 31;
    return s ? (lo >> s) | (hi << (32 - s)) : lo;
}

#include "mpf.cuh"

using namespace ozlu;

template <int L>
static void put(const MPF<L>& a) {
    printf(" %d %d", a.neg, a.e);
    for (int i = L - 1; i >= 0; --i) printf(" %08x", a.m[i]);
}

template <int L>
static MPF<L> rnd(std::mt19937_64& g, int emin, int emax) {
    MPF<L> v;
    for (int i = 0; i < L; ++i) v.m[i] = (uint32_t)g();
    v.m[L - 1] |= 0x80000000u;
    v.e = emin + (int)(g() % (uint64_t)(emax - emin + 1));
    v.neg = (int)(g() & 1);
    return v;
}

template <int L>
static void run(int n, uint64_t seed) {
    std::mt19937_64 g(seed);
    for (int i = 0; i < n; ++i) {
        MPF<L> a = rnd<L>(g, -3, 3), b, c = rnd<L>(g, -6, 6);
        const int kind = i % 8;
        if (kind == 0) { b = a; b.m[0] ^= (uint32_t)g(); b.neg ^= 1; }                 // cancellation
        else if (kind == 1) { b = a; b.neg ^= 1; }                                      // exact zero sum
        else if (kind == 2) { b = a; b.m[L - 2] ^= 1u; b.neg ^= 1; }                    // deep cancellation
        else if (kind == 3) { b = rnd<L>(g, -3 - 32 * (L + 3), 3); }                    // far apart
        else if (kind == 4) { b = a; b.e -= 1 + (int)(g() % 70); }
        else b = rnd<L>(g, -40, 40);
        if (i % 97 == 0) b = mpf_make_zero<L>();
        if (i % 5 == 0) { c = a; c.e = a.e + b.e; }                                      // c ~ a b
        printf("mul %d", L); put<L>(a); put<L>(b); put<L>(mpf_mul<L>(a, b)); printf("\n");
        printf("add %d", L); put<L>(a); put<L>(b); put<L>(mpf_add<L>(a, b)); printf("\n");
        printf("fms %d", L); put<L>(c); put<L>(a); put<L>(b); put<L>(mpf_fms<L>(c, a, b)); printf("\n");
        // exact cancellation: c = a b exactly (a, b with few significant bits)
        if (i % 4 == 0) {
            const double x = (double)(g() % 100000 + 1) * ((g() & 1) ? -1.0 : 1.0);
            const double y = (double)(g() % 100000 + 1);
            const MPF<L> xa = mpf_from_double<L>(x), yb = mpf_from_double<L>(y);
            const MPF<L> cc = mpf_from_double<L>(x * y);
            printf("fms %d", L); put<L>(cc); put<L>(xa); put<L>(yb); put<L>(mpf_fms<L>(cc, xa, yb)); printf("\n");
        }
        // reciprocal: random, f = 1/2, all-ones, a single low bit
        MPF<L> r = rnd<L>(g, -2000, 2000);
        if (i % 7 == 1) { for (int k = 0; k < L; ++k) r.m[k] = 0; r.m[L - 1] = 0x80000000u; }
        if (i % 7 == 2) { for (int k = 0; k < L; ++k) r.m[k] = 0xffffffffu; }
        if (i % 7 == 3) { for (int k = 0; k < L - 1; ++k) r.m[k] = 0; r.m[0] = 1u; r.m[L - 1] = 0x80000000u; }
        printf("recip %d", L); put<L>(r); put<L>(mpf_recip<L>(r)); printf("\n");
    }
}

// conversions between N-component binary64 expansions and L-word floats
static double rnd_exp_component(std::mt19937_64& g, double prev) {
    // below a quarter ulp of the previous component, random sign and size
    const int e = std::ilogb(prev) - 54 - (int)(g() % 30);
    const double m = 1.0 + (double)(g() >> 12) * 0x1p-52;
    return ((g() & 1) ? -1.0 : 1.0) * std::ldexp(m, e);
}

template <int L, int N>
static void run_conv(int n, uint64_t seed) {
    std::mt19937_64 g(seed);
    for (int i = 0; i < n; ++i) {
        double x[N];
        x[0] = ((g() & 1) ? -1.0 : 1.0) * std::ldexp(1.0 + (double)(g() >> 12) * 0x1p-52, (int)(g() % 81) - 40);
        for (int c = 1; c < N; ++c) x[c] = rnd_exp_component(g, x[c - 1]);
        if (i % 9 == 1) x[N - 1] = 0.0;                      // trailing zero component
        if (i % 9 == 2) x[0] = std::ldexp(1.0, (int)(g() % 20));  // power-of-two leader
        if (i % 9 == 3 && N > 2) { x[1] = 0.0; }              // interior zero
        printf("fromexp %d %d", L, N);
        for (int c = 0; c < N; ++c) printf(" %a", x[c]);
        put<L>(mpf_from_exp<L, N>(x));
        printf("\n");
        const MPF<L> a = rnd<L>(g, -60, 60);
        double out[N];
        mpf_to_exp<L, N>(a, out);
        printf("toexp %d %d", L, N);
        put<L>(a);
        for (int c = 0; c < N; ++c) printf(" %a", out[c]);
        printf("\n");
    }
}

// x mod m by one high multiply (mp_device.cuh mod_small, used for residues and
// t values) against the % operator: every modulus m <= 255 and every m of the
// extended table's range up to 16191 (odd m from 257, the primes among them
// included), x over edges and a seeded sample of [0, 2^32)
static void run_mod() {
    std::mt19937_64 g(7);
    long long n = 0, bad = 0;
    for (uint32_t m = 2; m <= 16191; m += (m < 255 ? 1 : 2)) {
        const uint32_t magic = (uint32_t)(((1ull << 32) + m - 1) / m);
        auto check = [&](uint32_t x) {
            ++n;
            bad += mod_small(x, m, magic) != x % m;
        };
        for (uint32_t x = 0; x < 4096; ++x) check(x);
        for (uint32_t k = 1; k < 64; ++k) {
            const uint64_t top = (1ull << 32) - 1;
            check((uint32_t)(top - k));
            const uint64_t mult = (top / m - k) * m;
            check((uint32_t)mult);
            check((uint32_t)(mult - 1));
            check((uint32_t)(mult + 1));
        }
        for (int i = 0; i < (m <= 255 ? 20000 : 1500); ++i) check((uint32_t)g());
    }
    printf("mod %lld %lld\n", n, bad);
}

int main(int argc, char** argv) {
    const int n = argc > 1 ? atoi(argv[1]) : 1000;
    run<4>(n, 1);
    run<6>(n, 2);
    run<7>(n, 7);
    run<8>(n, 3);
    run_conv<4, 2>(n, 4);
    run_conv<6, 3>(n, 5);
    run_conv<7, 4>(n, 8);
    run_conv<8, 4>(n, 6);
    run_mod();
    return 0;
}
