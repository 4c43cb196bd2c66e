// Host build of the binary64 expansion arithmetic (paper_2609_29554_gb300/csrc/expansion.cuh),
// which serves the native per-element LU comparison and the non-cooperative panel
// column kernels, for CPU tests: seeded operands and results printed as hex
// floats for an exact check in Python.
//
// Output, one case per line: "op N" then the operands' and the result's
// components (N each).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>

#define __device__
#define __forceinline__ inline
using std::fma;

#include "expansion.cuh"

using namespace ozlu;

template <int N>
static Exp<N> rnd(std::mt19937_64& g, int emin, int emax) {
    Exp<N> a;
    a.x[0] = ((g() & 1) ? -1.0 : 1.0) * std::ldexp(1.0 + (double)(g() >> 12) * 0x1p-52,
                                                    emin + (int)(g() % (uint64_t)(emax - emin + 1)));
    for (int c = 1; c < N; ++c) {
        const int e = std::ilogb(a.x[c - 1]) - 54 - (int)(g() % 4);
        a.x[c] = ((g() & 1) ? -1.0 : 1.0) * std::ldexp(1.0 + (double)(g() >> 12) * 0x1p-52, e);
    }
    return a;
}

template <int N>
static void put(const Exp<N>& a) {
    for (int c = 0; c < N; ++c) printf(" %a", a.x[c]);
}

template <int N>
static void run(int n, uint64_t seed) {
    std::mt19937_64 g(seed);
    for (int i = 0; i < n; ++i) {
        const Exp<N> a = rnd<N>(g, -20, 20);
        Exp<N> b = rnd<N>(g, -20, 20);
        if (i % 4 == 0) {  // near cancellation in a + b
            b = a;
            b.x[0] = -a.x[0];
            for (int c = 1; c < N; ++c) b.x[c] = -a.x[c] * (1.0 + 0x1p-40 * (double)(g() % 7));
        }
        const Exp<N> c = rnd<N>(g, -20, 20);
        printf("add %d", N); put<N>(a); put<N>(b); put<N>(add<N>(a, b)); printf("\n");
        printf("mul %d", N); put<N>(a); put<N>(b); put<N>(mul<N>(a, b)); printf("\n");
        printf("div %d", N); put<N>(a); put<N>(c); put<N>(div<N>(a, c)); printf("\n");
        printf("fms %d", N); put<N>(c); put<N>(a); put<N>(b); put<N>(fms<N>(c, a, b)); printf("\n");
    }
}

int main(int argc, char** argv) {
    const int n = argc > 1 ? atoi(argv[1]) : 500;
    run<2>(n, 1);
    run<3>(n, 2);
    run<4>(n, 3);
    return 0;
}
