// Planner of the allocation-free GEMM (ozlu_gemm_noalloc): the INT8 plan of
// Sec. 3.2 "Determining w and N" (the 54 maximal prime powers <= 255 in
// descending order, slack = ceil(log2 2K) + 16, w = ceil((p + slack)/S),
// need = 2w + log2 K + log2 S + 5, the smallest S with enough capacity under
// K_pad S 127^2 < 2^31) and the CRT constants of Eq. (11), written straight
// into the kernels' constant table with fixed-size arrays: it allocates no
// memory, host or device.  Host code only.
#include <math.h>
#include <string.h>

#include "ozlu_internal.h"

namespace ozlu {
namespace {

constexpr int PW = 16;  // words of P (54 moduli of <= 8 bits: <= 432 bits)

bool is_prime_na(int v) {
    if (v < 2) return false;
    for (int d = 2; d * d <= v; ++d)
        if (v % d == 0) return false;
    return true;
}

// the 54 maximal prime powers <= 255, descending (Sec. 3.2)
int int8_moduli_na(int* out) {
    int cnt = 0;
    for (int q = 2; q <= 255; ++q) {
        if (!is_prime_na(q)) continue;
        int v = q;
        while (v * q <= 255) v *= q;
        out[cnt++] = v;
    }
    for (int i = 0; i < cnt; ++i)
        for (int j = i + 1; j < cnt; ++j)
            if (out[j] > out[i]) { const int t = out[i]; out[i] = out[j]; out[j] = t; }
    return cnt;
}

int inv_mod_na(int a, int m) {
    long long t = 0, nt = 1, r = m, nr = a % m;
    while (nr) {
        const long long q = r / nr;
        long long tmp = t - q * nt; t = nt; nt = tmp;
        tmp = r - q * nr; r = nr; nr = tmp;
    }
    return (int)(t < 0 ? t + m : t);
}

}  // namespace

// INT8 plan of Sec. 3.2 into a DevTable, fixed-size arrays only
int plan_noalloc(int p, int K, DevTable& t, int& Kpad_out) {
    memset(&t, 0, sizeof t);
    if (p < 1 || K < 1) return OZLU_ERR_CAPACITY;
    int mods[64];
    const int nm = int8_moduli_na(mods);
    const int slack = (int)ceil(log2(2.0 * K) - 1e-12) + 16;
    const int Kpad = (K + 127) / 128 * 128;
    for (int S = 1; S <= 64; ++S) {
        if ((double)Kpad * S * 127.0 * 127.0 >= ldexp(1.0, 31)) continue;
        const int w = (p + slack + S - 1) / S;
        const double need = 2.0 * w + log2((double)K) + log2((double)S) + 5.0;
        double cum = 0.0;
        int N = 0;
        for (int i = 0; i < nm; ++i) {
            cum += log2((double)mods[i]);
            if (cum > need) { N = i + 1; break; }
        }
        if (N == 0) continue;
        const int g0 = S - 1, G = S;
        const int sbar_bits = 2 * w - 1 + (int)ceil(log2((double)S * K) - 1e-12) + 1;
        const int WG = (sbar_bits + 31) / 32;
        const int pint_bits = w * (2 * S - 2 - g0) + sbar_bits;
        const int WX = (w * S + 1 + 31) / 32;
        const int H = (w + 1 + 15) / 16;
        if (WG > MAXWG || WX > MAXWX || H > MAXH || G > MAXG || pint_bits + 2 > WINDOW_BITS)
            return OZLU_ERR_CAPACITY;
        // P and M_l as little-endian 32-bit words
        uint32_t P[PW] = {1};
        for (int i = 0; i < N; ++i) {
            uint64_t c = 0;
            for (int wd = 0; wd < PW; ++wd) {
                const uint64_t v = (uint64_t)P[wd] * (uint32_t)mods[i] + c;
                P[wd] = (uint32_t)v;
                c = v >> 32;
            }
        }
        t.N = N; t.WG = WG; t.H = H; t.S = S; t.w = w; t.g0 = g0; t.G = G; t.Q = w * S; t.WX = WX;
        for (int l = 0; l < N; ++l) {
            const uint32_t m = (uint32_t)mods[l];
            uint32_t M[PW];
            uint64_t rem = 0;
            for (int wd = PW - 1; wd >= 0; --wd) {
                const uint64_t cur = (rem << 32) | P[wd];
                M[wd] = (uint32_t)(cur / m);
                rem = cur % m;
            }
            uint64_t mm = 0;
            for (int wd = PW - 1; wd >= 0; --wd) mm = ((mm << 32) | M[wd]) % m;
            t.mod[l] = (int)m;
            t.y[l] = inv_mod_na((int)mm, (int)m);
            t.magic[l] = (uint32_t)(((1ull << 32) + m - 1) / m);
            t.invm[l] = 1.0f / (float)m;
            uint64_t r = 1 % m;
            for (int j = 0; j < MAXH; ++j) {
                t.pow16[l][j] = (uint32_t)r;
                r = (r << 16) % m;
            }
            for (int wd = 0; wd < MAXWG; ++wd) t.Mlow[l][wd] = wd < PW ? M[wd] : 0u;
        }
        for (int wd = 0; wd < MAXWG; ++wd) t.Plow[wd] = wd < PW ? P[wd] : 0u;
        Kpad_out = Kpad;
        return OZLU_OK;
    }
    return OZLU_ERR_CAPACITY;
}

}  // namespace ozlu
