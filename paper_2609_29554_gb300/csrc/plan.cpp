// Host planner: modulus set, CRT constants and the (S, w, N_mod) rule.
//
// Sec. 3.2: the 54 pairwise-coprime maximal prime powers <= 255 (taken in
// descending order), slack = ceil(log2 2K) + 16 + g_ex, and for S = 1, 2, ...
// w = ceil((p + slack)/S), need = 2w + log2 K + log2 S + 5, N_mod = the
// number of moduli whose cumulative log2 first exceeds need; the smallest S
// that has such an N_mod and meets the accumulator condition is taken.
// CRT constants M_l = P/m_l and y_l = M_l^-1 mod m_l (Eq. (11)).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "ozlu_internal.h"

namespace ozlu {
namespace {

bool is_prime(int v) {
    if (v < 2) return false;
    for (int d = 2; (long long)d * d <= v; ++d)
        if (v % d == 0) return false;
    return true;
}

std::vector<int> int8_set() {
    std::vector<int> ms;
    for (int q = 2; q <= 255; ++q) {
        if (!is_prime(q)) continue;
        int v = q;
        while (v * q <= 255) v *= q;
        ms.push_back(v);
    }
    std::sort(ms.begin(), ms.end(), [](int a, int b) { return a > b; });
    return ms;
}

// Eq. (17): K (m/2)^2 < 2^53, largest primes first.
std::vector<int> fp64_set(int K, int count) {
    const unsigned __int128 lim = (unsigned __int128)1 << 55;
    long long b = (long long)floor(sqrt(ldexp(1.0, 55) / K));
    while (b > 1 && (unsigned __int128)K * b * b >= lim) --b;
    while ((unsigned __int128)K * (b + 1) * (b + 1) < lim) ++b;
    std::vector<int> ms;
    for (long long v = b; v > 2 && (int)ms.size() < count; --v)
        if (is_prime((int)v)) ms.push_back((int)v);
    return ms;
}

void mul_small(std::vector<uint32_t>& a, uint32_t f) {
    uint64_t carry = 0;
    for (auto& w : a) {
        uint64_t v = (uint64_t)w * f + carry;
        w = (uint32_t)v;
        carry = v >> 32;
    }
    if (carry) a.push_back((uint32_t)carry);
}

std::vector<uint32_t> div_small(const std::vector<uint32_t>& a, uint32_t d) {
    std::vector<uint32_t> q(a.size());
    uint64_t rem = 0;
    for (int i = (int)a.size() - 1; i >= 0; --i) {
        uint64_t cur = (rem << 32) | a[i];
        q[i] = (uint32_t)(cur / d);
        rem = cur % d;
    }
    while (q.size() > 1 && q.back() == 0) q.pop_back();
    return q;
}

uint32_t mod_small(const std::vector<uint32_t>& a, uint32_t d) {
    uint64_t rem = 0;
    for (int i = (int)a.size() - 1; i >= 0; --i) rem = ((rem << 32) | a[i]) % d;
    return (uint32_t)rem;
}

int inv_mod(int a, int m) {
    long long t = 0, nt = 1, r = m, nr = a % m;
    while (nr) {
        long long q = r / nr;
        long long tmp = t - q * nt; t = nt; nt = tmp;
        tmp = r - q * nr; r = nr; nr = tmp;
    }
    if (t < 0) t += m;
    return (int)t;
}

int ceil_log2(double v) { return (int)ceil(log2(v) - 1e-12); }

}  // namespace

// Eq. (Lhint): the cost-model estimate of the slice count,
// S* = ceil(sqrt(r n_d (M + N) / (M N))), n_d = ceil(t / 16), with r the ratio
// of per-digit residue cost to per-flop GEMM cost (30 for INT8, 17.9 for
// binary64 in the paper) and t the width of one unsplit pass (p + slack)
int lhint_S(double r, int t, int M, int N) {
    if (M < 1 || N < 1 || t < 1) return 1;
    const double nd = (double)((t + 15) / 16);
    const int s = (int)ceil(sqrt(r * nd * ((double)M + N) / ((double)M * N)) - 1e-12);
    return s < 1 ? 1 : s;
}

int make_plan(int p, int K, const ozlu_opts* o, Plan& out) {
    ozlu_opts d;
    memset(&d, 0, sizeof d);
    if (!o) o = &d;
    const int be = o->backend == OZLU_BE_AUTO ? OZLU_BE_INT8 : o->backend;
    if (p < 1 || K < 1) return OZLU_ERR_CAPACITY;
    if (be != OZLU_BE_INT8 && be != OZLU_BE_FP8 && be != OZLU_BE_FP64 && be != OZLU_BE_FP16) return -1;
    const int slack = ceil_log2(2.0 * K) + 16 + o->g_ex;
    const int Kpad = (K + 127) / 128 * 128;
    std::vector<int> mods = be == OZLU_BE_FP64 ? fp64_set(K, MAXMOD) : int8_set();
    int s_lo = o->nslice > 0 ? o->nslice : 1;
    int s_hi = o->nslice > 0 ? o->nslice : 64;
    for (int S = s_lo; S <= s_hi; ++S) {
        // accumulator conditions: INT32 (Sec. 3.2), FP32 for the base-17
        // Karatsuba planes (|digit sums| <= 15)
        if (be == OZLU_BE_INT8 && (double)Kpad * S * 127.0 * 127.0 >= ldexp(1.0, 31)) continue;
        if (be == OZLU_BE_FP8 && (double)Kpad * S * 225.0 >= ldexp(1.0, 24)) continue;
        // Eq. (14): binary16 residues with an fp32 accumulator
        if (be == OZLU_BE_FP16 && (double)Kpad * S * 127.0 * 127.0 >= ldexp(1.0, 24)) continue;
        const int w = (p + slack + S - 1) / S;
        const double need = 2.0 * w + log2((double)K) + log2((double)S) + 5.0;
        double cum = 0.0;
        int N = 0;
        for (int i = 0; i < (int)mods.size(); ++i) {
            cum += log2((double)mods[i]);
            if (cum > need) { N = i + 1; break; }
        }
        if (N == 0) continue;
        Plan pl;
        pl.p = p; pl.K = K; pl.Kpad = Kpad; pl.backend = be; pl.g_ex = o->g_ex;
        pl.extra = o->extra_groups < 0 ? 0 : o->extra_groups;
        pl.S = S; pl.w = w; pl.Q = w * S; pl.N = N; pl.need = need;
        pl.g0 = std::max(0, S - 1 - pl.extra);
        pl.G = 2 * S - 1 - pl.g0;
        pl.pair_terms = 0;
        for (int g = pl.g0; g <= 2 * S - 2; ++g) pl.pair_terms += std::min(g, 2 * S - 2 - g) + 1;
        std::vector<uint32_t> P{1};
        for (int i = 0; i < N; ++i) { pl.mod[i] = mods[i]; mul_small(P, (uint32_t)mods[i]); }
        pl.P = P;
        pl.M.resize(N);
        for (int i = 0; i < N; ++i) {
            pl.M[i] = div_small(P, (uint32_t)mods[i]);
            pl.y[i] = inv_mod((int)mod_small(pl.M[i], (uint32_t)mods[i]), mods[i]);
        }
        // |S_g| <= pairs K 2^(2w-2), pairs <= S: two's complement width
        pl.sbar_bits = 2 * w - 1 + ceil_log2((double)S * K) + 1;
        pl.WG = (pl.sbar_bits + 31) / 32;
        pl.pint_bits = w * (2 * S - 2 - pl.g0) + pl.sbar_bits;
        pl.WX = (pl.Q + 1 + 31) / 32;
        pl.H = (w + 1 + 15) / 16;
        // 32-bit t values of the binary64 back-end: sum t M_l < 2^64 needs N <= 32
        if (be == OZLU_BE_FP64 && N > 32) return OZLU_ERR_CAPACITY;
        if (N > MAXMOD || pl.WG > MAXWG || pl.WX > MAXWX || pl.H > MAXH || pl.G > MAXG ||
            pl.pint_bits + 2 > WINDOW_BITS)
            return OZLU_ERR_CAPACITY;
        out = pl;
        return OZLU_OK;
    }
    return OZLU_ERR_CAPACITY;
}

// The same rule for p-bit multi-limb inputs (INT8 residues): S is not
// bounded by the expansion kernels' fixed windows (S digits are produced one
// at a time from the limbs and the CRT accumulates in a window sized from
// the plan), only by the device tables (N_mod, words of S_g, 16-bit chunks
// of a digit) and the INT32 accumulator condition.
int make_plan_mp(int p, int K, Plan& out) {
    if (p < 1 || K < 1) return OZLU_ERR_CAPACITY;
    const int slack = ceil_log2(2.0 * K) + 16;
    const int Kpad = (K + 127) / 128 * 128;
    const std::vector<int> mods = int8_set();
    for (int S = 1; S <= 4096; ++S) {
        if ((double)Kpad * S * 127.0 * 127.0 >= ldexp(1.0, 31)) break;
        const int w = (p + slack + S - 1) / S;
        const double need = 2.0 * w + log2((double)K) + log2((double)S) + 5.0;
        double cum = 0.0;
        int N = 0;
        for (int i = 0; i < (int)mods.size(); ++i) {
            cum += log2((double)mods[i]);
            if (cum > need) { N = i + 1; break; }
        }
        if (N == 0) continue;
        Plan pl;
        pl.p = p; pl.K = K; pl.Kpad = Kpad; pl.backend = OZLU_BE_INT8;
        pl.S = S; pl.w = w; pl.Q = w * S; pl.N = N; pl.need = need;
        pl.g0 = S - 1;
        pl.G = S;
        pl.pair_terms = 0;
        for (int g = pl.g0; g <= 2 * S - 2; ++g) pl.pair_terms += std::min(g, 2 * S - 2 - g) + 1;
        std::vector<uint32_t> P{1};
        for (int i = 0; i < N; ++i) { pl.mod[i] = mods[i]; mul_small(P, (uint32_t)mods[i]); }
        pl.P = P;
        pl.M.resize(N);
        for (int i = 0; i < N; ++i) {
            pl.M[i] = div_small(P, (uint32_t)mods[i]);
            pl.y[i] = inv_mod((int)mod_small(pl.M[i], (uint32_t)mods[i]), mods[i]);
        }
        pl.sbar_bits = 2 * w - 1 + ceil_log2((double)S * K) + 1;
        pl.WG = (pl.sbar_bits + 31) / 32;
        pl.pint_bits = w * (2 * S - 2 - pl.g0) + pl.sbar_bits;
        pl.WX = 0;
        pl.H = (w + 1 + 15) / 16;
        if (N > MAXMOD || pl.WG > MAXWG || pl.H > MAXH) return OZLU_ERR_CAPACITY;
        out = pl;
        return OZLU_OK;
    }
    return OZLU_ERR_CAPACITY;
}

namespace {
// Sec. 4.2.4: the 54 INT8 moduli and the primes in (255, 16191], descending
const std::vector<int>& ext_set() {
    static const std::vector<int> ms = [] {
        std::vector<int> v = int8_set();
        for (int q = 257; q <= 16191; q += 2)
            if (is_prime(q)) v.push_back(q);
        std::sort(v.begin(), v.end(), [](int a, int b) { return a > b; });
        return v;
    }();
    return ms;
}
}  // namespace

// The rule of Sec. 3.2 with the extended table of Sec. 4.2.4: the moduli are
// taken from the 1882-entry table (largest first), every modulus costs three
// int8 Karatsuba planes whose products are bounded like INT8 residues
// (|r0|, |q|, |r0 + q| <= 127), so the accumulator condition is unchanged.
int make_plan_mp_ext(int p, int K, int S_req, Plan& out) {
    if (p < 1 || K < 1 || S_req < 0) return OZLU_ERR_CAPACITY;
    const int slack = ceil_log2(2.0 * K) + 16;
    const int Kpad = (K + 127) / 128 * 128;
    const std::vector<int>& mods = ext_set();
    const int s_lo = S_req > 0 ? S_req : 1, s_hi = S_req > 0 ? S_req : 4096;
    for (int S = s_lo; S <= s_hi; ++S) {
        if ((double)Kpad * S * 127.0 * 127.0 >= ldexp(1.0, 31)) break;
        const int w = (p + slack + S - 1) / S;
        const double need = 2.0 * w + log2((double)K) + log2((double)S) + 5.0;
        double cum = 0.0;
        int N = 0;
        for (int i = 0; i < (int)mods.size(); ++i) {
            cum += log2((double)mods[i]);
            if (cum > need) { N = i + 1; break; }
        }
        if (N == 0) continue;
        Plan pl;
        pl.p = p; pl.K = K; pl.Kpad = Kpad; pl.backend = OZLU_BE_INT8;
        pl.S = S; pl.w = w; pl.Q = w * S; pl.N = N; pl.need = need;
        pl.g0 = S - 1;
        pl.G = S;
        pl.pair_terms = 0;
        for (int g = pl.g0; g <= 2 * S - 2; ++g) pl.pair_terms += std::min(g, 2 * S - 2 - g) + 1;
        pl.ext = true;
        pl.ext_mod.assign(mods.begin(), mods.begin() + N);
        std::vector<uint32_t> P{1};
        for (int i = 0; i < N; ++i) {
            if (i < MAXMOD) pl.mod[i] = mods[i];
            mul_small(P, (uint32_t)mods[i]);
        }
        pl.P = P;
        pl.M.resize(N);
        pl.ext_y.resize(N);
        for (int i = 0; i < N; ++i) {
            pl.M[i] = div_small(P, (uint32_t)mods[i]);
            pl.ext_y[i] = inv_mod((int)mod_small(pl.M[i], (uint32_t)mods[i]), mods[i]);
            if (i < MAXMOD) pl.y[i] = pl.ext_y[i];
        }
        pl.sbar_bits = 2 * w - 1 + ceil_log2((double)S * K) + 1;
        pl.WG = (pl.sbar_bits + 31) / 32;
        pl.pint_bits = w * (2 * S - 2 - pl.g0) + pl.sbar_bits;
        pl.WX = 0;
        pl.H = 0;
        out = pl;
        return OZLU_OK;
    }
    return OZLU_ERR_CAPACITY;
}

void build_ext_image(const Plan& pl, ExtImage& img) {
    const int N = pl.N, WG = pl.WG;
    const int WD = (pl.w + 2 + 31) / 32;  // words of one digit with its carry
    img.WD = WD;
    size_t off = 0;
    auto take = [&](size_t words) {
        const size_t o = off;
        off += (words + 63) / 64 * 64;
        return o;
    };
    img.o_mod = take(N);
    img.o_y = take(N);
    img.o_magic = take(N);
    img.o_coef = take(3 * (size_t)N);
    img.o_pw = take(N);
    img.o_two32 = take(N);
    img.o_inv40 = take(2 * (size_t)N);
    img.o_pow32 = take((size_t)WD * N);
    img.o_Mw = take((size_t)WG * N);
    img.o_Pw = take(WG);
    img.words.assign(off, 0u);
    uint32_t* w = img.words.data();
    for (int l = 0; l < N; ++l) {
        const uint32_t m = (uint32_t)pl.ext_mod[l];
        w[img.o_mod + l] = m;
        w[img.o_y + l] = (uint32_t)pl.ext_y[l];
        w[img.o_magic + l] = (uint32_t)(((1ull << 32) + m - 1) / m);
        // C = P00 + 128 (Pss - P00 - P11) + 16384 P11 = (1 - 128) P00 + (16384 - 128) P11 + 128 Pss
        w[img.o_coef + l] = (uint32_t)((m + (1 % m) - (128 % m)) % m);
        w[img.o_coef + N + l] = (uint32_t)((16384 - 128) % m);
        w[img.o_coef + 2 * N + l] = (uint32_t)(128 % m);
        uint64_t r = 1 % m;
        for (int k = 0; k < pl.w; ++k) r = (r * 2) % m;
        w[img.o_pw + l] = (uint32_t)r;
        w[img.o_two32 + l] = (uint32_t)((1ull << 32) % m);
        const uint64_t inv = (uint64_t)(((unsigned __int128)1 << 40) / m +
                                        ((((unsigned __int128)1 << 40) % m) * 2 >= m ? 1 : 0));
        w[img.o_inv40 + 2 * l] = (uint32_t)inv;
        w[img.o_inv40 + 2 * l + 1] = (uint32_t)(inv >> 32);
        uint64_t pj = 1 % m;
        for (int j = 0; j < WD; ++j) {
            w[img.o_pow32 + (size_t)j * N + l] = (uint32_t)pj;
            pj = (pj << 32) % m;
        }
        for (int j = 0; j < WG; ++j)
            w[img.o_Mw + (size_t)j * N + l] = j < (int)pl.M[l].size() ? pl.M[l][j] : 0u;
    }
    for (int j = 0; j < WG; ++j) w[img.o_Pw + j] = j < (int)pl.P.size() ? pl.P[j] : 0u;
}

void fill_table(const Plan& pl, DevTable& t) {
    memset(&t, 0, sizeof t);
    t.N = pl.N; t.WG = pl.WG; t.H = pl.H; t.S = pl.S; t.w = pl.w; t.g0 = pl.g0;
    t.G = pl.G; t.Q = pl.Q; t.WX = pl.WX;
    for (int l = 0; l < pl.N; ++l) {
        const uint32_t m = (uint32_t)pl.mod[l];
        t.mod[l] = (int)m;
        t.y[l] = pl.y[l];
        t.magic[l] = (uint32_t)(((1ull << 32) + m - 1) / m);
        t.invm[l] = 1.0f / (float)m;
        uint64_t r = 1 % m;
        for (int j = 0; j < MAXH; ++j) {
            t.pow16[l][j] = (uint32_t)r;
            r = (r << 16) % m;
        }
        // all MAXWG low words: a kernel may work modulo 2^(32 W) for any W >= WG
        for (int wd = 0; wd < MAXWG; ++wd)
            t.Mlow[l][wd] = wd < (int)pl.M[l].size() ? pl.M[l][wd] : 0u;
    }
    for (int wd = 0; wd < MAXWG; ++wd) t.Plow[wd] = wd < (int)pl.P.size() ? pl.P[wd] : 0u;
}

}  // namespace ozlu

extern "C" int ozlu_plan(int p, int k, const ozlu_opts* opts, ozlu_plan_info* out) {
    if (!out) return -4;
    ozlu::Plan pl;
    int rc = ozlu::make_plan(p, k, opts, pl);
    if (rc) return rc;
    memset(out, 0, sizeof *out);
    out->p = pl.p; out->K = pl.K; out->backend = pl.backend; out->S = pl.S; out->w = pl.w;
    out->Q = pl.Q; out->n_mod = pl.N; out->g0 = pl.g0; out->n_groups = pl.G;
    out->pair_terms = pl.pair_terms;
    for (int i = 0; i < pl.N && i < 64; ++i) out->moduli[i] = pl.mod[i];
    return OZLU_OK;
}

extern "C" int ozlu_mp_plan(int p, int k, ozlu_plan_info* out) {
    if (p < 1) return -1;
    if (k < 1) return -2;
    if (!out) return -3;
    ozlu::Plan pl;
    int rc = ozlu::make_plan_mp(p, k, pl);
    if (rc) return rc;
    memset(out, 0, sizeof *out);
    out->p = pl.p; out->K = pl.K; out->backend = pl.backend; out->S = pl.S; out->w = pl.w;
    out->Q = pl.Q; out->n_mod = pl.N; out->g0 = pl.g0; out->n_groups = pl.G;
    out->pair_terms = pl.pair_terms;
    for (int i = 0; i < pl.N && i < 64; ++i) out->moduli[i] = pl.mod[i];
    return OZLU_OK;
}

extern "C" int ozlu_mp_plan_opts(int p, int k, const ozlu_opts* opts, ozlu_plan_info* out) {
    if (p < 1) return -1;
    if (k < 1) return -2;
    if (!out) return -4;
    const bool ext = opts && opts->modset == OZLU_MODSET_EXT;
    if (opts && (opts->modset < 0 || opts->modset > OZLU_MODSET_EXT || opts->nslice < 0)) return -3;
    ozlu::Plan pl;
    const int rc = ext ? ozlu::make_plan_mp_ext(p, k, opts->nslice, pl) : ozlu::make_plan_mp(p, k, pl);
    if (rc) return rc;
    memset(out, 0, sizeof *out);
    out->p = pl.p; out->K = pl.K; out->backend = pl.backend; out->S = pl.S; out->w = pl.w;
    out->Q = pl.Q; out->n_mod = pl.N; out->g0 = pl.g0; out->n_groups = pl.G;
    out->pair_terms = pl.pair_terms;
    for (int i = 0; i < pl.N && i < 64; ++i) out->moduli[i] = ext ? pl.ext_mod[i] : pl.mod[i];
    return OZLU_OK;
}
