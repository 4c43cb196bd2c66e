// p-bit multi-limb matrices: the Ozaki-II GEMM (ozlu_mp_gemm) with INT8
// residues, for the arbitrary-precision LU of Sec. 3.4 / Sec. 4.4.
//
// The steps are those of Sec. 3.1 with a p-bit significand in place of the
// expansion:
//   (S1) mu_i = (Q - 1) - max_h exps(a_ih) (0 for an all-zero row), nu_j likewise
//   (S2) X = trunc(a 2^mu) read directly from the limbs, S balanced w-bit
//        digits (Eq. (2)) formed one after the other with the carry between
//        them (the digits of a negative X follow from those of |X|)
//   (S3) centered residues of each digit by 16-bit chunks and the 2^(16 j)
//        mod m table, stored as the INT8 planes of ozlu_gemm
//   (S4)-(S5) the INT8 residue GEMMs and their modular epilogue (shared with
//        ozlu_gemm; G = S digit groups g = S-1 .. 2S-2)
//   (S6) one thread per output: every S_g (Eq. (11), modulo 2^(32 WG)) is
//        added at bit w (g - g0) of an accumulator of NW words in shared
//        memory, streamed through a short register window of signed 64-bit
//        word sums (the sign of each S_g only reaches one word above it);
//        the old C is truncated onto the grid and added; the exact sum is
//        rounded once to p bits (round to nearest even).  The accumulator
//        holds the largest P_int with 64 bits to spare; an old C reaching
//        above it raises the grid (the product integer is truncated onto it).
// The output is processed in column chunks that bound the t values.
#include <limits.h>
#include <string.h>

#include "mp_device.cuh"
#include "ozlu_handle.h"

namespace ozlu {
namespace {

constexpr int MPD = 9;      // words of one digit with its carry (w <= 254)
constexpr int MPCT = 64;    // threads per block of the CRT kernel

struct MPView {
    uint32_t* limbs;
    int* exps;
    int* signs;
    long long ld, plane;
    int L;
};

MPView view_of(const ozlu_mp_matrix& M, long long off) {
    return MPView{M.limbs + off, M.exps + off, M.signs + off, M.ld, M.plane, M.L};
}

__device__ __forceinline__ bool mp_zero(const MPView& X, long long x) {
    return X.limbs[(long long)(X.L - 1) * X.plane + x] == 0;
}

// bits [pos, pos + 32) of the magnitude of element x (zeros outside [0, 32 L))
__device__ __forceinline__ uint32_t mant32(const MPView& X, long long x, long long pos) {
    if (pos >= 32LL * X.L || pos <= -32) return 0;
    const long long q = pos >= 0 ? (pos >> 5) : -((-pos + 31) >> 5);
    const int r = (int)(pos - 32 * q);
    const uint32_t lo = (q >= 0 && q < X.L) ? X.limbs[q * X.plane + x] : 0u;
    const uint32_t hi = (q + 1 >= 0 && q + 1 < X.L) ? X.limbs[(q + 1) * X.plane + x] : 0u;
    return r ? (lo >> r) | (hi << (32 - r)) : lo;
}

// (S1) shared exponents over rows (is_col = 0: row a, h < len) or columns
__global__ void mp_shift_kernel(MPView X, int count, int len, int is_col, int Q, int* out) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= count) return;
    int emax = INT_MIN;
    for (int h = 0; h < len; ++h) {
        const long long x = is_col ? (long long)h + (long long)a * X.ld : (long long)a + (long long)h * X.ld;
        if (!mp_zero(X, x)) emax = max(emax, X.exps[x]);
    }
    out[a] = emax == INT_MIN ? 0 : (Q - 1) - emax;
}

// centered residue of sign * mag modulo m_l, mag < 2^(16 H)
template <int H>
__device__ __forceinline__ int mp_residue(const uint32_t (&mag)[MPD], bool neg, const DevTable& tab, int l) {
    const uint32_t m = (uint32_t)tab.mod[l];
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < H; ++j) acc += ((mag[j >> 1] >> (16 * (j & 1))) & 0xffffu) * tab.pow16[l][j];
    uint32_t r = mod_small(acc, m, tab.magic[l]);
    if (neg && r) r = m - r;
    int c = (int)r;
    if (c > (int)(m - 1) / 2) c -= (int)m;
    return c;
}

// (S2)+(S3): one element per thread; A side: element (r, h), B side: (h, r);
// planes [l][t][r][h] (Rpad x Kpad; zeros in the K padding, the padded rows
// untouched).  A threads run along r (consecutive elements of a column), B
// threads along h.
template <int H>
__global__ void __launch_bounds__(256) mp_convert_kernel(MPView X, int R, int Kc, int is_b,
                                                         const int* __restrict__ shifts,
                                                         const __grid_constant__ DevTable tab, int Kpad,
                                                         int Rpad, int8_t* __restrict__ planes) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)R * Kpad) return;
    const int r = is_b ? (int)(idx / Kpad) : (int)(idx % R);
    const int h = is_b ? (int)(idx % Kpad) : (int)(idx / R);
    const size_t plane = (size_t)Rpad * Kpad, off = (size_t)r * Kpad + h;
    const int S = tab.S, w = tab.w;
    const long long x = is_b ? (long long)h + (long long)r * X.ld : (long long)r + (long long)h * X.ld;
    if (h >= Kc || mp_zero(X, x)) {
        for (int l = 0; l < tab.N; ++l)
            for (int t = 0; t < S; ++t) planes[(size_t)(l * S + t) * plane + off] = 0;
        return;
    }
    const bool neg = X.signs[x] != 0;
    // bit b of |X| = trunc(|a| 2^mu) is bit b + sh of the magnitude
    const long long sh = 32LL * X.L - X.exps[x] - shifts[r];
    const int nw = (w + 2 + 31) >> 5;
    uint32_t carry = 0;
    for (int t = 0; t < S; ++t) {
        uint32_t D[MPD];
#pragma unroll
        for (int k = 0; k < MPD; ++k) D[k] = k < nw ? mant32(X, x, (long long)t * w + 32 * k + sh) : 0u;
        mask_below<MPD>(D, w);
        uint64_t c = carry;
#pragma unroll
        for (int k = 0; k < MPD; ++k) {
            const uint64_t s = (uint64_t)D[k] + c;
            D[k] = (uint32_t)s;
            c = s >> 32;
        }
        // u = D <= 2^w; X >= 0: u >= 2^(w-1) gives the digit u - 2^w;
        // X < 0: u > 2^(w-1) gives 2^w - u, else -u (Eq. (2) on the signed X)
        bool dneg = neg;
        if (t < S - 1) {
            const bool ge = bit_at<MPD>(D, w - 1) || bit_at<MPD>(D, w);
            const bool half = bit_at<MPD>(D, w - 1) && !bit_at<MPD>(D, w) && !any_below<MPD>(D, w - 1);
            const bool wrap = neg ? (ge && !half) : ge;
            if (wrap) {
                complement_below<MPD>(D, w);
                dneg = !neg;
                carry = 1;
            } else {
                carry = 0;
            }
        }
        for (int l = 0; l < tab.N; ++l)
            planes[(size_t)(l * S + t) * plane + off] = (int8_t)mp_residue<H>(D, dneg, tab, l);
    }
}

// ---- (S5)/(S6): CRT, recombination, fused update, rounding to p bits ----
struct Acc {  // NW-word integer of this thread in shared memory, word k at w[k * MPCT]
    uint32_t* w;
    int NW;
    __device__ __forceinline__ uint32_t& operator[](int k) const { return w[k * MPCT]; }
};

__device__ void acc_negate(const Acc& A) {
    uint64_t c = 1;
    for (int k = 0; k < A.NW; ++k) {
        const uint64_t s = (uint64_t)(~A[k]) + c;
        A[k] = (uint32_t)s;
        c = s >> 32;
    }
}

__device__ int acc_bitlen(const Acc& A) {
    for (int k = A.NW - 1; k >= 0; --k)
        if (A[k]) return 32 * k + 32 - __clz(A[k]);
    return 0;
}

__device__ __forceinline__ uint32_t acc_word(const Acc& A, long long k) { return (k >= 0 && k < A.NW) ? A[(int)k] : 0u; }

// bits [pos, pos + 32) (zeros outside)
__device__ __forceinline__ uint32_t acc_bits32(const Acc& A, long long pos) {
    const long long q = pos >= 0 ? (pos >> 5) : -((-pos + 31) >> 5);
    const int r = (int)(pos - 32 * q);
    const uint32_t lo = acc_word(A, q), hi = acc_word(A, q + 1);
    return r ? (lo >> r) | (hi << (32 - r)) : lo;
}

// A >>= s (non-negative value, truncation)
__device__ void acc_shr(const Acc& A, int s) {
    for (int k = 0; k < A.NW; ++k) A[k] = acc_bits32(A, (long long)k * 32 + s);
}

// A += sign * (mant of element x of C) * 2^s, truncating bits below 2^0
// (two's complement over NW words)
__device__ void acc_add_mp(const Acc& A, const MPView& C, long long x, long long s, bool neg) {
    uint64_t c = neg ? 1u : 0u;
    for (int k = 0; k < A.NW; ++k) {
        uint32_t v = mant32(C, x, 32LL * k - s);
        if (neg) v = ~v;
        const uint64_t t = (uint64_t)A[k] + v + c;
        A[k] = (uint32_t)t;
        c = t >> 32;
    }
}

template <int WG>
__global__ void __launch_bounds__(MPCT) mp_crt_kernel(const uint8_t* __restrict__ T, int m, int nchunk, int j0,
                                                      const int* __restrict__ mu, const int* __restrict__ nu,
                                                      const __grid_constant__ DevTable tab, int NW, int alpha,
                                                      int beta, MPView C, int p) {
    extern __shared__ uint32_t accsm[];
    const long long e = (long long)blockIdx.x * MPCT + threadIdx.x;
    const long long mn = (long long)m * nchunk;
    if (e >= mn) return;
    const int i = (int)(e % m), jj = (int)(e / m), j = j0 + jj;
    const Acc A{accsm + threadIdx.x, NW};
    constexpr int WIN = WG + 2;
    long long win[WIN];
#pragma unroll
    for (int k = 0; k < WIN; ++k) win[k] = 0;
    int base = 0;
    long long carry = 0;
    auto retire = [&]() {
        const long long v = win[0] + carry;
        if (base < NW) A[base] = (uint32_t)v;
        carry = v >> 32;  // arithmetic
#pragma unroll
        for (int k = 0; k < WIN - 1; ++k) win[k] = win[k + 1];
        win[WIN - 1] = 0;
        ++base;
    };
    for (int gi = 0; gi < tab.G; ++gi) {
        uint64_t a[WG];
#pragma unroll
        for (int w = 0; w < WG; ++w) a[w] = 0;
        float F = 0.0f;
        const uint8_t* tp = T + (size_t)gi * tab.N * mn + e;
        for (int l = 0; l < tab.N; ++l) {
            const uint32_t t = tp[(size_t)l * mn];
#pragma unroll
            for (int w = 0; w < WG; ++w) a[w] += (uint64_t)t * tab.Mlow[l][w];
            F = fmaf((float)t, tab.invm[l], F);
        }
        const uint32_t R = (uint32_t)rintf(F);
        uint32_t Sg[WG];
        long long cy = 0;
#pragma unroll
        for (int w = 0; w < WG; ++w) {
            const long long cur = (long long)a[w] + cy - (long long)((uint64_t)R * tab.Plow[w]);
            Sg[w] = (uint32_t)cur;
            cy = cur >> 32;
        }
        const long long pos = (long long)tab.w * gi;
        const int q = (int)(pos >> 5), r = (int)(pos & 31);
        while (base < q) retire();
        // S_g 2^r as WG unsigned words and one signed word above them
#pragma unroll
        for (int k = 0; k < WG; ++k) {
            const uint32_t lo = k ? Sg[k - 1] : 0u;
            win[k] += (long long)(r ? (Sg[k] << r) | (lo >> (32 - r)) : Sg[k]);
        }
        win[WG] += r ? (long long)((int)Sg[WG - 1] >> (32 - r)) : ((Sg[WG - 1] >> 31) ? -1LL : 0LL);
    }
    while (base < NW) retire();
    // P_int (two's complement, NW words) on the grid 2^E
    bool neg = (A[NW - 1] >> 31) != 0;
    if (neg) acc_negate(A);
    if (alpha < 0) neg = !neg;
    long long E = (long long)tab.w * tab.g0 - mu[i] - nu[j];
    const long long xc = (long long)i + (long long)j * C.ld;
    if (beta && !mp_zero(C, xc)) {
        const int ctop = C.exps[xc];
        const int Lp = acc_bitlen(A);
        const long long etop = max(E + Lp, (long long)ctop) + 1;
        const long long Wb = 32LL * NW - 2;
        if (etop - E > Wb) {
            const long long E2 = etop - Wb;
            acc_shr(A, (int)(E2 - E));  // truncation toward zero of the product
            E = E2;
        }
        if (neg) acc_negate(A);
        // trunc(C 2^-E): magnitude bit b at bit b + (exps - 32 L) - E of the grid
        acc_add_mp(A, C, xc, (long long)C.exps[xc] - 32LL * C.L - E, C.signs[xc] != 0);
        neg = (A[NW - 1] >> 31) != 0;
        if (neg) acc_negate(A);
    }
    // round |total| 2^E to p bits and store
    const int Lt = acc_bitlen(A);
    if (Lt == 0) {
        for (int k = 0; k < C.L; ++k) C.limbs[(long long)k * C.plane + xc] = 0;
        C.exps[xc] = 0;
        C.signs[xc] = 0;
        return;
    }
    int Lo = Lt;
    if (Lt > p) {
        const int sh = Lt - p;
        const bool rb = (acc_bits32(A, sh - 1) & 1u) != 0;
        bool sticky = false;
        for (int k = 0; k < NW && 32 * k < sh - 1; ++k) {
            const int lo = 32 * k, hiw = min(32 * k + 32, sh - 1);
            const uint32_t mask = hiw - lo >= 32 ? 0xffffffffu : ((1u << (hiw - lo)) - 1u);
            sticky |= (A[k] & mask) != 0;
        }
        const bool up = rb && (sticky || (acc_bits32(A, sh) & 1u));
        // clear the bits below sh, then add 2^sh if rounding up
        for (int k = 0; k < NW; ++k) {
            if (32 * k + 32 <= sh) A[k] = 0;
            else if (32 * k < sh) A[k] &= ~((1u << (sh - 32 * k)) - 1u);
        }
        if (up) {
            uint64_t c = 0;
            for (int k = sh >> 5; k < NW; ++k) {
                const uint64_t add = (k == (sh >> 5)) ? (1ull << (sh & 31)) : 0ull;
                const uint64_t t = (uint64_t)A[k] + add + c;
                A[k] = (uint32_t)t;
                c = t >> 32;
                if (k > (sh >> 5) && !c) break;
            }
            Lo = acc_bitlen(A);
        }
    }
    const long long first = (long long)Lo - 32LL * C.L;  // bit of A at limb 0, bit 0
    for (int k = 0; k < C.L; ++k) C.limbs[(long long)k * C.plane + xc] = acc_bits32(A, first + 32LL * k);
    C.exps[xc] = (int)(Lo + E);
    C.signs[xc] = neg ? 1 : 0;
}

template <int H>
void convert_h(const MPView& X, int R, int Kc, int is_b, const int* shifts, const DevTable& tab, int Kpad, int Rpad,
               int8_t* planes, cudaStream_t s) {
    // rows [0, R) only (padded rows reach discarded outputs); zeros in the K padding
    const long long total = (long long)R * Kpad;
    if (total == 0) return;
    mp_convert_kernel<H><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, R, Kc, is_b, shifts, tab, Kpad, Rpad,
                                                                         planes);
}

void mp_convert(const MPView& X, int R, int Kc, int is_b, const int* shifts, const DevTable& tab, int Kpad, int Rpad,
                int8_t* planes, cudaStream_t s) {
    switch (tab.H) {
#define OZ_H(HH) case HH: convert_h<HH>(X, R, Kc, is_b, shifts, tab, Kpad, Rpad, planes, s); break;
        OZ_H(1) OZ_H(2) OZ_H(3) OZ_H(4) OZ_H(5) OZ_H(6) OZ_H(7) OZ_H(8) OZ_H(9) OZ_H(10) OZ_H(11) OZ_H(12)
        OZ_H(13) OZ_H(14) OZ_H(15)
#undef OZ_H
        default: convert_h<16>(X, R, Kc, is_b, shifts, tab, Kpad, Rpad, planes, s); break;
    }
}

template <int WG>
void crt_wg(const uint8_t* T, int m, int nchunk, int j0, const int* mu, const int* nu, const DevTable& tab, int NW,
            int alpha, int beta, const MPView& C, int p, cudaStream_t s) {
    const long long mn = (long long)m * nchunk;
    const size_t smem = sizeof(uint32_t) * (size_t)NW * MPCT;
    cudaFuncSetAttribute(mp_crt_kernel<WG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    mp_crt_kernel<WG><<<(unsigned)((mn + MPCT - 1) / MPCT), MPCT, smem, s>>>(T, m, nchunk, j0, mu, nu, tab, NW,
                                                                            alpha, beta, C, p);
}

void mp_crt(const uint8_t* T, int m, int nchunk, int j0, const int* mu, const int* nu, const DevTable& tab, int NW,
            int alpha, int beta, const MPView& C, int p, cudaStream_t s) {
    switch (tab.WG) {
#define OZ_W(WW) case WW: crt_wg<WW>(T, m, nchunk, j0, mu, nu, tab, NW, alpha, beta, C, p, s); break;
        OZ_W(1) OZ_W(2) OZ_W(3) OZ_W(4) OZ_W(5) OZ_W(6) OZ_W(7) OZ_W(8) OZ_W(9) OZ_W(10) OZ_W(11) OZ_W(12)
        OZ_W(13) OZ_W(14) OZ_W(15)
#undef OZ_W
        default: crt_wg<16>(T, m, nchunk, j0, mu, nu, tab, NW, alpha, beta, C, p, s); break;
    }
}

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// accumulator words for a plan: the largest P_int plus 64 bits, one sign bit spare
int mp_window_words(const Plan& pl) { return (pl.pint_bits + 64 + 31) / 32 + 1; }

int mp_plan_for(ozlu_handle* h, int p, int K, const Plan** pl, const DevTable** tab) {
    const auto key = std::make_tuple(p, K, 1000, 0, 0, 0);  // backend code 1000: p-bit
    auto it = h->plans.find(key);
    if (it == h->plans.end()) {
        PlanEntry e;
        const int rc = make_plan_mp(p, K, e.plan);
        if (rc) return rc;
        fill_table(e.plan, e.table);
        it = h->plans.emplace(key, e).first;
    }
    *pl = &it->second.plan;
    *tab = &it->second.table;
    return OZLU_OK;
}

// C = beta C + alpha A B, device views (m x k, k x n, m x n)
int mp_gemm_device(ozlu_handle* h, int p, int m, int n, int k, int alpha, const ozlu_mp_matrix& A,
                   const ozlu_mp_matrix& B, int beta, const ozlu_mp_matrix& C) {
    if (m == 0 || n == 0) return OZLU_OK;
    const Plan* pl;
    const DevTable* tab;
    int rc = mp_plan_for(h, p, k, &pl, &tab);
    if (rc) return rc;
    cudaStream_t s = h->stream;
    const int Kpad = pl->Kpad, Mpad = (m + 127) / 128 * 128;
    const size_t planesN = (size_t)pl->N * pl->S;
    // column chunk: t values of one chunk below 4 GiB and B planes below 2 GiB
    const size_t tcol = (size_t)pl->G * pl->N * m;
    long long nch = (long long)(((size_t)4 << 30) / (tcol ? tcol : 1));
    const long long bcap = (long long)(((size_t)2 << 30) / (planesN * Kpad)) / 128 * 128;
    if (nch > bcap) nch = bcap;
    nch = nch / 128 * 128;
    if (nch < 128) nch = 128;
    if (nch > n) nch = n;
    const int Ncpad = (int)((nch + 127) / 128 * 128);
    size_t off = 0;
    const size_t o_mu = off; off = up256(off + sizeof(int) * (size_t)m);
    const size_t o_nu = off; off = up256(off + sizeof(int) * (size_t)n);
    const size_t o_ra = off; off = up256(off + planesN * Mpad * Kpad);
    const size_t o_rb = off; off = up256(off + planesN * (size_t)Ncpad * Kpad);
    const size_t o_t = off;  off = up256(off + tcol * (size_t)nch);
    if ((rc = h->ws.ensure(off))) return rc;
    char* base = (char*)h->ws.base;
    int* mu = (int*)(base + o_mu);
    int* nu = (int*)(base + o_nu);
    int8_t* RA = (int8_t*)(base + o_ra);
    int8_t* RB = (int8_t*)(base + o_rb);
    uint8_t* T = (uint8_t*)(base + o_t);
    const MPView vA = view_of(A, 0), vB = view_of(B, 0), vC = view_of(C, 0);
    const int NW = mp_window_words(*pl);
    const int prev = h->open_phase;
    h->phase(PH_CONVERT);
    mp_shift_kernel<<<(m + 127) / 128, 128, 0, s>>>(vA, m, k, 0, pl->Q, mu);
    mp_shift_kernel<<<(n + 127) / 128, 128, 0, s>>>(vB, n, k, 1, pl->Q, nu);
    mp_convert(vA, m, k, 0, mu, *tab, Kpad, Mpad, RA, s);
    h->count(3);
    for (long long j0 = 0; j0 < n; j0 += nch) {
        const int nc = (int)(n - j0 < nch ? n - j0 : nch);
        const int ncp = (nc + 127) / 128 * 128;
        h->phase(PH_CONVERT);
        mp_convert(view_of(B, j0 * B.ld), nc, k, 1, nu + j0, *tab, Kpad, ncp, RB, s);
        h->phase(PH_GEMM);
        launch_gemm_imma(RA, RB, m, nc, Mpad, ncp, Kpad, *tab, T, s);
        h->phase(PH_CRT);
        mp_crt(T, m, nc, (int)j0, mu, nu, *tab, NW, alpha, beta, vC, p, s);
        h->count(3);
        h->stats.gemm_launches += 1;
        h->stats.crt_launches += 1;
        h->stats.gemm_ops += 2.0 * m * nc * (double)k * pl->N * pl->pair_terms;
    }
    h->phase(prev);
    return cudaGetLastError() == cudaSuccess ? OZLU_OK : OZLU_ERR_CUDA;
}

}  // namespace ozlu

using namespace ozlu;

namespace {
bool mp_valid(const ozlu_mp_matrix* M, int p, int rows, int cols) {
    if (!M || M->L < 1 || 32LL * M->L < p) return false;
    if (rows == 0 || cols == 0) return true;
    if (!M->limbs || !M->exps || !M->signs) return false;
    if (M->ld < (rows > 1 ? rows : 1) || M->plane < M->ld * (long long)cols) return false;
    return is_device_ptr(M->limbs) && is_device_ptr(M->exps) && is_device_ptr(M->signs);
}
}  // namespace

extern "C" int ozlu_mp_gemm(ozlu_handle* h, int p, int m, int n, int k, int alpha, const ozlu_mp_matrix* A,
                            const ozlu_mp_matrix* B, int beta, const ozlu_mp_matrix* C) {
    if (!h) return -1;
    if (p < 1) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 1) return -5;
    if (alpha != 1 && alpha != -1) return -6;
    if (!mp_valid(A, p, m, k)) return -7;
    if (!mp_valid(B, p, k, n)) return -8;
    if (beta != 0 && beta != 1) return -9;
    if (!mp_valid(C, p, m, n)) return -10;
    if (cudaSetDevice(h->device) != cudaSuccess) return OZLU_ERR_CUDA;
    return mp_gemm_device(h, p, m, n, k, alpha, *A, *B, beta, *C);
}
