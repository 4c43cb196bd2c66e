// ozlu_gemm_noalloc: the Ozaki-II GEMM without any allocation.
//
// Some callers must not allocate: a host that has handed nearly all device
// memory to its own pool allocator before calling in, or a latency-critical
// caller that cannot afford the device-wide synchronisation cudaMalloc may
// imply.  This entry point serves them.  It uses no handle and allocates
// neither device nor host memory: its intermediates (shared exponents,
// residue planes, t values) live in one file-scope device array of fixed
// size, NOALLOC_SCRATCH_BYTES, which every GPU that loads the library holds
// until the process exits.  The caller passes device pointers for A, B, C.
//
// The first call on a device looks up the device address of the array with
// cudaGetSymbolAddress, with that device current, and caches it; that first
// call should come before any stream capture.  Every call reuses the same
// array and leaves its contents behind; the kernels overwrite every byte they
// later read (padding included), so nothing needs clearing between calls.
// Calls that overlap on the GPU (on different streams, or from different
// host threads) race on the array: serialise them.
//
// Back-end: INT8 residues on mma.sync (the same kernels as ozlu_gemm's INT8
// path), so results equal ozlu_gemm with backend OZLU_BE_INT8 bit for bit.
// The plan follows the same rule as the handle's planner, recomputed here
// with fixed-size arrays so that no host memory is allocated either.
#include <math.h>
#include <string.h>

#include <mutex>

#include "ozlu_internal.h"

namespace ozlu {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 16u << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAXDEV = 64;
constexpr int PW = 16;  // words of P (54 moduli of <= 8 bits: <= 432 bits)

std::mutex g_mutex;
void* g_scratch_ptr[MAXDEV] = {nullptr};

// device address of the scratch array for the current device (set-up once)
int scratch_ptr(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return OZLU_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return OZLU_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return OZLU_OK;
}

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

// INT8 plan of Sec. 3.2 into a DevTable, fixed-size arrays only
int plan_na(int p, int K, DevTable& t, int& Kpad_out) {
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

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace ozlu

using namespace ozlu;

extern "C" int ozlu_gemm_noalloc(int nc, int p, int m, int n, int k, int alpha, const double* A,
                                 long long lda, const double* B, long long ldb, int beta, double* C,
                                 long long ldc, void* stream) {
    if (nc < 2 || nc > 4) return -1;
    if (p == 0) p = 53 * nc;
    if (p < 1 || p > 53 * nc) return -2;
    if (m < 0) return -3;
    if (n < 0) return -4;
    if (k < 1) return -5;
    if (alpha != 1 && alpha != -1) return -6;
    if (!A || !on_device(A)) return -7;
    if (lda < (m > 1 ? m : 1)) return -8;
    if (!B || !on_device(B)) return -9;
    if (ldb < (k > 1 ? k : 1)) return -10;
    if (beta != 0 && beta != 1) return -11;
    if (!C || !on_device(C)) return -12;
    if (ldc < (m > 1 ? m : 1)) return -13;
    if (m == 0 || n == 0) return OZLU_OK;
    DevTable tab;
    int Kpad = 0;
    int rc = plan_na(p, k, tab, Kpad);
    if (rc) return rc;
    const int Mpad = (m + 127) / 128 * 128, Npad = (n + 127) / 128 * 128;
    size_t off = 0;
    const size_t o_mu = off; off = up256(off + sizeof(int) * (size_t)m);
    const size_t o_nu = off; off = up256(off + sizeof(int) * (size_t)n);
    const size_t o_ra = off; off = up256(off + (size_t)tab.N * tab.S * Mpad * Kpad);
    const size_t o_rb = off; off = up256(off + (size_t)tab.N * tab.S * Npad * Kpad);
    const size_t o_t = off;  off = up256(off + (size_t)tab.G * tab.N * m * n);
    if (off > NOALLOC_SCRATCH_BYTES) return OZLU_ERR_CAPACITY;  // problem too large for the array
    void* base = nullptr;
    if ((rc = scratch_ptr(&base))) return rc;
    char* sb = (char*)base;
    int* mu = (int*)(sb + o_mu);
    int* nu = (int*)(sb + o_nu);
    int8_t* RA = (int8_t*)(sb + o_ra);
    int8_t* RB = (int8_t*)(sb + o_rb);
    uint8_t* T = (uint8_t*)(sb + o_t);
    cudaStream_t s = (cudaStream_t)stream;
    launch_row_shifts(A, lda, nc, m, k, tab.Q, mu, s);
    launch_col_shifts(B, ldb, nc, k, n, tab.Q, nu, s);
    launch_convert(A, lda, nc, m, k, false, mu, tab, Kpad, Mpad, RA, 0, s);
    launch_convert(B, ldb, nc, k, n, true, nu, tab, Kpad, Npad, RB, 0, s);
    launch_gemm_imma(RA, RB, m, n, Mpad, Npad, Kpad, tab, T, s);
    launch_crt(T, false, m, n, mu, nu, tab, nc, alpha, beta, C, ldc, s);
    return cudaGetLastError() == cudaSuccess ? OZLU_OK : OZLU_ERR_CUDA;
}
