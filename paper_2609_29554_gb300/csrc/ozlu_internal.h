// Internal declarations shared by the ozlu host code and kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ozlu.h"

namespace ozlu {

constexpr int MAXMOD = 64;       // moduli per plan (INT8 set has 54)
constexpr int MAXH = 16;         // 16-bit halves of one balanced digit (w < 256)
constexpr int MAXWG = 16;        // 32-bit words of one digit-group integer S_g
constexpr int WACC = 16;         // 32-bit words of the fused output window
constexpr int WINDOW_BITS = 510; // window width above the grid 2^E (sign bit spare)
constexpr int MAXWX = 12;        // 32-bit words of one Q-bit fixed-point input
constexpr int MAXG = 8;          // retained digit groups

// Host-side plan (Sec. 3.2 "Determining w and N").
struct Plan {
    int p = 0, K = 0, Kpad = 0, backend = OZLU_BE_INT8, g_ex = 0, extra = 0;
    int S = 0, w = 0, Q = 0, N = 0, g0 = 0, G = 0, pair_terms = 0;
    double need = 0.0;
    int mod[MAXMOD] = {0};
    int y[MAXMOD] = {0};
    std::vector<uint32_t> P;               // P = prod m_l, little-endian words
    std::vector<std::vector<uint32_t>> M;  // M_l = P / m_l
    int sbar_bits = 0, WG = 0, pint_bits = 0, WX = 0, H = 0;
    // extended modulus table (Sec. 4.2.4): the moduli and y_l of all N
    // entries (mod[] / y[] hold at most MAXMOD), three int8 planes each
    bool ext = false;
    std::vector<int> ext_mod, ext_y;
};

// Constant tables of an extended-table plan, in device memory (too large for
// a kernel parameter); word-indexed arrays are [word][modulus] so that the
// lanes of a warp, one modulus each, read consecutive addresses.
struct ExtDev {
    int N, S, w, g0, G, WG, WD;
    const int* mod;                    // [N]
    const uint32_t* y;                 // [N]  M_l^-1 mod m_l
    const uint32_t* magic;             // [N]  ceil(2^32 / m_l)
    const uint32_t* coef;              // [3][N] plane weights mod m_l: 1 - 128, 16384 - 128, 128
    const uint32_t* pw;                // [N]  2^w mod m_l
    const uint32_t* two32;             // [N]  2^32 mod m_l
    const unsigned long long* inv40;   // [N]  round(2^40 / m_l)
    const uint32_t* pow32;             // [WD][N] 2^(32 j) mod m_l
    const uint32_t* Mw;                // [WG][N] word j of M_l
    const uint32_t* Pw;                // [WG]    word j of P
};

// Constant table of one plan, passed to kernels by value (__grid_constant__).
struct DevTable {
    int N, WG, H, S, w, g0, G, Q, WX;
    int mod[MAXMOD];
    int y[MAXMOD];
    uint32_t magic[MAXMOD];   // ceil(2^32 / m): x mod m by one __umulhi
    float invm[MAXMOD];       // 1/m for F = sum t_l / m_l (Eq. (11))
    uint32_t pow16[MAXMOD][MAXH];  // 2^(16 j) mod m
    uint32_t Mlow[MAXMOD][MAXWG];  // M_l mod 2^(32 WG)
    uint32_t Plow[MAXWG];          // P mod 2^(32 WG)
};

// device memory of the library: cudaMalloc unless a test has asked for the
// next allocations to fail (ozlu_debug_fail_alloc); returns false on failure
bool dev_alloc(void** p, size_t bytes);
// raise a kernel's dynamic shared-memory limit on the current device (the
// attribute is per device; each (kernel, device) pair is set once)
void raise_smem_limit(const void* kernel, int bytes);
// SM count of the current device (cached per device)
int device_sms();

int make_plan(int p, int K, const ozlu_opts* o, Plan& out);
// Eq. (Lhint) cost-model slice count (the autotuner's seed)
int lhint_S(double r, int t, int M, int N);
int make_plan_mp(int p, int K, Plan& out);  // p-bit multi-limb inputs, INT8
// p-bit inputs with the extended modulus table (Sec. 4.2.4): S = S_req, or
// the smallest feasible S when S_req = 0
int make_plan_mp_ext(int p, int K, int S_req, Plan& out);
// host image of an extended plan's device tables: the word arrays in the
// order of ExtDev (offsets in 32-bit words, 64-word aligned)
struct ExtImage {
    std::vector<uint32_t> words;
    size_t o_mod, o_y, o_magic, o_coef, o_pw, o_two32, o_inv40, o_pow32, o_Mw, o_Pw;
    int WD;
};
void build_ext_image(const Plan& pl, ExtImage& img);
void fill_table(const Plan& pl, DevTable& t);
// the allocation-free GEMM's planner: the INT8 plan straight into a table,
// fixed-size arrays only (no host allocation)
int plan_noalloc(int p, int K, DevTable& t, int& Kpad);

// ---------------------------------------------------------------- kernels --
// (S1) shared exponents: mu[i] over rows of A (m x k), nu[j] over columns of B.
void launch_row_shifts(const double* A, long long lda, int nc, int m, int k, int Q,
                       int* mu, cudaStream_t s);
void launch_col_shifts(const double* B, long long ldb, int nc, int k, int n, int Q,
                       int* nu, cudaStream_t s);
// (S2)+(S3) fused: expansions -> Q-bit integers -> S digits -> residue planes.
// A side: planes [l][t][Mpad][Kpad] (row i, K contiguous); B side: [l][t][Npad][Kpad].
// mode 0: int8 residues (1 plane); 1: E4M3 base-17 digits d0, d1, d0+d1 (3 planes);
// 2: binary16 residues (1 plane, 2-byte elements); 3: binary64 residues (8-byte).
// Plane index (l * S + t) * P + p.
void launch_convert(const double* X, long long ld, int nc, int rows, int cols,
                    bool is_b, const int* shifts, const DevTable& tab, int Kpad,
                    int Rpad, void* planes, int mode, cudaStream_t s);
// (S4) on tcgen05: FP8 base-17 Karatsuba (fp8 = true) or FP16 residues
int launch_gemm_tc05(bool fp8, const void* RA, const void* RB, int m, int n, int Mpad, int Npad,
                     int Kpad, const DevTable& tab, uint8_t* T, int* err, cudaStream_t s);
// (S4)+(S5 t_l) INT8 residue GEMMs with the modular epilogue; T[gi][l][j][i].
void launch_gemm_imma(const int8_t* RA, const int8_t* RB, int m, int n, int Mpad,
                      int Npad, int Kpad, const DevTable& tab, uint8_t* T,
                      cudaStream_t s);
// the same for n <= 16 outputs per column block: 128 x 16 tiles, B planes with
// Npad = n rounded up to 16 rows
void launch_gemm_imma_narrow(const int8_t* RA, const int8_t* RB, int m, int n, int Mpad, int Npad, int Kpad,
                             const DevTable& tab, uint8_t* T, cudaStream_t s);
// (S4)+(S5 t_l) with the extended table: three int8 Karatsuba planes per
// modulus (plane (l, t, c) at (l S + t) 3 + c), 16-bit t values T[gi][l][j][i]
void launch_gemm_imma_ext(const int8_t* RA, const int8_t* RB, int m, int n, int Mpad, int Npad, int Kpad,
                          const DevTable& tab, const ExtDev& ext, uint16_t* T, cudaStream_t s);
// (S4) binary64 residue GEMMs; t values as 32-bit words
void launch_gemm_f64(const double* RA, const double* RB, int m, int n, int Mpad, int Npad, int Kpad,
                     const DevTable& tab, uint32_t* T, cudaStream_t s);
// (S5)+(S6): CRT per digit group, recombination, fused beta*C + alpha*AB, rounding.
// t values are bytes (INT8/FP8/FP16 moduli <= 255) or 32-bit words (t32, binary64).
void launch_crt(const void* T, bool t32, int m, int n, const int* mu, const int* nu,
                const DevTable& tab, int nc, int alpha, int beta, double* C,
                long long ldc, cudaStream_t s);

}  // namespace ozlu
