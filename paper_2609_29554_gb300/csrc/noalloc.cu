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
// array and leaves its contents behind.  Each call writes the parts of the
// array its results depend on before reading them: shared exponents, the
// residue rows of A and B with their zero K padding, and the t values.  The
// padding rows of the residue planes (row m to the next multiple of 128, and
// likewise for n) are not written and may hold bytes of an earlier call; the
// GEMM reads them, but they only reach output tiles outside m x n, which are
// discarded.  So nothing needs clearing between calls.  Calls that overlap
// on the GPU (on different streams, or from different host threads) race on
// the array: serialise them.
//
// Back-end: INT8 residues on mma.sync (the same kernels as ozlu_gemm's INT8
// path), so results equal ozlu_gemm with backend OZLU_BE_INT8 bit for bit.
// The plan follows the same rule as the handle's planner, recomputed with
// fixed-size arrays so that no host memory is allocated either
// (plan_noalloc, noalloc_plan.cpp).
#include <math.h>
#include <string.h>

#include <mutex>

#include "ozlu_internal.h"

namespace ozlu {
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = 16u << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAXDEV = 64;

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

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// device (or managed) memory of the current device: a pointer into another
// GPU's memory is rejected like a host pointer
bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    if (a.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    return a.device == dev;
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
    int rc = plan_noalloc(p, k, tab, Kpad);
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
