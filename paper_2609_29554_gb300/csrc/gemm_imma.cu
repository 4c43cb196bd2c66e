// (S4) exact INT8 x INT8 -> INT32 residue GEMMs with the (S5) modular epilogue.
//
// Sec. 3.1 (S4) and Sec. 3.2: for every modulus m_l and retained digit group
// g, C_g^(l) = sum_{ta + tb = g} A_ta^(l) B_tb^(l); the pair terms of one group
// are fused by concatenating their K loops into one int32 accumulation
// (Eq. (8)).  The epilogue forms t_l = (C mod m_l) y_l mod m_l (Eq. (11)) and
// stores it as one byte.
//
// sm_103a has no tcgen05 INT8 MMA (ptxas rejects .kind::i8 there), so this
// back-end runs on the warp-level mma.sync.m16n8k32 s8 instruction.
//   CTA tile 128 x 128, K step 64 bytes, 8 warps (2 x 4), warp tile 64 x 32,
//   cp.async 16-byte copies into a 4-stage ring, XOR-swizzled 64-byte rows so
//   ldmatrix reads are bank-conflict free.
// Operand planes are K-contiguous: A plane (l, t) is Mpad x Kpad, B plane
// (l, t) is Npad x Kpad (B stored as N x K, the "col" operand of mma.sync).
//
// Extended modulus table (Sec. 4.2.4, moduli up to 16191): a centered
// residue r is split into balanced base-128 digits r = 128 q + r0 and stored
// as the three int8 planes r0, q, r0 + q (plane (l, t, c) at index
// (l S + t) 3 + c).  The CTA of (l, g) runs the three plane products one after
// the other through the same pipeline and folds each into a residue mod m_l
// with its Karatsuba weight: C = P00 + 128 (Pss - P00 - P11) + 16384 P11
//                             = (1 - 128) P00 + (16384 - 128) P11 + 128 Pss,
// so the int32 accumulators stay exact (K_pad S 127^2 < 2^31) and only
// residues are combined.  t_l (< 2^14) is stored as 16 bits.
#include <string.h>

#include "mp_device.cuh"
#include "ozlu_internal.h"

namespace ozlu {
namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4, THREADS = 256;
constexpr int TILE_BYTES = BM * BK;  // one operand stage (== BN * BK)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t& r0, uint32_t& r1,
                                            uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_s8(int (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                       uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// byte offset of 16-byte chunk `ch` of row `row` in a swizzled 64-byte-row tile
__device__ __forceinline__ int swz(int row, int ch) { return row * BK + ((ch ^ ((row >> 1) & 3)) << 4); }

// t = ((c mod m) y) mod m for |c| < 2^31
__device__ __forceinline__ uint32_t t_value(int c, uint32_t m, uint32_t y, uint32_t magic) {
    const uint32_t a = c < 0 ? (uint32_t)(-(long long)c) : (uint32_t)c;
    uint32_t r = mod_small(a, m, magic);
    if (c < 0 && r) r = m - r;
    return mod_small(r * y, m, magic);
}

// x mod m in [0, m) for a signed 32-bit x
__device__ __forceinline__ uint32_t smod(int c, uint32_t m, uint32_t magic) {
    const uint32_t a = c < 0 ? (uint32_t)(-(long long)c) : (uint32_t)c;
    uint32_t r = mod_small(a, m, magic);
    if (c < 0 && r) r = m - r;
    return r;
}

template <bool EXT>
__global__ void __launch_bounds__(THREADS) gemm_imma_kernel(
    const int8_t* __restrict__ RA, const int8_t* __restrict__ RB, int m, int n, int Mpad,
    int Npad, int Kpad, const __grid_constant__ DevTable tab, const ExtDev ext, void* __restrict__ Tout) {
    extern __shared__ __align__(128) uint8_t smem[];
    constexpr int P = EXT ? 3 : 1;  // residue planes per modulus
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tm = blockIdx.x, tn = blockIdx.y;
    const int NM = EXT ? ext.N : tab.N;
    const int l = blockIdx.z % NM, gi = blockIdx.z / NM;
    const int S = EXT ? ext.S : tab.S, g = (EXT ? ext.g0 : tab.g0) + gi;
    const int ta0 = max(0, g - (S - 1)), ta1 = min(g, S - 1);
    const int KT = Kpad / BK;
    const int per_plane = (ta1 - ta0 + 1) * KT;
    const int iters = P * per_plane;
    const size_t aplane = (size_t)Mpad * Kpad, bplane = (size_t)Npad * Kpad;

    auto load_stage = [&](int stage, int it) {
        const int pq = it / per_plane, rest = it - pq * per_plane;
        const int pr = rest / KT, kt = rest - pr * KT;
        const int ta = ta0 + pr, tb = g - ta;
        const size_t ia = EXT ? (size_t)((l * S + ta) * 3 + pq) : (size_t)(l * S + ta);
        const size_t ib = EXT ? (size_t)((l * S + tb) * 3 + pq) : (size_t)(l * S + tb);
        const int8_t* a = RA + ia * aplane + (size_t)tm * BM * Kpad + kt * BK;
        const int8_t* b = RB + ib * bplane + (size_t)tn * BN * Kpad + kt * BK;
        uint8_t* sa = smem + stage * 2 * TILE_BYTES;
        uint8_t* sb = sa + TILE_BYTES;
#pragma unroll
        for (int rep = 0; rep < 2; ++rep) {
            const int c = tid + rep * THREADS;  // 512 chunks of 16 bytes per operand
            const int row = c >> 2, ch = c & 3;
            cp_async16(smem_u32(sa + swz(row, ch)), a + (size_t)row * Kpad + ch * 16);
            cp_async16(smem_u32(sb + swz(row, ch)), b + (size_t)row * Kpad + ch * 16);
        }
    };

    const uint32_t md = EXT ? (uint32_t)ext.mod[l] : (uint32_t)tab.mod[l];
    const uint32_t yd = EXT ? ext.y[l] : (uint32_t)tab.y[l];
    const uint32_t mg = EXT ? ext.magic[l] : tab.magic[l];

    int acc[4][4][4];
    uint32_t part[EXT ? 4 : 1][EXT ? 4 : 1][EXT ? 4 : 1];  // EXT: residue of the planes folded so far
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0;
    if (EXT) {
#pragma unroll
        for (int i = 0; i < (EXT ? 4 : 1); ++i)
#pragma unroll
            for (int j = 0; j < (EXT ? 4 : 1); ++j)
#pragma unroll
                for (int r = 0; r < (EXT ? 4 : 1); ++r) part[i][j][r] = 0;
    }

#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < iters) load_stage(s, s);
        cp_async_commit();
    }

    const int wm = warp & 1, wn = warp >> 1;  // 2 x 4 warps
    for (int it = 0; it < iters; ++it) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        {
            const int nxt = it + STAGES - 1;
            if (nxt < iters) load_stage(nxt % STAGES, nxt);
            cp_async_commit();
        }
        const uint8_t* sa = smem + (it % STAGES) * 2 * TILE_BYTES;
        const uint8_t* sb = sa + TILE_BYTES;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            uint32_t af[4][4], bf[4][2];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                const int row = wm * 64 + mi * 16 + (lane & 15);
                const int ch = kk * 2 + (lane >> 4);
                ldmatrix_x4(smem_u32(sa + swz(row, ch)), af[mi][0], af[mi][1], af[mi][2], af[mi][3]);
            }
#pragma unroll
            for (int nj = 0; nj < 2; ++nj) {
                const int id = lane >> 3;
                const int row = wn * 32 + (nj * 2 + (id >> 1)) * 8 + (lane & 7);
                const int ch = kk * 2 + (id & 1);
                ldmatrix_x4(smem_u32(sb + swz(row, ch)), bf[2 * nj][0], bf[2 * nj][1],
                            bf[2 * nj + 1][0], bf[2 * nj + 1][1]);
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni) mma_s8(acc[mi][ni], af[mi], bf[ni][0], bf[ni][1]);
        }
        if (EXT && (it + 1) % per_plane == 0) {
            // one plane product complete: fold its residue with the plane's weight
            const uint32_t cf = ext.coef[(it / per_plane) * NM + l];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        uint32_t& pv = part[EXT ? mi : 0][EXT ? ni : 0][EXT ? r : 0];
                        pv = mod_small(pv + cf * smod(acc[mi][ni][r], md, mg), md, mg);
                        acc[mi][ni][r] = 0;
                    }
        }
    }
    cp_async_wait<0>();
    __syncthreads();

    const int gid = lane >> 2, tig = lane & 3;
    const int i0 = tm * BM, j0 = tn * BN;
    if (!EXT) {
        // epilogue: t values into a column-major 128 x 128 byte tile, then out
        uint8_t* st = smem;  // [col][row]
#pragma unroll
        for (int mi = 0; mi < 4; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int r0 = wm * 64 + mi * 16 + gid;
                const int c0 = wn * 32 + ni * 8 + 2 * tig;
                st[c0 * BM + r0] = (uint8_t)t_value(acc[mi][ni][0], md, yd, mg);
                st[(c0 + 1) * BM + r0] = (uint8_t)t_value(acc[mi][ni][1], md, yd, mg);
                st[c0 * BM + r0 + 8] = (uint8_t)t_value(acc[mi][ni][2], md, yd, mg);
                st[(c0 + 1) * BM + r0 + 8] = (uint8_t)t_value(acc[mi][ni][3], md, yd, mg);
            }
        __syncthreads();
        uint8_t* out = (uint8_t*)Tout + ((size_t)gi * NM + l) * (size_t)m * n;
        // 128 columns x 8 segments of 16 rows
        for (int s = tid; s < BN * (BM / 16); s += THREADS) {
            const int col = s >> 3, seg = s & 7;
            const int j = j0 + col, i = i0 + seg * 16;
            if (j >= n || i >= m) continue;
            const uint8_t* src = st + col * BM + seg * 16;
            uint8_t* dst = out + (size_t)j * m + i;
            if (i + 16 <= m && (((uintptr_t)dst) & 15) == 0) {
                *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
            } else {
                const int cnt = min(16, m - i);
                for (int q = 0; q < cnt; ++q) dst[q] = src[q];
            }
        }
    } else {
        // t = (folded residue) y mod m, 16 bits, through a column-major tile
        uint16_t* st = reinterpret_cast<uint16_t*>(smem);  // [col][row]
#pragma unroll
        for (int mi = 0; mi < 4; ++mi)
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int r0 = wm * 64 + mi * 16 + gid;
                const int c0 = wn * 32 + ni * 8 + 2 * tig;
                const int q0 = EXT ? mi : 0, q1 = EXT ? ni : 0;
                st[c0 * BM + r0] = (uint16_t)mod_small(part[q0][q1][0] * yd, md, mg);
                st[(c0 + 1) * BM + r0] = (uint16_t)mod_small(part[q0][q1][EXT ? 1 : 0] * yd, md, mg);
                st[c0 * BM + r0 + 8] = (uint16_t)mod_small(part[q0][q1][EXT ? 2 : 0] * yd, md, mg);
                st[(c0 + 1) * BM + r0 + 8] = (uint16_t)mod_small(part[q0][q1][EXT ? 3 : 0] * yd, md, mg);
            }
        __syncthreads();
        uint16_t* out = (uint16_t*)Tout + ((size_t)gi * NM + l) * (size_t)m * n;
        // 128 columns x 16 segments of 8 rows (16 bytes)
        for (int s = tid; s < BN * (BM / 8); s += THREADS) {
            const int col = s >> 4, seg = s & 15;
            const int j = j0 + col, i = i0 + seg * 8;
            if (j >= n || i >= m) continue;
            const uint16_t* src = st + col * BM + seg * 8;
            uint16_t* dst = out + (size_t)j * m + i;
            if (i + 8 <= m && (((uintptr_t)dst) & 15) == 0) {
                *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
            } else {
                const int cnt = min(8, m - i);
                for (int q = 0; q < cnt; ++q) dst[q] = src[q];
            }
        }
    }
}

// Narrow outputs (n <= 16, the p-bit LU's column scalings and the bottom of
// its recursion): a 128 x 16 CTA tile, 4 warps of 32 x 16, the same K step,
// ring and swizzle, so that a one-column product does not pay for 128.
constexpr int NBN = 16, NTHREADS = 128;
constexpr int NTILE_B = NBN * BK;  // 1 KiB

__global__ void __launch_bounds__(NTHREADS) gemm_imma_narrow_kernel(
    const int8_t* __restrict__ RA, const int8_t* __restrict__ RB, int m, int n, int Mpad, int Npad, int Kpad,
    const __grid_constant__ DevTable tab, uint8_t* __restrict__ T) {
    extern __shared__ __align__(128) uint8_t smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tm = blockIdx.x, tn = blockIdx.y;
    const int l = blockIdx.z % tab.N, gi = blockIdx.z / tab.N;
    const int S = tab.S, g = tab.g0 + gi;
    const int ta0 = max(0, g - (S - 1)), ta1 = min(g, S - 1);
    const int KT = Kpad / BK;
    const int iters = (ta1 - ta0 + 1) * KT;
    const size_t aplane = (size_t)Mpad * Kpad, bplane = (size_t)Npad * Kpad;
    constexpr int STAGE = TILE_BYTES + NTILE_B;

    auto load_stage = [&](int stage, int it) {
        const int pr = it / KT, kt = it - pr * KT;
        const int ta = ta0 + pr, tb = g - ta;
        const int8_t* a = RA + (size_t)(l * S + ta) * aplane + (size_t)tm * BM * Kpad + kt * BK;
        const int8_t* b = RB + (size_t)(l * S + tb) * bplane + (size_t)tn * NBN * Kpad + kt * BK;
        uint8_t* sa = smem + stage * STAGE;
        uint8_t* sb = sa + TILE_BYTES;
#pragma unroll
        for (int rep = 0; rep < 4; ++rep) {
            const int c = tid + rep * NTHREADS;  // 512 chunks of 16 bytes of A
            const int row = c >> 2, ch = c & 3;
            cp_async16(smem_u32(sa + swz(row, ch)), a + (size_t)row * Kpad + ch * 16);
        }
        if (tid < NBN * 4) {
            const int row = tid >> 2, ch = tid & 3;
            cp_async16(smem_u32(sb + swz(row, ch)), b + (size_t)row * Kpad + ch * 16);
        }
    };

    int acc[2][2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0;
#pragma unroll
    for (int s = 0; s < STAGES - 1; ++s) {
        if (s < iters) load_stage(s, s);
        cp_async_commit();
    }
    for (int it = 0; it < iters; ++it) {
        cp_async_wait<STAGES - 2>();
        __syncthreads();
        {
            const int nxt = it + STAGES - 1;
            if (nxt < iters) load_stage(nxt % STAGES, nxt);
            cp_async_commit();
        }
        const uint8_t* sa = smem + (it % STAGES) * STAGE;
        const uint8_t* sb = sa + TILE_BYTES;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            uint32_t af[2][4], bf[2][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int row = warp * 32 + mi * 16 + (lane & 15);
                const int ch = kk * 2 + (lane >> 4);
                ldmatrix_x4(smem_u32(sa + swz(row, ch)), af[mi][0], af[mi][1], af[mi][2], af[mi][3]);
            }
            {
                const int id = lane >> 3;
                const int row = (id >> 1) * 8 + (lane & 7);
                const int ch = kk * 2 + (id & 1);
                ldmatrix_x4(smem_u32(sb + swz(row, ch)), bf[0][0], bf[0][1], bf[1][0], bf[1][1]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 2; ++ni) mma_s8(acc[mi][ni], af[mi], bf[ni][0], bf[ni][1]);
        }
    }
    cp_async_wait<0>();
    __syncthreads();
    const uint32_t md = (uint32_t)tab.mod[l], yd = (uint32_t)tab.y[l], mg = tab.magic[l];
    uint8_t* st = smem;  // [col][row], 16 x 128 bytes
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) {
            const int r0 = warp * 32 + mi * 16 + gid;
            const int c0 = ni * 8 + 2 * tig;
            st[c0 * BM + r0] = (uint8_t)t_value(acc[mi][ni][0], md, yd, mg);
            st[(c0 + 1) * BM + r0] = (uint8_t)t_value(acc[mi][ni][1], md, yd, mg);
            st[c0 * BM + r0 + 8] = (uint8_t)t_value(acc[mi][ni][2], md, yd, mg);
            st[(c0 + 1) * BM + r0 + 8] = (uint8_t)t_value(acc[mi][ni][3], md, yd, mg);
        }
    __syncthreads();
    uint8_t* out = T + ((size_t)gi * tab.N + l) * (size_t)m * n;
    const int i0 = tm * BM, j0 = tn * NBN;
    for (int s2 = tid; s2 < NBN * (BM / 16); s2 += NTHREADS) {
        const int col = s2 >> 3, seg = s2 & 7;
        const int j = j0 + col, i = i0 + seg * 16;
        if (j >= n || i >= m) continue;
        const uint8_t* src = st + col * BM + seg * 16;
        uint8_t* dst = out + (size_t)j * m + i;
        if (i + 16 <= m && (((uintptr_t)dst) & 15) == 0) {
            *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
        } else {
            const int cnt = min(16, m - i);
            for (int q = 0; q < cnt; ++q) dst[q] = src[q];
        }
    }
}

}  // namespace

void launch_gemm_imma(const int8_t* RA, const int8_t* RB, int m, int n, int Mpad, int Npad,
                      int Kpad, const DevTable& tab, uint8_t* T, cudaStream_t s) {
    const int smem = STAGES * 2 * TILE_BYTES;  // 64 KB
    raise_smem_limit((const void*)gemm_imma_kernel<false>, smem);
    dim3 grid(Mpad / BM, Npad / BN, tab.N * tab.G);
    ExtDev none;
    memset(&none, 0, sizeof none);
    gemm_imma_kernel<false><<<grid, THREADS, smem, s>>>(RA, RB, m, n, Mpad, Npad, Kpad, tab, none, T);
}

// n <= 16: the B planes hold Npad = n rounded up to 16 rows
void launch_gemm_imma_narrow(const int8_t* RA, const int8_t* RB, int m, int n, int Mpad, int Npad, int Kpad,
                             const DevTable& tab, uint8_t* T, cudaStream_t s) {
    const int smem = STAGES * (TILE_BYTES + NTILE_B);  // 36 KB
    dim3 grid(Mpad / BM, Npad / NBN, tab.N * tab.G);
    gemm_imma_narrow_kernel<<<grid, NTHREADS, smem, s>>>(RA, RB, m, n, Mpad, Npad, Kpad, tab, T);
}

void launch_gemm_imma_ext(const int8_t* RA, const int8_t* RB, int m, int n, int Mpad, int Npad, int Kpad,
                          const DevTable& tab, const ExtDev& ext, uint16_t* T, cudaStream_t s) {
    const int smem = STAGES * 2 * TILE_BYTES;  // 64 KB (the 32 KB t tile reuses it)
    raise_smem_limit((const void*)gemm_imma_kernel<true>, smem);
    dim3 grid(Mpad / BM, Npad / BN, ext.N * ext.G);
    gemm_imma_kernel<true><<<grid, THREADS, smem, s>>>(RA, RB, m, n, Mpad, Npad, Kpad, tab, ext, T);
}

}  // namespace ozlu
