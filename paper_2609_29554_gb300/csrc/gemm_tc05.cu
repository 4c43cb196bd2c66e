// (S4) residue GEMMs on the fifth-generation tensor cores of sm_103a, with
// the (S5) modular epilogue.
//
// Back-ends (Sec. 4.2.3):
//   FP8  E4M3, balanced base-17 digits of each centered residue, Eq. (15):
//        r = 17 d1 + d0, |d0| <= 8, |d1| <= 7, |d0 + d1| <= 15.  Three digit
//        planes per residue (d0, d1, d0 + d1) and three fp32 accumulators
//        P00, P11, Pss give the exact product by Karatsuba,
//        r r' summed = P00 + 17 (Pss - P00 - P11) + 289 P11.
//   FP16 the centered residue itself (|r| <= 127 is exact in binary16), one
//        plane, one fp32 accumulator; exact while K_pad S 127^2 < 2^24
//        (Eq. (14)).
// Both rely on the fp32 tensor-core accumulation being exact for integer
// sums below 2^24; the parity tests check it bit for bit.
//
// Kernel: persistent, one CTA per SM over the 128 x 128 output tiles of all
// (modulus, digit group) pairs.
//   warp 0: TMA producer (cp.async.bulk.tensor, SWIZZLE_128B, no multicast)
//   warp 1: one thread issues tcgen05.mma (M = 128, N = 128, K = 32 bytes
//           per instruction) into TMEM, tcgen05.commit frees smem stages and
//           hands a finished accumulator to the epilogue
//   warps 2-9 (FP8) or 2-17 (FP16): epilogue (two or four warps per TMEM
//           lane quarter, each on a half or a quarter of the columns),
//           tcgen05.ld 32x32b, combine, t_l = (C mod m) y mod m, then free the
//           accumulator buffer for the MMA warp
// Every mbarrier wait has an iteration limit; on expiry the CTA records
// OZLU_ERR_TIMEOUT, stops issuing work, and releases its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "mp_device.cuh"
#include "ozlu_internal.h"

namespace ozlu {
namespace {

constexpr int BM = 128, BN = 128, BK = 128;  // BK in bytes: one 128-byte swizzle row
constexpr int STAGES = 6;
// producer, MMA and the epilogue warps: 8 for FP8 (three accumulators per
// output keep the registers of one epilogue thread high), 16 for FP16
template <bool FP8>
struct Cfg {
    static constexpr int THREADS = FP8 ? 320 : 576;
    static constexpr int EPI = THREADS - 64;      // epilogue threads
    static constexpr int SPLIT = (THREADS - 64) / 128;  // column parts per TMEM lane quarter
};
constexpr int TILE = BM * BK;                // 16 KiB per operand stage
constexpr long long WAIT_LIMIT = 1ll << 24;  // iterations of ~100 ns

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(su32(b)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(su32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false (and the error word set) after `limit` tries
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err, volatile int* abort,
                                          long long limit = WAIT_LIMIT) {
    long long it = 0;
    while (!mbar_try_wait(b, parity)) {
        if (*abort) return false;
        if (++it > limit) {
            atomicExch(err, OZLU_ERR_TIMEOUT);
            *abort = 1;
            return false;
        }
        __nanosleep(64);
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
            "r"(su32(dst)),
        "l"(tm), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// shared-memory matrix descriptor: K-major, SWIZZLE_128B, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
    const uint64_t addr = su32(p);
    return ((addr & 0x3ffff) >> 4) | (1ull << 16) | (64ull << 32) | (1ull << 46) | (2ull << 61);
}

template <bool FP8>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    if (FP8)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(su32(b))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ uint32_t t_value(int c, uint32_t m, uint32_t y, uint32_t magic) {
    const uint32_t a = c < 0 ? (uint32_t)(-(long long)c) : (uint32_t)c;
    uint32_t r = mod_small(a, m, magic);
    if (c < 0 && r) r = m - r;
    return mod_small(r * y, m, magic);
}

// Persistent kernel: one CTA per SM walks the tiles (tm, tn, l, gi) with
// stride gridDim.x, tn fastest, so the CTAs in flight share A row panels and
// B column panels of one modulus in L2.  The smem ring runs across tiles; the
// accumulators are double-buffered in TMEM (FP16: 2 x 128 columns; FP8 keeps
// one 384-column buffer), so the epilogue of one tile overlaps the MMAs of
// the next.
template <bool FP8>
__global__ void __launch_bounds__(Cfg<FP8>::THREADS, 1) gemm_tc05_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int m, int n,
    int Mpad, int Npad, int KB, const __grid_constant__ DevTable tab, uint8_t* __restrict__ T,
    int* __restrict__ err) {
    constexpr int P = FP8 ? 3 : 1;                // planes (accumulators)
    constexpr int NBUF = FP8 ? 1 : 2;             // accumulator buffers
    constexpr uint32_t TMEM_COLS = FP8 ? 512 : 256;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sa = sm;
    uint8_t* sb = sm + STAGES * TILE;
    uint64_t* full = (uint64_t*)(sm + 2 * STAGES * TILE);
    uint64_t* empty = full + STAGES;
    uint64_t* accf = empty + STAGES;   // [NBUF] accumulator ready (MMA -> epilogue)
    uint64_t* acce = accf + 2;         // [NBUF] accumulator free (epilogue -> MMA)
    uint32_t* tmem_slot = (uint32_t*)(acce + 2);
    volatile int* abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int TM = Mpad / BM, TN = Npad / BN;
    const int tiles = TM * TN * tab.N * tab.G;
    const int S = tab.S;
    // tile t -> (tm, tn, l, gi) and its work items (pair terms x K blocks x planes)
    auto decode = [&](int t, int& tm, int& tn, int& l, int& gi, int& ta0, int& items) {
        tn = t % TN;
        int r = t / TN;
        tm = r % TM;
        r /= TM;
        l = r % tab.N;
        gi = r / tab.N;
        const int g = tab.g0 + gi;
        ta0 = max(0, g - (S - 1));
        const int ta1 = min(g, S - 1);
        items = (ta1 - ta0 + 1) * KB * P;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], Cfg<FP8>::EPI);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            long long it = 0;       // global item counter (smem ring position)
            long long issued = 0;
            for (int t = blockIdx.x; t < tiles && !*abort; t += gridDim.x) {
                int tm, tn, l, gi, ta0, items;
                decode(t, tm, tn, l, gi, ta0, items);
                const int g = tab.g0 + gi;
                for (int i = 0; i < items && !*abort; ++i, ++it) {
                    const int s = (int)(it % STAGES);
                    const long long round = it / STAGES;
                    if (!mbar_wait(&empty[s], (uint32_t)((round & 1) ^ 1), err, abort)) break;
                    const int p = i % P, rest = i / P;
                    const int kb = rest % KB, pr = rest / KB;
                    const int ta = ta0 + pr, tb = g - ta;
                    mbar_expect_tx(&full[s], 2 * TILE);
                    const int ya = ((l * S + ta) * P + p) * Mpad + tm * BM;
                    const int yb = ((l * S + tb) * P + p) * Npad + tn * BN;
                    const int x = FP8 ? kb * BK : kb * (BK / 2);  // element units of the map
                    tma_load_2d(sa + s * TILE, &tmA, x, ya, &full[s]);
                    tma_load_2d(sb + s * TILE, &tmB, x, yb, &full[s]);
                    issued = it + 1;
                }
            }
            if (*abort) {
                // let the copies already issued land before the CTA exits (bounded)
                for (long long q = issued - STAGES < 0 ? 0 : issued - STAGES; q < issued; ++q) {
                    long long w = 0;
                    while (!mbar_try_wait(&full[q % STAGES], (uint32_t)((q / STAGES) & 1)) && ++w < WAIT_LIMIT)
                        __nanosleep(64);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // kind::f8f6f4 E4M3 x E4M3 or kind::f16 F16 x F16 (format code 0 in both),
            // fp32 accumulate, K-major A and B, N = 128, M = 128
            const uint32_t idesc = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
            long long it = 0;
            int j = 0;  // local tile count
            for (int t = blockIdx.x; t < tiles && !*abort; t += gridDim.x, ++j) {
                int tm, tn, l, gi, ta0, items;
                decode(t, tm, tn, l, gi, ta0, items);
                const int b = j % NBUF;
                const uint32_t use = (uint32_t)(j / NBUF);
                if (!mbar_wait(&acce[b], (use & 1) ^ 1, err, abort)) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n");
                const uint32_t acc = tmem + (uint32_t)(b * P * BN);
                bool ok = true;
                for (int i = 0; i < items; ++i, ++it) {
                    const int s = (int)(it % STAGES);
                    const long long round = it / STAGES;
                    if (!mbar_wait(&full[s], (uint32_t)(round & 1), err, abort)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;\n");
                    const int p = i % P;
                    const int first_of_plane = i < P;  // first item of each accumulator
                    const uint64_t ad = smem_desc(sa + s * TILE), bd = smem_desc(sb + s * TILE);
#pragma unroll
                    for (int k = 0; k < BK / 32; ++k)
                        mma<FP8>(acc + p * BN, ad + 2 * k, bd + 2 * k, idesc, (first_of_plane && k == 0) ? 0u : 1u);
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&accf[b]);
            }
        }
    } else {
        // epilogue warps: TMEM lane quarter = warp % 4; the k-th group of four
        // warps (from warp 2) takes the k-th of SPLIT parts of the tile's columns
        const int q = warp & 3;
        const int half = (warp - 2) >> 2;
        constexpr int CPP = (BN / 32) / Cfg<FP8>::SPLIT;  // 32-column chunks per part
        int j = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++j) {
            int tm, tn, l, gi, ta0, items;
            decode(t, tm, tn, l, gi, ta0, items);
            const int b = j % NBUF;
            const uint32_t use = (uint32_t)(j / NBUF);
            if (!mbar_wait(&accf[b], use & 1, err, abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const uint32_t md = (uint32_t)tab.mod[l], yd = (uint32_t)tab.y[l], mg = tab.magic[l];
            const int i = tm * BM + q * 32 + lane;
            uint8_t* out = T + ((size_t)gi * tab.N + l) * (size_t)m * n;
            const uint32_t lane_addr = tmem + (uint32_t)(b * P * BN) + ((uint32_t)(q * 32) << 16);
            for (int ch = half * CPP; ch < (half + 1) * CPP; ++ch) {
                uint32_t r0[32];
                tmem_ld32(lane_addr + ch * 32, r0);
                int c[32];
                if (FP8) {
                    uint32_t r1[32], r2[32];
                    tmem_ld32(lane_addr + BN + ch * 32, r1);
                    tmem_ld32(lane_addr + 2 * BN + ch * 32, r2);
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        const int p00 = (int)__uint_as_float(r0[jj]);
                        const int p11 = (int)__uint_as_float(r1[jj]);
                        const int pss = (int)__uint_as_float(r2[jj]);
                        c[jj] = p00 + 17 * (pss - p00 - p11) + 289 * p11;
                    }
                } else {
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) c[jj] = (int)__uint_as_float(r0[jj]);
                }
                if (i < m) {
#pragma unroll
                    for (int jj = 0; jj < 32; ++jj) {
                        const int col = tn * BN + ch * 32 + jj;
                        if (col < n) out[(size_t)col * m + i] = (uint8_t)t_value(c[jj], md, yd, mg);
                    }
                }
            }
            // the accumulator buffer may be overwritten by the next tile's MMAs
            asm volatile("tcgen05.fence::before_thread_sync;\n");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(su32(&acce[b])) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
    }
}

// Self-test of the bounded mbarrier wait: one thread waits with the kernel's
// own wait routine on a barrier nothing ever arrives at (phase 0 of a fresh
// barrier), with a short iteration limit; out[0] = 1 if the wait gave up.
// No TMA, MMA or TMEM is involved.
__global__ void mbar_expiry_selftest_kernel(long long limit, int* err, int* out) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    const bool ok = mbar_wait(&bar, 0, err, &abort_flag, limit);
    out[0] = ok ? 0 : 1;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D map over a plane stack: inner dimension = Kpad elements, outer = rows
bool make_map(CUtensorMap* tm, const void* base, bool fp8, int Kpad, long long rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int esz = fp8 ? 1 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)Kpad, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)Kpad * esz};
    cuuint32_t box[2] = {(cuuint32_t)(BK / esz), (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    return fn(tm, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, (void*)base, dims,
              strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int launch_mbar_expiry_selftest(long long limit, int* err, int* out, cudaStream_t s) {
    mbar_expiry_selftest_kernel<<<1, 32, 0, s>>>(limit, err, out);
    return cudaGetLastError() == cudaSuccess ? OZLU_OK : OZLU_ERR_CUDA;
}

size_t tc05_smem_bytes() { return 2 * STAGES * TILE + 2 * STAGES * 8 + 4 * 8 + 16 + 1024; }

int launch_gemm_tc05(bool fp8, const void* RA, const void* RB, int m, int n, int Mpad, int Npad, int Kpad,
                     const DevTable& tab, uint8_t* T, int* err, cudaStream_t s) {
    const int P = fp8 ? 3 : 1;
    CUtensorMap ta, tb;
    if (!make_map(&ta, RA, fp8, Kpad, (long long)tab.N * tab.S * P * Mpad)) return OZLU_ERR_UNSUPPORTED;
    if (!make_map(&tb, RB, fp8, Kpad, (long long)tab.N * tab.S * P * Npad)) return OZLU_ERR_UNSUPPORTED;
    const int KB = Kpad * (fp8 ? 1 : 2) / BK;
    const size_t smem = tc05_smem_bytes();
    const int sms = device_sms();
    const long long tiles = (long long)(Mpad / BM) * (Npad / BN) * tab.N * tab.G;
    dim3 grid((unsigned)(tiles < sms ? tiles : sms));
    if (fp8) {
        raise_smem_limit((const void*)gemm_tc05_kernel<true>, (int)smem);
        gemm_tc05_kernel<true><<<grid, Cfg<true>::THREADS, smem, s>>>(ta, tb, m, n, Mpad, Npad, KB, tab, T, err);
    } else {
        raise_smem_limit((const void*)gemm_tc05_kernel<false>, (int)smem);
        gemm_tc05_kernel<false><<<grid, Cfg<false>::THREADS, smem, s>>>(ta, tb, m, n, Mpad, Npad, KB, tab, T, err);
    }
    return cudaGetLastError() == cudaSuccess ? OZLU_OK : OZLU_ERR_CUDA;
}

}  // namespace ozlu
