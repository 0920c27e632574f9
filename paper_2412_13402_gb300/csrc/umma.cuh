// umma.cuh -- a BF16 GEMM on the fifth-generation tensor cores (tcgen05) for the surrogate's
// training and batched forward passes:
//     C[M x N] = A[M x K] * B[N x K]^T   (+ bias[n], tanh, BF16 copy of C)
// A and B are BF16 matrices in global memory (row stride lda / ldb elements, a multiple of 8),
// K-major ([M][K], [N][K]) or MN-major ([K][M], [K][N]; then bn is a multiple of 64), C is
// row-major FP32; a split of K over blockIdx.z writes its partial product to its own slice of C.
// One CTA of four warps computes a 128 x bn tile (bn = N rounded up to a multiple of 16, at most
// 256; wider N takes several tiles):
//   - TMA (cp.async.bulk.tensor, 128-byte swizzle) brings 64-column K slices of the A tile
//     (128 x 64) and the B tile (bn x 64) into a shared-memory ring of four stages (two when bn is
//     above 128), completing on an mbarrier with the transaction byte count;
//   - one thread issues four tcgen05.mma (M 128, N bn, K 16) per slice with the FP32 accumulator
//     in tensor memory, and tcgen05.commit releases the slice's stage (and, after the last
//     slice, the accumulator) through an mbarrier;
//   - the four warps read their 32 accumulator rows with tcgen05.ld and apply the epilogue.
// Out-of-range rows and columns of a tile are zero-filled by TMA and not stored.  Every mbarrier
// wait is bounded: on timeout the kernel writes a nonzero code to *err, stops issuing, waits
// (bounded) for the copies it started, frees its tensor memory and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace rtbte {
namespace umma {

constexpr int kTM = 128;        // tile rows (accumulator lanes)
constexpr int kTK = 64;         // K per stage: 64 BF16 = 128 bytes = one swizzle span
constexpr int kThreads = 128;
constexpr long long kWaitLimit = 1LL << 24;  // polls of an mbarrier before giving up
// MN-major tiles with 128-byte swizzle: blocks of 64 M (or N) elements x kTK K rows; the leading
// byte offset is the distance between such blocks, the stride byte offset the distance between
// 8-row K groups inside one (checked against a host reference)
constexpr uint32_t kMnLbo = kTK * 128, kMnSbo = 1024;

struct Args {
    int M, N, K, bn;
    int ldc, act;
    const float *bias;
    float *C;
    __nv_bfloat16 *Cb;
    int *err;
    int a_mn, b_mn;       // operand stored MN-major (M or N contiguous) instead of K-major
    int k_base;           // first K of this CTA's range (split-K over blockIdx.z: K range k_base + z * K)
    long long c_split;    // element stride of C between split-K slices
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// true when the phase with `parity` completed within the poll limit
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (long long i = 0; i < kWaitLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 64-bit shared-memory matrix descriptor of a K-major tile with 128-byte swizzle: rows of 128
// bytes, 8-row atoms of 1024 bytes (stride byte offset), version 1, swizzle mode 2.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr, uint32_t lbo = 16u, uint32_t sbo = 1024u) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);         // start address
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;    // leading byte offset
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;                         // descriptor version
    d |= (uint64_t)2 << 61;                         // 128-byte swizzle
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, M x N; a_mn / b_mn select
// the MN-major (transposed) layout of an operand
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn = 0, int b_mn = 0) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
            dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// NS-stage ring (NS = 2 or 4) of A and B slices; stage s holds A at base + s*a_bytes and B at
// base + NS*a_bytes + s*b_bytes, then the mbarriers full[NS], empty[NS], done and the TMEM slot.
template <int NCOLS, int NS>
__global__ void __launch_bounds__(kThreads) gemm_tc(const __grid_constant__ CUtensorMap tA,
                                                   const __grid_constant__ CUtensorMap tB, Args a) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // 128-byte swizzled tiles sit on 1024-byte boundaries
    const int bn = a.bn;
    const uint32_t a_bytes = kTM * kTK * 2, b_bytes = (uint32_t)bn * kTK * 2;
    uint32_t sA[NS], sB[NS], full[NS], empty[NS];
    const uint32_t bars = base + NS * (a_bytes + b_bytes);
#pragma unroll
    for (int i = 0; i < NS; ++i) {
        sA[i] = base + i * a_bytes;
        sB[i] = base + NS * a_bytes + i * b_bytes;
        full[i] = bars + 8 * i;
        empty[i] = bars + 8 * (NS + i);
    }
    const uint32_t done = bars + 16 * NS, tslot = done + 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kTM, n0 = blockIdx.y * bn;
    const int nk = (a.K + kTK - 1) / kTK;
    const int kb = a.k_base + blockIdx.z * a.K;  // this CTA's first K
    // one stage's copies: a K-major tile is one box {64 K, rows}; an MN-major tile is boxes of
    // {64 M or N, 64 K}, one per 64 rows, kTK * 128 bytes apart
    auto load_stage = [&](int s, int kt) {
        const int k0 = kb + kt * kTK;
        mbar_expect_tx(full[s], a_bytes + b_bytes);
        if (a.a_mn) {
            for (int h = 0; h < kTM / 64; ++h) tma_load_2d(sA[s] + h * (kTK * 128), &tA, m0 + 64 * h, k0, full[s]);
        } else {
            tma_load_2d(sA[s], &tA, k0, m0, full[s]);
        }
        if (a.b_mn) {
            for (int h = 0; h < bn / 64; ++h) tma_load_2d(sB[s] + h * (kTK * 128), &tB, n0 + 64 * h, k0, full[s]);
        } else {
            tma_load_2d(sB[s], &tB, k0, n0, full[s]);
        }
    };

    if (threadIdx.x == 0) {
        for (int i = 0; i < NS; ++i) {
            mbar_init(full[i], 1);
            mbar_init(empty[i], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {  // tensor memory for the accumulator: NCOLS columns x 128 lanes
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(tslot), "r"(NCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    uint32_t tmem;
    asm volatile("ld.shared.b32 %0, [%1];\n" : "=r"(tmem) : "r"(tslot) : "memory");

    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        s_fail = 0;
        const uint32_t idesc = idesc_bf16(kTM, bn, a.a_mn, a.b_mn);
        int issued = 0;  // slices whose TMA was started
        for (int s = 0; s < NS && s < nk; ++s) {
            load_stage(s, s);
            ++issued;
        }
        bool ok = true;
        for (int kt = 0; kt < nk && ok; ++kt) {
            const int s = kt % NS;
            const uint32_t par = (uint32_t)((kt / NS) & 1);
            if (!(ok = mbar_wait(full[s], par))) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int k16 = 0; k16 < kTK / 16; ++k16) {
                // K step of 16: 32 bytes along a K-major row, or two 8-row K groups of an MN-major block
                const uint64_t da = a.a_mn ? sw128_desc(sA[s] + 2048u * k16, kMnLbo, kMnSbo)
                                           : sw128_desc(sA[s] + 32u * k16);
                const uint64_t db = a.b_mn ? sw128_desc(sB[s] + 2048u * k16, kMnLbo, kMnSbo)
                                           : sw128_desc(sB[s] + 32u * k16);
                const uint32_t acc = (kt > 0 || k16 > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(empty[s])
                         : "memory");
            if (kt + NS < nk) {  // refill this stage once its MMAs have read it
                if (!(ok = mbar_wait(empty[s], par))) break;
                load_stage(s, kt + NS);
                ++issued;
            }
        }
        if (ok) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(done)
                         : "memory");
        } else {  // give up: record it, let the copies already started land before the CTA leaves
            s_fail = 1;
            atomicExch(a.err, 1);
            for (int kt = 0; kt < issued; ++kt) mbar_wait(full[kt % NS], (uint32_t)((kt / NS) & 1));
        }
    }
    __syncthreads();
    const bool failed = s_fail != 0;
    if (!failed && !mbar_wait(done, 0)) {
        if (lane == 0) atomicExch(a.err, 2);
    } else if (!failed) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int row = m0 + 32 * warp + lane;
        for (int c0 = 0; c0 < bn; c0 += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (row >= a.M) continue;
            const int col0 = n0 + c0;
            float v[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                v[j] = __uint_as_float(r[j]);
                if (a.bias && col0 + j < a.N) v[j] += a.bias[col0 + j];
                if (a.act) v[j] = tanhf(v[j]);
            }
            float *cr = a.C + (long long)blockIdx.z * a.c_split + (long long)row * a.ldc + col0;
            __nv_bfloat16 *br = a.Cb ? a.Cb + (long long)row * a.ldc + col0 : nullptr;
            // 16-byte stores where the 16 columns are in range and the row is 16-byte aligned
            if (col0 + 16 <= a.N && (a.ldc & 3) == 0 && (col0 & 3) == 0) {
#pragma unroll
                for (int j = 0; j < 16; j += 4) *reinterpret_cast<float4 *>(cr + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                if (br && (a.ldc & 7) == 0 && (col0 & 7) == 0) {
#pragma unroll
                    for (int j = 0; j < 16; j += 8) {
                        uint4 u;
                        __nv_bfloat162 h0 = __floats2bfloat162_rn(v[j], v[j + 1]), h1 = __floats2bfloat162_rn(v[j + 2], v[j + 3]),
                                       h2 = __floats2bfloat162_rn(v[j + 4], v[j + 5]), h3 = __floats2bfloat162_rn(v[j + 6], v[j + 7]);
                        u.x = *reinterpret_cast<uint32_t *>(&h0);
                        u.y = *reinterpret_cast<uint32_t *>(&h1);
                        u.z = *reinterpret_cast<uint32_t *>(&h2);
                        u.w = *reinterpret_cast<uint32_t *>(&h3);
                        *reinterpret_cast<uint4 *>(br + j) = u;
                    }
                } else if (br) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) br[j] = __float2bfloat16(v[j]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (col0 + j >= a.N) break;
                    cr[j] = v[j];
                    if (br) br[j] = __float2bfloat16(v[j]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOLS) : "memory");
}

// Stages of the ring: four while they fit beside each other in 128 KB, else two.
inline int stages_for(int bn) { return 4 * ((size_t)(kTM * kTK * 2) + (size_t)bn * kTK * 2) <= 131072 ? 4 : 2; }
// Dynamic shared memory of one CTA: the ring's A and B tiles, barriers, alignment slack.
inline size_t smem_bytes(int bn) {
    const int ns = stages_for(bn);
    return 1024 + (size_t)ns * ((size_t)(kTM * kTK * 2) + (size_t)bn * kTK * 2) + 16 * (size_t)ns + 64;
}

}  // namespace umma
}  // namespace rtbte
