// gemm_tc.cu -- low-precision products of the gradient (Section 4.1) on the
// sm_103a tensor cores: tcgen05.mma with the accumulator in tensor memory,
// operands staged into shared memory by TMA (cp.async.bulk.tensor, 128-byte
// swizzle).  Operands are BF16 (kind::f16, K = 16 per MMA), E4M3
// (kind::f8f6f4, K = 32 per MMA) with one scale per operand row, applied to
// the accumulator in the epilogue, or FP32 split in two (kind::tf32, K = 8
// per MMA): every operand is stored as its TF32 part (the value rounded to
// 10 mantissa bits, low 13 bits zero) and the FP32 remainder, and each K
// step issues hi*hi into one FP32 accumulator and hi*lo + lo*hi into a
// second one, added in the epilogue -- the dropped lo*lo term and the tensor
// core's truncation of the remainders to TF32 leave about 2^-21 of each
// product, so these are the FP32 products of the solve at tensor-core speed.
// (Keeping the small terms apart matters: each MMA's addition into its
// accumulator loses about 2^-26 of it on average, always downwards, which
// over the ~3 K/8 additions of one accumulator came to 1.2e-5 of the result
// at K = 1000; the main accumulator now takes a third of them.)  Every kind's K stage is 128 bytes per
// row (and an MMA's K step 32 bytes), so the shared-memory layout, the
// descriptors and the ring are the same; the element count per stage (64,
// 128 or 32), the instruction and, for the split kind, the two operand
// parts per stage differ.
//
// Both products are "TN": C[i, j] = sum_k A[i, k] * B[j, k] with A and B
// stored K-major (row-major with the reduction index contiguous):
//   T = A X        A: adjacency (N x N), B: X^T (m x N), written by the blend
//   Y = T A' + lK  A: T (N x m),         B: A' itself (m x m) -- A' is
//                  symmetric, so its rows are the K-major columns and no
//                  transpose is ever formed.
// FP32 accumulation in TMEM; the epilogue writes T as BF16 (or, for the
// split kind, as its TF32 part and remainder) for the second product, or Y
// as FP32 with lambda K added.
//
// Persistent: one CTA per SM walks the 128 x BN output tiles of every
// problem of the group.  BN = 256 (the default) halves the shared-memory
// operand bytes per flop of a 128 x 128 tile, which would otherwise saturate
// shared memory; BN = 128 doubles the tile count, which keeps more SMs busy
// when a group has few small problems (fastpfp_autotune picks per size
// class).  Warp 0 issues the TMA loads of a 4-stage ring continuously across
// tiles, warp 1 owns the TMEM allocation (two BN-column accumulators) and one
// lane issues the MMAs (K = 16 each, four per 64-wide stage) into one
// accumulator while warps 2..5 drain the other with tcgen05.ld, so a tile's
// epilogue overlaps the next tile's main loop.
// Every mbarrier wait is bounded: on expiry the CTA records
// FASTPFP_ERR_TIMEOUT, every role stops, the TMEM is freed and it returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "internal.h"

namespace fpfp {
namespace {

constexpr int BM = kTcTileM;
constexpr int kRowBytes = 128;                 // bytes of one operand row per K stage
constexpr int kTileBytesA = BM * kRowBytes;
constexpr int kThreads = 192;
// Shapes that depend on the tile width BN (128 or 256) and the operand kind.
template <int BN, int KIND>
struct TcShape {
    static constexpr bool kSplit = KIND == kTcTf32x3;
    static constexpr int BK = KIND == kTcE4m3 ? 128 : KIND == kTcTf32x3 ? 32 : 64;   // K elements per stage
    static constexpr int kTileBytesB = BN * kRowBytes;
    static constexpr int kPartBytes = kTileBytesA + kTileBytesB;   // the A and B tiles of one part
    // a split stage holds both parts: [A hi][B hi][A lo][B lo]
    static constexpr int kStageBytes = kSplit ? 2 * kPartBytes : kPartBytes;
    static constexpr int kStages = kSplit ? (BN == 256 ? 2 : 3) : 4;
    // two tiles' accumulators (double buffering); a split tile has two, the
    // products of the TF32 parts and the corrections
    static constexpr uint32_t kAccCols = kSplit ? 2 * BN : BN;
    static constexpr uint32_t kTmemCols = 2 * kAccCols;
    static_assert(kTmemCols <= 512, "tensor memory has 512 columns");
    // Instruction descriptor: FP32 accumulate (bits 4-5), A and B types
    // (bits 7-9, 10-12: BF16 = 1 and TF32 = 2 for kind::f16 / kind::tf32,
    // E4M3 = 0 for kind::f8f6f4), both K-major, N >> 3 (bits 17-22),
    // M >> 4 (bits 24-28).
    static constexpr uint32_t kFmt = KIND == kTcBf16 ? 1u : KIND == kTcTf32x3 ? 2u : 0u;
    static constexpr uint32_t kIdesc = (1u << 4) | (kFmt << 7) | (kFmt << 10) | ((uint32_t)(BN >> 3) << 17) |
                                       ((uint32_t)(BM >> 4) << 24);
};
constexpr long long kWaitNs = 2000ll * 1000000ll;
static_assert(sizeof(TcGroup) <= 32000, "a TcGroup is passed as one kernel parameter (at most 32 KB)");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on phase `parity`; false (and *abort set) on expiry or when
// another role of the CTA has already given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (unsigned it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63u) == 0u) {
            if (*abort) return false;
            if ((long long)(globaltimer_ns() - t0) > kWaitNs) {
                *abort = 1;
                return false;
            }
        }
    }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor (tcgen05): K-major operand, 128-byte
// swizzle, 8-row core groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride byte offset
    d |= (uint64_t)1 << 46;                     // fixed 0b001
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}
template <int KIND>
__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t acc) {
    if (KIND == kTcTf32x3)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    else if (KIND == kTcE4m3)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Output tile t of the group: problem g, tile row / column, or false when
// the solve that owns the problem is not running in the group's phase (its
// low-precision phase, or its FP32 phase for the split products; every role
// of every CTA decides the same way: the flags do not change during a
// launch).
template <int BN>
__device__ __forceinline__ bool tile_of(const TcGroup& G, int t, int* g, int* m0, int* n0) {
    int p = 0;
    while (p + 1 < G.count && G.tile0[p + 1] <= t) ++p;
    const int local = t - G.tile0[p];
    *g = p;
    *m0 = (local / G.ntn[p]) * BM;
    *n0 = (local % G.ntn[p]) * BN;
    const TcProblem& pr = G.prob[p];
    if (pr.ctrl) {
        if (ld_relaxed_i32(&pr.ctrl->done) != 0 || ld_relaxed_i32(&pr.ctrl->error) != 0 ||
            ld_relaxed_i32(&pr.ctrl->idle) != 0)
            return false;
        if ((ld_relaxed_i32(&pr.ctrl->lowp) != 0) != (G.phase == 0)) return false;
    }
    return true;
}

// The TF32 part of an FP32 value: rounded to 10 mantissa bits (to nearest,
// ties away from zero), low 13 bits zero.
__device__ __forceinline__ float tf32_hi(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Epilogue of one tile: warp `quarter` of the four epilogue warps drains TMEM
// lanes 32 * quarter .. + 31 (tile rows) of accumulator column base `tcol`
// (and adds the correction accumulator `BN` columns after it when `split`).
template <int BN>
__device__ __forceinline__ void drain_tile(const TcGroup& G, const TcProblem& pr, uint32_t tmem, uint32_t tcol,
                                           int quarter, int lane, int m0, int n0, bool split) {
    const int row = m0 + quarter * 32 + lane;
    const float rsc = (pr.rs && row < pr.M) ? __ldg(pr.rs + row) : 1.f;
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
        uint32_t r[32];
        const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + tcol + (uint32_t)c;
        tmem_ld32(ta, r);
        if (split) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t q[16];
                tmem_ld16(ta + (uint32_t)BN + (uint32_t)(16 * h), q);
#pragma unroll
                for (int v = 0; v < 16; ++v)
                    r[16 * h + v] = __float_as_uint(__uint_as_float(r[16 * h + v]) + __uint_as_float(q[v]));
            }
        }
        const int col = n0 + c;
        if (row >= pr.M || col >= pr.N) continue;
        const int nv = min(32, pr.N - col);
        if (pr.rs) {   // dequantisation: rs[row] * cs[col + v]
#pragma unroll
            for (int v = 0; v < 32; ++v) {
                const float cv = (pr.cs && v < nv) ? __ldg(pr.cs + col + v) : 1.f;
                r[v] = __float_as_uint(__uint_as_float(r[v]) * (rsc * cv));
            }
        }
        if (G.mode == kTcOutBf16) {
            __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(pr.out) + (size_t)row * pr.ldo + col;
            if (nv == 32) {
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    uint4 pk;
                    __nv_bfloat162 h0 = __floats2bfloat162_rn(__uint_as_float(r[8 * v + 0]), __uint_as_float(r[8 * v + 1]));
                    __nv_bfloat162 h1 = __floats2bfloat162_rn(__uint_as_float(r[8 * v + 2]), __uint_as_float(r[8 * v + 3]));
                    __nv_bfloat162 h2 = __floats2bfloat162_rn(__uint_as_float(r[8 * v + 4]), __uint_as_float(r[8 * v + 5]));
                    __nv_bfloat162 h3 = __floats2bfloat162_rn(__uint_as_float(r[8 * v + 6]), __uint_as_float(r[8 * v + 7]));
                    pk.x = *reinterpret_cast<uint32_t*>(&h0);
                    pk.y = *reinterpret_cast<uint32_t*>(&h1);
                    pk.z = *reinterpret_cast<uint32_t*>(&h2);
                    pk.w = *reinterpret_cast<uint32_t*>(&h3);
                    reinterpret_cast<uint4*>(out)[v] = pk;
                }
            } else {
                for (int v = 0; v < nv; ++v) out[v] = __float2bfloat16_rn(__uint_as_float(r[v]));
            }
        } else if (G.mode == kTcOutSplit) {
            float* hi = reinterpret_cast<float*>(pr.out) + (size_t)row * pr.ldo + col;
            float* lo = pr.out_lo + (size_t)row * pr.ldo + col;
            if (nv == 32) {
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const float4 x = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                                 __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
                    const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
                    reinterpret_cast<float4*>(hi)[v] = h;
                    reinterpret_cast<float4*>(lo)[v] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
                }
            } else {
                for (int v = 0; v < nv; ++v) {
                    const float x = __uint_as_float(r[v]), h = tf32_hi(x);
                    hi[v] = h;
                    lo[v] = x - h;
                }
            }
        } else {
            float* out = reinterpret_cast<float*>(pr.out) + (size_t)row * pr.ldo + col;
            const float* kk = pr.Kmat ? pr.Kmat + (size_t)row * pr.ldk + col : nullptr;
            if (pr.addend) {   // projected gradient step: addend + scale * acc
                const float* ad = pr.addend + (size_t)row * pr.ld_add + col;
#pragma unroll
                for (int v = 0; v < 32; ++v)
                    if (v < nv) r[v] = __float_as_uint(fmaf(pr.scale, __uint_as_float(r[v]), __ldg(ad + v)));
            }
            if (nv == 32) {
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    float4 o = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                           __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
                    if (kk) {
                        const float4 kv = __ldg(reinterpret_cast<const float4*>(kk) + v);
                        o.x = fmaf(pr.lambda, kv.x, o.x);
                        o.y = fmaf(pr.lambda, kv.y, o.y);
                        o.z = fmaf(pr.lambda, kv.z, o.z);
                        o.w = fmaf(pr.lambda, kv.w, o.w);
                    }
                    reinterpret_cast<float4*>(out)[v] = o;
                }
            } else {
                for (int v = 0; v < nv; ++v) {
                    float o = __uint_as_float(r[v]);
                    if (kk) o = fmaf(pr.lambda, kk[v], o);
                    out[v] = o;
                }
            }
        }
    }
}

template <int BN, int KIND>
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(const __grid_constant__ TcGroup G) {
    using S = TcShape<BN, KIND>;
    constexpr int BK = S::BK;
    constexpr int STAGES = S::kStages;
    constexpr int kStageBytes = S::kStageBytes;
    constexpr uint32_t kTmemCols = S::kTmemCols;
    const int ntiles = G.tile0[G.count];
    if ((int)blockIdx.x >= ntiles) return;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment of the tile ring (required by the 128-byte swizzle)
    unsigned char* base = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char* tiles = base;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * kStageBytes);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;   // [2]
    uint64_t* acc_empty = acc_full + 2;    // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);   // one arrival per epilogue warp
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer: the k-blocks of this CTA's tiles, one ring across tiles
        uint32_t it = 0;
        for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
            int g, m0, n0;
            if (!tile_of<BN>(G, t, &g, &m0, &n0)) continue;
            const int nk = (G.prob[g].K + BK - 1) / BK;
            for (int kb = 0; kb < nk; ++kb, ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (it / STAGES) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u, abort)) break;
                unsigned char* a = tiles + s * kStageBytes;
                unsigned char* b = a + kTileBytesA;
                mbar_expect_tx(&full[s], kStageBytes);
                tma_load_2d(a, &G.map_a[g], kb * BK, m0, &full[s]);
                tma_load_2d(b, &G.map_b[g], kb * BK, n0, &full[s]);
                if (S::kSplit) {
                    tma_load_2d(a + S::kPartBytes, &G.map_a_lo[g], kb * BK, m0, &full[s]);
                    tma_load_2d(b + S::kPartBytes, &G.map_b_lo[g], kb * BK, n0, &full[s]);
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: accumulator tc & 1 of the CTA's tc-th tile
        uint32_t it = 0, tc = 0;
        for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
            int g, m0, n0;
            if (!tile_of<BN>(G, t, &g, &m0, &n0)) continue;
            const int nk = (G.prob[g].K + BK - 1) / BK;
            const uint32_t buf = tc & 1u, aph = (tc >> 1) & 1u;
            if (!mbar_wait(&acc_empty[buf], aph ^ 1u, abort)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + buf * S::kAccCols;
            bool ok = true;
            for (int kb = 0; kb < nk; ++kb, ++it) {
                const int s = it % STAGES;
                const uint32_t ph = (it / STAGES) & 1u;
                if (!mbar_wait(&full[s], ph, abort)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a = smem_u32(tiles + s * kStageBytes);
                const uint32_t b = a + kTileBytesA;
                const uint64_t ad = smem_desc(a), bd = smem_desc(b);
                if (S::kSplit) {
                    const uint64_t adl = smem_desc(a + S::kPartBytes), bdl = smem_desc(b + S::kPartBytes);
                    const uint32_t corr = acc + (uint32_t)BN;   // the correction accumulator
#pragma unroll
                    for (int j = 0; j < 4; ++j) {   // 32 bytes of K per MMA (8 TF32)
                        const uint64_t o = (uint64_t)(2 * j);
                        const uint32_t first = (kb > 0 || j > 0) ? 1u : 0u;
                        mma_issue<KIND>(corr, ad + o, bdl + o, S::kIdesc, first);   // hi * lo
                        mma_issue<KIND>(corr, adl + o, bd + o, S::kIdesc, 1u);      // lo * hi
                        mma_issue<KIND>(acc, ad + o, bd + o, S::kIdesc, first);     // hi * hi
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j)   // 32 bytes of K per MMA (16 BF16 or 32 E4M3)
                        mma_issue<KIND>(acc, ad + (uint64_t)(2 * j), bd + (uint64_t)(2 * j), S::kIdesc,
                                        (kb > 0 || j > 0) ? 1u : 0u);
                }
                mma_commit(&empty[s]);
            }
            if (!ok) break;
            mma_commit(&acc_full[buf]);
            ++tc;
        }
    } else if (warp >= 2) {
        // epilogue: warp w drains TMEM lanes 32 * (w % 4) .. + 31 = tile rows
        const int quarter = warp & 3;
        uint32_t tc = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            int g, m0, n0;
            if (!tile_of<BN>(G, t, &g, &m0, &n0)) continue;
            const uint32_t buf = tc & 1u, aph = (tc >> 1) & 1u;
            // one lane waits; tcgen05.ld is warp-collective, so the outcome is broadcast
            int okl = 0;
            if (lane == 0) okl = mbar_wait(&acc_full[buf], aph, abort) ? 1 : 0;
            if (__shfl_sync(0xffffffffu, okl, 0) == 0) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            drain_tile<BN>(G, G.prob[g], tmem, buf * S::kAccCols, quarter, lane, m0, n0, S::kSplit);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[buf]))
                             : "memory");
            }
            ++tc;
        }
    }
    __syncthreads();
    if (*abort && threadIdx.x == 0) {
        // every problem of the group gets the timeout (their solves stop)
        for (int g = 0; g < G.count; ++g)
            if (G.prob[g].err) atomicCAS(G.prob[g].err, 0, FASTPFP_ERR_TIMEOUT);
    }
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

}  // namespace

template <int BN, int KIND>
constexpr size_t tc_smem_of() {
    return (size_t)TcShape<BN, KIND>::kStages * TcShape<BN, KIND>::kStageBytes + 1024 + 256;
}

size_t tc_smem_bytes(int bn, int kind) {
    if (kind == kTcTf32x3) return tc_smem_of<128, kTcTf32x3>();
    if (kind == kTcE4m3) return bn == 128 ? tc_smem_of<128, kTcE4m3>() : tc_smem_of<256, kTcE4m3>();
    return bn == 128 ? tc_smem_of<128, kTcBf16>() : tc_smem_of<256, kTcBf16>();
}

static int g_tc_sms = 0;

cudaError_t tc_configure() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_tc_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const void* fns[6] = {(const void*)tc_gemm_kernel<256, kTcBf16>,   (const void*)tc_gemm_kernel<128, kTcBf16>,
                          (const void*)tc_gemm_kernel<256, kTcE4m3>,   (const void*)tc_gemm_kernel<128, kTcE4m3>,
                          (const void*)tc_gemm_kernel<128, kTcTf32x3>, (const void*)tc_gemm_kernel<128, kTcTf32x3>};
    for (int i = 0; i < 6; ++i) {
        e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tc_smem_bytes((i & 1) ? 128 : 256, i / 2));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// rows x cols matrix, row-major with leading dimension ld elements (BF16,
// ld a multiple of 8; E4M3 bytes, ld a multiple of 16; FP32, ld a multiple
// of 4), read as boxes of 128 bytes along K by box_rows rows (128 for the A
// operand, the group's tile width for B) with 128-byte swizzle.
bool tc_make_map(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int box_rows, int kind) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    const int esize = kind == kTcE4m3 ? 1 : kind == kTcTf32x3 ? 4 : 2;
    if (!fn || ((size_t)ld * esize) % 16 != 0 || (reinterpret_cast<uintptr_t>(ptr) & 15) != 0) return false;
    if (box_rows != 128 && box_rows != 256) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
    const cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esize), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt = kind == kTcE4m3   ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                   : kind == kTcTf32x3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                       : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const CUresult r = fn(map, dt, 2,
                          const_cast<void*>(ptr), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

cudaError_t tc_gemm(const TcGroup& G0, cudaStream_t s) {
    if (G0.count <= 0) return cudaSuccess;
    TcGroup G = G0;
    // split products keep two accumulators per tile: 128-column tiles only
    // (their B tensor maps carry a 128-row box)
    if (G.kind == kTcTf32x3 && G.bn != 128) return cudaErrorInvalidValue;
    const int bn = G.bn == 128 ? 128 : 256;
    G.tile0[0] = 0;
    for (int i = 0; i < G.count; ++i) {
        G.ntn[i] = (G.prob[i].N + bn - 1) / bn;
        G.tile0[i + 1] = G.tile0[i] + ((G.prob[i].M + BM - 1) / BM) * G.ntn[i];
    }
    const int ntiles = G.tile0[G.count];
    if (ntiles <= 0) return cudaSuccess;
    const int grid = min(ntiles, g_tc_sms > 0 ? g_tc_sms : 148);
    const size_t smem = tc_smem_bytes(bn, G.kind);
    if (G.kind == kTcTf32x3) {
        tc_gemm_kernel<128, kTcTf32x3><<<grid, kThreads, smem, s>>>(G);
    } else if (G.kind == kTcE4m3) {
        if (bn == 128) tc_gemm_kernel<128, kTcE4m3><<<grid, kThreads, smem, s>>>(G);
        else tc_gemm_kernel<256, kTcE4m3><<<grid, kThreads, smem, s>>>(G);
    } else if (bn == 128) {
        tc_gemm_kernel<128, kTcBf16><<<grid, kThreads, smem, s>>>(G);
    } else {
        tc_gemm_kernel<256, kTcBf16><<<grid, kThreads, smem, s>>>(G);
    }
    return cudaGetLastError();
}

}  // namespace fpfp
