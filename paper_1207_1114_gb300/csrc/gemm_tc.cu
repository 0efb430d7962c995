// gemm_tc.cu -- low-precision products of the gradient (Section 4.1) on the
// sm_103a tensor cores: tcgen05.mma with the accumulator in tensor memory,
// operands staged into shared memory by TMA (cp.async.bulk.tensor, 128-byte
// swizzle).  Operands are BF16 (kind::f16, K = 16 per MMA) or E4M3
// (kind::f8f6f4, K = 32 per MMA) with one scale per operand row, applied to
// the accumulator in the epilogue.  Either way a K stage is 128 bytes per
// row, so the shared-memory layout, the descriptors and the ring are the
// same; only the element count per stage (64 or 128) and the instruction
// differ.
//
// Both products are "TN": C[i, j] = sum_k A[i, k] * B[j, k] with A and B
// stored K-major (row-major with the reduction index contiguous):
//   T = A X        A: adjacency (N x N), B: X^T (m x N), written by the blend
//   Y = T A' + lK  A: T (N x m),         B: A' itself (m x m) -- A' is
//                  symmetric, so its rows are the K-major columns and no
//                  transpose is ever formed.
// FP32 accumulation in TMEM; the epilogue writes T as BF16 for the second
// product, or Y as FP32 with lambda K added.
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

constexpr int BM = kTcTileM, STAGES = 4;
constexpr int kRowBytes = 128;                 // bytes of one operand row per K stage
constexpr int kTileBytesA = BM * kRowBytes;
constexpr int kThreads = 192;
// Shapes that depend on the tile width BN (128 or 256) and the operand type.
template <int BN, bool F8>
struct TcShape {
    static constexpr int BK = F8 ? 128 : 64;       // K elements per stage
    static constexpr int kTileBytesB = BN * kRowBytes;
    static constexpr int kStageBytes = kTileBytesA + kTileBytesB;
    static constexpr uint32_t kTmemCols = 2 * BN;   // two BN-column FP32 accumulators
    // Instruction descriptor: FP32 accumulate (bits 4-5), A and B types
    // (bits 7-9, 10-12: BF16 = 1 for kind::f16, E4M3 = 0 for kind::f8f6f4),
    // both K-major, N >> 3 (bits 17-22), M >> 4 (bits 24-28).
    static constexpr uint32_t kIdesc = (1u << 4) | (F8 ? 0u : (1u << 7) | (1u << 10)) |
                                       ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};
constexpr long long kWaitNs = 2000ll * 1000000ll;

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
template <bool F8>
__device__ __forceinline__ void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t acc) {
    if (F8)
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
// the solve that owns the problem is not in its BF16 phase (every role of
// every CTA decides the same way: the flags do not change during a launch).
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
        if (ld_relaxed_i32(&pr.ctrl->lowp) == 0) return false;
    }
    return true;
}

// Epilogue of one tile: warp `quarter` of the four epilogue warps drains TMEM
// lanes 32 * quarter .. + 31 (tile rows) of accumulator column base `tcol`.
template <int BN>
__device__ __forceinline__ void drain_tile(const TcGroup& G, const TcProblem& pr, uint32_t tmem, uint32_t tcol,
                                           int quarter, int lane, int m0, int n0) {
    const int row = m0 + quarter * 32 + lane;
    const float rsc = (pr.rs && row < pr.M) ? __ldg(pr.rs + row) : 1.f;
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + tcol + (uint32_t)c, r);
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

template <int BN, bool F8>
__global__ void __launch_bounds__(kThreads, 1) tc_gemm_kernel(const __grid_constant__ TcGroup G) {
    using S = TcShape<BN, F8>;
    constexpr int BK = S::BK;
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
            const uint32_t acc = tmem + buf * (uint32_t)BN;
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
#pragma unroll
                for (int j = 0; j < 4; ++j)   // 32 bytes of K per MMA (16 BF16 or 32 E4M3)
                    mma_issue<F8>(acc, ad + (uint64_t)(2 * j), bd + (uint64_t)(2 * j), S::kIdesc,
                                  (kb > 0 || j > 0) ? 1u : 0u);
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
            drain_tile<BN>(G, G.prob[g], tmem, buf * (uint32_t)BN, quarter, lane, m0, n0);
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

size_t tc_smem_bytes(int bn) {
    return (size_t)STAGES * (bn == 128 ? TcShape<128, false>::kStageBytes : TcShape<256, false>::kStageBytes) +
           1024 + 256;
}

static int g_tc_sms = 0;

cudaError_t tc_configure() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g_tc_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const void* fns[4] = {(const void*)tc_gemm_kernel<256, false>, (const void*)tc_gemm_kernel<128, false>,
                          (const void*)tc_gemm_kernel<256, true>, (const void*)tc_gemm_kernel<128, true>};
    for (int i = 0; i < 4; ++i) {
        e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tc_smem_bytes((i & 1) ? 128 : 256));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// rows x cols matrix, row-major with leading dimension ld elements (BF16,
// ld a multiple of 8; or E4M3 bytes, ld a multiple of 16), read as boxes of
// 128 bytes along K by box_rows rows (128 for the A operand, the group's
// tile width for B) with 128-byte swizzle.
bool tc_make_map(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int box_rows, bool fp8) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    const int esize = fp8 ? 1 : 2;
    if (!fn || ((size_t)ld * esize) % 16 != 0 || (reinterpret_cast<uintptr_t>(ptr) & 15) != 0) return false;
    if (box_rows != 128 && box_rows != 256) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * esize};
    const cuuint32_t box[2] = {(cuuint32_t)(kRowBytes / esize), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                          const_cast<void*>(ptr), dims,
                          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

cudaError_t tc_gemm(const TcGroup& G0, cudaStream_t s) {
    if (G0.count <= 0) return cudaSuccess;
    TcGroup G = G0;
    const int bn = G.bn == 128 ? 128 : 256;
    G.tile0[0] = 0;
    for (int i = 0; i < G.count; ++i) {
        G.ntn[i] = (G.prob[i].N + bn - 1) / bn;
        G.tile0[i + 1] = G.tile0[i] + ((G.prob[i].M + BM - 1) / BM) * G.ntn[i];
    }
    const int ntiles = G.tile0[G.count];
    if (ntiles <= 0) return cudaSuccess;
    const int grid = min(ntiles, g_tc_sms > 0 ? g_tc_sms : 148);
    if (G.fp8) {
        if (bn == 128)
            tc_gemm_kernel<128, true><<<grid, kThreads, tc_smem_bytes(128), s>>>(G);
        else
            tc_gemm_kernel<256, true><<<grid, kThreads, tc_smem_bytes(256), s>>>(G);
    } else if (bn == 128) {
        tc_gemm_kernel<128, false><<<grid, kThreads, tc_smem_bytes(128), s>>>(G);
    } else {
        tc_gemm_kernel<256, false><<<grid, kThreads, tc_smem_bytes(256), s>>>(G);
    }
    return cudaGetLastError();
}

}  // namespace fpfp
