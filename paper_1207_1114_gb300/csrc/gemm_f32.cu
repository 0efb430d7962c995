// gemm_f32.cu -- exact-FP32 products of the gradient (Section 4.1):
//   T = A X  and  Y[:, :m] = T A' + lambda K,
// as a shared-memory tiled SIMT GEMM (FP32 FMA, FP32 accumulation).  This is
// the "plain" precision of the solver and its refinement phase; the BF16
// tensor-core path lives in gemm_tc.cu.
#include "common.cuh"
#include "internal.h"

namespace fpfp {
namespace {

constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
constexpr int kThreads = (BM / TM) * (BN / TN);  // 256

__global__ void __launch_bounds__(kThreads) gemm_f32_kernel(const __grid_constant__ GemmF32Group grp) {
    if ((int)blockIdx.z >= grp.count) return;
    const GemmF32Args& g = grp.a[blockIdx.z];
    if ((int)blockIdx.y * BM >= g.M || (int)blockIdx.x * BN >= g.Nc) return;
    if (g.ctrl) {
        if (ld_relaxed_i32(&g.ctrl->done) != 0 || ld_relaxed_i32(&g.ctrl->error) != 0 ||
            ld_relaxed_i32(&g.ctrl->idle) != 0)
            return;
        if (ld_relaxed_i32(&g.ctrl->lowp) != 0) return;
    }
    __shared__ __align__(16) float As[2][BK][BM];
    __shared__ __align__(16) float Bs[2][BK][BN];
    const int tid = threadIdx.x;
    const int tr = tid / (BN / TN);   // 0..15
    const int tc = tid % (BN / TN);   // 0..15
    const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;

    // global -> shared mapping: A tile BM x BK (1024 values, 4 per thread),
    // B tile BK x BN (1024 values, 4 per thread)
    const int a_r = tid >> 1, a_k = (tid & 1) * 4;        // rows 0..127, k 0 or 4
    const int b_k = tid >> 5, b_c = (tid & 31) * 4;       // k 0..7, cols 0..124

    float acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

    float ra[4], rb[4];
    auto load_tiles = [&](int k0) {
        const int gr = row0 + a_r;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int gk = k0 + a_k + e;
            ra[e] = (gr < g.M && gk < g.K) ? __ldg(g.A + (size_t)gr * g.lda + gk) : 0.f;
        }
        const int gk = k0 + b_k;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int gc = col0 + b_c + e;
            rb[e] = (gk < g.K && gc < g.Nc) ? __ldg(g.B + (size_t)gk * g.ldb + gc) : 0.f;
        }
    };
    auto store_tiles = [&](int buf) {
#pragma unroll
        for (int e = 0; e < 4; ++e) As[buf][a_k + e][a_r] = ra[e];
        *reinterpret_cast<float4*>(&Bs[buf][b_k][b_c]) = make_float4(rb[0], rb[1], rb[2], rb[3]);
    };

    load_tiles(0);
    store_tiles(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < g.K; k0 += BK) {
        const bool more = k0 + BK < g.K;
        if (more) load_tiles(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[TM], b[TN];
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tr * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + tr * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tc * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tc * 4]);
            a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
            a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
            b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
            b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        if (more) {
            store_tiles(buf ^ 1);
            __syncthreads();
            buf ^= 1;
        }
    }

    // epilogue: rows {tr*4 + i, 64 + tr*4 + i}, cols {tc*4 + j, 64 + tc*4 + j}
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = row0 + (i < 4 ? tr * 4 + i : 64 + tr * 4 + (i - 4));
        if (r >= g.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int c = col0 + (j < 4 ? tc * 4 + j : 64 + tc * 4 + (j - 4));
            if (c >= g.Nc) continue;
            float v = acc[i][j];
            if (g.Kmat) v = fmaf(g.lambda, __ldg(g.Kmat + (size_t)r * g.ldk + c), v);
            g.C[(size_t)r * g.ldc + c] = v;
        }
    }
}

// ---------------------------------------------------------------------------
// The solve's products with the left operand supplied transposed (K x M
// row-major) and both operands 16-byte aligned with leading dimensions that
// are multiples of 4: every shared-memory tile row is a contiguous run of
// global memory, copied with cp.async into a three-stage ring.  BMT x 128 x
// 16 tiles (BMT = 128 or 64, picked per problem size by fastpfp_autotune),
// 256 threads, (BMT / 16) x 8 outputs per thread, packed f32x2 FMAs (two
// accumulators per instruction), FP32 accumulation in a fixed order per
// output.
constexpr int TBK = 16, TSTAGES = 3;
template <int BMT>
constexpr size_t tile_stage_floats() { return (size_t)TBK * (BMT + BN); }

__device__ __forceinline__ void cp_async16_zfill(void* smem_dst, const void* gmem_src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gmem_src), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

template <int BMT>
__global__ void __launch_bounds__(kThreads) gemm_f32t_kernel(const __grid_constant__ GemmF32TGroup grp) {
    constexpr int TMT = BMT / 16;                                // rows per thread: 8 or 4
    constexpr size_t kStage = tile_stage_floats<BMT>();
    if ((int)blockIdx.z >= grp.count) return;
    const GemmF32TArgs& g = grp.a[blockIdx.z];
    if ((int)blockIdx.y * BMT >= g.M || (int)blockIdx.x * BN >= g.Nc) return;
    if (g.ctrl) {
        if (ld_relaxed_i32(&g.ctrl->done) != 0 || ld_relaxed_i32(&g.ctrl->error) != 0 ||
            ld_relaxed_i32(&g.ctrl->idle) != 0)
            return;
        if (ld_relaxed_i32(&g.ctrl->lowp) != 0) return;
    }
    extern __shared__ __align__(16) float tsm[];
    const int tid = threadIdx.x;
    const int tr = tid / (BN / TN), tc = tid % (BN / TN);
    const int row0 = blockIdx.y * BMT, col0 = blockIdx.x * BN;
    const int KT = (g.K + TBK - 1) / TBK;

    // stage st: As = tsm + st * stage (TBK x BMT), Bs = As + TBK * BMT (TBK x BN)
    auto issue = [&](int st, int kt) {
        float* As = tsm + (size_t)st * kStage;
        float* Bs = As + TBK * BMT;
        const int k0 = kt * TBK;
#pragma unroll
        for (int idx = tid; idx < TBK * BMT / 4; idx += kThreads) {
            const int kk = idx / (BMT / 4), c4 = (idx % (BMT / 4)) * 4;
            const int gk = k0 + kk;
            const bool va = gk < g.K && row0 + c4 < g.M;
            cp_async16_zfill(As + kk * BMT + c4, va ? g.AT + (size_t)gk * g.lda + row0 + c4 : g.AT, va);
        }
#pragma unroll
        for (int idx = tid; idx < TBK * BN / 4; idx += kThreads) {
            const int kk = idx >> 5, c4 = (idx & 31) * 4;
            const int gk = k0 + kk;
            const bool vb = gk < g.K && col0 + c4 < g.Nc;
            cp_async16_zfill(Bs + kk * BN + c4, vb ? g.B + (size_t)gk * g.ldb + col0 + c4 : g.B, vb);
        }
    };

    unsigned long long acc[TMT][TN / 2];
#pragma unroll
    for (int i = 0; i < TMT; ++i)
#pragma unroll
        for (int j = 0; j < TN / 2; ++j) acc[i][j] = 0ull;   // (+0.0f, +0.0f)

#pragma unroll
    for (int st = 0; st < TSTAGES - 1; ++st) {
        if (st < KT) issue(st, st);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int kt = 0; kt < KT; ++kt) {
        asm volatile("cp.async.wait_group %0;" ::"n"(TSTAGES - 2) : "memory");
        __syncthreads();   // tile kt is in place; every thread is done with tile kt - 1
        if (kt + TSTAGES - 1 < KT) issue((kt + TSTAGES - 1) % TSTAGES, kt + TSTAGES - 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
        const float* As = tsm + (size_t)(kt % TSTAGES) * kStage;
        const float* Bs = As + TBK * BMT;
#pragma unroll
        for (int kk = 0; kk < TBK; ++kk) {
            float a[TMT];
            const float4 a0 = *reinterpret_cast<const float4*>(As + kk * BMT + tr * 4);
            a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
            if (TMT == 8) {
                const float4 a1 = *reinterpret_cast<const float4*>(As + kk * BMT + 64 + tr * 4);
                a[TMT > 4 ? 4 : 0] = a1.x; a[TMT > 5 ? 5 : 0] = a1.y;
                a[TMT > 6 ? 6 : 0] = a1.z; a[TMT > 7 ? 7 : 0] = a1.w;
            }
            const float4 b0 = *reinterpret_cast<const float4*>(Bs + kk * BN + tc * 4);
            const float4 b1 = *reinterpret_cast<const float4*>(Bs + kk * BN + 64 + tc * 4);
            const unsigned long long b[TN / 2] = {pk2(b0.x, b0.y), pk2(b0.z, b0.w), pk2(b1.x, b1.y),
                                                  pk2(b1.z, b1.w)};
#pragma unroll
            for (int i = 0; i < TMT; ++i) {
                const unsigned long long ai = pk2(a[i], a[i]);
#pragma unroll
                for (int j = 0; j < TN / 2; ++j) acc[i][j] = ffma2(ai, b[j], acc[i][j]);
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");

#pragma unroll
    for (int i = 0; i < TMT; ++i) {
        const int r = row0 + (i < 4 ? tr * 4 + i : 64 + tr * 4 + (i - 4));
        if (r >= g.M) continue;
#pragma unroll
        for (int j = 0; j < TN; ++j) {
            const int c = col0 + (j < 4 ? tc * 4 + j : 64 + tc * 4 + (j - 4));
            if (c >= g.Nc) continue;
            const unsigned long long pr = acc[i][j >> 1];
            float v = __uint_as_float((unsigned)((j & 1) ? (pr >> 32) : (pr & 0xffffffffull)));
            if (g.addend) v = fmaf(g.scale, v, __ldg(g.addend + (size_t)r * g.ld_add + c));
            if (g.Kmat) v = fmaf(g.lambda, __ldg(g.Kmat + (size_t)r * g.ldk + c), v);
            g.C[(size_t)r * g.ldc + c] = v;
        }
    }
}

}  // namespace

template <int BMT>
static size_t f32t_smem() { return (size_t)TSTAGES * tile_stage_floats<BMT>() * sizeof(float); }

cudaError_t gemm_f32t_configure() {
    cudaError_t e = cudaFuncSetAttribute((const void*)gemm_f32t_kernel<128>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)f32t_smem<128>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void*)gemm_f32t_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)f32t_smem<64>());
}

cudaError_t gemm_f32t_group(const GemmF32TGroup& g, cudaStream_t s) {
    const int bm = g.tile_m == 64 ? 64 : 128;
    int mt = 0, nt = 0;
    for (int i = 0; i < g.count; ++i) {
        mt = max(mt, (g.a[i].M + bm - 1) / bm);
        nt = max(nt, (g.a[i].Nc + BN - 1) / BN);
    }
    if (g.count <= 0 || mt == 0 || nt == 0) return cudaSuccess;
    if (bm == 64)
        gemm_f32t_kernel<64><<<dim3(nt, mt, g.count), kThreads, f32t_smem<64>(), s>>>(g);
    else
        gemm_f32t_kernel<128><<<dim3(nt, mt, g.count), kThreads, f32t_smem<128>(), s>>>(g);
    return cudaGetLastError();
}

cudaError_t gemm_f32_group(const GemmF32Group& g, cudaStream_t s) {
    int mt = 0, nt = 0;
    for (int i = 0; i < g.count; ++i) {
        mt = max(mt, (g.a[i].M + BM - 1) / BM);
        nt = max(nt, (g.a[i].Nc + BN - 1) / BN);
    }
    if (g.count <= 0 || mt == 0 || nt == 0) return cudaSuccess;
    gemm_f32_kernel<<<dim3(nt, mt, g.count), kThreads, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t gemm_f32(const GemmF32Args& a, cudaStream_t s) {
    GemmF32Group g{};
    g.a[0] = a;
    g.count = 1;
    return gemm_f32_group(g, s);
}

}  // namespace fpfp
