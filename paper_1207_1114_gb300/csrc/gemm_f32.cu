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
        if (ld_relaxed_i32(&g.ctrl->done) != 0 || ld_relaxed_i32(&g.ctrl->error) != 0) return;
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

}  // namespace

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
