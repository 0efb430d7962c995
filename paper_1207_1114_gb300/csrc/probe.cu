// probe.cu -- bandwidth of the memory levels that hold the slacked matrix Y
// during the projection rounds, and throughput of the gradient's product
// kernels, measured on the device the solver runs on.
//
// The P1/P2 rounds read and write every entry of Y once per round.  When a
// wave's matrices fit in shared memory they never leave it, so the level
// that bounds a round's traffic is shared memory; a single large pair
// streams its band through L2.  These probes run the same access pattern
// with no arithmetic besides one add per float: every thread reads a float4
// and writes it back, row after row, for a number of sweeps.
#include "common.cuh"
#include "internal.h"

namespace fpfp {
namespace {

constexpr int kProbeThreads = 512;

// Shared memory: each CTA sweeps `floats` floats of its own shared memory.
__global__ void __launch_bounds__(kProbeThreads, 1) smem_probe_kernel(int floats, int sweeps, float* sink) {
    extern __shared__ __align__(16) float4 buf[];
    const int q = floats >> 2;
    for (int i = threadIdx.x; i < q; i += blockDim.x) buf[i] = make_float4(0.f, 1.f, 2.f, 3.f);
    __syncthreads();
    for (int s = 0; s < sweeps; ++s) {
        for (int i = threadIdx.x; i < q; i += blockDim.x) {
            float4 v = buf[i];
            v.x += 1.f; v.y += 1.f; v.z += 1.f; v.w += 1.f;
            buf[i] = v;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) sink[blockIdx.x] = buf[0].x + buf[q - 1].w;
}

// Tensor memory used as plain storage, as the wave kernel holds band rows:
// every CTA (one per SM) allocates all 512 TMEM columns, and each warp
// sweeps its 32-lane quarter of one 128-column block with 16-column
// tcgen05.ld / tcgen05.st accesses (64 bytes per thread per access, the
// wave kernel's x16 form), adding one to every word.
__global__ void __launch_bounds__(kProbeThreads, 1) tmem_probe_kernel(int sweeps, float* sink) {
    __shared__ uint32_t s_tmem;
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (unsigned)__cvta_generic_to_shared(&s_tmem)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t t = s_tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(128 * (warp >> 2));
    float acc = 0.f;
    for (int s = 0; s < sweeps; ++s) {
        for (int c = 0; c < 128; c += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(t + c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + 1.0f);
            asm volatile(
                "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                ::"r"(t + c), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                  "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                : "memory");
            acc += __uint_as_float(r[0]);
        }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem), "r"(512) : "memory");
    if ((threadIdx.x & 31) == 0) sink[blockIdx.x * (kProbeThreads / 32) + warp] = acc;
}

// Global memory: the grid sweeps `bytes` of one buffer (L2-resident when it
// is small enough), each sweep a read-modify-write of every float4.
__global__ void __launch_bounds__(kProbeThreads) gmem_probe_kernel(float4* buf, size_t q, int sweeps) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int s = 0; s < sweeps; ++s) {
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < q; i += stride) {
            float4 v = __ldcg(buf + i);
            v.x += 1.f; v.y += 1.f; v.z += 1.f; v.w += 1.f;
            __stcg(buf + i, v);
        }
        __threadfence();
    }
}

// Pseudo-random values in [-1, 1) (a 32-bit integer hash of the index), so
// the timed products see data-dependent switching like real operands.
__global__ void fill_kernel(float* p, size_t n, unsigned seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        unsigned h = (unsigned)i * 0x9E3779B1u ^ seed;
        h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
        p[i] = (float)(h >> 8) * (2.0f / 16777216.0f) - 1.0f;
    }
}

}  // namespace

cudaError_t probe_gemm(int precision, int n, int reps, cudaStream_t s, float* best_ms) {
    const size_t nn = (size_t)n * n;
    float *a = nullptr, *b = nullptr, *c = nullptr;
    void *a16 = nullptr, *b16 = nullptr;
    float *sa = nullptr, *sb = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaSuccess;
    auto check = [&](cudaError_t r) { if (e == cudaSuccess) e = r; return e == cudaSuccess; };
    check(cudaMalloc(&a, nn * 4));
    check(cudaMalloc(&b, nn * 4));
    check(cudaMalloc(&c, nn * 4));
    check(cudaMalloc(&a16, nn * 2));
    check(cudaMalloc(&b16, nn * 2));
    check(cudaMalloc(&sa, (size_t)n * 4));
    check(cudaMalloc(&sb, (size_t)n * 4));
    check(cudaEventCreate(&e0));
    check(cudaEventCreate(&e1));
    if (e == cudaSuccess) {
        fill_kernel<<<1024, 256, 0, s>>>(a, nn, 1u);
        fill_kernel<<<1024, 256, 0, s>>>(b, nn, 2u);
        check(cudaGetLastError());
    }
    // one product C = A B^T (TN, both K-major) of the precision under test
    TcGroup g{};
    GemmF32TGroup f{};
    float *alo = nullptr, *blo = nullptr;
    if (e == cudaSuccess && precision == FASTPFP_FP32_SIMT) {
        f.count = 1;
        f.a[0] = GemmF32TArgs{a, n, b, n, c, n, nullptr, 0, 0.f, n, n, n, nullptr};
    } else if (e == cudaSuccess && precision == FASTPFP_FP32) {
        // split TF32: a and b become their TF32 parts, alo / blo the remainders
        check(cudaMalloc(&alo, nn * 4));
        check(cudaMalloc(&blo, nn * 4));
        if (e == cudaSuccess) {
            SplitGroup sg{};
            sg.count = 2;
            sg.q[0] = SplitRows{a, n, n, n, a, alo, n, 0, nullptr};
            sg.q[1] = SplitRows{b, n, n, n, b, blo, n, 0, nullptr};
            check(split_tf32_group(sg, s));
        }
        g.count = 1;
        g.mode = kTcOutF32;
        g.bn = kTcSplitBN;
        g.kind = kTcTf32x3;
        if (e == cudaSuccess &&
            (!tc_make_map(&g.map_a[0], a, n, n, n, kTcTileM, kTcTf32x3) ||
             !tc_make_map(&g.map_a_lo[0], alo, n, n, n, kTcTileM, kTcTf32x3) ||
             !tc_make_map(&g.map_b[0], b, n, n, n, kTcSplitBN, kTcTf32x3) ||
             !tc_make_map(&g.map_b_lo[0], blo, n, n, n, kTcSplitBN, kTcTf32x3)))
            e = cudaErrorInvalidValue;
        g.prob[0] = TcProblem{n, n, n, c, n, nullptr, 0, 0.f, nullptr, nullptr};
    } else if (e == cudaSuccess) {
        const bool fp8 = precision == FASTPFP_FP8;
        if (fp8) {
            QuantGroup q{};
            q.count = 2;
            q.q[0] = QuantRows{a, 0, n, n, n, (uint8_t*)a16, n, sa, nullptr};
            q.q[1] = QuantRows{b, 0, n, n, n, (uint8_t*)b16, n, sb, nullptr};
            check(quant_fp8_group(q, s));
        } else {
            check(to_bf16(a, n, n, n, (__nv_bfloat16*)a16, n, s));
            check(to_bf16(b, n, n, n, (__nv_bfloat16*)b16, n, s));
        }
        g.count = 1;
        g.mode = kTcOutF32;
        g.bn = 256;
        g.kind = fp8 ? kTcE4m3 : kTcBf16;
        if (!tc_make_map(&g.map_a[0], a16, n, n, n, kTcTileM, g.kind) ||
            !tc_make_map(&g.map_b[0], b16, n, n, n, 256, g.kind))
            e = cudaErrorInvalidValue;
        g.prob[0] = TcProblem{n, n, n, c, n, nullptr, 0, 0.f, nullptr, nullptr, fp8 ? sa : nullptr,
                              fp8 ? sb : nullptr};
    }
    auto launch = [&]() { return precision == FASTPFP_FP32_SIMT ? gemm_f32t_group(f, s) : tc_gemm(g, s); };
    if (e == cudaSuccess) check(launch());   // warm-up
    *best_ms = 0.f;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        check(cudaEventRecord(e0, s));
        check(launch());
        check(cudaEventRecord(e1, s));
        check(cudaEventSynchronize(e1));
        float ms = 0.f;
        check(cudaEventElapsedTime(&ms, e0, e1));
        if (r == 0 || ms < *best_ms) *best_ms = ms;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(a); cudaFree(b); cudaFree(c); cudaFree(a16); cudaFree(b16); cudaFree(sa); cudaFree(sb);
    if (alo) cudaFree(alo);
    if (blo) cudaFree(blo);
    return e;
}

cudaError_t probe_smem(int num_sms, int sweeps, cudaStream_t s, float* ms, double* bytes) {
    const int floats = (int)((kPdMaxSmem - 1024) / sizeof(float)) & ~3;
    cudaError_t e = cudaFuncSetAttribute((const void*)smem_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kPdMaxSmem);
    if (e != cudaSuccess) return e;
    float* sink = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(float) * num_sms)) != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    smem_probe_kernel<<<num_sms, kProbeThreads, (size_t)floats * 4, s>>>(floats, 1, sink);   // warm
    cudaEventRecord(a, s);
    smem_probe_kernel<<<num_sms, kProbeThreads, (size_t)floats * 4, s>>>(floats, sweeps, sink);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) {
        cudaEventElapsedTime(ms, a, b);
        *bytes = 8.0 * (double)floats * (double)num_sms * (double)sweeps;   // read + write
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return e;
}

cudaError_t probe_tmem(int num_sms, int sweeps, cudaStream_t s, float* ms, double* bytes) {
    // more than half an SM's shared memory per CTA: one CTA (one 512-column
    // TMEM allocation) per SM
    const int one_per_sm = 120 * 1024;
    cudaError_t e = cudaFuncSetAttribute((const void*)tmem_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         one_per_sm);
    if (e != cudaSuccess) return e;
    float* sink = nullptr;
    if ((e = cudaMalloc(&sink, sizeof(float) * num_sms * (kProbeThreads / 32))) != cudaSuccess) return e;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    tmem_probe_kernel<<<num_sms, kProbeThreads, one_per_sm, s>>>(1, sink);   // warm
    cudaEventRecord(a, s);
    tmem_probe_kernel<<<num_sms, kProbeThreads, one_per_sm, s>>>(sweeps, sink);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) {
        cudaEventElapsedTime(ms, a, b);
        // 128 lanes x 512 columns x 4 bytes per SM, read and written per sweep
        *bytes = 2.0 * 128.0 * 512.0 * 4.0 * (double)num_sms * (double)sweeps;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return e;
}

cudaError_t probe_gmem(size_t buf_bytes, int num_sms, int sweeps, cudaStream_t s, float* ms, double* bytes) {
    float4* buf = nullptr;
    cudaError_t e = cudaMalloc(&buf, buf_bytes);
    if (e != cudaSuccess) return e;
    const size_t q = buf_bytes / sizeof(float4);
    cudaMemsetAsync(buf, 0, buf_bytes, s);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int grid = num_sms * 2;
    gmem_probe_kernel<<<grid, kProbeThreads, 0, s>>>(buf, q, 1);   // warm (brings it into L2 when it fits)
    cudaEventRecord(a, s);
    gmem_probe_kernel<<<grid, kProbeThreads, 0, s>>>(buf, q, sweeps);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) {
        cudaEventElapsedTime(ms, a, b);
        *bytes = 2.0 * (double)buf_bytes * (double)sweeps;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    return e;
}

}  // namespace fpfp
