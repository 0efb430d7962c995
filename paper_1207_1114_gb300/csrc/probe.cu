// probe.cu -- bandwidth of the memory levels that hold the slacked matrix Y
// during the projection rounds, measured on the device the solver runs on.
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

}  // namespace

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
