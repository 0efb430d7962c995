// common.cuh -- device helpers shared by the FastPFP kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/fastpfp.h"
#include "exact.cuh"

namespace fpfp {

constexpr int kMaxOuterTrace = 4096;  // per-solve trace capacity (outer iterations)
constexpr int kObjBlocks = 256;       // blocks of the objective kernel

// Device control block of one solve.  Zeroed (except the fields the host
// sets) before the first outer iteration.
struct Ctrl {
    int done;              // 1 once the outer loop has stopped
    int outer;             // outer iterations completed
    int error;             // FASTPFP_ERR_* raised on the device, 0 if none
    int converged;         // 1 if max|dX| < tol_outer was reached
    int inner_total;       // sum of P1/P2 rounds
    int inner_max;         // largest round count of one outer iteration
    int lowp;              // 1 while the BF16 phase runs
    int lowp_iters;        // outer iterations run in BF16
    int refine_left;       // FP32 iterations left after the BF16 phase
    int last_inner;        // rounds of the latest P_D call
    double last_delta;     // latest max|dX| (outer) or max|dY| (P_D only)
    double objective;      // Eq. (3) at the discrete result
    unsigned long long dx_bits;  // max|dX| of the running outer iteration (double bits)
    unsigned xmax_bits;    // max(X) of the running outer iteration (ordered float bits)
    unsigned bar;          // grid-barrier arrival counter (grows within a solve)
    unsigned bar_base;     // counter value at the start of the next cooperative launch
    int matched;           // discretisation: columns matched so far
    unsigned obj_ticket;   // objective: blocks that have stored their partial sum
    int idle;              // 1 while a streamed batch keeps this pair out of the running wave:
                           // its product and projection launches skip it
    int wave_pairs;        // largest wave the pair ran in (device-planned waves)
    int inner_trace[kMaxOuterTrace];
    double delta_trace[kMaxOuterTrace];
    double obj_part[kObjBlocks];   // objective: one partial sum per block, folded in block order
};

// ---------------------------------------------------------------- ordering
// Order-preserving map of a float onto uint32 (larger float -> larger uint).
__device__ __forceinline__ unsigned float_to_ordered(float f) {
    unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(unsigned u) {
    unsigned b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
    return __uint_as_float(b);
}

// --------------------------------------------------------------- reductions
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// ------------------------------------------------------------ memory model
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Vector reduction-add of four floats into global memory (sm_90+).
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a),
                 "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// Reduction-add of one double into global memory.
__device__ __forceinline__ void red_add_f64(double* p, double v) {
    asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

// ------------------------------------------------------- order-free sums
// The column sums and totals of the projection rounds are added across CTAs
// by atomics, in an order that changes from run to run.  They are made exact
// -- and so independent of that order -- by rounding every contribution to a
// multiple of a power-of-two quantum q chosen from a bound that every CTA
// computes identically before it adds: if every partial sum stays below
// 2^24 q (FP32) or 2^53 q (FP64), every addition is exact.  The rounding
// error of one contribution is at most q/2, about one unit in the last place
// of the bound.
//
// FP32: scales of the quantum for a bound b >= 1 (finite): with
// E = floor(log2 b), b < 2^(E+1) = 2^24 q for q = 2^(E-23); dn = 1/q, up = q.
struct Quant32 {
    float dn, up;
};
__device__ __forceinline__ Quant32 quant32_for(float bound) {
    int E = ((__float_as_int(bound) >> 23) & 0xff) - 127;
    E = E < 0 ? 0 : (E > 100 ? 100 : E);
    return Quant32{__int_as_float((127 + 23 - E) << 23), __int_as_float((127 - 23 + E) << 23)};
}
__device__ __forceinline__ float quant32(float v, Quant32 q) { return rintf(v * q.dn) * q.up; }
__device__ __forceinline__ float4 quant32x4(float4 v, Quant32 a, Quant32 b, Quant32 c, Quant32 d) {
    return make_float4(quant32(v.x, a), quant32(v.y, b), quant32(v.z, c), quant32(v.w, d));
}
// Margin on every bound: covers the FP32 rounding of the bound itself and of
// the updates it bounds.
constexpr float kBoundMargin = 1.0f + 1.0f / 1024.0f;

// FP64: Quant64 and its helpers (exact.cuh), shared with host builds.

// Asynchronous 16-byte global -> shared copy through L2 only (the source is
// written by other CTAs' reductions, so L1 must not hold a stale copy), and
// the wait for all of this thread's copies.  Both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async_cg16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Grid-wide barrier for a cooperative launch.  `counter` only ever grows
// within a solve: every CTA adds 1 per barrier, and a barrier is passed once
// the counter reaches `target` (the value after all CTAs of the grid have
// arrived).  The arrive is a release and the wait an acquire, so writes made
// by any thread of a CTA before the barrier are visible to every thread of
// every CTA after it.  The wait is bounded: after `timeout_ns` (or as soon as
// another CTA has raised an error) it records FASTPFP_ERR_TIMEOUT in *err and
// returns false; every caller then leaves the kernel.  Must be reached by all
// threads of the CTA.  `arrive` = false (fault-injection tests only) waits
// without arriving, so the barrier can never complete and every wait runs out.
__device__ __forceinline__ bool grid_barrier(unsigned* counter, unsigned target, int* err,
                                             long long timeout_ns, bool arrive = true) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (arrive) red_release_add_u32(counter, 1u);
        uint64_t t0 = 0;
        unsigned spins = 0;
        while (ld_acquire_u32(counter) < target) {
            if ((++spins & 255u) == 0u) {
                const uint64_t now = globaltimer_ns();
                if (t0 == 0) t0 = now;
                if (ld_relaxed_i32(err) != 0 || (long long)(now - t0) > timeout_ns ||
                    spins > (1u << 30)) {
                    atomicCAS(err, 0, FASTPFP_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Split-phase form of grid_barrier: grid_arrive publishes the CTA's prior
// writes and counts it in; grid_wait (later, after unrelated work) waits until
// the counter reaches `target`.  Same bounds and error handling as above.
__device__ __forceinline__ void grid_arrive(unsigned* counter) {
    __syncthreads();
    if (threadIdx.x == 0) red_release_add_u32(counter, 1u);
}
__device__ __forceinline__ bool grid_wait(unsigned* counter, unsigned target, int* err,
                                          long long timeout_ns) {
    __shared__ int s_ok_w;
    if (threadIdx.x == 0) {
        int ok = 1;
        uint64_t t0 = 0;
        unsigned spins = 0;
        while (ld_acquire_u32(counter) < target) {
            if ((++spins & 255u) == 0u) {
                const uint64_t now = globaltimer_ns();
                if (t0 == 0) t0 = now;
                if (ld_relaxed_i32(err) != 0 || (long long)(now - t0) > timeout_ns ||
                    spins > (1u << 30)) {
                    atomicCAS(err, 0, FASTPFP_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        s_ok_w = ok;
    }
    __syncthreads();
    return s_ok_w != 0;
}

}  // namespace fpfp
