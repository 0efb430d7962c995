// fastga.cu -- FastGA: graduated assignment with C = A (x) A' (Appendix,
// Eqs. GAO3/GAO4), the comparison method of Section 5, run with a fixed
// beta (the paper gives no schedule).
//
// One outer iteration is the gradient products (the same launches FastPFP
// uses, Y[:, :m] = A X A' + lambda K) followed by one cooperative launch of
// ga_kernel over the pair's N x N slacked matrix (slack columns Q = 0),
// with beta acting on Q scaled by its largest magnitude s (one beta for
// pairs whose products differ in scale; the paper gives no beta):
//
//   Y(0)   = max(exp(beta (Q/s - rowmax Q/s)), 2^-100)
//   repeat: Z = R(Y) rows to unit sums, Y' = C(Z) columns to unit sums (each
//           floored at 2^-100), until max|Y' - Y| < eps_2 or I_1 steps
//   X      = Y[:, :m], max|dX| for the outer stop (eps_1, I_0).
//
// A CTA owns a contiguous block of rows; Y and Z stay in global memory (an
// N x N FP32 matrix of N <= 4096 is L2-resident).  Row sums are warp sums in
// a fixed order.  Column sums are two-stage, in a fixed order: every CTA
// stores the partial of its rows per column, then (after a grid barrier)
// CTA c adds up all CTAs' partials of its block of columns, so every run
// gives the same bits (and a column whose entries all sit at the floor still
// sums to a positive number).  Three grid barriers per normalisation step:
// after the partials, after the sums, after the step's max|dY|; one more per
// launch for s.
#include "common.cuh"
#include "internal.h"

namespace fpfp {
namespace {

constexpr float kGaFloor = 0x1p-100f;   // positivity floor of the normalised iterates

__device__ __forceinline__ float block_max(float v, float* red) {
    v = warp_max(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    float t = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    return t;
}
__device__ __forceinline__ double block_max_dbl(double v, double* red) {
    v = warp_max_d(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    return t;
}

__global__ void __launch_bounds__(kGaThreads, 1) ga_kernel(const GaParams P) {
    extern __shared__ __align__(16) float cN[];   // ldy floats: this step's column sums
    __shared__ float s_red[32];
    __shared__ double s_dred[32];
    Ctrl* C = P.ctrl;
    if (ld_relaxed_i32(&C->done) != 0 || ld_relaxed_i32(&C->error) != 0) return;
    const int N = P.N, m = P.m, ldy = P.ldy, ldx = P.ldx;
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const unsigned G = gridDim.x;
    const int r0 = blockIdx.x * P.rpc, r1 = min(N, r0 + P.rpc);
    const unsigned bar_base = C->bar_base;
    unsigned gen = 0;
    int* err = &C->error;
    float* Y = P.Y;
    float* Z = P.Z;
    float* part = P.part;   // G x ldy: the CTAs' column partials of the running step
    float* csum = P.csum;   // ldy: the step's column sums
    unsigned* dmax = P.dbuf;           // [0], [1]: the step's max|dY| (float bits), by parity;
                                       // [2]: max|Q| of the launch (float bits)

    // ---- s = max|Q| over the pair (slack columns hold Q = 0)
    float qa = 0.f;
    for (int i = r0 + warp; i < r1; i += nwarp) {
        const float* y = Y + (size_t)i * ldy;
        for (int j = lane; j < m; j += 32) qa = fmaxf(qa, fabsf(y[j]));
    }
    qa = block_max(qa, s_red);
    if (tid == 0 && r1 > r0 && qa > 0.f) atomicMax(dmax + 2, __float_as_uint(qa));
    if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, P.timeout_ns)) return;
    ++gen;
    float sq = __uint_as_float(__ldcg(dmax + 2));
    if (!isfinite(sq)) {
        if (blockIdx.x == 0 && tid == 0) atomicCAS(err, 0, FASTPFP_ERR_NONFINITE);
        return;
    }
    if (!(sq > 0.f)) sq = 1.f;

    // ---- Y(0): exp of beta Q/s shifted by the row maximum (slack columns
    // hold Q = 0 whatever Y stores there), floored; padding columns 0
    for (int i = r0 + warp; i < r1; i += nwarp) {
        float* y = Y + (size_t)i * ldy;
        float mx = m < N ? 0.f : -INFINITY;
        for (int j = lane; j < m; j += 32) mx = fmaxf(mx, y[j] / sq);
        mx = warp_max(mx);
        for (int j = lane; j < ldy; j += 32) {
            const float q = j < m ? y[j] / sq : 0.f;
            y[j] = j < N ? fmaxf(expf(P.beta * (q - mx)), kGaFloor) : 0.f;
        }
    }

    // ---- the normalisation loop
    const int cb = (N + (int)G - 1) / (int)G;   // columns summed by each CTA
    const int c0 = (int)blockIdx.x * cb, c1 = min(N, c0 + cb);
    int k = 0;
    while (true) {
        const int par = k & 1;
        // rows to unit sums (Y -> Z)
        for (int i = r0 + warp; i < r1; i += nwarp) {
            const float* y = Y + (size_t)i * ldy;
            float* z = Z + (size_t)i * ldy;
            float s = 0.f;
            for (int j = lane; j < N; j += 32) s += y[j];
            s = warp_sum(s);
            for (int j = lane; j < N; j += 32) z[j] = fmaxf(y[j] / s, kGaFloor);
        }
        __syncthreads();   // the block's Z rows are in before its column pass reads them
        // the block's column partials, its rows in order
        for (int j = tid; j < N; j += nthr) {
            float c = 0.f;
            for (int i = r0; i < r1; ++i) c += Z[(size_t)i * ldy + j];
            part[(size_t)blockIdx.x * ldy + j] = c;
        }
        if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, P.timeout_ns)) return;
        ++gen;
        // this CTA's block of column sums, the CTAs' partials in order
        for (int j = c0 + tid; j < c1; j += nthr) {
            float c = 0.f;
            for (unsigned g = 0; g < G; ++g) c += __ldcg(part + (size_t)g * ldy + j);
            csum[j] = c;
        }
        // step k - 1's maximum (the other parity) was read by every CTA before
        // it arrived at this step's first barrier; step k + 1 raises it after
        // this step's third barrier, which this zero precedes
        if (blockIdx.x == 0 && tid == 0) dmax[par ^ 1] = 0u;
        if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, P.timeout_ns)) return;
        ++gen;
        for (int j = tid; j < N; j += nthr) cN[j] = __ldcg(csum + j);
        __syncthreads();
        // columns to unit sums (Z -> Y) and the step's max|dY|
        float dm = 0.f;
        for (int i = r0 + warp; i < r1; i += nwarp) {
            const float* z = Z + (size_t)i * ldy;
            float* y = Y + (size_t)i * ldy;
            for (int j = lane; j < N; j += 32) {
                const float v = fmaxf(z[j] / cN[j], kGaFloor);
                dm = fmaxf(dm, fabsf(v - y[j]));
                y[j] = v;
            }
        }
        dm = block_max(dm, s_red);
        if (tid == 0 && r1 > r0) atomicMax(dmax + par, __float_as_uint(dm));
        if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, P.timeout_ns)) return;
        ++gen;
        const float d = __uint_as_float(__ldcg(dmax + par));
        ++k;
        if (!isfinite(d)) {
            if (blockIdx.x == 0 && tid == 0) atomicCAS(err, 0, FASTPFP_ERR_NONFINITE);
            return;
        }
        if ((double)d < P.tol_inner || k >= P.max_inner) break;
    }

    // ---- X(t+1) = Y[:, :m] and max|dX| (FP64, like FastPFP's)
    AbsDiffMax dxm;
    for (int i = r0 + warp; i < r1; i += nwarp) {
        const float* y = Y + (size_t)i * ldy;
        float* x = P.X + (size_t)i * ldx;
        for (int j = lane; j < ldx; j += 32) {
            const float v = j < m ? y[j] : 0.f;
            dxm.add(v, x[j]);
            x[j] = v;
        }
    }
    const double dx = block_max_dbl(dxm.value(), s_dred);
    if (tid == 0 && r1 > r0) atomicMax(&C->dx_bits, (unsigned long long)__double_as_longlong(dx));
    if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, P.timeout_ns)) return;
    ++gen;

    // ---- no CTA reads the maxima any more: zero them for the next launch;
    // loop control of Algorithm 1's repeat loop (CTA 0)
    if (blockIdx.x == 0 && tid == 0) {
        dmax[0] = 0u;
        dmax[1] = 0u;
        dmax[2] = 0u;
        const double d = __longlong_as_double((long long)__ldcg(&C->dx_bits));
        if (!isfinite(d)) atomicCAS(err, 0, FASTPFP_ERR_NONFINITE);
        C->dx_bits = 0ull;
        const int t = C->outer;
        if (t < kMaxOuterTrace) {
            C->inner_trace[t] = k;
            C->delta_trace[t] = d;
        }
        C->outer = t + 1;
        C->inner_total += k;
        C->inner_max = max(C->inner_max, k);
        C->last_inner = k;
        C->last_delta = d;
        if (d < P.tol_outer) {
            C->converged = 1;
            C->done = 1;
        }
        if (t + 1 >= P.max_outer) C->done = 1;
        C->bar_base = bar_base + G * gen;
    }
}

}  // namespace

int ga_rows_per_cta(int N, int num_sms) {
    const int G = N < num_sms ? N : num_sms;
    return (N + G - 1) / (G > 0 ? G : 1);
}

cudaError_t ga_configure() {
    return cudaFuncSetAttribute((const void*)ga_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(kPdbMaxN * sizeof(float)));
}

cudaError_t ga_launch(const GaParams& P, cudaStream_t s) {
    if (P.N < 1 || P.rpc < 1 || P.ldy < P.N || P.ldy > kPdbMaxN) return cudaErrorInvalidValue;
    const int grid = (P.N + P.rpc - 1) / P.rpc;
    void* args[] = {const_cast<GaParams*>(&P)};
    return cudaLaunchCooperativeKernel((const void*)ga_kernel, dim3(grid), dim3(kGaThreads), args,
                                       (size_t)P.ldy * sizeof(float), s);
}

}  // namespace fpfp
