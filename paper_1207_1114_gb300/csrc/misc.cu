// misc.cu -- small kernels around the solve: control-block set-up, the
// attribute affinity K = B B'^T (below Eq. 4), the initial X (after
// Algorithm 1), BF16 and E4M3 operand copies, caller-orientation outputs and
// the objective of Eq. (3) at the discrete result.
#include "common.cuh"
#include "internal.h"

namespace fpfp {
namespace {

__global__ void init_ctrl_kernel(Ctrl* c, int lowp) {
    c->lowp = lowp;
    c->refine_left = 0;
}

// K[i, j] = sum_c B[i, c] B2[j, c]; one thread per entry, attributes of the
// block's rows staged in shared memory.
__global__ void affinity_kernel(const float* __restrict__ B, const float* __restrict__ B2, int N,
                                int m, int k, float* __restrict__ K, int ldk) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    extern __shared__ float brow[];
    for (int c = threadIdx.x; c < k; c += blockDim.x) brow[c] = B[(size_t)i * k + c];
    __syncthreads();
    if (j >= m) return;
    float acc = 0.f;
    for (int c = 0; c < k; ++c) acc = fmaf(brow[c], __ldg(B2 + (size_t)j * k + c), acc);
    K[(size_t)i * ldk + j] = acc;
}

__global__ void init_x_kernel(float* X, int N, int m, int ldx, const float* X0, int transposed,
                              __nv_bfloat16* Xt16, int ldxt) {
    const size_t total = (size_t)N * ldx;
    const float u = (float)(1.0 / ((double)N * (double)m));
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / ldx), j = (int)(e % ldx);
        float v = 0.f;
        if (j < m) {
            if (X0) v = transposed ? X0[(size_t)j * N + i] : X0[(size_t)i * m + j];
            else v = u;
        }
        X[e] = v;
        if (Xt16 && j < m) Xt16[(size_t)j * ldxt + i] = __float2bfloat16_rn(v);
    }
}

__global__ void to_bf16_kernel(const float* src, int r, int c, int lds, __nv_bfloat16* dst,
                               int ldd) {
    const size_t total = (size_t)r * ldd;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / ldd), j = (int)(e % ldd);
        dst[e] = __float2bfloat16_rn(j < c ? src[(size_t)i * lds + j] : 0.f);
    }
}

// Two floats to two E4M3 bytes (round to nearest even, saturating at
// +-448): the lower byte holds lo.
__device__ __forceinline__ unsigned short e4m3x2(float lo, float hi) {
    unsigned short r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
    return r;
}

// One warp per row of one matrix of the group (blockIdx.y): the row's
// largest magnitude, its power-of-two scale, then the E4M3 bytes, four per
// lane and store.
__global__ void __launch_bounds__(256) quant_fp8_kernel(const __grid_constant__ QuantGroup G) {
    if ((int)blockIdx.y >= G.count) return;
    const QuantRows& q = G.q[blockIdx.y];
    const int row = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (row >= q.rows) return;
    if (q.ctrl) {
        if (ld_relaxed_i32(&q.ctrl->done) != 0 || ld_relaxed_i32(&q.ctrl->error) != 0 ||
            ld_relaxed_i32(&q.ctrl->idle) != 0)
            return;
        if (ld_relaxed_i32(&q.ctrl->lowp) == 0) return;
    }
    const float* f = q.src_bf16 ? nullptr : reinterpret_cast<const float*>(q.src) + (size_t)row * q.lds;
    const __nv_bfloat16* h = q.src_bf16 ? reinterpret_cast<const __nv_bfloat16*>(q.src) + (size_t)row * q.lds
                                        : nullptr;
    auto at = [&](int c) { return c < q.cols ? (h ? __bfloat162float(h[c]) : f[c]) : 0.f; };
    float mx = 0.f;
    for (int c = lane; c < q.cols; c += 32) mx = fmaxf(mx, fabsf(at(c)));
    mx = warp_max(mx);
    // the largest e with mx * 2^e <= 448 = 0.875 * 2^9 (mx = fr * 2^ex, fr in [0.5, 1))
    int e = 0;
    if (mx > 0.f && isfinite(mx)) {
        int ex;
        const float fr = frexpf(mx, &ex);
        e = (fr <= 0.875f ? 9 : 8) - ex;
        e = max(-126, min(126, e));
    }
    const float up = ldexpf(1.f, e);
    if (lane == 0) q.scale[row] = ldexpf(1.f, -e);
    uint8_t* d = q.dst + (size_t)row * q.ldd;
    for (int c = 4 * lane; c < q.cols; c += 128) {
        const unsigned lo = e4m3x2(at(c) * up, at(c + 1) * up);
        const unsigned hi = e4m3x2(at(c + 2) * up, at(c + 3) * up);
        if (c + 3 < q.cols) {
            *reinterpret_cast<unsigned*>(d + c) = lo | (hi << 16);
        } else {
            const unsigned w = lo | (hi << 16);
            for (int t = 0; c + t < q.cols; ++t) d[c + t] = (uint8_t)(w >> (8 * t));
        }
    }
}

// dst (c x ldd, BF16) = src^T for an r x c FP32 src (leading dimension lds).
__global__ void transpose_bf16_kernel(const float* src, int r, int c, int lds, __nv_bfloat16* dst, int ldd) {
    __shared__ float tile[32][33];
    const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int i = bi + y, j = bj + threadIdx.x;
        tile[y][threadIdx.x] = (i < r && j < c) ? src[(size_t)i * lds + j] : 0.f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int j = bj + y, i = bi + threadIdx.x;
        if (j < c && i < r) dst[(size_t)j * ldd + i] = __float2bfloat16_rn(tile[threadIdx.x][y]);
    }
}

// The FP32 products' operands on the tensor cores: every value split into
// its TF32 part (rounded to 10 mantissa bits, low 13 bits zero) and the FP32
// remainder.  One 32 x 32 tile of one matrix of the group (blockIdx.z) per
// block, through shared memory when the matrix is transposed; pad columns
// of the destination are written as zero.  A matrix with ctrl set is split
// only while its solve runs its FP32 phase.
__device__ __forceinline__ void split_tf32(float x, float* hi, float* lo) {
    const float h = __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
    *hi = h;
    *lo = x - h;
}
__global__ void split_tf32_kernel(const __grid_constant__ SplitGroup G) {
    if ((int)blockIdx.z >= G.count) return;
    const SplitRows& q = G.q[blockIdx.z];
    if (q.ctrl) {
        if (ld_relaxed_i32(&q.ctrl->done) != 0 || ld_relaxed_i32(&q.ctrl->error) != 0 ||
            ld_relaxed_i32(&q.ctrl->idle) != 0 || ld_relaxed_i32(&q.ctrl->lowp) != 0)
            return;
    }
    // destination extent: rows x ldd (pad columns zero)
    const int drows = q.transpose ? q.cols : q.rows, dcols = q.transpose ? q.rows : q.cols;
    const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
    if (bi >= drows || bj >= q.ldd) return;
    __shared__ float tile[32][33];
    if (q.transpose) {
        for (int y = threadIdx.y; y < 32; y += blockDim.y) {
            const int i = bj + y, j = bi + threadIdx.x;   // source row bj + y, column bi + x
            tile[y][threadIdx.x] = (i < q.rows && j < q.cols) ? q.src[(size_t)i * q.lds + j] : 0.f;
        }
        __syncthreads();
    }
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int i = bi + y, j = bj + threadIdx.x;
        if (i >= drows || j >= q.ldd) continue;
        float x = 0.f;
        if (j < dcols) x = q.transpose ? tile[threadIdx.x][y] : q.src[(size_t)i * q.lds + j];
        split_tf32(x, q.hi + (size_t)i * q.ldd + j, q.lo + (size_t)i * q.ldd + j);
    }
}

__global__ void perm_fill_kernel(int32_t* perm, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[i] = -1;
}

__global__ void perm_scatter_kernel(const int32_t* row_of_col, int m, int transposed,
                                    int32_t* perm) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int r = row_of_col[j];
    if (transposed) perm[j] = r;          // graph 1 indexes the columns
    else if (r >= 0) perm[r] = j;         // graph 1 indexes the rows
}

// X_out (caller orientation) from the canonical N x m X.
__global__ void x_out_kernel(const float* X, int N, int m, int ldx, int transposed, float* out) {
    __shared__ float tile[32][33];
    const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = bi + r, j = bj + threadIdx.x;
        if (i < N && j < m) {
            const float v = X[(size_t)i * ldx + j];
            if (!transposed) out[(size_t)i * m + j] = v;
            else tile[r][threadIdx.x] = v;
        }
    }
    if (!transposed) return;
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int j = bj + r, i = bi + threadIdx.x;   // out is m x N
        if (i < N && j < m) out[(size_t)j * N + i] = tile[threadIdx.x][r];
    }
}

// 1/2 sum_{j,l} A[r(j), r(l)] A2[l, j] + lambda sum_j K[r(j), j], in FP64.
// Every block stores its partial sum; the last block to finish adds them in
// block order, so the result does not depend on the blocks' timing.
__global__ void objective_kernel(const float* A, int N, const float* A2, int m, const float* K,
                                 int ldk, float lambda, const int32_t* row_of_col, Ctrl* ctrl) {
    double acc = 0.0;
    const size_t total = (size_t)m * m;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total;
         e += (size_t)gridDim.x * blockDim.x) {
        const int l = (int)(e / m), j = (int)(e % m);
        const int rj = row_of_col[j], rl = row_of_col[l];
        if (rj < 0 || rl < 0) continue;   // an aborted discretisation leaves -1 entries
        acc += 0.5 * (double)A[(size_t)rj * N + rl] * (double)A2[(size_t)l * m + j];
    }
    if (K && lambda != 0.f) {
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x)
            if (row_of_col[j] >= 0) acc += (double)lambda * (double)K[(size_t)row_of_col[j] * ldk + j];
    }
    __shared__ double red[32];
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    __shared__ int last;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        ctrl->obj_part[blockIdx.x] = t;
        __threadfence();
        last = atomicAdd(&ctrl->obj_ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(&ctrl->obj_part[b]);
        ctrl->objective = t;
        ctrl->obj_ticket = 0u;
    }
}

// Condition of the outer loop's CUDA-graph while node, run after every outer
// iteration: continue while neither the stop word (words[done_idx]) nor the
// error word (words[err_idx]) is set and fewer than max_iter iterations have
// run.  The iteration count in *iter bounds the loop even if no kernel of the
// body ever sets the stop word.
__global__ void loop_cond_kernel(const int* words, int done_idx, int err_idx, int* iter, int max_iter,
                                 cudaGraphConditionalHandle handle) {
    const int t = *iter + 1;
    *iter = t;
    const volatile int* w = words;
    const bool go = w[done_idx] == 0 && w[err_idx] == 0 && t < max_iter;
    cudaGraphSetConditional(handle, go ? 1u : 0u);
}

// Runs once before the while node: clears the iteration count and opens the
// loop.  The handle's default is 0 (closed), so the body runs only if device
// code set the condition; a condition that never gets set cannot loop.
__global__ void loop_init_kernel(int* iter, cudaGraphConditionalHandle handle) {
    *iter = 0;
    cudaGraphSetConditional(handle, 1u);
}

__global__ void flags_kernel(const FlagList f, int* out) {
    const int i = threadIdx.x;
    if (i < f.n) out[i] = (f.ctrl[i]->done != 0 ? 1 : 0) | (f.ctrl[i]->error != 0 ? 2 : 0);
    if (i == 0) out[kMaxWavePairs] = f.wave->error;
}

inline int grid_for(size_t total, int block, int cap = 4096) {
    size_t g = (total + block - 1) / block;
    if (g < 1) g = 1;
    if (g > (size_t)cap) g = cap;
    return (int)g;
}

}  // namespace

// Segment blockIdx.y of the list, 16 bytes per thread and step (four in
// flight), the last bytes of a size that is not a multiple of 16 in words.
constexpr int kCopyThreads = 256, kCopyBlocksPerSeg = 16;
__global__ void __launch_bounds__(kCopyThreads) gather_copy_kernel(const __grid_constant__ CopyList L) {
    const CopySeg sg = L.seg[blockIdx.y];
    const size_t n16 = sg.bytes / 16;
    const float4* src = reinterpret_cast<const float4*>(sg.src);
    float4* dst = reinterpret_cast<float4*>(sg.dst);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {
        const float4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
        dst[i] = a;
        dst[i + stride] = b;
        dst[i + 2 * stride] = c;
        dst[i + 3 * stride] = d;
    }
    for (; i < n16; i += stride) dst[i] = src[i];
    if (blockIdx.x == 0) {
        const size_t w0 = n16 * 4, nw = sg.bytes / 4;
        const float* s4 = reinterpret_cast<const float*>(sg.src);
        float* d4 = reinterpret_cast<float*>(sg.dst);
        for (size_t w = w0 + threadIdx.x; w < nw; w += blockDim.x) d4[w] = s4[w];
    }
}

cudaError_t gather_copy(const CopyList& L, cudaStream_t s) {
    if (L.count <= 0) return cudaSuccess;
    if (L.count > kMaxCopySegs) return cudaErrorInvalidValue;
    gather_copy_kernel<<<dim3(kCopyBlocksPerSeg, L.count), kCopyThreads, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t init_ctrl(Ctrl* c, int lowp, cudaStream_t s) {
    init_ctrl_kernel<<<1, 1, 0, s>>>(c, lowp);
    return cudaGetLastError();
}

cudaError_t loop_cond(const int* words, int done_idx, int err_idx, int* iter, int max_iter,
                      cudaGraphConditionalHandle handle, cudaStream_t s) {
    loop_cond_kernel<<<1, 1, 0, s>>>(words, done_idx, err_idx, iter, max_iter, handle);
    return cudaGetLastError();
}

cudaError_t loop_init(int* iter, cudaGraphConditionalHandle handle, cudaStream_t s) {
    loop_init_kernel<<<1, 1, 0, s>>>(iter, handle);
    return cudaGetLastError();
}

cudaError_t gather_flags(const FlagList& f, int* out, cudaStream_t s) {
    flags_kernel<<<1, kMaxWavePairs, 0, s>>>(f, out);
    return cudaGetLastError();
}

cudaError_t affinity(const float* B, const float* B2, int N, int m, int k, float* K, int ldk,
                     cudaStream_t s) {
    if (N <= 0 || m <= 0) return cudaSuccess;
    dim3 grid((m + 255) / 256, N);
    affinity_kernel<<<grid, 256, (size_t)k * sizeof(float), s>>>(B, B2, N, m, k, K, ldk);
    return cudaGetLastError();
}

cudaError_t init_x(float* X, int N, int m, int ldx, const float* X0, int transposed,
                   __nv_bfloat16* Xt16, int ldxt, cudaStream_t s) {
    const size_t total = (size_t)N * ldx;
    init_x_kernel<<<grid_for(total, 256), 256, 0, s>>>(X, N, m, ldx, X0, transposed, Xt16, ldxt);
    return cudaGetLastError();
}

cudaError_t to_bf16(const float* src, int r, int c, int lds, __nv_bfloat16* dst, int ldd,
                    cudaStream_t s) {
    const size_t total = (size_t)r * ldd;
    to_bf16_kernel<<<grid_for(total, 256), 256, 0, s>>>(src, r, c, lds, dst, ldd);
    return cudaGetLastError();
}

cudaError_t split_tf32_group(const SplitGroup& g, cudaStream_t s) {
    int rows = 0, cols = 0;
    for (int i = 0; i < g.count; ++i) {
        rows = max(rows, g.q[i].transpose ? g.q[i].cols : g.q[i].rows);
        cols = max(cols, g.q[i].ldd);
    }
    if (g.count <= 0 || rows <= 0 || cols <= 0) return cudaSuccess;
    split_tf32_kernel<<<dim3((cols + 31) / 32, (rows + 31) / 32, g.count), dim3(32, 8), 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t quant_fp8_group(const QuantGroup& g, cudaStream_t s) {
    int rows = 0;
    for (int i = 0; i < g.count; ++i) rows = max(rows, g.q[i].rows);
    if (g.count <= 0 || rows <= 0) return cudaSuccess;
    quant_fp8_kernel<<<dim3((rows + 7) / 8, g.count), 256, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t transpose_to_bf16(const float* src, int r, int c, int lds, __nv_bfloat16* dst, int ldd,
                              cudaStream_t s) {
    dim3 grid((c + 31) / 32, (r + 31) / 32);
    transpose_bf16_kernel<<<grid, dim3(32, 8), 0, s>>>(src, r, c, lds, dst, ldd);
    return cudaGetLastError();
}

cudaError_t write_outputs(const int32_t* row_of_col, int N, int m, int transposed, int32_t* perm_out,
                          const float* X, int ldx, float* X_out, cudaStream_t s) {
    if (perm_out) {
        if (!transposed) perm_fill_kernel<<<(N + 255) / 256, 256, 0, s>>>(perm_out, N);
        perm_scatter_kernel<<<(m + 255) / 256, 256, 0, s>>>(row_of_col, m, transposed, perm_out);
    }
    if (X_out) {
        dim3 grid((m + 31) / 32, (N + 31) / 32);
        x_out_kernel<<<grid, dim3(32, 8), 0, s>>>(X, N, m, ldx, transposed, X_out);
    }
    return cudaGetLastError();
}

cudaError_t objective(const float* A, int N, const float* A2, int m, const float* K, int ldk,
                      float lambda, const int32_t* row_of_col, Ctrl* ctrl, cudaStream_t s) {
    const size_t total = (size_t)m * m;
    objective_kernel<<<grid_for(total, 256, kObjBlocks), 256, 0, s>>>(A, N, A2, m, K, ldk, lambda,
                                                                      row_of_col, ctrl);
    return cudaGetLastError();
}

}  // namespace fpfp
