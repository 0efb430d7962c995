// warmstart.cu -- kernels of the learned warm start (X(0) from a learned
// similarity; the paper recommends the uniform start and notes that the
// result depends on the initialisation, discussion after Algorithm 1).
//
//   features  F_i = [zscore(deg)_i, hist_i[0..15], zscore(B)_i[0..14]]
//   MLP       H = relu(F W1 + b1), E = H W2 + b2     (32 -> 128 -> 64, shared)
//   S         E_big E_small^T / 8,  X(0) = Sinkhorn(max(exp(S - rowmax S), 2^-100))
//             (every normalised entry floored at 2^-100 too: a trained S can
//             be so peaked that whole columns would underflow to zero)
//   training  row + column softmax cross-entropy of S against a solved
//             matching; analytic backward through S and the MLP; Adam.
//
// Every reduction is deterministic (fixed order): warp trees, or two-phase
// column reductions over fixed row chunks.
#include "common.cuh"
#include "internal.h"

namespace fpfp {
namespace {

constexpr int kChunkRows = 64;   // rows per partial of the two-phase column reductions

__device__ __forceinline__ int hist_bin(float w) {
    const float t = floorf(16.0f * w);   // exact: 16 w is a power-of-two scaling
    return t < 0.f ? 0 : (t > 15.f ? 15 : (int)t);
}

// Raw features: F[i, 0] = deg_i, F[i, 1..16] = histogram of incident weights
// (normalised by the incident-edge count), F[i, 17 + c] = B[i, c] for c < k.
// One warp per node.
__global__ void node_stats_kernel(const float* __restrict__ W, int n, const float* __restrict__ B, int k,
                                  float* __restrict__ F) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n) return;
    const float* row = W + (size_t)warp * n;
    float deg = 0.f;
    int cnt = 0;
    int h[16];
#pragma unroll
    for (int b = 0; b < 16; ++b) h[b] = 0;
    for (int j = lane; j < n; j += 32) {
        const float w = __ldg(row + j);
        deg += w;
        if (w != 0.f) {
            ++cnt;
            const int b = hist_bin(w);
#pragma unroll
            for (int q = 0; q < 16; ++q) h[q] += (q == b);
        }
    }
    deg = warp_sum(deg);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) h[q] += __shfl_xor_sync(0xffffffffu, h[q], o);
    }
    float* f = F + (size_t)warp * kMlpIn;
    if (lane == 0) {
        f[0] = deg;
        const float inv = 1.0f / (float)(cnt > 0 ? cnt : 1);
#pragma unroll
        for (int q = 0; q < 16; ++q) f[1 + q] = (float)h[q] * inv;
    }
    if (lane < 15) f[17 + lane] = lane < k ? B[(size_t)warp * k + lane] : 0.f;
}

// z-score of feature columns 0 and 17..16+k over the n nodes (population
// std + 1e-6); one block per column, FP32 block reductions in fixed order.
__global__ void zscore_kernel(float* F, int n, int k) {
    const int col = blockIdx.x == 0 ? 0 : 16 + blockIdx.x;
    if (blockIdx.x > 0 && blockIdx.x > k) return;
    __shared__ float red[32];
    __shared__ float mean_s, std_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float s = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += F[(size_t)i * kMlpIn + col];
    s = warp_sum(s);
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < nw; ++w) t += red[w];
        mean_s = t / (float)n;
    }
    __syncthreads();
    const float mu = mean_s;
    float q = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float d = F[(size_t)i * kMlpIn + col] - mu;
        q += d * d;
    }
    q = warp_sum(q);
    __syncthreads();
    if (lane == 0) red[warp] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < nw; ++w) t += red[w];
        std_s = sqrtf(t / (float)n) + 1e-6f;
    }
    __syncthreads();
    const float sd = std_s;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        float& v = F[(size_t)i * kMlpIn + col];
        v = (v - mu) / sd;
    }
}

// Y[n x no] = act(X[n x ki] W[ki x no] + b) * scale; one thread per output.
__global__ void linear_kernel(const float* __restrict__ X, int n, int ki, const float* __restrict__ W,
                              const float* __restrict__ b, float* __restrict__ Y, int no, int relu,
                              float scale) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (o >= no || i >= n) return;
    float acc = b ? b[o] : 0.f;
    const float* x = X + (size_t)i * ki;
    for (int q = 0; q < ki; ++q) acc = fmaf(x[q], W[(size_t)q * no + o], acc);
    if (relu) acc = fmaxf(acc, 0.f);
    Y[(size_t)i * no + o] = acc * scale;
}

// dst[c x ldd] = src[r x c]^T (FP32).
__global__ void transpose_kernel(const float* src, int r, int c, int lds, float* dst, int ldd) {
    __shared__ float tile[32][33];
    const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int i = bi + y, j = bj + threadIdx.x;
        tile[y][threadIdx.x] = (i < r && j < c) ? src[(size_t)i * lds + j] : 0.f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int j = bj + y, i = bi + threadIdx.x;
        if (j < c && i < r) dst[(size_t)j * ldd + i] = tile[threadIdx.x][y];
    }
}

constexpr float kSinkFloor = 0x1p-100f;   // positivity floor of the Sinkhorn iterates

// S <- max(exp(S - max of its row), kSinkFloor); one warp per row.
__global__ void row_exp_kernel(float* S, int r, int c, int ld) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= r) return;
    float* row = S + (size_t)warp * ld;
    float m = -INFINITY;
    for (int j = lane; j < c; j += 32) m = fmaxf(m, row[j]);
    m = warp_max(m);
    for (int j = lane; j < c; j += 32) row[j] = fmaxf(expf(row[j] - m), kSinkFloor);
}

// Each row divided by its sum (floored); one warp per row.
__global__ void row_normalize_kernel(float* S, int r, int c, int ld) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= r) return;
    float* row = S + (size_t)warp * ld;
    float s = 0.f;
    for (int j = lane; j < c; j += 32) s += row[j];
    s = warp_sum(s);
    const float inv = 1.0f / s;
    for (int j = lane; j < c; j += 32) row[j] = fmaxf(row[j] * inv, kSinkFloor);
}

// Column partial sums over row chunks: part[chunk][j].
__global__ void col_partial_kernel(const float* S, int r, int c, int ld, float* part) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, ch = blockIdx.y;
    if (j >= c) return;
    const int i1 = min(r, (ch + 1) * kChunkRows);
    float s = 0.f;
    for (int i = ch * kChunkRows; i < i1; ++i) s += S[(size_t)i * ld + j];
    part[(size_t)ch * c + j] = s;
}

// Each column divided by its sum (the chunk partials added in order).
__global__ void col_normalize_kernel(float* S, int r, int c, int ld, const float* part, int nch) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= c) return;
    float s = 0.f;
    for (int ch = 0; ch < nch; ++ch) s += part[(size_t)ch * c + j];
    const float inv = 1.0f / s;
    const int i0 = blockIdx.y * kChunkRows, i1 = min(r, i0 + kChunkRows);
    for (int i = i0; i < i1; ++i) S[(size_t)i * ld + j] = fmaxf(S[(size_t)i * ld + j] * inv, kSinkFloor);
}

// Column log-sum-exp of S: phase 1, per chunk (max, sum exp) with an online update.
__global__ void col_lse_partial_kernel(const float* S, int r, int c, int ld, float2* part) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, ch = blockIdx.y;
    if (j >= c) return;
    const int i1 = min(r, (ch + 1) * kChunkRows);
    float m = -INFINITY, s = 0.f;
    for (int i = ch * kChunkRows; i < i1; ++i) {
        const float v = S[(size_t)i * ld + j];
        if (v > m) {
            s = s * expf(m - v) + 1.f;
            m = v;
        } else {
            s += expf(v - m);
        }
    }
    part[(size_t)ch * c + j] = make_float2(m, s);
}
__global__ void col_lse_final_kernel(const float2* part, int nch, int c, float* lse) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= c) return;
    float m = -INFINITY;
    for (int ch = 0; ch < nch; ++ch) m = fmaxf(m, part[(size_t)ch * c + j].x);
    float s = 0.f;
    for (int ch = 0; ch < nch; ++ch) {
        const float2 p = part[(size_t)ch * c + j];
        s += p.y * expf(p.x - m);
    }
    lse[j] = m + logf(s);
}

// Row log-sum-exp of the matched rows t[j] (one warp per column j).
__global__ void row_lse_kernel(const float* S, int c, int ld, const int32_t* t, float* lse) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= c) return;
    const float* row = S + (size_t)t[warp] * ld;
    float m = -INFINITY;
    for (int q = lane; q < c; q += 32) m = fmaxf(m, row[q]);
    m = warp_max(m);
    float s = 0.f;
    for (int q = lane; q < c; q += 32) s += expf(row[q] - m);
    s = warp_sum(s);
    if (lane == 0) lse[warp] = m + logf(s);
}

// dS = (softmax_col(S) - 1[i = t(j)]) / m + for matched rows i = t(j'):
//      (softmax_row(S)[i, :] - 1[col = j']) / m.   tinv[i] = j' or -1.
__global__ void dS_kernel(const float* S, int r, int c, int ld, const float* lse_c, const float* lse_r,
                          const int32_t* t, const int32_t* tinv, float* dS, int ldd) {
    const float inv_m = 1.0f / (float)c;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)r * c;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / c), j = (int)(e % c);
        const float s = S[(size_t)i * ld + j];
        float g = expf(s - lse_c[j]) - (t[j] == i ? 1.f : 0.f);
        const int jp = tinv[i];
        if (jp >= 0) g += expf(s - lse_r[jp]) - (j == jp ? 1.f : 0.f);
        dS[(size_t)i * ldd + j] = g * inv_m;
    }
}

// loss = -(1/m) sum_j (2 S[t(j), j] - lse_c[j] - lse_r[j]), FP64 accumulation.
__global__ void loss_kernel(const float* S, int c, int ld, const int32_t* t, const float* lse_c,
                            const float* lse_r, double* out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int j = threadIdx.x; j < c; j += blockDim.x)
        acc += 2.0 * (double)S[(size_t)t[j] * ld + j] - (double)lse_c[j] - (double)lse_r[j];
    acc = warp_sum_d(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *out = -s / (double)c;
    }
}

// G[a x b] (+)= X[n x a]^T D[n x b]; one thread per output, rows in order.
__global__ void at_b_kernel(const float* X, int n, int a, const float* D, int b, float* G, int accumulate) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= a * b) return;
    const int p = o / b, q = o % b;
    float s = 0.f;
    for (int i = 0; i < n; ++i) s = fmaf(X[(size_t)i * a + p], D[(size_t)i * b + q], s);
    G[o] = accumulate ? G[o] + s : s;
}

// g[b] (+)= sum_i D[i, b]; one thread per column, rows in order.
__global__ void colsum_kernel(const float* D, int n, int b, float* g, int accumulate) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= b) return;
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += D[(size_t)i * b + q];
    g[q] = accumulate ? g[q] + s : s;
}

// dH[n x hid] = (dE[n x out] W2^T) * [H > 0].
__global__ void dh_kernel(const float* dE, int n, const float* W2, const float* H, float* dH) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (a >= kMlpHidden || i >= n) return;
    float s = 0.f;
    for (int q = 0; q < kMlpOut; ++q) s = fmaf(dE[(size_t)i * kMlpOut + q], W2[(size_t)a * kMlpOut + q], s);
    dH[(size_t)i * kMlpHidden + a] = H[(size_t)i * kMlpHidden + a] > 0.f ? s : 0.f;
}

__global__ void adam_kernel(float* p, float* m, float* v, const float* g, int np, float lr, float bc1,
                            float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
}

__global__ void scale_kernel(float* x, size_t n, float s) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        x[e] *= s;
}

inline int blocks_for(size_t total, int block, int cap = 4096) {
    size_t g = (total + block - 1) / block;
    return (int)(g < 1 ? 1 : (g > (size_t)cap ? cap : g));
}

}  // namespace

#define WS_CHECK()                                   \
    do {                                             \
        cudaError_t e_ = cudaGetLastError();         \
        if (e_ != cudaSuccess) return e_;            \
    } while (0)

cudaError_t ws_features(const float* W, int n, const float* B, int k, float* F, cudaStream_t s) {
    node_stats_kernel<<<(n + 7) / 8, 256, 0, s>>>(W, n, B, k, F);
    WS_CHECK();
    zscore_kernel<<<1 + (k < 15 ? k : 15), 256, 0, s>>>(F, n, k < 15 ? k : 15);
    WS_CHECK();
    return cudaSuccess;
}

cudaError_t ws_mlp_forward(const float* F, int n, const float* params, float* H, float* E, float escale,
                           cudaStream_t s) {
    const float* W1 = params;
    const float* b1 = W1 + kMlpIn * kMlpHidden;
    const float* W2 = b1 + kMlpHidden;
    const float* b2 = W2 + kMlpHidden * kMlpOut;
    linear_kernel<<<dim3((kMlpHidden + 127) / 128, n), 128, 0, s>>>(F, n, kMlpIn, W1, b1, H, kMlpHidden, 1, 1.f);
    WS_CHECK();
    linear_kernel<<<dim3((kMlpOut + 63) / 64, n), 64, 0, s>>>(H, n, kMlpHidden, W2, b2, E, kMlpOut, 0, escale);
    WS_CHECK();
    return cudaSuccess;
}

cudaError_t ws_transpose(const float* src, int r, int c, int lds, float* dst, int ldd, cudaStream_t s) {
    transpose_kernel<<<dim3((c + 31) / 32, (r + 31) / 32), dim3(32, 8), 0, s>>>(src, r, c, lds, dst, ldd);
    return cudaGetLastError();
}

cudaError_t ws_scale(float* x, size_t n, float v, cudaStream_t s) {
    scale_kernel<<<blocks_for(n, 256), 256, 0, s>>>(x, n, v);
    return cudaGetLastError();
}

cudaError_t ws_sinkhorn(float* S, int r, int c, int ld, int iters, float* part, float* scalar,
                        cudaStream_t s) {
    (void)scalar;
    row_exp_kernel<<<(r + 7) / 8, 256, 0, s>>>(S, r, c, ld);
    WS_CHECK();
    const int nch = (r + kChunkRows - 1) / kChunkRows;
    for (int it = 0; it < iters; ++it) {
        row_normalize_kernel<<<(r + 7) / 8, 256, 0, s>>>(S, r, c, ld);
        WS_CHECK();
        col_partial_kernel<<<dim3((c + 127) / 128, nch), 128, 0, s>>>(S, r, c, ld, part);
        WS_CHECK();
        col_normalize_kernel<<<dim3((c + 127) / 128, nch), 128, 0, s>>>(S, r, c, ld, part, nch);
        WS_CHECK();
    }
    return cudaSuccess;
}

cudaError_t ws_loss_grad_S(const float* S, int r, int c, int ld, const int32_t* t, const int32_t* tinv,
                           float* lse_c, float* lse_r, float2* part, float* dS, int ldd, double* loss,
                           cudaStream_t s) {
    const int nch = (r + kChunkRows - 1) / kChunkRows;
    col_lse_partial_kernel<<<dim3((c + 127) / 128, nch), 128, 0, s>>>(S, r, c, ld, part);
    WS_CHECK();
    col_lse_final_kernel<<<(c + 127) / 128, 128, 0, s>>>(part, nch, c, lse_c);
    WS_CHECK();
    row_lse_kernel<<<(c + 7) / 8, 256, 0, s>>>(S, c, ld, t, lse_r);
    WS_CHECK();
    dS_kernel<<<blocks_for((size_t)r * c, 256), 256, 0, s>>>(S, r, c, ld, lse_c, lse_r, t, tinv, dS, ldd);
    WS_CHECK();
    loss_kernel<<<1, 256, 0, s>>>(S, c, ld, t, lse_c, lse_r, loss);
    WS_CHECK();
    return cudaSuccess;
}

cudaError_t ws_mlp_backward(const float* F, const float* H, const float* dE, int n, const float* params,
                            float* dH, float* grad, int accumulate, cudaStream_t s) {
    const float* W2 = params + kMlpIn * kMlpHidden + kMlpHidden;
    float* gW1 = grad;
    float* gb1 = gW1 + kMlpIn * kMlpHidden;
    float* gW2 = gb1 + kMlpHidden;
    float* gb2 = gW2 + kMlpHidden * kMlpOut;
    at_b_kernel<<<(kMlpHidden * kMlpOut + 127) / 128, 128, 0, s>>>(H, n, kMlpHidden, dE, kMlpOut, gW2, accumulate);
    WS_CHECK();
    colsum_kernel<<<1, kMlpOut, 0, s>>>(dE, n, kMlpOut, gb2, accumulate);
    WS_CHECK();
    dh_kernel<<<dim3(1, n), kMlpHidden, 0, s>>>(dE, n, W2, H, dH);
    WS_CHECK();
    at_b_kernel<<<(kMlpIn * kMlpHidden + 127) / 128, 128, 0, s>>>(F, n, kMlpIn, dH, kMlpHidden, gW1, accumulate);
    WS_CHECK();
    colsum_kernel<<<1, kMlpHidden, 0, s>>>(dH, n, kMlpHidden, gb1, accumulate);
    WS_CHECK();
    return cudaSuccess;
}

namespace {
// Out-of-range entries of perm are ignored (their column keeps target row 0).
__global__ void targets_kernel(const int32_t* perm, int n_a, int transposed, int N, int m, int32_t* t,
                               int32_t* tinv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_a) return;
    const int j = perm[i];
    if (transposed) {          // graph 1 indexes the columns: column i -> row perm[i]
        if (i < m && j >= 0 && j < N) {
            t[i] = j;
            tinv[j] = i;
        }
    } else if (i < N && j >= 0 && j < m) {   // graph 1 indexes the rows: row i -> column perm[i]
        t[j] = i;
        tinv[i] = j;
    }
}
}  // namespace

cudaError_t ws_targets(const int32_t* perm, int n_a, int transposed, int N, int m, int32_t* t,
                       int32_t* tinv, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(tinv, 0xff, (size_t)N * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(t, 0, (size_t)m * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    targets_kernel<<<(n_a + 255) / 256, 256, 0, s>>>(perm, n_a, transposed, N, m, t, tinv);
    return cudaGetLastError();
}

cudaError_t ws_adam(float* p, float* m, float* v, const float* g, int step, float lr, cudaStream_t s) {
    const float bc1 = 1.0f - powf(0.9f, (float)step), bc2 = 1.0f - powf(0.999f, (float)step);
    adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(p, m, v, g, kMlpParams, lr, bc1, bc2);
    return cudaGetLastError();
}

}  // namespace fpfp
