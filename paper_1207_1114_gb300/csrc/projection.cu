// projection.cu -- persistent successive-projection kernel (Section 4.3) with
// the FastPFP update and max-normalisation of Algorithm 1 fused at its end.
//
// One cooperative launch runs every P1/P2 round of one outer iteration.  CTA
// b owns a contiguous band of rows of the slacked N x N matrix Y for the
// whole launch, so row sums r = Y 1 never leave the CTA.  Column sums
// c = Y^T 1 and the total s = 1^T Y 1 are the only cross-CTA quantities:
// each round every CTA adds its column partials into one of three rotating
// global accumulators (vector red.add) and its FP64 share of s, then one
// bounded grid barrier ends the round.  Every partial is rounded first to a
// power-of-two quantum from a bound all CTAs share (common.cuh), so the sums
// are exact whatever order the atomics land in; the input's sums are taken
// in FP64 the same way after a first barrier that agrees on max|y|.  Round u reads the sums of round u-1,
// applies Eq. (P1) elementwise
//      y <- y + 1/N + s/N^2 - r_i/N - c_j/N
// then Eq. (P2) y <- max(y, 0), measures max|dy|, and accumulates the sums
// of its own output for round u+1 in the same pass.  When the band fits in
// shared memory (RES) it stays on chip for all rounds; otherwise it is
// streamed from global memory (L2-resident up to ~100 MB).
#include "common.cuh"
#include "internal.h"

namespace fpfp {

namespace {

constexpr int kQptMax = 4;  // float4 column quads owned by one thread: N <= 4 * 4 * 1024

struct Smem {
    float4* rows;      // RES: rpc x Q quads of the CTA's band
    float* rsum;       // rpc row sums of the previous round
    float* arow;       // rpc offsets 1/N + s/N^2 - r_i/N of the next round
    float* rowpart;    // rpc x 32 per-warp row partials
    double* dred;      // 32 doubles of block-reduction scratch
    float* fred;       // 32 floats of block-reduction scratch
    int* ictl;         // [0] non-finite total, [1] stop the rounds, [2] bound mode of the next pass
    float* fctl;       // [0] max|dY| of the last round, [1] bound of the next pass's column sums
    double* qd;        // [0], [1] quantum (dn, up) of the next pass's share of s
};

// Shared-memory layout; pd_smem_bytes() below must mirror it.
__device__ __forceinline__ Smem carve(char* base, int rpc, int Q, bool res) {
    Smem s;
    size_t off = 0;
    s.rows = reinterpret_cast<float4*>(base);
    off += res ? (size_t)rpc * Q * sizeof(float4) : 0;
    s.rsum = reinterpret_cast<float*>(base + off);
    off += (size_t)rpc * sizeof(float);
    s.arow = reinterpret_cast<float*>(base + off);
    off += (size_t)rpc * sizeof(float);
    s.rowpart = reinterpret_cast<float*>(base + off);
    off += (size_t)rpc * 32 * sizeof(float);
    off = (off + 15) & ~size_t(15);
    s.dred = reinterpret_cast<double*>(base + off);
    off += 32 * sizeof(double);
    s.fred = reinterpret_cast<float*>(base + off);
    off += 32 * sizeof(float);
    s.ictl = reinterpret_cast<int*>(base + off);
    off += 4 * sizeof(int);
    s.fctl = reinterpret_cast<float*>(base + off);
    off += 4 * sizeof(float);
    s.qd = reinterpret_cast<double*>(base + off);
    return s;
}

__device__ __forceinline__ float sum4(float4 v) { return (v.x + v.y) + (v.z + v.w); }

__device__ __forceinline__ float block_max_f(float v, float* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    float t = scratch[0];
    for (int w = 1; w < nw; ++w) t = fmaxf(t, scratch[w]);
    return t;
}
__device__ __forceinline__ double block_max_d(double v, double* scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_max_d(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double t = scratch[0];
    for (int w = 1; w < nw; ++w) t = fmax(t, scratch[w]);
    return t;
}

// Keeps components of quad q that lie in columns < limit; zeroes the rest.
__device__ __forceinline__ float4 mask_cols(float4 v, int q, int limit) {
    const int c0 = 4 * q;
    if (c0 + 4 <= limit) return v;
    if (c0 + 0 >= limit) v.x = 0.f;
    if (c0 + 1 >= limit) v.y = 0.f;
    if (c0 + 2 >= limit) v.z = 0.f;
    if (c0 + 3 >= limit) v.w = 0.f;
    return v;
}

template <bool RES, int kQpt>
__global__ void __launch_bounds__(1024, 1) pd_kernel(const PdParams P) {
    extern __shared__ __align__(16) char smem_raw[];
    Ctrl* C = P.ctrl;
    if (P.mode == kPdOuterStep) {
        if (ld_relaxed_i32(&C->done) != 0 || ld_relaxed_i32(&C->error) != 0) return;
    }
    const int N = P.N, ldy = P.ldy, Q = ldy >> 2;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
    const unsigned G = gridDim.x;
    const int rpc = P.rpc;
    const int r0 = blockIdx.x * rpc;
    const int nr = max(0, min(N, r0 + rpc) - r0);
    Smem S = carve(smem_raw, rpc, Q, RES);
    const unsigned bar_base = C->bar_base;
    unsigned gen = 0;
    int* err = &C->error;

    float4* Yg = reinterpret_cast<float4*>(P.Y);
    auto row_ptr = [&](int rr) -> float4* {
        return RES ? S.rows + (size_t)rr * Q : Yg + (size_t)(r0 + rr) * Q;
    };

    // Column quads owned by this thread: q_k = tid + k * nthr.
    float4 cpart[kQpt];
    float4 cN[kQpt];

    // ---- prologue: optional slack reset, band load, sums of the input Y.
    const bool reset_slack = (P.mode == kPdOuterStep) && P.slack_reset && P.m < N;
    float ym = 0.f;   // max|y| of the band, for the quanta of the exact input sums
    for (int rr = 0; rr < nr; ++rr) {
        float4* src = Yg + (size_t)(r0 + rr) * Q;
        float4* dst = row_ptr(rr);
        for (int q = tid; q < Q; q += nthr) {
            float4 v = src[q];
            ym = fmaxf(ym, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            if (reset_slack) {
                // keep columns < m, zero the slack columns m..N-1
                const int c0 = 4 * q;
                if (c0 + 0 >= P.m) v.x = 0.f;
                if (c0 + 1 >= P.m) v.y = 0.f;
                if (c0 + 2 >= P.m) v.z = 0.f;
                if (c0 + 3 >= P.m) v.w = 0.f;
                if (!RES) src[q] = v;
            }
            if (RES) dst[q] = v;
        }
    }
    // zero accumulator 1 (used by round 1); accumulator 0 is zero on entry
    {
        float* c1 = P.colbuf + (size_t)1 * ldy;
        for (int q = blockIdx.x * nthr + tid; q < Q; q += G * nthr)
            reinterpret_cast<float4*>(c1)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (blockIdx.x == 0 && tid == 0) {
            P.sbuf[1] = 0.0;
            P.dbuf[1] = 0u;
        }
    }
    {
        const float bm = block_max_f(ym, S.fred);
        if (tid == 0 && bm > 0.f) atomicMax(P.dbuf + 3, __float_as_uint(bm));
    }
    if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, P.timeout_ns)) return;
    ++gen;
    // quanta of the input's sums: every column partial is at most N max|y|,
    // the total at most N^2 max|y|
    const float ymax = __uint_as_float(__ldcg(P.dbuf + 3));
    const Quant64 q_in = quant64_for((double)N * (double)ymax * (double)kBoundMargin);
    if (tid == 0) {
        const Quant64 qs = quant64_for((double)N * (double)N * (double)ymax * (double)kBoundMargin);
        S.qd[0] = qs.dn;
        S.qd[1] = qs.up;
    }
    __syncthreads();

    // End of a pass over the band: fold row sums (FP32), publish the CTA's
    // share of s (FP64, one warp), of max|dY| and of the column sums, wait at
    // the grid barrier, then let warp 0 turn the new total s into the per-row
    // offsets a_i = 1/N + s/N^2 - r_i/N of Eq. (P1) for the next pass.  Only
    // warp 0 touches FP64, once per pass.
    const double invN_d = 1.0 / (double)N;
    const double invN2_d = invN_d * invN_d;
    const float invN = 1.0f / (float)N;
    auto finish_pass = [&](int cur, float dmax, int u, bool arrive) -> bool {
        __syncthreads();
        for (int rr = tid; rr < nr; rr += nthr) {
            float r = 0.f;
            for (int w = 0; w < (nthr >> 5); ++w) r += S.rowpart[rr * 32 + w];
            S.rsum[rr] = r;
        }
        dmax = warp_max(dmax);
        if (lane == 0) S.fred[warp] = dmax;
        __syncthreads();
        if (warp == 0) {
            double sp = 0.0;
            for (int rr = lane; rr < nr; rr += 32) sp += (double)S.rsum[rr];
            sp = warp_sum_d(sp);
            float bm = lane < (nthr >> 5) ? S.fred[lane] : 0.f;
            bm = warp_max(bm);
            if (lane == 0) {
                atomicAdd(&P.sbuf[cur], quant64(sp, Quant64{S.qd[0], S.qd[1]}));
                if (bm > 0.f) atomicMax(&P.dbuf[cur], __float_as_uint(bm));
            }
        }
        float* ccur = P.colbuf + (size_t)cur * ldy;
        double* cin = colbuf64(P.colbuf, ldy);
        if (u == 0) {
            // the input's column sums, FP64
#pragma unroll
            for (int k = 0; k < kQpt; ++k) {
                const int q = tid + k * nthr;
                if (q < Q) {
                    red_add_f64(cin + 4 * q + 0, quant64((double)cpart[k].x, q_in));
                    red_add_f64(cin + 4 * q + 1, quant64((double)cpart[k].y, q_in));
                    red_add_f64(cin + 4 * q + 2, quant64((double)cpart[k].z, q_in));
                    red_add_f64(cin + 4 * q + 3, quant64((double)cpart[k].w, q_in));
                }
            }
        } else {
            // this pass's output is >= 0: column j's sum is at most
            // c_j + 1 + s/N (previous c_j, s; cN holds c_j / N) or, after the
            // input round, the one bound in fctl[1]
            const bool one = S.ictl[2] != 0;
            const float cb = S.fctl[1], Nf = (float)N;
#pragma unroll
            for (int k = 0; k < kQpt; ++k) {
                const int q = tid + k * nthr;
                if (q < Q) {
                    float4 v = cpart[k];
                    // one quantum for the quad, from the largest of its bounds
                    const float cm = fmaxf(fmaxf(cN[k].x, cN[k].y), fmaxf(cN[k].z, cN[k].w));
                    const Quant32 a = quant32_for(one ? cb : fmaf(cm, kBoundMargin * Nf, cb));
                    v = quant32x4(v, a, a, a, a);
                    red_add_v4(ccur + 4 * q, v.x, v.y, v.z, v.w);
                }
            }
        }
        if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, P.timeout_ns, arrive)) return false;
        ++gen;
        // column sums of this pass, scaled by 1/N, for the next round (issued
        // together with warp 0's loads of s and max|dY| below)
#pragma unroll
        for (int k = 0; k < kQpt; ++k) {
            const int q = tid + k * nthr;
            if (q < Q) {
                float4 c;
                if (u == 0) {
                    const double2 a = __ldcg(reinterpret_cast<const double2*>(cin) + 2 * q);
                    const double2 b = __ldcg(reinterpret_cast<const double2*>(cin) + 2 * q + 1);
                    c = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
                } else {
                    c = __ldcg(reinterpret_cast<const float4*>(ccur) + q);
                }
                cN[k] = make_float4(c.x * invN, c.y * invN, c.z * invN, c.w * invN);
            }
        }
        if (warp == 0) {
            const double s = __ldcg(&P.sbuf[cur]);
            const float d = __uint_as_float(__ldcg(&P.dbuf[cur]));
            const double a_base = invN_d + s * invN2_d;
            for (int rr = lane; rr < nr; rr += 32)
                S.arow[rr] = (float)(a_base - (double)S.rsum[rr] * invN_d);
            if (lane == 0) {
                S.ictl[0] = isfinite(s) ? 0 : 1;
                S.ictl[1] = (u > 0 && ((double)d < P.tol_inner || u >= P.max_inner)) ? 1 : 0;
                S.fctl[0] = d;
                // bounds of the next pass's sums: after the input every column
                // sum is at most 4 N max|y| + 1 (input, row offsets and column
                // offset of P1 each at most N max|y| per column); after a round
                // column j's at most c_j + 1 + s/N, the total at most 2 s + N
                const float mg = kBoundMargin, Nf = (float)N, sf = (float)s;
                float sb;
                if (u == 0) {
                    const float b1 = fmaf(4.0f * Nf, ymax, 1.0f) * mg;
                    S.ictl[2] = 1;
                    S.fctl[1] = b1;
                    sb = b1 * Nf * mg;
                } else {
                    S.ictl[2] = 0;
                    S.fctl[1] = fmaf(sf, invN, 1.0f) * mg;
                    sb = fmaf(2.0f, sf, Nf) * (mg * mg);
                }
                const Quant64 qs = quant64_for_f(sb);
                S.qd[0] = qs.dn;
                S.qd[1] = qs.up;
            }
        }
        __syncthreads();
        return true;
    };

#pragma unroll
    for (int k = 0; k < kQpt; ++k) cpart[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int rr = 0; rr < nr; ++rr) {
        const float4* row = row_ptr(rr);
        float racc = 0.f;
#pragma unroll
        for (int k = 0; k < kQpt; ++k) {
            const int q = tid + k * nthr;
            if (q < Q) {
                const float4 y = row[q];
                racc += sum4(y);
                cpart[k].x += y.x; cpart[k].y += y.y; cpart[k].z += y.z; cpart[k].w += y.w;
            }
        }
        racc = warp_sum(racc);
        if (lane == 0) S.rowpart[rr * 32 + warp] = racc;
    }
    const bool arrive0 = !(P.skip_arrive && blockIdx.x == 0 && C->outer == 0);
    if (!finish_pass(0, 0.f, 0, arrive0)) return;
    if (S.ictl[0]) {
        if (tid == 0) atomicCAS(err, 0, FASTPFP_ERR_NONFINITE);
        return;
    }

    // Zeroes every accumulator of the launch (after its last cross-CTA read):
    // the rotating column sums, totals and maxima, the FP64 input sums and
    // the input's max|y|.
    auto clear_sums = [&]() {
        for (int b = 0; b < 3; ++b) {
            float* cb = P.colbuf + (size_t)b * ldy;
            for (int q = blockIdx.x * nthr + tid; q < Q; q += G * nthr)
                reinterpret_cast<float4*>(cb)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        double2* c64 = reinterpret_cast<double2*>(colbuf64(P.colbuf, ldy));
        for (int q = blockIdx.x * nthr + tid; q < Q; q += G * nthr) {
            c64[2 * q] = make_double2(0.0, 0.0);
            c64[2 * q + 1] = make_double2(0.0, 0.0);
        }
        if (blockIdx.x == 0 && tid == 0) {
            for (int b = 0; b < 3; ++b) { P.sbuf[b] = 0.0; P.dbuf[b] = 0u; }
            P.dbuf[3] = 0u;
        }
    };

    // ---- P1/P2 rounds (cN holds c/N of the previous pass, S.arow its a_i)
    int u = 0;
    float delta = 0.f;
    while (true) {
        ++u;
        const int cur = u % 3, nxt = (u + 1) % 3;
#pragma unroll
        for (int k = 0; k < kQpt; ++k) cpart[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        // clear the accumulator of round u+1 (last read in round u-1)
        {
            float* cn = P.colbuf + (size_t)nxt * ldy;
            for (int q = blockIdx.x * nthr + tid; q < Q; q += G * nthr)
                reinterpret_cast<float4*>(cn)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (blockIdx.x == 0 && tid == 0) {
                P.sbuf[nxt] = 0.0;
                P.dbuf[nxt] = 0u;
            }
        }
        float dmax = 0.f;
        // rows in groups of four so the four row-sum shuffle chains overlap
        for (int rg = 0; rg < nr; rg += 4) {
            float racc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int rr = rg + j;
                if (rr >= nr) break;
                float4* row = row_ptr(rr);
                const float ai = S.arow[rr];
#pragma unroll
                for (int k = 0; k < kQpt; ++k) {
                    const int q = tid + k * nthr;
                    if (q < Q) {
                        const float4 y = row[q];
                        float4 z;
                        z.x = fmaxf((y.x + ai) - cN[k].x, 0.f);
                        z.y = fmaxf((y.y + ai) - cN[k].y, 0.f);
                        z.z = fmaxf((y.z + ai) - cN[k].z, 0.f);
                        z.w = fmaxf((y.w + ai) - cN[k].w, 0.f);
                        z = mask_cols(z, q, N);
                        dmax = fmaxf(dmax, fmaxf(fmaxf(fabsf(z.x - y.x), fabsf(z.y - y.y)),
                                                 fmaxf(fabsf(z.z - y.z), fabsf(z.w - y.w))));
                        row[q] = z;
                        racc[j] += sum4(z);
                        cpart[k].x += z.x; cpart[k].y += z.y; cpart[k].z += z.z; cpart[k].w += z.w;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) racc[j] = warp_sum(racc[j]);
            if (lane == 0) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (rg + j < nr) S.rowpart[(rg + j) * 32 + warp] = racc[j];
            }
        }
        if (!finish_pass(cur, dmax, u, true)) return;
        delta = S.fctl[0];
        if (S.ictl[1]) break;
    }

    if (P.mode == kPdProjectOnly) {
        if (RES) {
            for (int rr = 0; rr < nr; ++rr) {
                const float4* src = row_ptr(rr);
                float4* dst = Yg + (size_t)(r0 + rr) * Q;
                for (int q = tid; q < Q; q += nthr) dst[q] = src[q];
            }
        }
        if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, P.timeout_ns)) return;
        ++gen;
        clear_sums();
        if (blockIdx.x == 0 && tid == 0) {
            C->last_inner = u;
            C->last_delta = (double)delta;
            C->bar_base = bar_base + G * gen;
        }
        return;
    }

    // ---- blend and normalise (Algorithm 1): X <- ((1-a) X + a Y[:, :m]) / max
    const int m = P.m, ldx = P.ldx, Qx = ldx >> 2;
    const float alpha = P.alpha, beta = 1.0f - P.alpha;
    float4* Xg = reinterpret_cast<float4*>(P.X);
    float mx = 1.0f;
    if (P.normalize) {
        float lmax = -INFINITY;
        for (int rr = 0; rr < nr; ++rr) {
            const float4* row = row_ptr(rr);
            const float4* xr = Xg + (size_t)(r0 + rr) * Qx;
            for (int q = tid; q < Qx; q += nthr) {
                const float4 x = xr[q], y = row[q];
                float4 v = make_float4(beta * x.x + alpha * y.x, beta * x.y + alpha * y.y,
                                       beta * x.z + alpha * y.z, beta * x.w + alpha * y.w);
                const int c0 = 4 * q;
                lmax = fmaxf(lmax, v.x);
                if (c0 + 1 < m) lmax = fmaxf(lmax, v.y);
                if (c0 + 2 < m) lmax = fmaxf(lmax, v.z);
                if (c0 + 3 < m) lmax = fmaxf(lmax, v.w);
            }
        }
        const float bm = block_max_f(lmax, S.fred);
        if (tid == 0 && nr > 0) atomicMax(&C->xmax_bits, float_to_ordered(bm));
        if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, P.timeout_ns)) return;
        ++gen;
        mx = ordered_to_float(__ldcg(&C->xmax_bits));
    }
    AbsDiffMax dxm;   // max|dX| in FP64, as the oracle takes it
    const bool write16 = (P.Xt16 != nullptr);
    for (int rr = 0; rr < nr; ++rr) {
        const int i = r0 + rr;
        const float4* row = row_ptr(rr);
        float4* xr = Xg + (size_t)i * Qx;
        for (int q = tid; q < Qx; q += nthr) {
            const float4 x = xr[q], y = row[q];
            float4 v = make_float4(beta * x.x + alpha * y.x, beta * x.y + alpha * y.y,
                                   beta * x.z + alpha * y.z, beta * x.w + alpha * y.w);
            if (P.normalize) { v.x /= mx; v.y /= mx; v.z /= mx; v.w /= mx; }
            v = mask_cols(v, q, m);
            dxm.add4(v, x);
            xr[q] = v;
            if (write16) {
                const int c0 = 4 * q;
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (c0 + e < m) P.Xt16[(size_t)(c0 + e) * P.ldxt + i] = __float2bfloat16_rn(vv[e]);
            }
        }
    }
    if (RES) {
        // the slack columns m..N-1 carry over to the next outer iteration
        const int qs = m >> 2;
        for (int rr = 0; rr < nr; ++rr) {
            const float4* src = row_ptr(rr);
            float4* dst = Yg + (size_t)(r0 + rr) * Q;
            for (int q = qs + tid; q < Q; q += nthr) dst[q] = src[q];
        }
    }
    const double bdx = block_max_d(dxm.value(), S.dred);
    if (tid == 0 && nr > 0) atomicMax(&C->dx_bits, (unsigned long long)__double_as_longlong(bdx));
    if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, P.timeout_ns)) return;
    ++gen;

    // all cross-CTA reads of this launch are done: clear the accumulators
    clear_sums();
    if (blockIdx.x == 0 && tid == 0) {
        const double d = __longlong_as_double((long long)__ldcg(&C->dx_bits));
        if (!isfinite(d)) atomicCAS(err, 0, FASTPFP_ERR_NONFINITE);
        C->dx_bits = 0ull;
        C->xmax_bits = 0u;
        const int t = C->outer;
        if (t < kMaxOuterTrace) {
            C->inner_trace[t] = u;
            C->delta_trace[t] = d;
        }
        C->outer = t + 1;
        C->inner_total += u;
        C->inner_max = max(C->inner_max, u);
        C->last_inner = u;
        C->last_delta = d;
        if (C->lowp) {
            C->lowp_iters += 1;
            // the phase ends at switch_tol, when max|dX| shrinks by less than half
            // (the products' rounding noise is near; from the fourth iteration on) or
            // when only the refinement iterations are left
            const double dprev = (t >= 1 && t - 1 < kMaxOuterTrace) ? C->delta_trace[t - 1] : d;
            if (d < P.switch_tol || (t >= 3 && d > 0.5 * dprev) || t + 1 >= P.max_outer - P.refine_iters) {
                C->lowp = 0;
                C->refine_left = P.refine_iters;
            }
        } else {
            if (d < P.tol_outer) {
                C->converged = 1;
                C->done = 1;
            }
            if (C->refine_left > 0) {
                C->refine_left -= 1;
                if (C->refine_left == 0) C->done = 1;
            }
        }
        if (t + 1 >= P.max_outer) C->done = 1;
        C->bar_base = bar_base + G * gen;
    }
}

}  // namespace

size_t pd_smem_bytes(int rpc, int Q, bool res) {
    size_t off = res ? (size_t)rpc * Q * 16 : 0;
    off += (size_t)rpc * 4 * 2;
    off += (size_t)rpc * 32 * 4;
    off = (off + 15) & ~size_t(15);
    off += 32 * 8 + 32 * 4 + 4 * 4 + 4 * 4 + 2 * 8;
    return off;
}

cudaError_t pd_configure() {
    const void* fns[] = {(const void*)pd_kernel<true, 1>, (const void*)pd_kernel<false, 1>,
                         (const void*)pd_kernel<true, kQptMax>, (const void*)pd_kernel<false, kQptMax>};
    for (const void* f : fns) {
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, kPdMaxSmem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

void pd_plan(int N, int num_sms, PdLaunch* L) {
    const int ldy = (N + 3) & ~3;
    const int Q = ldy >> 2;
    int thr = ((Q + 31) / 32) * 32;
    if (thr < 64) thr = 64;
    if (thr > 1024) thr = 1024;
    // enough CTAs that each owns a modest band, at most one per SM
    long long elems = (long long)N * ldy;
    int G = (int)((elems + kPdElemsPerCta - 1) / kPdElemsPerCta);
    if (G < 1) G = 1;
    if (G > num_sms) G = num_sms;
    if (G > N) G = N;
    const int rpc = (N + G - 1) / G;
    G = (N + rpc - 1) / rpc;
    L->grid = G;
    L->block = thr;
    L->rpc = rpc;
    L->ldy = ldy;
    const size_t res_bytes = pd_smem_bytes(rpc, Q, true);
    L->resident = res_bytes <= (size_t)kPdMaxSmem;
    L->smem = L->resident ? res_bytes : pd_smem_bytes(rpc, Q, false);
}

cudaError_t pd_launch(const PdLaunch& L, const PdParams& P, cudaStream_t s) {
    void* args[] = {const_cast<PdParams*>(&P)};
    const bool one = (L.ldy >> 2) <= L.block;
    const void* f = L.resident ? (one ? (const void*)pd_kernel<true, 1> : (const void*)pd_kernel<true, kQptMax>)
                               : (one ? (const void*)pd_kernel<false, 1> : (const void*)pd_kernel<false, kQptMax>);
    return cudaLaunchCooperativeKernel(f, dim3(L.grid), dim3(L.block), args, L.smem, s);
}

}  // namespace fpfp
