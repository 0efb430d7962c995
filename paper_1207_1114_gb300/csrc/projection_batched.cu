// projection_batched.cu -- one cooperative launch runs the successive
// projection (Section 4.3) and the blend / normalisation / loop control of
// Algorithm 1 for a whole wave of graph pairs at once.
//
// The projection rounds are bound by grid-synchronisation latency, not by
// bandwidth.  A wave therefore shares every barrier between many pairs.
// All rows of all pairs are concatenated and cut into one band
// per CTA of about the same cost (entries plus a measured cost per pair the
// band spans); a band may span several pairs ("segments") and stays on chip
// for all rounds: the first rows of every thread in tensor memory (all 512
// columns of the SM, used as storage through tcgen05.ld/st), the rest in
// shared memory.  A round
// applies Eq. (P1) and Eq. (P2) elementwise to every segment of the band,
// measures max|dY|, and publishes the pairs' column partials (vector
// red.add), FP64 shares of the totals s and round maxima.  Every partial is
// first rounded to a power-of-two quantum (common.cuh) from a bound all CTAs
// share, so the sums are exact and do not depend on the order in which the
// atomics land: a solve gives the same bits every run.  After the grid
// barrier every CTA reads every pair's round maximum, so all CTAs take the
// same stop decision for each pair (max|dY| < eps_2 or I_1 rounds) and leave
// the loop together.  Pairs whose outer loop has finished are skipped.
#include <type_traits>

#include "band_plan.cuh"
#include "common.cuh"
#include "internal.h"

namespace fpfp {
namespace {

struct Seg {
    int pair;       // index into the wave's pair table
    int lr0;        // first row of the segment inside its pair
    int nrows;      // rows of the segment
    int brow0;      // first row of the segment inside the band (rsum/rowpart index)
    int soff;       // float offset of the segment's shared-memory rows in the band storage
    int coff;       // float offset of the segment's column sums
    int tm;         // thread-rows per row group held in TMEM (band rows 0 .. ntm - 1)
    int tcol;       // first TMEM column of the segment in every thread's share
    int ntm;        // band rows of the segment in TMEM; rows ntm .. nrows - 1 are in shared memory
    int qpg;        // thread layout of the pair (pdb_shape): threads per row,
    int rpkq;       // row groups * 4 + quads per thread
};

// Per-pair fields used every round, copied to shared memory once per launch.
struct PairS {
    float* colbuf;
    double* sbuf;
    unsigned* dbuf;
    float invNf;    // (float)(1/N), for the FP32 bounds
    int bmode;      // quanta of the next pass's column partials: 0 per column, 1 one for the pair
    int N, ldy;
    float abase;    // 1/N + s/N^2 of the last finished pass (the row offset is abase - r_i/N)
    float cb;       // bmode 0: column j's bound is c_j * margin + cb; bmode 1: every column's bound
    double invN;    // 1/N
    float ymax;     // max|y| of the launch's input
    Quant64 sq;     // quantum of the next pass's contributions to s
};

static_assert(sizeof(Seg) == kSegBytes, "pdb_smem_bytes sizes the segment table");
static_assert(kPdbThreads <= 16 * 32, "a segment's fred slots hold 16 warps' maxima and 16 warps' totals");
static_assert(sizeof(PairS) == kPairBytes, "pdb_smem_bytes sizes the pair table");

struct Shared {
    Seg* seg;            // L.max_segs
    PairS* pair;         // L.npairs
    int* pstate;         // L.npairs: bit0 active this launch, bit1 stopped
    int* pstop;          // L.npairs: round at which the pair stopped
    int* ictl;           // [2] n segments, [3] non-finite, [4] running pairs
    int* qpref;          // L.npairs + 1: prefix sums of the pairs' column quads
    float* fred;         // L.max_segs x 32: per-warp maxima (0 .. 15), per-warp row-partial totals (16 .. 31)
    float* rsum;         // band rows
    float* rowpart;      // band rows x rp_stride per-warp row partials
    float* cN;           // sum over segments of ldy floats: the column sums c_j of the last round
    float* band;         // band rows of every segment (16-byte aligned)
};

__device__ __forceinline__ Shared carve_b(char* base, const PdbLayout& L, int nthr) {
    Shared s;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base + off;
        off = (off + bytes + 15) & ~size_t(15);
        return p;
    };
    s.seg = reinterpret_cast<Seg*>(take(sizeof(Seg) * L.max_segs));
    s.pair = reinterpret_cast<PairS*>(take(sizeof(PairS) * L.npairs));
    s.pstate = reinterpret_cast<int*>(take(sizeof(int) * L.npairs));
    s.pstop = reinterpret_cast<int*>(take(sizeof(int) * L.npairs));
    s.ictl = reinterpret_cast<int*>(take(sizeof(int) * 8));
    s.qpref = reinterpret_cast<int*>(take(sizeof(int) * (L.npairs + 1)));
    s.fred = reinterpret_cast<float*>(take(sizeof(float) * L.max_segs * 32));
    s.rsum = reinterpret_cast<float*>(take(sizeof(float) * L.max_band_rows));
    s.rowpart = reinterpret_cast<float*>(take(sizeof(float) * L.max_band_rows * L.rp_stride));
    s.cN = reinterpret_cast<float*>(take(sizeof(float) * L.max_band_cols));
    s.band = reinterpret_cast<float*>(take(sizeof(float) * L.max_band_elems));
    return s;
}

// Thread -> (row group, quads) mapping of one segment (pdb_shape): QP
// threads cover a row, RP row groups work on different rows at once, and a
// thread owns quads q0 and (kq = 2) q0 + QP of its group's rows.  Threads
// past RP * QP have no rows (grp >= RP).
struct Map {
    int QP, RP, grp, q0, kq;
};
__device__ __forceinline__ Map make_map(int qpg, int rpkq, int tid) {
    Map m;
    m.QP = qpg;
    m.RP = rpkq >> 2;
    m.kq = rpkq & 3;
    m.grp = tid / qpg;
    m.q0 = tid - m.grp * qpg;
    return m;
}

// The column term of P1 on padding columns: far below any offset a_i, so
// their update max(a_i - kPadB, -0) is -0 (finite: no infinity enters).
constexpr float kPadB = 1.0e30f;

// float4 loads of X and of Y each thread issues before it uses any in the
// blend: with one CTA of 16 warps per SM, one load pair per thread leaves
// the blend latency-bound far below the HBM rate.
constexpr int kBlendLoads = 4;

// Two-lane FP32 arithmetic (sm_100 packed f32x2): one instruction updates
// two floats held in a register pair.
__device__ __forceinline__ unsigned long long pk(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// One column quad of one row held in registers: Eq. (P1) then Eq. (P2).
// With t = a_i + b_j the offset P1 adds (a_i = 1/N + s/N^2 - r_i/N per row,
// b = -c_j/N per column, passed in `b`), max(y + t, 0) = y + max(t, -y)
// exactly (an FP32 y - y is +0), so the round's change d = max(t, -y) comes
// out of the update itself and max|dY| costs one three-way max per two
// entries.  Padding columns (>= N) hold y = 0 and b = -kPadB, so t is
// hugely negative there and d = max(t, -0) = -0: they stay zero with no
// test in the loop.  Returns the quad's contribution to the row sum and adds
// the new y to the column partials cp.  Packed f32x2 additions, two lanes
// per op.
template <bool UPDATE>
__device__ __forceinline__ float quad_upd(float4& y, float ai, float4 b, float4& cp, float& dmax) {
    if (UPDATE) {
        const unsigned long long A = pk(ai, ai);
        const float2 t01 = upk(add2(A, pk(b.x, b.y)));
        const float2 t23 = upk(add2(A, pk(b.z, b.w)));
        const float4 d =
            make_float4(fmaxf(t01.x, -y.x), fmaxf(t01.y, -y.y), fmaxf(t23.x, -y.z), fmaxf(t23.y, -y.w));
        dmax = max3f(dmax, fabsf(d.x), fabsf(d.y));
        dmax = max3f(dmax, fabsf(d.z), fabsf(d.w));
        const float2 z01 = upk(add2(pk(y.x, y.y), pk(d.x, d.y)));
        const float2 z23 = upk(add2(pk(y.z, y.w), pk(d.z, d.w)));
        y = make_float4(z01.x, z01.y, z23.x, z23.y);
    }
    const float2 c01 = upk(add2(pk(cp.x, cp.y), pk(y.x, y.y)));
    const float2 c23 = upk(add2(pk(cp.z, cp.w), pk(y.z, y.w)));
    cp = make_float4(c01.x, c01.y, c23.x, c23.y);
    const float2 r = upk(add2(pk(y.x, y.y), pk(y.z, y.w)));
    return r.x + r.y;
}

// The same for a quad in shared memory.
template <bool UPDATE>
__device__ __forceinline__ float quad_step(float4* __restrict__ p, float ai, float4 b, float4& cp, float& dmax) {
    float4 y = *p;
    const float s = quad_upd<UPDATE>(y, ai, b, cp, dmax);
    if (UPDATE) *p = y;
    return s;
}

// Tensor memory as storage (no MMA): warp-collective 32-lane x N-column
// loads and stores of 32-bit words, each lane its own TMEM lane.
__device__ __forceinline__ void tm_ld16(uint32_t taddr, float4 (&q)[4]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 4; ++j)
        q[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]), __uint_as_float(r[4 * j + 2]),
                           __uint_as_float(r[4 * j + 3]));
}
__device__ __forceinline__ void tm_st16(uint32_t taddr, const float4 (&q)[4]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(__float_as_uint(q[0].x)), "r"(__float_as_uint(q[0].y)), "r"(__float_as_uint(q[0].z)),
          "r"(__float_as_uint(q[0].w)), "r"(__float_as_uint(q[1].x)), "r"(__float_as_uint(q[1].y)),
          "r"(__float_as_uint(q[1].z)), "r"(__float_as_uint(q[1].w)), "r"(__float_as_uint(q[2].x)),
          "r"(__float_as_uint(q[2].y)), "r"(__float_as_uint(q[2].z)), "r"(__float_as_uint(q[2].w)),
          "r"(__float_as_uint(q[3].x)), "r"(__float_as_uint(q[3].y)), "r"(__float_as_uint(q[3].z)),
          "r"(__float_as_uint(q[3].w))
        : "memory");
}
// Two 16-column loads behind one wait (the wait names their registers, so
// no use of them can be scheduled before it): half the load round trips of
// one wait per load.
__device__ __forceinline__ void tm_ld16x2(uint32_t ta, uint32_t tb, float4 (&q)[8]) {
    uint32_t a[16], b[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(a[0]), "=r"(a[1]), "=r"(a[2]), "=r"(a[3]), "=r"(a[4]), "=r"(a[5]), "=r"(a[6]), "=r"(a[7]),
          "=r"(a[8]), "=r"(a[9]), "=r"(a[10]), "=r"(a[11]), "=r"(a[12]), "=r"(a[13]), "=r"(a[14]), "=r"(a[15])
        : "r"(ta));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(b[0]), "=r"(b[1]), "=r"(b[2]), "=r"(b[3]), "=r"(b[4]), "=r"(b[5]), "=r"(b[6]), "=r"(b[7]),
          "=r"(b[8]), "=r"(b[9]), "=r"(b[10]), "=r"(b[11]), "=r"(b[12]), "=r"(b[13]), "=r"(b[14]), "=r"(b[15])
        : "r"(tb));
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                   "+r"(a[8]), "+r"(a[9]), "+r"(a[10]), "+r"(a[11]), "+r"(a[12]), "+r"(a[13]), "+r"(a[14]),
                   "+r"(a[15]), "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]),
                   "+r"(b[6]), "+r"(b[7]), "+r"(b[8]), "+r"(b[9]), "+r"(b[10]), "+r"(b[11]), "+r"(b[12]),
                   "+r"(b[13]), "+r"(b[14]), "+r"(b[15])
                 :: "memory");
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        q[j] = make_float4(__uint_as_float(a[4 * j]), __uint_as_float(a[4 * j + 1]), __uint_as_float(a[4 * j + 2]),
                           __uint_as_float(a[4 * j + 3]));
        q[4 + j] = make_float4(__uint_as_float(b[4 * j]), __uint_as_float(b[4 * j + 1]),
                               __uint_as_float(b[4 * j + 2]), __uint_as_float(b[4 * j + 3]));
    }
}
__device__ __forceinline__ float4 tm_ld4(uint32_t taddr) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    return make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]), __uint_as_float(r[3]));
}
__device__ __forceinline__ void tm_st4(uint32_t taddr, float4 v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(taddr),
                 "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
                 "r"(__float_as_uint(v.w))
                 : "memory");
}
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Four rows' warp sums in one shuffle tree: bit 4 of the lane picks rows
// {0,1} or {2,3}, bit 3 the row within the pair; lanes 0, 8, 16, 24 end
// with rows 0, 1, 2, 3.
__device__ __forceinline__ float sum4_rows(const float (&s)[4], int lane) {
    const bool b4 = (lane & 16) != 0, b3 = (lane & 8) != 0;
    float x0 = b4 ? s[2] : s[0], x1 = b4 ? s[3] : s[1];
    x0 += __shfl_xor_sync(0xffffffffu, b4 ? s[0] : s[2], 16);
    x1 += __shfl_xor_sync(0xffffffffu, b4 ? s[1] : s[3], 16);
    float z = b3 ? x1 : x0;
    z += __shfl_xor_sync(0xffffffffu, b3 ? x0 : x1, 8);
    z += __shfl_xor_sync(0xffffffffu, z, 4);
    z += __shfl_xor_sync(0xffffffffu, z, 2);
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    return z;
}

// The TMEM rows of one segment for this thread's row group: thread-rows
// k < tm (band rows grp + RP k) at TMEM columns taddr + 4 k, four rows per
// load/store.  Rows past nrows (the group's last thread-rows) are carried
// but not updated or counted.  Warp-collective: whole warps call it.
template <bool UPDATE>
__device__ __forceinline__ void seg_rows_tmem(uint32_t taddr, int tm, int nrows, int Q, int N, const Map& mp,
                                              int lane, const float* __restrict__ rsum, float abase,
                                              float* __restrict__ rowpart, int rps, float4 c0v, float ninvN,
                                              float4& cp0, float& dmax, float& tot) {
    const bool h0 = mp.q0 < Q;
    const int RP = mp.RP;
    int k = 0;
    // eight thread-rows per wait
    for (; k + 7 < tm; k += 8) {
        float4 q[8];
        tm_ld16x2(taddr + 4 * k, taddr + 4 * k + 16, q);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float s[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = mp.grp + RP * (k + 4 * h + j);
                s[j] = 0.f;
                if (r < nrows && h0) {
                    const float a = UPDATE ? fmaf(ninvN, rsum[r], abase) : 0.f;
                    s[j] = quad_upd<UPDATE>(q[4 * h + j], a, c0v, cp0, dmax);
                }
            }
            const float z = sum4_rows(s, lane);
            const int rj = mp.grp + RP * (k + 4 * h + 2 * (lane >> 4) + ((lane >> 3) & 1));
            if ((lane & 7) == 0 && rj < nrows) { rowpart[(size_t)rj * rps] = z; tot += z; }
        }
        if (UPDATE) {
            const float4 qa[4] = {q[0], q[1], q[2], q[3]}, qb[4] = {q[4], q[5], q[6], q[7]};
            tm_st16(taddr + 4 * k, qa);
            tm_st16(taddr + 4 * k + 16, qb);
        }
    }
    for (; k + 3 < tm; k += 4) {
        float4 q[4];
        tm_ld16(taddr + 4 * k, q);
        float s[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = mp.grp + RP * (k + j);
            s[j] = 0.f;
            if (r < nrows && h0) {
                const float a = UPDATE ? fmaf(ninvN, rsum[r], abase) : 0.f;
                s[j] = quad_upd<UPDATE>(q[j], a, c0v, cp0, dmax);
            }
        }
        if (UPDATE) tm_st16(taddr + 4 * k, q);
        const float z = sum4_rows(s, lane);
        const int rj = mp.grp + RP * (k + 2 * (lane >> 4) + ((lane >> 3) & 1));
        if ((lane & 7) == 0 && rj < nrows) { rowpart[(size_t)rj * rps] = z; tot += z; }
    }
    for (; k < tm; ++k) {
        const int r = mp.grp + RP * k;
        float4 y = tm_ld4(taddr + 4 * k);
        float s0 = 0.f;
        if (r < nrows && h0) {
            const float a = UPDATE ? fmaf(ninvN, rsum[r], abase) : 0.f;
            s0 = quad_upd<UPDATE>(y, a, c0v, cp0, dmax);
        }
        if (UPDATE) tm_st4(taddr + 4 * k, y);
        s0 = warp_sum(s0);
        if (lane == 0 && r < nrows) { rowpart[(size_t)r * rps] = s0; tot += s0; }
    }
}

// The TMEM rows of a segment whose threads own two quads per row (kq = 2):
// thread-row k holds quads q0 and q0 + QP at TMEM columns taddr + 8 k and
// + 8 k + 4, two rows per 16-column load/store.  Warp-collective.
template <bool UPDATE>
__device__ __forceinline__ void seg_rows_tmem2(uint32_t taddr, int tm, int nrows, int Q, int N, const Map& mp,
                                               int lane, const float* __restrict__ rsum, float abase,
                                               float* __restrict__ rowpart, int rps, float4 c0v, float4 c1v,
                                               float ninvN, float4& cp0, float4& cp1, float& dmax, float& tot) {
    const int q1 = mp.q0 + mp.QP;
    const bool h0 = mp.q0 < Q, h1 = q1 < Q;
    const int RP = mp.RP;
    int k = 0;
    // four thread-rows per wait, their four row sums in one shuffle tree
    for (; k + 3 < tm; k += 4) {
        float4 q[8];   // row k + j: quads 0, 1 at q[2 j], q[2 j + 1]
        tm_ld16x2(taddr + 8 * k, taddr + 8 * k + 16, q);
        float s[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = mp.grp + RP * (k + j);
            s[j] = 0.f;
            if (r < nrows) {
                const float a = UPDATE ? fmaf(ninvN, rsum[r], abase) : 0.f;
                if (h0) s[j] += quad_upd<UPDATE>(q[2 * j], a, c0v, cp0, dmax);
                if (h1) s[j] += quad_upd<UPDATE>(q[2 * j + 1], a, c1v, cp1, dmax);
            }
        }
        if (UPDATE) {
            const float4 qa[4] = {q[0], q[1], q[2], q[3]}, qb[4] = {q[4], q[5], q[6], q[7]};
            tm_st16(taddr + 8 * k, qa);
            tm_st16(taddr + 8 * k + 16, qb);
        }
        const float z = sum4_rows(s, lane);
        const int rj = mp.grp + RP * (k + 2 * (lane >> 4) + ((lane >> 3) & 1));
        if ((lane & 7) == 0 && rj < nrows) { rowpart[(size_t)rj * rps] = z; tot += z; }
    }
    for (; k + 1 < tm; k += 2) {
        float4 q[4];   // row k: quads 0, 1; row k + 1: quads 0, 1
        tm_ld16(taddr + 8 * k, q);
        float s[2] = {0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int r = mp.grp + RP * (k + j);
            if (r < nrows) {
                const float a = UPDATE ? fmaf(ninvN, rsum[r], abase) : 0.f;
                if (h0) s[j] += quad_upd<UPDATE>(q[2 * j], a, c0v, cp0, dmax);
                if (h1) s[j] += quad_upd<UPDATE>(q[2 * j + 1], a, c1v, cp1, dmax);
            }
        }
        if (UPDATE) tm_st16(taddr + 8 * k, q);
        // both rows' warp sums in five shuffles (lower half-warp row k)
        const bool hi = (lane & 16) != 0;
        float keep = hi ? s[1] : s[0];
        keep += __shfl_xor_sync(0xffffffffu, hi ? s[0] : s[1], 16);
        keep += __shfl_xor_sync(0xffffffffu, keep, 8);
        keep += __shfl_xor_sync(0xffffffffu, keep, 4);
        keep += __shfl_xor_sync(0xffffffffu, keep, 2);
        keep += __shfl_xor_sync(0xffffffffu, keep, 1);
        const int r0 = mp.grp + RP * k, r1 = r0 + RP;
        if (lane == 0 && r0 < nrows) { rowpart[(size_t)r0 * rps] = keep; tot += keep; }
        if (lane == 16 && r1 < nrows) { rowpart[(size_t)r1 * rps] = keep; tot += keep; }
    }
    if (k < tm) {
        const int r = mp.grp + RP * k;
        float4 y0 = tm_ld4(taddr + 8 * k), y1 = tm_ld4(taddr + 8 * k + 4);
        float s0 = 0.f;
        if (r < nrows) {
            const float a = UPDATE ? fmaf(ninvN, rsum[r], abase) : 0.f;
            if (h0) s0 += quad_upd<UPDATE>(y0, a, c0v, cp0, dmax);
            if (h1) s0 += quad_upd<UPDATE>(y1, a, c1v, cp1, dmax);
        }
        if (UPDATE) {
            tm_st4(taddr + 8 * k, y0);
            tm_st4(taddr + 8 * k + 4, y1);
        }
        s0 = warp_sum(s0);
        if (lane == 0 && r < nrows) { rowpart[(size_t)r * rps] = s0; tot += s0; }
    }
}

// All rows of one segment handled by this thread's row group: four rows in
// flight, then two, then one.  KQ = column quads per thread (1 or 2).  The
// row offset of Eq. (P1) is abase - r_i / N (one FMA from the row sums of
// the last pass; abase = 1/N + s/N^2 is formed in FP64 once per pair).
// Must be called by whole warps (a row group is whole warps).
template <bool UPDATE, int KQ>
__device__ __forceinline__ void seg_rows(float4* __restrict__ band, int nrows, int Q, int N,
                                         const Map& mp, int nthr, int lane,
                                         const float* __restrict__ rsum, float abase,
                                         float* __restrict__ rowpart, int rps, float4 c0v, float4 c1v, float ninvN,
                                         float4& cp0, float4& cp1, float& dmax, float& tot) {
    const bool h0 = mp.q0 < Q;
    const int q1 = mp.q0 + mp.QP;   // the second quad (kq = 2)
    const bool h1 = KQ > 1 && q1 < Q;
    const int RP = mp.RP;
    const int stride = RP * Q;
    int r = mp.grp;
    float4* p = band + (size_t)mp.grp * Q + mp.q0;
    for (; r + 3 * RP < nrows; r += 4 * RP, p += 4 * stride) {
        float a[4], s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 4; ++k) a[k] = UPDATE ? fmaf(ninvN, rsum[r + k * RP], abase) : 0.f;
        // per column quad, every load of the four rows before any store (the
        // rows are distinct, which the compiler cannot prove), so their
        // latencies overlap
#pragma unroll
        for (int j = 0; j < KQ; ++j) {
            if (!(j == 0 ? h0 : h1)) continue;
            float4* pj = p + j * mp.QP;
            const float4 cv = j == 0 ? c0v : c1v;
            float4& cpj = j == 0 ? cp0 : cp1;
            float4 y[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) y[k] = pj[k * stride];
#pragma unroll
            for (int k = 0; k < 4; ++k) s[k] += quad_upd<UPDATE>(y[k], a[k], cv, cpj, dmax);
            if (UPDATE) {
#pragma unroll
                for (int k = 0; k < 4; ++k) pj[k * stride] = y[k];
            }
        }
        const float z = sum4_rows(s, lane);
        if ((lane & 7) == 0) { rowpart[(size_t)(r + (2 * (lane >> 4) + ((lane >> 3) & 1)) * RP) * rps] = z; tot += z; }
    }
    for (; r + RP < nrows; r += 2 * RP, p += 2 * stride) {
        const float a0 = UPDATE ? fmaf(ninvN, rsum[r], abase) : 0.f;
        const float a1 = UPDATE ? fmaf(ninvN, rsum[r + RP], abase) : 0.f;
        float s0 = 0.f, s1 = 0.f;
        if (h0) {
            s0 += quad_step<UPDATE>(p, a0, c0v, cp0, dmax);
            s1 += quad_step<UPDATE>(p + stride, a1, c0v, cp0, dmax);
        }
        if (KQ > 1 && h1) {
            s0 += quad_step<UPDATE>(p + mp.QP, a0, c1v, cp1, dmax);
            s1 += quad_step<UPDATE>(p + stride + mp.QP, a1, c1v, cp1, dmax);
        }
        // both rows' warp sums in five shuffles: the lower half-warp folds
        // row r, the upper half row r + RP
        const bool hi = (lane & 16) != 0;
        float keep = hi ? s1 : s0;
        keep += __shfl_xor_sync(0xffffffffu, hi ? s0 : s1, 16);
        keep += __shfl_xor_sync(0xffffffffu, keep, 8);
        keep += __shfl_xor_sync(0xffffffffu, keep, 4);
        keep += __shfl_xor_sync(0xffffffffu, keep, 2);
        keep += __shfl_xor_sync(0xffffffffu, keep, 1);
        if (lane == 0) { rowpart[(size_t)r * rps] = keep; tot += keep; }
        if (lane == 16) { rowpart[(size_t)(r + RP) * rps] = keep; tot += keep; }
    }
    if (r < nrows) {
        const float a0 = UPDATE ? fmaf(ninvN, rsum[r], abase) : 0.f;
        float s0 = 0.f;
        if (h0) s0 += quad_step<UPDATE>(p, a0, c0v, cp0, dmax);
        if (KQ > 1 && h1) s0 += quad_step<UPDATE>(p + mp.QP, a0, c1v, cp1, dmax);
        s0 = warp_sum(s0);
        if (lane == 0) { rowpart[(size_t)r * rps] = s0; tot += s0; }
    }
}

__global__ void __launch_bounds__(kPdbThreads, 1) pdb_kernel(const PdbParams P) {
    extern __shared__ __align__(16) char smem_raw[];
    WaveCtrl* W = P.wave;
    if (ld_relaxed_i32(&W->all_done) != 0 || ld_relaxed_i32(&W->error) != 0) return;
    // a wave planned on the device (dyn) finds its pair count and layout in
    // the wave control block, written by the planner kernel before the launch
    const int npairs = P.dyn ? W->npairs : P.npairs;
    const PdbLayout Lay = P.dyn ? W->layout : P.layout;
    // the per-pair tables are sized for layout.npairs pairs and the layout
    // for the launch's shared memory: a launch outside them would overrun,
    // so every CTA leaves (the same decision everywhere, before any barrier)
    unsigned dyn_smem;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_smem));
    if (npairs > Lay.npairs || Lay.max_segs < 1 || pdb_smem_bytes(Lay, kPdbThreads) > dyn_smem) {
        if (threadIdx.x == 0 && blockIdx.x == 0) atomicCAS(&W->error, 0, FASTPFP_ERR_ARG);
        return;
    }
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const unsigned G = gridDim.x;
    Shared S = carve_b(smem_raw, Lay, nthr);
    int* err = &W->error;
    const unsigned base = W->bar_base;
    unsigned gen = 0u;
    const int RPS = Lay.rp_stride;
    // testing only (debug_flags bit 0): CTA 0 skips its first arrival of the
    // first launch of a solve, so every wait of that launch runs out
    bool skip_first = P.skip_arrive && blockIdx.x == 0 && ld_relaxed_i32(&P.pairs[0].ctrl->outer) == 0;

    // ---- the band -> segments, pair states and per-pair fields
    if (tid == 0) {
        int nseg = 0, brow = 0, soff = 0, coff = 0, tcol = 0;
        const int b0 = P.band_row[blockIdx.x], b1 = P.band_row[blockIdx.x + 1];
        for (int p = 0; p < npairs && nseg < Lay.max_segs; ++p) {
            const PairDesc& d = P.pairs[p];
            const int lo = max(b0, d.row0), hi = min(b1, d.row0 + d.N);
            if (lo >= hi) continue;
            Seg s;
            s.pair = p;
            s.lr0 = lo - d.row0;
            s.nrows = hi - lo;
            s.brow0 = brow;
            s.soff = soff;
            s.coff = coff;
            s.tcol = tcol;
            s.tm = pdb_tmem_rows(s.nrows, d.ldy, nthr, tcol, &s.ntm, &tcol, Lay.two_quad_ties);
            const PdbShape sh = pdb_shape(d.ldy, nthr, Lay.two_quad_ties);
            s.qpg = sh.qpg;
            s.rpkq = 4 * sh.rp + sh.kq;
            S.seg[nseg++] = s;
            brow += s.nrows;
            soff += (s.nrows - s.ntm) * d.ldy;
            coff += d.ldy;
        }
        S.ictl[2] = nseg;
        S.ictl[3] = 0;
        int* qp = S.qpref;
        qp[0] = 0;
        for (int p = 0; p < npairs; ++p) qp[p + 1] = qp[p] + (P.pairs[p].ldy >> 2);
    }
    for (int p = tid; p < npairs; p += nthr) {
        const PairDesc& d = P.pairs[p];
        const int done = ld_relaxed_i32(&d.ctrl->done);
        S.pstate[p] = done ? 0 : 1;
        S.pstop[p] = 0;
        PairS ps;
        ps.colbuf = d.colbuf;
        ps.sbuf = d.sbuf;
        ps.dbuf = d.dbuf;
        ps.N = d.N;
        ps.ldy = d.ldy;
        ps.abase = 0.f;
        ps.bmode = 0;
        ps.invN = 1.0 / (double)d.N;
        ps.invNf = (float)ps.invN;
        ps.cb = 0.f;
        ps.ymax = 0.f;
        ps.sq = Quant64{1.0, 1.0};
        S.pair[p] = ps;
    }
    __syncthreads();
    const int nseg = S.ictl[2];

    // ---- tensor memory: all 512 columns of this SM hold the first rows of
    // every row group (one quad per thread and row); shared memory the rest
    __shared__ uint32_t s_tmem;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (unsigned)__cvta_generic_to_shared(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    // this thread's share: its warp's 32-lane quarter, one of four column blocks
    const uint32_t tme = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(kTmemColsPerThread * (warp >> 2));

    auto slack_mask = [&](float4 v, int c0, int m) {
        if (c0 + 0 >= m) v.x = 0.f;
        if (c0 + 1 >= m) v.y = 0.f;
        if (c0 + 2 >= m) v.z = 0.f;
        if (c0 + 3 >= m) v.w = 0.f;
        return v;
    };

    // ---- prologue: load the band (optional slack reset), with max|y| of
    // every segment for the quanta of the exact input sums below
    for (int si = 0; si < nseg; ++si) {
        const Seg sg = S.seg[si];
        const PairDesc& d = P.pairs[sg.pair];
        if (!(S.pstate[sg.pair] & 1)) continue;
        float ym = 0.f;
        auto absmax = [&ym](float4 v) { ym = fmaxf(ym, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)))); };
        const int Q = d.ldy >> 2, m = d.m;
        const bool reset = P.slack_reset && m < d.N;
        const float4* src = reinterpret_cast<const float4*>(d.Y) + (size_t)sg.lr0 * Q;
        // TMEM rows: thread-row k of the row group is band row grp + RP k
        // (eight float4 loads in flight per thread before any is used)
        if (sg.tm > 0) {
            const Map mp = make_map(sg.qpg, sg.rpkq, tid);
            if (mp.grp < mp.RP) {
                for (int k0 = 0; k0 < sg.tm; k0 += 4) {
                    float4 v[8];   // thread-rows k0 .. k0 + 3, quads j = 0, 1
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int k = k0 + (i >> 1), j = i & 1;
                        const int r = mp.grp + mp.RP * k, q = mp.q0 + j * mp.QP;
                        v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (k < sg.tm && j < mp.kq && r < sg.nrows && q < Q) v[i] = src[(size_t)r * Q + q];
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int k = k0 + (i >> 1), j = i & 1;
                        if (k >= sg.tm || j >= mp.kq) continue;   // warp-uniform
                        const int r = mp.grp + mp.RP * k, q = mp.q0 + j * mp.QP;
                        if (r < sg.nrows && q < Q) {
                            if (reset) v[i] = slack_mask(v[i], 4 * q, m);
                            absmax(v[i]);
                        }
                        tm_st4(tme + sg.tcol + 4 * (mp.kq * k + j), v[i]);
                    }
                }
            }
        }
        // shared-memory rows ntm .. nrows - 1
        const float4* src2 = src + (size_t)sg.ntm * Q;
        float4* dst = reinterpret_cast<float4*>(S.band + sg.soff);
        const int ne = (sg.nrows - sg.ntm) * Q;
        for (int e0 = tid; e0 < ne; e0 += 4 * nthr) {
            float4 v[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (e0 + i * nthr < ne) v[i] = src2[e0 + i * nthr];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int e = e0 + i * nthr;
                if (e >= ne) break;
                if (reset) v[i] = slack_mask(v[i], 4 * (e % Q), m);
                absmax(v[i]);
                dst[e] = v[i];
            }
        }
        ym = warp_max(ym);
        if (lane == 0) S.fred[si * 32 + warp] = ym;
    }
    tm_wait_st();
    __syncthreads();
    if (warp < 2) {
        for (int si = warp; si < nseg; si += 2) {
            const Seg sg = S.seg[si];
            if (!(S.pstate[sg.pair] & 1)) continue;
            float bm = lane < (nthr >> 5) ? S.fred[si * 32 + lane] : 0.f;
            bm = warp_max(bm);
            if (lane == 0 && bm > 0.f) atomicMax(S.pair[sg.pair].dbuf + 3, __float_as_uint(bm));
        }
    }
    grid_arrive(&W->bar);   // waited for at the start of body()

    // One pass over the active segments.  UPDATE = false only sums.  Row
    // partials go to rowpart, per-segment per-warp maxima and totals of the
    // row partials to fred, column partials to the pairs' accumulator `cur`.
    auto pass = [&](auto update_tag, int cur) {
        constexpr bool UPDATE = decltype(update_tag)::value;
        for (int si = 0; si < nseg; ++si) {
            const Seg sg = S.seg[si];
            const int pst = S.pstate[sg.pair];
            if (!(pst & 1) || (pst & 2)) continue;   // inactive or stopped pair
            const PairS pr = S.pair[sg.pair];
            const int N = pr.N, Q = pr.ldy >> 2;
            const Map mp = make_map(sg.qpg, sg.rpkq, tid);
            const bool in_grp = mp.grp < mp.RP;
            // b = -c_j / N of this thread's column quads (the column term of
            // P1), -kPadB on padding columns
            float4 c0v = make_float4(0.f, 0.f, 0.f, 0.f), c1v = c0v;
            if (UPDATE && in_grp) {
                const float4* cN = reinterpret_cast<const float4*>(S.cN + sg.coff);
                const float ni = -1.0f / (float)N;
                auto scale = [ni, N](float4 v, int c) {
                    return make_float4(ni * v.x, c + 1 < N ? ni * v.y : -kPadB, c + 2 < N ? ni * v.z : -kPadB,
                                       c + 3 < N ? ni * v.w : -kPadB);
                };
                if (mp.q0 < Q) c0v = scale(cN[mp.q0], 4 * mp.q0);
                if (mp.kq > 1 && mp.q0 + mp.QP < Q) c1v = scale(cN[mp.q0 + mp.QP], 4 * (mp.q0 + mp.QP));
            }
            float4 cp0 = make_float4(0.f, 0.f, 0.f, 0.f), cp1 = cp0;
            float dmax = 0.f;
            float tot = 0.f;   // this lane's share of the warp's row partials of the segment
            if (in_grp) {
                const int wig = (tid % mp.QP) >> 5;
                float4* bp = reinterpret_cast<float4*>(S.band + sg.soff);
                float* rp = S.rowpart + (size_t)sg.brow0 * RPS + wig;
                const float* rs = S.rsum + sg.brow0;
                const float ninvN = -1.0f / (float)N;
                if (sg.tm > 0 && mp.kq == 1)
                    seg_rows_tmem<UPDATE>(tme + sg.tcol, sg.tm, sg.nrows, Q, N, mp, lane, rs, pr.abase, rp, RPS,
                                          c0v, ninvN, cp0, dmax, tot);
                else if (sg.tm > 0)
                    seg_rows_tmem2<UPDATE>(tme + sg.tcol, sg.tm, sg.nrows, Q, N, mp, lane, rs, pr.abase, rp, RPS,
                                           c0v, c1v, ninvN, cp0, cp1, dmax, tot);
                // rows ntm .. nrows - 1 (ntm is a multiple of RP, so row groups line up)
                const int ns = sg.nrows - sg.ntm;
                if (mp.kq == 1)
                    seg_rows<UPDATE, 1>(bp, ns, Q, N, mp, nthr, lane, rs + sg.ntm, pr.abase,
                                        rp + (size_t)sg.ntm * RPS, RPS, c0v, c1v, ninvN, cp0, cp1, dmax, tot);
                else
                    seg_rows<UPDATE, 2>(bp, ns, Q, N, mp, nthr, lane, rs + sg.ntm, pr.abase,
                                        rp + (size_t)sg.ntm * RPS, RPS, c0v, c1v, ninvN, cp0, cp1, dmax, tot);
            }
            if (UPDATE) tm_wait_st();
            dmax = warp_max(dmax);
            tot = warp_sum(tot);
            if (lane == 0) {
                S.fred[si * 32 + warp] = dmax;
                S.fred[si * 32 + 16 + warp] = tot;
            }
            // column partials: every row group adds its own (L2 folds the row
            // groups; no block-wide fold, no barrier), rounded to the column's
            // quantum so that the sums are exact in any order
            if (UPDATE && in_grp) {
                // the pass's output is >= 0, so column j's new sum is at most
                // c_j + 1 + s/N (previous round's c_j, s) or, after the input
                // round, the pair's bound cb (set in wait_post); one quantum
                // serves the thread's columns, from the largest of their bounds
                float bnd = pr.cb;
                if (!pr.bmode) {
                    const float4* cNq = reinterpret_cast<const float4*>(S.cN + sg.coff);
                    float cm = 0.f;
                    if (mp.q0 < Q) {
                        const float4 c = cNq[mp.q0];
                        cm = fmaxf(fmaxf(c.x, c.y), fmaxf(c.z, c.w));
                    }
                    if (mp.kq > 1 && mp.q0 + mp.QP < Q) {
                        const float4 c = cNq[mp.q0 + mp.QP];
                        cm = fmaxf(cm, fmaxf(fmaxf(c.x, c.y), fmaxf(c.z, c.w)));
                    }
                    bnd = fmaf(cm, kBoundMargin, pr.cb);
                }
                const Quant32 u = quant32_for(bnd);
                float* acc = pr.colbuf + (size_t)cur * pr.ldy;
                if (mp.q0 < Q) {
                    cp0 = quant32x4(cp0, u, u, u, u);
                    red_add_v4(acc + 4 * mp.q0, cp0.x, cp0.y, cp0.z, cp0.w);
                }
                if (mp.kq > 1 && mp.q0 + mp.QP < Q) {
                    cp1 = quant32x4(cp1, u, u, u, u);
                    red_add_v4(acc + 4 * (mp.q0 + mp.QP), cp1.x, cp1.y, cp1.z, cp1.w);
                }
            } else if (in_grp) {
                // the input's column sums in FP64: every partial is at most
                // N max|y| in magnitude
                const Quant64 q0 = quant64_for((double)N * (double)pr.ymax * (double)kBoundMargin);
                double* acc = colbuf64(pr.colbuf, pr.ldy);
                auto add4 = [&](float4 v, int q) {
                    double* a = acc + 4 * (size_t)q;
                    red_add_f64(a + 0, quant64((double)v.x, q0));
                    red_add_f64(a + 1, quant64((double)v.y, q0));
                    red_add_f64(a + 2, quant64((double)v.z, q0));
                    red_add_f64(a + 3, quant64((double)v.w, q0));
                };
                if (mp.q0 < Q) add4(cp0, mp.q0);
                if (mp.kq > 1 && mp.q0 + mp.QP < Q) add4(cp1, mp.q0 + mp.QP);
            }
        }
        // every warp's partials are in (publish folds them)
        __syncthreads();
    };

    // Zero accumulator `which` of the wave's pairs with threads t of nt
    // (which == 3: the FP64 input sums and the input's max|y|).  The column
    // quads are numbered consecutively over the pairs and dealt round-robin
    // over the CTAs, so every CTA zeroes about the same few.
    auto clear_acc = [&](int which, int t, int nt) {
        const int np = npairs;
        const int* qp = S.qpref;
        const int total = qp[np];
        for (int f = t * (int)G + (int)blockIdx.x; f < total; f += nt * (int)G) {
            int lo = 0, hi = np;   // the pair whose quads hold f: qp[lo] <= f < qp[lo + 1]
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (qp[mid] <= f) lo = mid; else hi = mid;
            }
            const PairS& pr = S.pair[lo];
            const int q = f - qp[lo];
            if (which == 3) {
                double2* a = reinterpret_cast<double2*>(colbuf64(pr.colbuf, pr.ldy)) + 2 * (size_t)q;
                a[0] = make_double2(0.0, 0.0);
                a[1] = make_double2(0.0, 0.0);
                if (q == 0) pr.dbuf[3] = 0u;
                continue;
            }
            reinterpret_cast<float4*>(pr.colbuf + (size_t)which * pr.ldy)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (q == 0) {
                pr.sbuf[which] = 0.0;
                pr.dbuf[which] = 0u;
            }
        }
    };

    // The row sum of band row r: its row group's per-warp partials, in order.
    auto row_sum = [&](const Seg& sg, int nw, int r) {
        const float* rpp = S.rowpart + (size_t)(sg.brow0 + r) * RPS;
        float t = 0.f;
        if ((RPS & 3) == 0) {   // float4 loads (rows 16-byte aligned), the same order of additions
            for (int w = 0; w < nw; w += 4) {
                const float4 v = *reinterpret_cast<const float4*>(rpp + w);
                t += v.x;
                if (w + 1 < nw) t += v.y;
                if (w + 2 < nw) t += v.z;
                if (w + 3 < nw) t += v.w;
            }
            return t;
        }
        for (int w = 0; w < nw; ++w) t += rpp[w];
        return t;
    };

    // End of a pass (every warp's partials in): warps 0 and 1 publish the
    // segments' totals and round maxima (alternate segments) while warps
    // 2.. fold the row sums for the next pass.  A band's total is the sum, in a fixed order, of the
    // per-warp totals of the row partials the pass stored (FP32), and is
    // accumulated over the CTAs in FP64.
    auto publish = [&](int cur) {
        if (tid == 0) S.ictl[4] = 0;   // the running-pair count of wait_post
        if (warp < 2) {
            for (int si = warp; si < nseg; si += 2) {
                const Seg sg = S.seg[si];
                const int pst = S.pstate[sg.pair];
                if (!(pst & 1) || (pst & 2)) continue;
                float sp = lane < (nthr >> 5) ? S.fred[si * 32 + 16 + lane] : 0.f;
                float bm = lane < (nthr >> 5) ? S.fred[si * 32 + lane] : 0.f;
                sp = warp_sum(sp);
                bm = warp_max(bm);
                if (lane == 0) {
                    const PairS& pr = S.pair[sg.pair];
                    atomicAdd(pr.sbuf + cur, quant64_of_f32(sp, pr.sq));
                    if (bm > 0.f) atomicMax(pr.dbuf + cur, __float_as_uint(bm));
                }
            }
        } else {
            for (int si = 0; si < nseg; ++si) {
                const Seg sg = S.seg[si];
                const int pst = S.pstate[sg.pair];
                if (!(pst & 1) || (pst & 2)) continue;
                const int nw = sg.qpg >> 5;
                for (int r = tid - 64; r < sg.nrows; r += nthr - 64) S.rsum[sg.brow0 + r] = row_sum(sg, nw, r);
            }
        }
        if (skip_first) {   // fault-injection test: this arrival is lost
            skip_first = false;
            __syncthreads();
        } else {
            grid_arrive(&W->bar);
        }
    };

    // Wait for the barrier of pass `cur` (round u), then take every pair's
    // stop decision (identical in every CTA), load the column sums c_j of the
    // segments and turn the new totals into the next row-offset bases
    // 1/N + s/N^2.
    auto wait_post = [&](int cur, int u, bool check_stop) -> bool {
        const unsigned target = base + G * (gen + 1u);
        if (!grid_wait(&W->bar, target, err, P.timeout_ns)) return false;
        ++gen;
        // the running pairs' totals and maxima first (one pair per thread of
        // the first four warps): their L2 round trip heads the chain below
        double s_pre = 0.0;
        unsigned d_pre = 0u;
        if (tid < 128 && tid < npairs) {
            const int ps = S.pstate[tid];
            if ((ps & 1) && !(ps & 2)) {
                s_pre = __ldcg(S.pair[tid].sbuf + cur);
                d_pre = __ldcg(S.pair[tid].dbuf + cur);
            }
        }
        // every segment's column sums in flight at once (copied, not loaded
        // and stored, so no segment waits for the previous one's latency);
        // the input's sums (u = 0) are FP64 and converted here
        for (int si = 0; si < nseg; ++si) {
            const Seg sg = S.seg[si];
            const int pst = S.pstate[sg.pair];
            if (!(pst & 1) || (pst & 2)) continue;
            const PairS pr = S.pair[sg.pair];
            float4* dst = reinterpret_cast<float4*>(S.cN + sg.coff);
            if (u == 0) {
                const double2* c = reinterpret_cast<const double2*>(colbuf64(pr.colbuf, pr.ldy));
                for (int q = tid; q < (pr.ldy >> 2); q += nthr) {
                    const double2 a = __ldcg(c + 2 * q), b = __ldcg(c + 2 * q + 1);
                    dst[q] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
                }
                continue;
            }
            const float4* c = reinterpret_cast<const float4*>(pr.colbuf + (size_t)cur * pr.ldy);
            for (int q = tid; q < (pr.ldy >> 2); q += nthr) cp_async_cg16(dst + q, c + q);
        }
        // the pairs, one per thread of the first four warps (totals and
        // maxima loaded above)
        int any = 0;
        for (int p = tid; p < npairs && tid < 128; p += 128) {
            int ps = S.pstate[p];
            if ((ps & 1) && !(ps & 2)) {
                PairS& pr = S.pair[p];
                const double s = p == tid ? s_pre : __ldcg(pr.sbuf + cur);
                const float dd = __uint_as_float(p == tid ? d_pre : __ldcg(pr.dbuf + cur));
                const double invN = pr.invN;
                pr.abase = (float)(invN + s * invN * invN);
                if (!f64_is_finite(s)) S.ictl[3] = 1;
                // bounds of the next pass's sums (its output is >= 0): after
                // the input, every column sum is at most 4 N max|y| + 1 (the
                // input, the row offsets and the column offset of P1 are each
                // at most N max|y| per column); after a round, column j's at
                // most c_j + 1 + s/N and the total at most 2 s + N
                // (FP32 bounds: the margin covers their rounding)
                const float mg = kBoundMargin, Nf = (float)pr.N, sf = f64_to_f32_rn(s);
                if (u == 0) {
                    const float b1 = fmaf(4.0f * Nf, pr.ymax, 1.0f) * mg;
                    pr.bmode = 1;
                    pr.cb = b1;
                    pr.sq = quant64_for_f(b1 * Nf * mg);
                } else {
                    pr.bmode = 0;
                    pr.cb = fmaf(sf, pr.invNf, 1.0f) * mg;
                    pr.sq = quant64_for_f(fmaf(2.0f, sf, Nf) * (mg * mg));
                }
                if (check_stop && (dd < P.tol_inner_f || u >= P.max_inner)) {
                    ps |= 2;
                    S.pstop[p] = u;
                }
                S.pstate[p] = ps;
                any |= !(ps & 2);
            }
        }
        // Accumulator (u + 2) % 3, which round u + 2 adds into, was last read
        // (column sums, total, maximum) in every CTA's wait_post of round
        // u - 1, before its arrival at the barrier just passed: the threads
        // the pair loop leaves idle zero it now, so the stores are done long
        // before this CTA's next arrival (a release, which would wait for
        // them) and visible before any CTA's round u + 2 reductions.
        if (tid >= 128) clear_acc((u + 2) % 3, tid - 128, nthr - 128);
        // ictl[4] counts the warps that still have a running pair (zeroed in publish)
        any = __any_sync(0xffffffffu, any);
        if (warp < 4 && lane == 0 && any) atomicAdd(&S.ictl[4], 1);
        cp_async_wait_all();
        __syncthreads();
        return true;
    };

    // Everything from here until the tensor memory is released; a timeout or
    // a non-finite total leaves it early (all threads of the CTA together).
    auto body = [&]() {
    // ---- max|y| of every pair's input (the prologue's barrier), the
    // quantum of the input's total, then the exact sums of the input
    if (!grid_wait(&W->bar, base + G * (gen + 1u), err, P.timeout_ns)) return;
    ++gen;
    for (int p = tid; p < npairs; p += nthr) {
        if (!(S.pstate[p] & 1)) continue;
        PairS& pr = S.pair[p];
        pr.ymax = __uint_as_float(__ldcg(pr.dbuf + 3));
        const double N = (double)pr.N;
        pr.sq = quant64_for(N * N * (double)pr.ymax * (double)kBoundMargin);   // |s| <= N^2 max|y|
    }
    __syncthreads();
    pass(std::false_type{}, 0);
    publish(0);
    if (!wait_post(0, 0, false)) return;
    if (S.ictl[3]) {
        if (tid == 0) atomicCAS(err, 0, FASTPFP_ERR_NONFINITE);
        return;
    }
    bool act = S.ictl[4] != 0;

    // ---- the rounds
    int u = 0;
    while (act) {
        ++u;
        pass(std::true_type{}, u % 3);
        publish(u % 3);
        if (!wait_post(u % 3, u, true)) return;
        act = S.ictl[4] != 0;
    }

    // ---- the band back to Y, every column: the slack columns carry over to
    // the next outer iteration, the first m feed the blend below
    for (int si = 0; si < nseg; ++si) {
        const Seg sg = S.seg[si];
        if (!(S.pstate[sg.pair] & 1)) continue;
        const PairDesc& d = P.pairs[sg.pair];
        const int Q = d.ldy >> 2;
        float4* Yg = reinterpret_cast<float4*>(d.Y) + (size_t)sg.lr0 * Q;
        if (sg.tm > 0) {
            const Map mp = make_map(sg.qpg, sg.rpkq, tid);
            if (mp.grp < mp.RP) {
                for (int k = 0; k < sg.tm; ++k) {
                    const int r = mp.grp + mp.RP * k;
                    for (int j = 0; j < mp.kq; ++j) {
                        const int q = mp.q0 + j * mp.QP;
                        const float4 v = tm_ld4(tme + sg.tcol + 4 * (mp.kq * k + j));
                        if (r < sg.nrows && q < Q) Yg[(size_t)r * Q + q] = v;
                    }
                }
            }
        }
        const float4* band = reinterpret_cast<const float4*>(S.band + sg.soff);
        float4* dst = Yg + (size_t)sg.ntm * Q;
        for (int e = tid; e < (sg.nrows - sg.ntm) * Q; e += nthr) dst[e] = band[e];
    }
    __syncthreads();

    // ---- blend and normalise every active pair
    const float alpha = P.alpha, beta = 1.0f - P.alpha;
    if (P.normalize) {
        for (int si = 0; si < nseg; ++si) {
            const Seg sg = S.seg[si];
            if (!(S.pstate[sg.pair] & 1)) continue;
            const PairDesc& d = P.pairs[sg.pair];
            const int Qy = d.ldy >> 2, Qx = d.ldx >> 2, m = d.m;
            const float4* Yg = reinterpret_cast<const float4*>(d.Y) + (size_t)sg.lr0 * Qy;
            const float4* X = reinterpret_cast<const float4*>(d.X) + (size_t)sg.lr0 * Qx;
            float lmax = -INFINITY;
            const int dr = nthr / Qx, dq = nthr % Qx;
            int r = tid / Qx, q = tid % Qx;
            while (r < sg.nrows) {
                int qk[kBlendLoads];
                float4 xk[kBlendLoads], yk[kBlendLoads];
#pragma unroll
                for (int k = 0; k < kBlendLoads; ++k) {
                    qk[k] = r < sg.nrows ? q : -1;
                    if (r < sg.nrows) { xk[k] = X[(size_t)r * Qx + q]; yk[k] = Yg[(size_t)r * Qy + q]; }
                    r += dr; q += dq;
                    if (q >= Qx) { q -= Qx; ++r; }
                }
#pragma unroll
                for (int k = 0; k < kBlendLoads; ++k) {
                    if (qk[k] < 0) break;
                    const float4 x = xk[k], y = yk[k];
                    const int c0 = 4 * qk[k];
                    lmax = fmaxf(lmax, beta * x.x + alpha * y.x);
                    if (c0 + 1 < m) lmax = fmaxf(lmax, beta * x.y + alpha * y.y);
                    if (c0 + 2 < m) lmax = fmaxf(lmax, beta * x.z + alpha * y.z);
                    if (c0 + 3 < m) lmax = fmaxf(lmax, beta * x.w + alpha * y.w);
                }
            }
            lmax = warp_max(lmax);
            if (lane == 0) S.fred[si * 32 + warp] = lmax;
        }
        __syncthreads();
        if (warp == 0) {
            for (int si = 0; si < nseg; ++si) {
                const Seg sg = S.seg[si];
                if (!(S.pstate[sg.pair] & 1)) continue;
                float bm = lane < (nthr >> 5) ? S.fred[si * 32 + lane] : -INFINITY;
                bm = warp_max(bm);
                if (lane == 0) atomicMax(&P.pairs[sg.pair].ctrl->xmax_bits, float_to_ordered(bm));
            }
        }
        grid_arrive(&W->bar);
        if (!grid_wait(&W->bar, base + G * (gen + 1u), err, P.timeout_ns)) return;
        ++gen;
    }
    for (int si = 0; si < nseg; ++si) {
        const Seg sg = S.seg[si];
        if (!(S.pstate[sg.pair] & 1)) continue;
        const PairDesc& d = P.pairs[sg.pair];
        const int Qy = d.ldy >> 2, Qx = d.ldx >> 2, m = d.m;
        const float mx = P.normalize ? ordered_to_float(__ldcg(&d.ctrl->xmax_bits)) : 1.0f;
        const float4* Yg = reinterpret_cast<const float4*>(d.Y) + (size_t)sg.lr0 * Qy;
        float4* X = reinterpret_cast<float4*>(d.X) + (size_t)sg.lr0 * Qx;
        __nv_bfloat16* Xt16 = d.Xt16;
        const int ldxt = d.ldxt;
        AbsDiffMax dxm;   // max|dX| in FP64, as the oracle takes it
        const int dr = nthr / Qx, dq = nthr % Qx;
        int rn = tid / Qx, qn = tid % Qx;
        while (rn < sg.nrows) {
            int rk[kBlendLoads], qk[kBlendLoads];
            float4 xk[kBlendLoads], yk[kBlendLoads];
#pragma unroll
            for (int k = 0; k < kBlendLoads; ++k) {
                rk[k] = rn;
                qk[k] = qn;
                if (rn < sg.nrows) { xk[k] = X[(size_t)rn * Qx + qn]; yk[k] = Yg[(size_t)rn * Qy + qn]; }
                rn += dr; qn += dq;
                if (qn >= Qx) { qn -= Qx; ++rn; }
            }
#pragma unroll
            for (int k = 0; k < kBlendLoads; ++k) {
                const int r = rk[k], q = qk[k];
                if (r >= sg.nrows) break;
                const float4 x = xk[k], y = yk[k];
                float4 v = make_float4(beta * x.x + alpha * y.x, beta * x.y + alpha * y.y,
                                       beta * x.z + alpha * y.z, beta * x.w + alpha * y.w);
                if (P.normalize) { v.x /= mx; v.y /= mx; v.z /= mx; v.w /= mx; }
                const int c0 = 4 * q;
                if (c0 + 4 > m) {
                    if (c0 + 1 >= m) v.y = 0.f;
                    if (c0 + 2 >= m) v.z = 0.f;
                    if (c0 + 3 >= m) v.w = 0.f;
                }
                dxm.add4(v, x);
                X[(size_t)r * Qx + q] = v;
                if (Xt16) {
                    const int i = sg.lr0 + r;
                    Xt16[(size_t)c0 * ldxt + i] = __float2bfloat16_rn(v.x);
                    if (c0 + 1 < m) Xt16[(size_t)(c0 + 1) * ldxt + i] = __float2bfloat16_rn(v.y);
                    if (c0 + 2 < m) Xt16[(size_t)(c0 + 2) * ldxt + i] = __float2bfloat16_rn(v.z);
                    if (c0 + 3 < m) Xt16[(size_t)(c0 + 3) * ldxt + i] = __float2bfloat16_rn(v.w);
                }
            }
        }
        // per-warp max|dX| of the segment, folded at L2 by the atomic
        const double dx = warp_max_d(dxm.value());
        if (lane == 0 && dx > 0.0) atomicMax(&d.ctrl->dx_bits, (unsigned long long)__double_as_longlong(dx));
    }
    grid_arrive(&W->bar);
    if (!grid_wait(&W->bar, base + G * (gen + 1u), err, P.timeout_ns)) return;
    ++gen;

    // ---- per-pair loop control, accumulator clean-up
    for (int b = 0; b < 4; ++b) clear_acc(b, tid, nthr);
    if (blockIdx.x == 0) {
        for (int p = tid; p < npairs; p += nthr) {
            if (!(S.pstate[p] & 1)) continue;
            Ctrl* C = P.pairs[p].ctrl;
            const int ui = S.pstop[p];
            const double d = __longlong_as_double((long long)__ldcg(&C->dx_bits));
            if (!isfinite(d)) atomicCAS(err, 0, FASTPFP_ERR_NONFINITE);
            C->dx_bits = 0ull;
            C->xmax_bits = 0u;
            const int t = C->outer;
            if (t < kMaxOuterTrace) {
                C->inner_trace[t] = ui;
                C->delta_trace[t] = d;
            }
            C->outer = t + 1;
            C->inner_total += ui;
            C->inner_max = max(C->inner_max, ui);
            C->last_inner = ui;
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
        }
        __syncthreads();
        if (tid == 0) {
            int all = 1;
            for (int p = 0; p < npairs; ++p) all &= (P.pairs[p].ctrl->done != 0);
            W->all_done = all;
            W->bar_base = base + G * gen;
        }
    }
    };
    body();

    // ---- release the tensor memory (every TMEM access of the CTA is complete)
    tm_wait_st();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

cudaError_t pdb_configure() {
    return cudaFuncSetAttribute((const void*)pdb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kPdMaxSmem);
}

cudaError_t pdb_launch(const PdbParams& P, int grid, size_t smem, cudaStream_t s) {
    void* args[] = {const_cast<PdbParams*>(&P)};
    // Every CTA allocates all 512 TMEM columns, so two CTAs must never share
    // an SM (the second's allocation would wait for the first, which waits
    // at the grid barrier): more than half an SM's shared memory per CTA
    // guarantees one CTA per SM whatever the band needs.
    const size_t one_per_sm = 120 * 1024;
    return cudaLaunchCooperativeKernel((const void*)pdb_kernel, dim3(grid), dim3(kPdbThreads), args,
                                       smem > one_per_sm ? smem : one_per_sm, s);
}

}  // namespace fpfp
