// fastpfp_api.cu -- the C ABI declared in include/fastpfp.h.
//
// A handle owns every device buffer the solver touches, allocated once in
// fastpfp_create: one "slot" of per-pair scratch (Y, X, T, K, accumulators,
// control block, discretisation buffers) for each pair that can be solved at
// the same time, sized for graphs of up to max_n nodes.
//
// Pairs run Algorithm 1 in waves: pairs whose slacked matrices fit on chip
// together (TMEM + shared memory of all SMs) share one cooperative launch of
// pdb_kernel per outer iteration, which runs every P1/P2 round of every pair
// with one grid barrier per round, blends, normalises and decides on the
// device whether each pair's loop continues; the pairs' gradient products
// are grouped launches.  A lone pair is a wave of one.  A batch larger than
// one wave is streamed (solve_stream): finished pairs leave and waiting pairs
// enter between outer iterations.  A pair too large for any wave runs
// through pd_kernel, which streams its band through L2.
//
// The repeat loop of Algorithm 1 runs in one of two ways.  By default one
// outer iteration is captured into the body of a CUDA-graph while node whose
// condition a one-thread kernel sets after every iteration from the device
// stop word, so a solve (or wave) is one graph launch with no host round
// trip until its end.  With loop_mode = 1 (and always with profile = 1) the
// host enqueues outer iterations in chunks and checks, one chunk behind so
// the GPU never idles, whether every pair has stopped; launches after a
// pair's stop return at once.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "band_plan.cuh"
#include "common.cuh"
#include "internal.h"

using namespace fpfp;

namespace {

constexpr int kMaxN = 16384;     // four float4 column quads per thread of a 1024-thread CTA
constexpr int kMaxK = 256;       // attribute dimension staged by fastpfp_match_host
constexpr size_t kCtrlHeader = offsetof(Ctrl, inner_trace);
constexpr int kProfIters = 128;                   // outer iterations timed when profile = 1
constexpr int kProfEvents = 2 * kProfIters + 3;   // iteration boundaries + discretisation
constexpr int kChunk = 4;                         // outer iterations enqueued between checks
constexpr size_t kTraceBytes = (size_t)kMaxOuterTrace * (sizeof(int) + sizeof(double));

inline int round4(int x) { return (x + 3) & ~3; }
inline int round8(int x) { return (x + 7) & ~7; }   // BF16 rows: 16-byte TMA strides
inline int round16(int x) { return (x + 15) & ~15; }   // E4M3 rows: 16-byte TMA strides
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Per-pair device scratch.
struct Slot {
    float *Y, *X, *T, *K;
    __nv_bfloat16 *A16, *A216, *Xt16, *T16;
    float* colbuf;
    double* sbuf;
    unsigned* dbuf;
    Ctrl* ctrl;
    DiscBuffers disc;
    // device staging of host-memory inputs and outputs (the *_host calls)
    float *sA, *sA2, *sB, *sB2, *sX0, *sXout;
    int32_t* sperm;
    // 16-byte-row copies of A and A' for the FP32 products when the caller's
    // rows are not 16-byte aligned
    float *A32, *A232;
    // FP8 products: E4M3 copies of A, A', X^T and T (leading dimension
    // round16 of the row length) and their per-row scales
    uint8_t *qA, *qA2, *qXt, *qT;
    float *scA, *scA2, *scX, *scT;
    // FP32 products on the tensor cores: TF32 parts and FP32 remainders of
    // A, A' (once per solve), X^T (per iteration) and T (the first product's
    // output), rows padded to multiples of 4 floats
    float *Ahi, *Alo, *A2hi, *A2lo, *Xthi, *Xtlo, *Thi, *Tlo;
};

}  // namespace

struct fastpfp_s {
    int device = 0, max_n = 0, max_batch = 0, num_sms = 0, ld = 0, nslots = 0;
    char* pool = nullptr;
    size_t pool_bytes = 0;
    std::vector<Slot> slots;
    // wave tables (device) and their pinned staging
    PairDesc* d_pairs = nullptr;
    int* d_band = nullptr;
    WaveCtrl* d_wave = nullptr;
    PairDesc* h_pairs = nullptr;
    int* h_band = nullptr;
    int* h_done = nullptr;       // pinned, 2 x 4 words: stop flags read one chunk behind
    Ctrl* host_ctrl = nullptr;   // pinned, max_batch control-block headers
    int last_count = 0;          // pairs of the last call; their traces are in trace_store
    char* trace_store = nullptr; // device, max_batch x kTraceBytes: per-pair inner counts and deltas
    int* d_flags = nullptr;      // device, kMaxWavePairs + 1 stop/error words of a streamed wave
    int* h_flags = nullptr;      // pinned copy of d_flags
    // a batch streamed inside one graph: per-pair wave-table templates and
    // the device planner's state (device), with pinned staging
    PairDesc* d_tmpl = nullptr;
    PairDesc* h_tmpl = nullptr;
    StreamState* d_stream = nullptr;
    StreamState* h_stream = nullptr;
    int host_syncs = 0;          // host synchronisations of the current call
    // FastGA: the N x N scratch of its normalisation (allocated on first use)
    float* ga_z = nullptr;

    cudaEvent_t ev[kProfEvents] = {};
    cudaEvent_t chunk_ev[2] = {};
    // graph-controlled outer loop: a capture stream, the loop's iteration
    // counter (device), and the graphs of the current call, released after
    // the call has synchronised
    cudaStream_t cap = nullptr;
    int* d_loop = nullptr;
    int loop_body = 0;          // kernels per iteration of the last graph loop (0: host loop)
    std::vector<cudaGraph_t> graphs;
    std::vector<cudaGraphExec_t> execs;
    // tile shapes of the gradient products per size and count class
    int tile_f32[FASTPFP_TUNE_SIZES][FASTPFP_TUNE_COUNTS];
    int tile_tc[FASTPFP_TUNE_SIZES][FASTPFP_TUNE_COUNTS];
    // learned warm start: features, activations, embeddings and gradients of
    // both graphs (big = canonical rows, small = columns)
    struct {
        float *Fb, *Fs, *Hb, *Hs, *Eb, *Es, *Eb8, *Es8, *EsT, *dEb, *dEs, *dH, *grad, *scalar;
        float *lse_c, *lse_r;
        float2* part;
        int32_t *t, *tinv;
        double* loss;
    } ws{};
};

namespace {

// Size class of a canonical N (2^(c+6) < N <= 2^(c+7)) and count class of a
// group of pairs, the indices of the handle's tile table.
int size_class(int N) {
    int c = 0;
    for (int u = 128; u < N && c < FASTPFP_TUNE_SIZES - 1; u <<= 1) ++c;
    return c;
}
int count_class(int count) { return count <= 1 ? 0 : count <= 4 ? 1 : count <= 16 ? 2 : 3; }
constexpr int kCountClassHi[FASTPFP_TUNE_COUNTS] = {1, 4, 16, 32};
int f32_tile(fastpfp_t h, int N, int count) { return h->tile_f32[size_class(N)][count_class(count)]; }
int tc_tile(fastpfp_t h, int N, int count) { return h->tile_tc[size_class(N)][count_class(count)]; }

#define FP_CUDA(x)                                         \
    do {                                                   \
        cudaError_t e_ = (x);                              \
        if (e_ != cudaSuccess) return FASTPFP_ERR_CUDA;    \
    } while (0)

bool params_ok(const fastpfp_params* p) {
    if (!p) return false;
    if (!(p->alpha >= 0.f && p->alpha <= 1.f)) return false;
    if (!(p->lambda >= 0.f) || !isfinite(p->lambda)) return false;
    if (p->max_outer < 1 || p->max_inner < 1) return false;
    if (p->max_outer > kMaxOuterTrace) return false;
    if (!(p->tol_outer >= 0.0) || !(p->tol_inner >= 0.0)) return false;
    if (p->precision != FASTPFP_FP32 && p->precision != FASTPFP_BF16 && p->precision != FASTPFP_FP8 &&
        p->precision != FASTPFP_FP32_SIMT)
        return false;
    if (p->refine_iters < 0) return false;
    if (p->loop_mode != 0 && p->loop_mode != 1) return false;
    if (p->algorithm != FASTPFP_ALG_FASTPFP && p->algorithm != FASTPFP_ALG_PG &&
        p->algorithm != FASTPFP_ALG_FASTGA)
        return false;
    if (p->algorithm == FASTPFP_ALG_FASTGA) {   // FP32 products; a positive, finite beta
        if (p->precision != FASTPFP_FP32 && p->precision != FASTPFP_FP32_SIMT) return false;
        if (!(p->beta > 0.f) || !isfinite(p->beta)) return false;
    }
    return true;
}

// A BF16 or FP8 phase before the FP32 iterations.
inline bool lowp_of(const fastpfp_params* p) {
    return p->precision == FASTPFP_BF16 || p->precision == FASTPFP_FP8;
}
// The FP32 phase's products on the FP32 FMA pipes instead of split TF32 on
// the tensor cores.
inline bool simt_of(const fastpfp_params* p) { return p->precision == FASTPFP_FP32_SIMT; }

long long timeout_ns(const fastpfp_params* p) {
    const int ms = (p && p->timeout_ms > 0) ? p->timeout_ms : 2000;
    return (long long)ms * 1000000ll;
}

// Arguments of one solve in canonical orientation (N >= m).
struct Problem {
    const float *A, *A2, *B, *B2;
    int N, m, k;
    int transposed;
    const float* X0;     // caller orientation
    int32_t* perm_out;   // caller orientation
    float* X_out;        // caller orientation
};

int check_pair(fastpfp_t h, const float* A, int n_a, const float* A2, int n_b, const float* B,
               const float* B2, int k, const fastpfp_params* p, int32_t* perm_out) {
    if (!h || !A || !A2 || !perm_out || !params_ok(p)) return FASTPFP_ERR_ARG;
    if (n_a < 1 || n_b < 1 || k < 0 || k > kMaxK) return FASTPFP_ERR_ARG;
    if (k > 0 && p->lambda != 0.f && (!B || !B2)) return FASTPFP_ERR_ARG;
    if (n_a > h->max_n || n_b > h->max_n) return FASTPFP_ERR_SIZE;
    return FASTPFP_OK;
}

Problem canonical(const float* A, int n_a, const float* A2, int n_b, const float* B,
                  const float* B2, int k, float lambda, const float* X0, int32_t* perm_out,
                  float* X_out) {
    Problem q;
    q.transposed = n_a < n_b;
    q.A = q.transposed ? A2 : A;
    q.A2 = q.transposed ? A : A2;
    q.B = q.transposed ? B2 : B;
    q.B2 = q.transposed ? B : B2;
    q.N = q.transposed ? n_b : n_a;
    q.m = q.transposed ? n_a : n_b;
    q.k = (k > 0 && lambda != 0.f) ? k : 0;
    q.X0 = X0;
    q.perm_out = perm_out;
    q.X_out = X_out;
    return q;
}

// ---- the per-pair pieces of a solve ---------------------------------------

// An n x n adjacency as an operand of the FP32 products: the caller's
// matrix when its rows start on 16-byte boundaries, else the padded copy
// made by enqueue_setup.
inline bool rows16(const float* p, int n) { return ((uintptr_t)p & 15u) == 0 && (n & 3) == 0; }
inline const float* f32_operand(const float* A, int n, float* padded, int* ld) {
    if (rows16(A, n)) {
        *ld = n;
        return A;
    }
    *ld = round4(n);
    return padded;
}


// Control block, accumulators and Y cleared; K and the initial X written.
// A solve that stopped on an error may leave the accumulators dirty, so every
// solve starts from cleared ones.  Returns the kernels launched or < 0.
int enqueue_setup(const Slot& sl, cudaStream_t s, const Problem& q, const fastpfp_params* p,
                  int ld) {
    const int ldy = round4(q.N), ldx = round4(q.m);
    const bool lowp = lowp_of(p);   // a BF16 or FP8 phase
    FP_CUDA(cudaMemsetAsync(sl.ctrl, 0, kCtrlHeader, s));
    FP_CUDA(cudaMemsetAsync(sl.colbuf, 0, colbuf_bytes(ld), s));
    FP_CUDA(cudaMemsetAsync(sl.sbuf, 0, 3 * sizeof(double), s));
    FP_CUDA(cudaMemsetAsync(sl.dbuf, 0, kDbufWords * sizeof(unsigned), s));
    FP_CUDA(cudaMemsetAsync(sl.Y, 0, (size_t)q.N * ldy * sizeof(float), s));
    FP_CUDA(init_ctrl(sl.ctrl, lowp ? 1 : 0, s));
    int nl = 2;
    if (q.k > 0) {
        FP_CUDA(affinity(q.B, q.B2, q.N, q.m, q.k, sl.K, ldx, s));
        ++nl;
    }
    FP_CUDA(init_x(sl.X, q.N, q.m, ldx, q.X0, q.transposed, lowp ? sl.Xt16 : nullptr, round8(q.N), s));
    // 16-byte rows of A and A' for the FP32 products (only when the caller's are not)
    if (!rows16(q.A, q.N))
        FP_CUDA(cudaMemcpy2DAsync(sl.A32, (size_t)round4(q.N) * 4, q.A, (size_t)q.N * 4, (size_t)q.N * 4, q.N,
                                  cudaMemcpyDeviceToDevice, s));
    if (!rows16(q.A2, q.m))
        FP_CUDA(cudaMemcpy2DAsync(sl.A232, (size_t)round4(q.m) * 4, q.A2, (size_t)q.m * 4, (size_t)q.m * 4, q.m,
                                  cudaMemcpyDeviceToDevice, s));
    if (!simt_of(p)) {
        // TF32 parts and remainders of A and A' for the FP32 products
        SplitGroup g{};
        g.count = 2;
        g.q[0] = SplitRows{q.A, q.N, q.N, q.N, sl.Ahi, sl.Alo, round4(q.N), 0, nullptr};
        g.q[1] = SplitRows{q.A2, q.m, q.m, q.m, sl.A2hi, sl.A2lo, round4(q.m), 0, nullptr};
        FP_CUDA(split_tf32_group(g, s));
        ++nl;
    }
    if (p->precision == FASTPFP_BF16) {
        // BF16 operand copies of A and A' for the tensor-core products
        FP_CUDA(to_bf16(q.A, q.N, q.N, q.N, sl.A16, round8(q.N), s));
        FP_CUDA(to_bf16(q.A2, q.m, q.m, q.m, sl.A216, round8(q.m), s));
        nl += 2;
    } else if (p->precision == FASTPFP_FP8) {
        // E4M3 copies of A and A' with per-row scales, once per solve
        QuantGroup g{};
        g.count = 2;
        g.q[0] = QuantRows{q.A, 0, q.N, q.N, q.N, sl.qA, round16(q.N), sl.scA, nullptr};
        g.q[1] = QuantRows{q.A2, 0, q.m, q.m, q.m, sl.qA2, round16(q.m), sl.scA2, nullptr};
        FP_CUDA(quant_fp8_group(g, s));
        ++nl;
    }
    return nl;
}

// The gradient products of Section 4.1 in FP32 for one pair, as the
// transposed-operand GEMM consumes them:
//   T^T (m x N, in slot T, ld round4(N)) = X^T A
//   Y[:, :m] = (T^T)^T A' + lambda K.
// Skipped on the device while the solve runs its BF16 phase.
void f32_products(const Slot& sl, const Problem& q, const fastpfp_params* p, GemmF32TArgs* g1, GemmF32TArgs* g2) {
    const int ldy = round4(q.N), ldx = round4(q.m), ldt = round4(q.N);
    int lda = 0, lda2 = 0;
    const float* A = f32_operand(q.A, q.N, sl.A32, &lda);
    const float* A2 = f32_operand(q.A2, q.m, sl.A232, &lda2);
    *g1 = GemmF32TArgs{sl.X, ldx, A, lda, sl.T, ldt, nullptr, 0, 0.f, q.m, q.N, q.N, sl.ctrl};
    *g2 = GemmF32TArgs{sl.T, ldt, A2, lda2, sl.Y, ldy, q.k ? sl.K : nullptr, ldx,
                       q.k ? (float)p->lambda : 0.f, q.N, q.m, q.m, sl.ctrl};
    if (p->algorithm == FASTPFP_ALG_PG) {   // Y[:, :m] = X + alpha (T A' + lambda K), Eq. (pg)
        g2->addend = sl.X;
        g2->ld_add = ldx;
        g2->scale = p->alpha;
        g2->lambda *= p->alpha;
    }
}

int enqueue_gradient(const Slot& sl, cudaStream_t s, const Problem& q, const fastpfp_params* p, int tile_m) {
    GemmF32TGroup g1{}, g2{};
    g1.count = g2.count = 1;
    g1.tile_m = g2.tile_m = tile_m;
    f32_products(sl, q, p, &g1.a[0], &g2.a[0]);
    FP_CUDA(gemm_f32t_group(g1, s));
    FP_CUDA(gemm_f32t_group(g2, s));
    return 2;
}

// The same gradient on the tensor cores for pairs in slots 0..count-1: one
// grouped launch for T = A X (BF16 out) and one for Y = T A' + lambda K (FP32
// out), each covering up to kTcMaxGroup pairs.  The tensor maps describe the
// slots' BF16 buffers and are built once per solve.  FP8 runs the same two
// launches on E4M3 copies: X^T (written in BF16 by the blend) and T are
// quantised per row just before the product that reads them (qx, qt), A and
// A' once at set-up, and the epilogues scale by the two operands' row scales.
struct TcPlan {
    std::vector<TcGroup> g1, g2;          // low-precision phase: BF16 or E4M3 products
    std::vector<QuantGroup> qx, qt;
    std::vector<SplitGroup> sx;           // FP32 phase: X^T split, then the split-TF32 products
    std::vector<TcGroup> f1, f2;
};

// The FP32 phase's products of problems qs[0..count) (slot slot_of[i], or
// i) on the tensor cores, split TF32: per iteration X^T is split from the
// blend's X, then T = A X (written as its TF32 part and remainder) and
// Y[:, :m] = T A' + lambda K; every launch skips solves outside their FP32
// phase.
bool plan_split(fastpfp_t h, const Problem* qs, int count, const fastpfp_params* p, TcPlan* plan,
                const int* slot_of = nullptr) {
    plan->sx.clear();
    plan->f1.clear();
    plan->f2.clear();
    for (int b = 0; b < count; b += kTcMaxGroup) {
        TcGroup a{}, c{};
        SplitGroup sx{};
        const int n = std::min(kTcMaxGroup, count - b);
        int nmax = 0;
        for (int i = 0; i < n; ++i) nmax = std::max(nmax, qs[b + i].N);
        (void)nmax;
        const int bn = kTcSplitBN;
        a.count = c.count = sx.count = n;
        a.mode = kTcOutSplit;
        c.mode = kTcOutF32;
        a.bn = c.bn = bn;
        a.kind = c.kind = kTcTf32x3;
        a.phase = c.phase = 1;
        for (int i = 0; i < n; ++i) {
            const Problem& q = qs[b + i];
            const Slot& sl = h->slots[slot_of ? slot_of[b + i] : b + i];
            const int l4N = round4(q.N), l4m = round4(q.m);
            if (!tc_make_map(&a.map_a[i], sl.Ahi, q.N, q.N, l4N, kTcTileM, kTcTf32x3) ||
                !tc_make_map(&a.map_a_lo[i], sl.Alo, q.N, q.N, l4N, kTcTileM, kTcTf32x3) ||
                !tc_make_map(&a.map_b[i], sl.Xthi, q.m, q.N, l4N, bn, kTcTf32x3) ||
                !tc_make_map(&a.map_b_lo[i], sl.Xtlo, q.m, q.N, l4N, bn, kTcTf32x3) ||
                !tc_make_map(&c.map_a[i], sl.Thi, q.N, q.m, l4m, kTcTileM, kTcTf32x3) ||
                !tc_make_map(&c.map_a_lo[i], sl.Tlo, q.N, q.m, l4m, kTcTileM, kTcTf32x3) ||
                !tc_make_map(&c.map_b[i], sl.A2hi, q.m, q.m, l4m, bn, kTcTf32x3) ||
                !tc_make_map(&c.map_b_lo[i], sl.A2lo, q.m, q.m, l4m, bn, kTcTf32x3))
                return false;
            sx.q[i] = SplitRows{sl.X, q.N, q.m, l4m, sl.Xthi, sl.Xtlo, l4N, 1, sl.ctrl};
            a.prob[i] = TcProblem{q.N, q.m, q.N, sl.Thi, l4m, nullptr, 0, 0.f, sl.ctrl, &sl.ctrl->error};
            a.prob[i].out_lo = sl.Tlo;
            c.prob[i] = TcProblem{q.N, q.m, q.m, sl.Y, l4N, q.k ? sl.K : nullptr, l4m, q.k ? (float)p->lambda : 0.f,
                                  sl.ctrl, &sl.ctrl->error};
            if (p->algorithm == FASTPFP_ALG_PG) {   // Y[:, :m] = X + alpha (T A' + lambda K), Eq. (pg)
                c.prob[i].addend = sl.X;
                c.prob[i].ld_add = l4m;
                c.prob[i].scale = p->alpha;
                c.prob[i].lambda *= p->alpha;
            }
        }
        plan->sx.push_back(sx);
        plan->f1.push_back(a);
        plan->f2.push_back(c);
    }
    return true;
}

int enqueue_fp32(const TcPlan& plan, cudaStream_t s) {
    for (const SplitGroup& g : plan.sx) FP_CUDA(split_tf32_group(g, s));
    for (const TcGroup& g : plan.f1) FP_CUDA(tc_gemm(g, s));
    for (const TcGroup& g : plan.f2) FP_CUDA(tc_gemm(g, s));
    return (int)(plan.sx.size() + plan.f1.size() + plan.f2.size());
}

bool plan_tc(fastpfp_t h, const Problem* qs, int count, const fastpfp_params* p, TcPlan* plan,
             const int* slot_of = nullptr) {
    plan->g1.clear();
    plan->g2.clear();
    plan->qx.clear();
    plan->qt.clear();
    const bool fp8 = p->precision == FASTPFP_FP8;
    for (int b = 0; b < count; b += kTcMaxGroup) {
        TcGroup a{}, c{};
        QuantGroup qx{}, qt{};
        const int n = std::min(kTcMaxGroup, count - b);
        int nmax = 0;
        for (int i = 0; i < n; ++i) nmax = std::max(nmax, qs[b + i].N);
        const int bn = tc_tile(h, nmax, n);
        a.count = c.count = n;
        a.mode = kTcOutBf16;
        c.mode = kTcOutF32;
        a.bn = c.bn = bn;
        a.kind = c.kind = fp8 ? kTcE4m3 : kTcBf16;
        qx.count = qt.count = fp8 ? n : 0;
        for (int i = 0; i < n; ++i) {
            const Problem& q = qs[b + i];
            const Slot& sl = h->slots[slot_of ? slot_of[b + i] : b + i];
            const int l16N = round8(q.N), l16m = round8(q.m);
            if (fp8) {
                const int l8N = round16(q.N), l8m = round16(q.m);
                if (!tc_make_map(&a.map_a[i], sl.qA, q.N, q.N, l8N, kTcTileM, kTcE4m3) ||
                    !tc_make_map(&a.map_b[i], sl.qXt, q.m, q.N, l8N, bn, kTcE4m3) ||
                    !tc_make_map(&c.map_a[i], sl.qT, q.N, q.m, l8m, kTcTileM, kTcE4m3) ||
                    !tc_make_map(&c.map_b[i], sl.qA2, q.m, q.m, l8m, bn, kTcE4m3))
                    return false;
                qx.q[i] = QuantRows{sl.Xt16, 1, q.m, q.N, l16N, sl.qXt, l8N, sl.scX, sl.ctrl};
                qt.q[i] = QuantRows{sl.T16, 1, q.N, q.m, l16m, sl.qT, l8m, sl.scT, sl.ctrl};
                a.prob[i] = TcProblem{q.N, q.m, q.N, sl.T16, l16m, nullptr, 0, 0.f, sl.ctrl, &sl.ctrl->error,
                                      sl.scA, sl.scX};
                c.prob[i] = TcProblem{q.N, q.m, q.m, sl.Y, round4(q.N), q.k ? sl.K : nullptr, round4(q.m),
                                      q.k ? (float)p->lambda : 0.f, sl.ctrl, &sl.ctrl->error, sl.scT, sl.scA2};
                continue;
            }
            if (!tc_make_map(&a.map_a[i], sl.A16, q.N, q.N, l16N, kTcTileM) ||
                !tc_make_map(&a.map_b[i], sl.Xt16, q.m, q.N, l16N, bn) ||
                !tc_make_map(&c.map_a[i], sl.T16, q.N, q.m, l16m, kTcTileM) ||
                !tc_make_map(&c.map_b[i], sl.A216, q.m, q.m, l16m, bn))
                return false;
            a.prob[i] = TcProblem{q.N, q.m, q.N, sl.T16, l16m, nullptr, 0, 0.f, sl.ctrl, &sl.ctrl->error};
            c.prob[i] = TcProblem{q.N, q.m, q.m, sl.Y, round4(q.N), q.k ? sl.K : nullptr, round4(q.m),
                                  q.k ? (float)p->lambda : 0.f, sl.ctrl, &sl.ctrl->error};
        }
        if (p->algorithm == FASTPFP_ALG_PG) {   // Y[:, :m] = X + alpha (T A' + lambda K), Eq. (pg)
            for (int i = 0; i < n; ++i) {
                const Slot& sl = h->slots[slot_of ? slot_of[b + i] : b + i];
                c.prob[i].addend = sl.X;
                c.prob[i].ld_add = round4(qs[b + i].m);
                c.prob[i].scale = p->alpha;
                c.prob[i].lambda *= p->alpha;
            }
        }
        plan->g1.push_back(a);
        plan->g2.push_back(c);
        if (fp8) {
            plan->qx.push_back(qx);
            plan->qt.push_back(qt);
        }
    }
    return true;
}

int enqueue_tc(const TcPlan& plan, cudaStream_t s) {
    for (const QuantGroup& g : plan.qx) FP_CUDA(quant_fp8_group(g, s));
    for (const TcGroup& g : plan.g1) FP_CUDA(tc_gemm(g, s));
    for (const QuantGroup& g : plan.qt) FP_CUDA(quant_fp8_group(g, s));
    for (const TcGroup& g : plan.g2) FP_CUDA(tc_gemm(g, s));
    return (int)(plan.g1.size() + plan.g2.size() + plan.qx.size() + plan.qt.size());
}

// Discretisation, objective, caller-orientation outputs, control header.
int enqueue_finish(const Slot& sl, cudaStream_t s, const Problem& q, const fastpfp_params* p,
                   int num_sms, Ctrl* host_slot) {
    const int ldx = round4(q.m);
    FP_CUDA(discretize(sl.X, q.N, q.m, ldx, sl.disc, sl.ctrl, timeout_ns(p), num_sms, s));
    FP_CUDA(objective(q.A, q.N, q.A2, q.m, q.k ? sl.K : nullptr, ldx, q.k ? (float)p->lambda : 0.f,
                      sl.disc.col_match, sl.ctrl, s));
    FP_CUDA(write_outputs(sl.disc.col_match, q.N, q.m, q.transposed, q.perm_out, sl.X, ldx, q.X_out, s));
    FP_CUDA(cudaMemcpyAsync(host_slot, sl.ctrl, kCtrlHeader, cudaMemcpyDeviceToHost, s));
    return 2 + (q.perm_out ? (q.transposed ? 1 : 2) : 0) + (q.X_out ? 1 : 0);
}

void release_graphs(fastpfp_t h) {
    for (cudaGraphExec_t e : h->execs) cudaGraphExecDestroy(e);
    for (cudaGraph_t g : h->graphs) cudaGraphDestroy(g);
    h->execs.clear();
    h->graphs.clear();
}

// The outer loop as a graph: loop_init (clears the iteration count in
// h->d_loop, opens the loop), then a while node whose body is one outer
// iteration (`step(0, cap)` captured on the handle's capture stream)
// followed by loop_cond, which reads the stop and error words at d_words and
// closes the loop when either is set or after max_outer iterations.  The
// condition's default is "closed", so the body can only repeat while device
// code keeps it open.  The graph is launched on `s`; it and its executable
// live until release_graphs.  Returns the kernels of one iteration (also
// stored in h->loop_body) or < 0.
template <typename Step>
int run_outer_graph(fastpfp_t h, cudaStream_t s, const int* d_words, int done_idx, int err_idx,
                    int max_outer, Step step) {
    cudaGraph_t g = nullptr;
    FP_CUDA(cudaGraphCreate(&g, 0));
    h->graphs.push_back(g);
    cudaGraphConditionalHandle hc;
    FP_CUDA(cudaGraphConditionalHandleCreate(&hc, g, 0, cudaGraphCondAssignDefault));
    FP_CUDA(cudaStreamBeginCaptureToGraph(h->cap, g, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    const cudaError_t ei = loop_init(h->d_loop, hc, h->cap);
    cudaGraph_t captured = nullptr;
    const cudaError_t e0 = cudaStreamEndCapture(h->cap, &captured);
    FP_CUDA(ei);
    FP_CUDA(e0);
    cudaGraphNode_t init = nullptr;
    size_t nn = 1;
    FP_CUDA(cudaGraphGetNodes(g, &init, &nn));
    if (nn != 1 || !init) return FASTPFP_ERR_CUDA;
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hc;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    FP_CUDA(cudaGraphAddNode(&node, g, &init, nullptr, 1, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    FP_CUDA(cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal));
    int r = step(0, h->cap);
    if (r >= 0)
        r = loop_cond(d_words, done_idx, err_idx, h->d_loop, max_outer, hc, h->cap) == cudaSuccess
                ? r + 1 : FASTPFP_ERR_CUDA;
    const cudaError_t ec = cudaStreamEndCapture(h->cap, &captured);
    if (r < 0) return r;
    FP_CUDA(ec);
    cudaGraphExec_t ex = nullptr;
    FP_CUDA(cudaGraphInstantiate(&ex, g, 0));
    h->execs.push_back(ex);
    FP_CUDA(cudaGraphLaunch(ex, s));
    h->loop_body = r;
    return r;
}

// Enqueues the outer loop; `step(t, stream)` enqueues outer iteration t on
// `stream` and returns the kernels it launched (or < 0).  Graph mode (see
// run_outer_graph) returns 0 here; the kernels it ran are counted after the
// call synchronised.  Host mode enqueues chunks of kChunk iterations: after
// every chunk four ints of the device control word at `d_words` are copied
// to pinned memory behind an event; the host checks the previous chunk's
// copy (words done_idx and err_idx), so one chunk is always queued ahead.
template <typename Step>
int run_outer(fastpfp_t h, cudaStream_t s, const fastpfp_params* p, const int* d_words, int done_idx,
              int err_idx, Step step) {
    const int max_outer = p->max_outer;
    h->loop_body = 0;
    if (p->loop_mode == 0 && !p->profile) {
        const int r = run_outer_graph(h, s, d_words, done_idx, err_idx, max_outer, step);
        return r < 0 ? r : 0;
    }
    int t = 0, chunk = 0, nl = 0;
    while (t < max_outer) {
        const int tc = std::min(kChunk, max_outer - t);
        for (int i = 0; i < tc; ++i, ++t) {
            const int r = step(t, s);
            if (r < 0) return r;
            nl += r;
        }
        if (t >= max_outer) break;
        const int slot = chunk & 1;
        FP_CUDA(cudaMemcpyAsync(&h->h_done[4 * slot], d_words, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
        FP_CUDA(cudaEventRecord(h->chunk_ev[slot], s));
        if (chunk >= 1) {
            FP_CUDA(cudaEventSynchronize(h->chunk_ev[slot ^ 1]));
            h->host_syncs += 1;
            const int* w = &h->h_done[4 * (slot ^ 1)];
            if (w[done_idx] || w[err_idx]) break;
        }
        ++chunk;
    }
    return nl;
}

// One pair through pd_kernel.  Returns the kernels launched or < 0.
int enqueue_single(fastpfp_t h, cudaStream_t s, const Slot& sl, const Problem& q,
                   const fastpfp_params* p, Ctrl* host_slot) {
    const int N = q.N, m = q.m;
    const int ldy = round4(N), ldx = round4(m);
    const bool lowp = lowp_of(p);   // a BF16 or FP8 phase
    TcPlan tc;
    if (lowp && !plan_tc(h, &q, 1, p, &tc)) return FASTPFP_ERR_UNSUPPORTED;
    const int slot = (int)(&sl - h->slots.data());
    if (!simt_of(p) && !plan_split(h, &q, 1, p, &tc, &slot)) return FASTPFP_ERR_UNSUPPORTED;
    int nl = enqueue_setup(sl, s, q, p, h->ld);
    if (nl < 0) return nl;
    PdLaunch L;
    pd_plan(N, h->num_sms, &L);
    PdParams P{};
    P.Y = sl.Y;
    P.N = N;
    P.ldy = ldy;
    P.m = m;
    P.X = sl.X;
    P.ldx = ldx;
    P.Xt16 = lowp ? sl.Xt16 : nullptr;
    P.ldxt = round8(N);
    P.alpha = p->algorithm == FASTPFP_ALG_PG ? 1.0f : p->alpha;   // PG keeps the projection itself
    P.normalize = p->normalize_max ? 1 : 0;
    P.slack_reset = p->slack_policy == 1 ? 1 : 0;
    P.tol_inner = p->tol_inner;
    P.max_inner = p->max_inner;
    P.tol_outer = p->tol_outer;
    P.max_outer = p->max_outer;
    P.refine_iters = p->refine_iters;
    P.switch_tol = p->switch_tol;
    P.colbuf = sl.colbuf;
    P.sbuf = sl.sbuf;
    P.dbuf = sl.dbuf;
    P.ctrl = sl.ctrl;
    P.timeout_ns = timeout_ns(p);
    P.rpc = L.rpc;
    P.mode = kPdOuterStep;
    P.skip_arrive = (p->debug_flags & 1) ? 1 : 0;
    const bool prof = p->profile != 0;
    static_assert(offsetof(Ctrl, done) == 0 && offsetof(Ctrl, error) == 8, "Ctrl head layout");
    const int r = run_outer(h, s, p, &sl.ctrl->done, 0, 2, [&](int t, cudaStream_t st) -> int {
        const bool pt = prof && t < kProfIters;
        if (pt && t == 0) FP_CUDA(cudaEventRecord(h->ev[0], st));
        int g = 0;
        if (lowp) {
            g = enqueue_tc(tc, st);
            if (g < 0) return g;
        }
        const int g32 = simt_of(p) ? enqueue_gradient(sl, st, q, p, f32_tile(h, q.N, 1)) : enqueue_fp32(tc, st);
        if (g32 < 0) return g32;
        if (pt) FP_CUDA(cudaEventRecord(h->ev[2 * t + 1], st));
        FP_CUDA(pd_launch(L, P, st));
        if (pt) FP_CUDA(cudaEventRecord(h->ev[2 * t + 2], st));
        return g + g32 + 1;
    });
    if (r < 0) return r;
    nl += r;
    if (prof) FP_CUDA(cudaEventRecord(h->ev[kProfEvents - 2], s));
    const int f = enqueue_finish(sl, s, q, p, h->num_sms, host_slot);
    if (f < 0) return f;
    if (prof) FP_CUDA(cudaEventRecord(h->ev[kProfEvents - 1], s));
    return nl + f;
}

// One pair through FastGA (fastga.cu): the gradient products of FastPFP
// (FP32: split TF32 on the tensor cores, or SIMT), then one ga_kernel launch
// per outer iteration; the same setup, loop control and finish as a
// single-pair FastPFP solve.
int enqueue_ga(fastpfp_t h, cudaStream_t s, const Slot& sl, const Problem& q, const fastpfp_params* p,
               Ctrl* host_slot) {
    const int N = q.N, m = q.m;
    const int slot = (int)(&sl - h->slots.data());
    TcPlan tc;
    if (!simt_of(p) && !plan_split(h, &q, 1, p, &tc, &slot)) return FASTPFP_ERR_UNSUPPORTED;
    // scratch: Z (max_n x ld), the CTAs' column partials (num_sms x ld), the column sums (ld)
    const size_t ld = (size_t)round4(h->max_n);
    if (!h->ga_z) FP_CUDA(cudaMalloc(&h->ga_z, ((size_t)h->max_n + h->num_sms + 1) * ld * sizeof(float)));
    int nl = enqueue_setup(sl, s, q, p, h->ld);
    if (nl < 0) return nl;
    GaParams P{};
    P.Y = sl.Y;
    P.Z = h->ga_z;
    P.X = sl.X;
    P.part = h->ga_z + (size_t)h->max_n * ld;
    P.csum = P.part + (size_t)h->num_sms * ld;
    P.dbuf = sl.dbuf;
    P.ctrl = sl.ctrl;
    P.N = N;
    P.m = m;
    P.ldy = round4(N);
    P.ldx = round4(m);
    P.rpc = ga_rows_per_cta(N, h->num_sms);
    P.beta = p->beta;
    P.tol_inner = p->tol_inner;
    P.tol_outer = p->tol_outer;
    P.max_inner = p->max_inner;
    P.max_outer = p->max_outer;
    P.timeout_ns = timeout_ns(p);
    const int r = run_outer(h, s, p, &sl.ctrl->done, 0, 2, [&](int, cudaStream_t st) -> int {
        const int g32 = simt_of(p) ? enqueue_gradient(sl, st, q, p, f32_tile(h, q.N, 1)) : enqueue_fp32(tc, st);
        if (g32 < 0) return g32;
        FP_CUDA(ga_launch(P, st));
        return g32 + 1;
    });
    if (r < 0) return r;
    nl += r;
    const int f = enqueue_finish(sl, s, q, p, h->num_sms, host_slot);
    if (f < 0) return f;
    return nl + f;
}

// Per-phase times of the last profiled solve (after the stream synced).
void read_profile(fastpfp_t h, int outer, float share, fastpfp_stats* st) {
    if (!st) return;
    float g = 0.f, pr = 0.f, d = 0.f, x = 0.f;
    const int T = outer < kProfIters ? outer : kProfIters;
    for (int t = 0; t < T; ++t) {
        if (cudaEventElapsedTime(&x, h->ev[2 * t], h->ev[2 * t + 1]) == cudaSuccess) g += x;
        if (cudaEventElapsedTime(&x, h->ev[2 * t + 1], h->ev[2 * t + 2]) == cudaSuccess) pr += x;
    }
    if (cudaEventElapsedTime(&x, h->ev[kProfEvents - 2], h->ev[kProfEvents - 1]) == cudaSuccess) d = x;
    st->ms_gemm = g * share;
    st->ms_proj = pr * share;
    st->ms_disc = d * share;
}

int fill_stats(const Ctrl& c, int transposed, int launches, int wave_pairs, fastpfp_stats* st,
               int host_syncs = 0) {
    const int status = c.error != 0 ? c.error : FASTPFP_OK;
    if (st) {
        st->host_syncs = host_syncs;
        st->launches = launches;
        st->wave_pairs = wave_pairs;
        st->ms_gemm = st->ms_proj = st->ms_disc = 0.f;
        st->outer_iters = c.outer;
        st->inner_iters_total = c.inner_total;
        st->inner_iters_max = c.inner_max;
        st->converged = c.converged;
        st->lowp_iters = c.lowp_iters;
        st->transposed = transposed;
        st->status = status;
        st->final_delta = c.last_delta;
        st->objective = c.objective;
    }
    return status;
}

// ---- waves of the batched path ---------------------------------------------

struct Wave {
    int first = 0, count = 0, grid = 0;
    size_t smem = 0;
    PdbLayout layout{};
    std::vector<int> band;   // grid + 1 row boundaries
};

// A wave planned by the shared band planner (band_plan.cuh) for pairs
// [first, first + count) of qs.
bool plan_bands(const std::vector<Problem>& qs, int first, int count, int num_sms, Wave* w,
                int max_level = 3) {
    std::vector<int> Ns(count);
    for (int i = 0; i < count; ++i) Ns[i] = qs[first + i].N;
    WavePlan wp;
    if (!plan_bands_seq(Ns.data(), count, num_sms, max_level, &wp)) return false;
    w->band.assign(wp.band, wp.band + wp.grid + 1);
    w->first = first;
    w->count = count;
    w->grid = wp.grid;
    w->layout = wp.layout;
    w->smem = wp.smem;
    return true;
}

// Largest wave starting at `first` (at least one pair when it fits at all).
bool plan_wave(const std::vector<Problem>& qs, int first, int nslots, int num_sms, Wave* w) {
    int best = 0;
    Wave cand;
    const int limit = std::min<int>({(int)qs.size() - first, nslots, kMaxWavePairs});
    for (int c = 1; c <= limit; ++c) {
        if (qs[first + c - 1].N > kPdbMaxN) break;
        if (!plan_bands(qs, first, c, num_sms, &cand)) break;
        *w = cand;
        best = c;
    }
    return best > 0;
}

// A pair of a wave and the slot whose buffers it uses.
struct Member {
    int pair;
    int slot;
    int last = -1;   // streamed waves: the launch that last ran the pair
};

// Wave tables of members mem (pair table in member order, band table of w)
// staged through pinned memory, the wave control word cleared.  The pinned
// staging is reused by the next wave, so callers synchronise in between.
// The wave-table entry of problem q in slot sl (row0 left 0).
PairDesc pair_desc(const Slot& sl, const Problem& q, bool lowp) {
    PairDesc d{};
    d.Y = sl.Y;
    d.X = sl.X;
    d.Xt16 = lowp ? sl.Xt16 : nullptr;
    d.colbuf = sl.colbuf;
    d.sbuf = sl.sbuf;
    d.dbuf = sl.dbuf;
    d.ctrl = sl.ctrl;
    d.N = q.N;
    d.ldy = round4(q.N);
    d.m = q.m;
    d.ldx = round4(q.m);
    d.ldxt = round8(q.N);
    return d;
}

int write_wave_tables(fastpfp_t h, cudaStream_t s, const std::vector<Problem>& qs,
                      const std::vector<Member>& mem, const Wave& w, bool lowp) {
    int row0 = 0;
    for (int i = 0; i < (int)mem.size(); ++i) {
        const Problem& q = qs[mem[i].pair];
        PairDesc d = pair_desc(h->slots[mem[i].slot], q, lowp);
        d.row0 = row0;
        row0 += q.N;
        h->h_pairs[i] = d;
    }
    for (int b = 0; b <= w.grid; ++b) h->h_band[b] = w.band[b];
    FP_CUDA(cudaMemcpyAsync(h->d_pairs, h->h_pairs, sizeof(PairDesc) * mem.size(), cudaMemcpyHostToDevice, s));
    FP_CUDA(cudaMemcpyAsync(h->d_band, h->h_band, sizeof(int) * (w.grid + 1), cudaMemcpyHostToDevice, s));
    FP_CUDA(cudaMemsetAsync(h->d_wave, 0, sizeof(WaveCtrl), s));
    return 0;
}

PdbParams wave_params(fastpfp_t h, const Wave& w, int npairs, const fastpfp_params* p) {
    PdbParams P{};
    P.pairs = h->d_pairs;
    P.npairs = npairs;
    P.band_row = h->d_band;
    P.wave = h->d_wave;
    P.layout = w.layout;
    P.alpha = p->algorithm == FASTPFP_ALG_PG ? 1.0f : p->alpha;   // PG keeps the projection itself
    P.normalize = p->normalize_max ? 1 : 0;
    P.slack_reset = p->slack_policy == 1 ? 1 : 0;
    P.tol_inner = p->tol_inner;
    P.tol_inner_f = float_at_least(p->tol_inner);
    P.max_inner = p->max_inner;
    P.tol_outer = p->tol_outer;
    P.max_outer = p->max_outer;
    P.refine_iters = p->refine_iters;
    P.switch_tol = p->switch_tol;
    P.timeout_ns = timeout_ns(p);
    P.skip_arrive = (p->debug_flags & 1) ? 1 : 0;
    return P;
}

// FP32 products of every member: one grouped launch per product and
// kF32MaxGroup members.
void f32_groups(fastpfp_t h, const std::vector<Problem>& qs, const std::vector<Member>& mem,
                const fastpfp_params* p, std::vector<GemmF32TGroup>& ga_out, std::vector<GemmF32TGroup>& gb_out) {
    ga_out.clear();
    gb_out.clear();
    if (!simt_of(p)) return;   // the FP32 products run on the tensor cores (plan_split)
    for (int b = 0; b < (int)mem.size(); b += kF32MaxGroup) {
        GemmF32TGroup ga{}, gb{};
        ga.count = gb.count = std::min(kF32MaxGroup, (int)mem.size() - b);
        int nmax = 0;
        for (int i = 0; i < ga.count; ++i) {
            f32_products(h->slots[mem[b + i].slot], qs[mem[b + i].pair], p, &ga.a[i], &gb.a[i]);
            nmax = std::max(nmax, qs[mem[b + i].pair].N);
        }
        ga.tile_m = gb.tile_m = f32_tile(h, nmax, ga.count);
        ga_out.push_back(ga);
        gb_out.push_back(gb);
    }
}

// The inner-round counts and deltas of the pair in `slot`, kept per pair
// of the call (the slot may be reused by a later pair).
int save_trace(fastpfp_t h, cudaStream_t s, int slot, int pair, int max_outer) {
    const Ctrl* c = h->slots[slot].ctrl;
    char* dst = h->trace_store + (size_t)pair * kTraceBytes;
    const size_t n = (size_t)std::min(max_outer, kMaxOuterTrace);
    FP_CUDA(cudaMemcpyAsync(dst, c->inner_trace, n * sizeof(int), cudaMemcpyDeviceToDevice, s));
    FP_CUDA(cudaMemcpyAsync(dst + (size_t)kMaxOuterTrace * sizeof(int), c->delta_trace, n * sizeof(double),
                            cudaMemcpyDeviceToDevice, s));
    return 0;
}

// One wave through pdb_kernel, the loop controlled as run_outer says; pair
// w.first + i uses slot i.  Returns the kernels launched or < 0.
int enqueue_wave(fastpfp_t h, cudaStream_t s, const std::vector<Problem>& qs, const Wave& w,
                 const fastpfp_params* p, Ctrl* host_slots) {
    int nl = 0;
    const bool lowp = lowp_of(p);   // a BF16 or FP8 phase
    std::vector<Member> mem(w.count);
    for (int i = 0; i < w.count; ++i) mem[i] = Member{w.first + i, i};
    TcPlan tc;
    if (lowp && !plan_tc(h, &qs[w.first], w.count, p, &tc)) return FASTPFP_ERR_UNSUPPORTED;
    if (!simt_of(p) && !plan_split(h, &qs[w.first], w.count, p, &tc)) return FASTPFP_ERR_UNSUPPORTED;
    for (int i = 0; i < w.count; ++i) {
        const int r = enqueue_setup(h->slots[i], s, qs[w.first + i], p, h->ld);
        if (r < 0) return r;
        nl += r;
    }
    const int wt = write_wave_tables(h, s, qs, mem, w, lowp);
    if (wt < 0) return wt;
    const PdbParams P = wave_params(h, w, w.count, p);
    std::vector<GemmF32TGroup> f32a, f32b;
    f32_groups(h, qs, mem, p, f32a, f32b);
    const bool prof = p->profile != 0;
    static_assert(offsetof(WaveCtrl, error) == 0 && offsetof(WaveCtrl, all_done) == 4,
                  "WaveCtrl layout");
    const int r = run_outer(h, s, p, reinterpret_cast<const int*>(h->d_wave), 1, 0,
                            [&](int t, cudaStream_t st) -> int {
        const bool pt = prof && t < kProfIters;
        if (pt && t == 0) FP_CUDA(cudaEventRecord(h->ev[0], st));
        int n = 0;
        if (lowp) {
            n = enqueue_tc(tc, st);
            if (n < 0) return n;
        }
        const int f = enqueue_fp32(tc, st);   // split-TF32 FP32 products (none with SIMT)
        if (f < 0) return f;
        n += f;
        for (const GemmF32TGroup& g : f32a) FP_CUDA(gemm_f32t_group(g, st));   // T^T = X^T A
        for (const GemmF32TGroup& g : f32b) FP_CUDA(gemm_f32t_group(g, st));   // Y = T A' + lambda K
        n += (int)(f32a.size() + f32b.size());
        if (pt) FP_CUDA(cudaEventRecord(h->ev[2 * t + 1], st));
        FP_CUDA(pdb_launch(P, w.grid, w.smem, st));
        if (pt) FP_CUDA(cudaEventRecord(h->ev[2 * t + 2], st));
        return n + 1;
    });
    if (r < 0) return r;
    nl += r;
    if (prof) FP_CUDA(cudaEventRecord(h->ev[kProfEvents - 2], s));
    for (int i = 0; i < w.count; ++i) {
        const int f = enqueue_finish(h->slots[i], s, qs[w.first + i], p, h->num_sms, &host_slots[i]);
        if (f < 0) return f;
        nl += f;
        const int tr = save_trace(h, s, i, w.first + i, p->max_outer);
        if (tr < 0) return tr;
    }
    if (prof) FP_CUDA(cudaEventRecord(h->ev[kProfEvents - 1], s));
    return nl;
}

int solve_batch(fastpfp_t h, cudaStream_t s, int count, const fastpfp_pair* pairs,
                const fastpfp_params* p, fastpfp_stats* st, bool host);

}  // namespace

extern "C" {

void fastpfp_default_params(fastpfp_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->lambda = 0.f;
    p->alpha = 0.5f;
    p->tol_outer = 1e-6;
    p->tol_inner = 1e-6;
    p->max_outer = 100;
    p->max_inner = 1000;
    p->precision = FASTPFP_FP32;
    p->refine_iters = 8;
    p->switch_tol = 1e-3;
    p->normalize_max = 1;
    p->slack_policy = 0;
    p->timeout_ms = 2000;
    p->profile = 0;
    p->loop_mode = 0;
    p->debug_flags = 0;
    p->algorithm = FASTPFP_ALG_FASTPFP;
    p->beta = 100.f;
}

const char* fastpfp_error_string(int code) {
    switch (code) {
        case FASTPFP_OK: return "ok";
        case FASTPFP_ERR_ARG: return "invalid argument";
        case FASTPFP_ERR_SIZE: return "graph larger than the handle's max_n";
        case FASTPFP_ERR_CUDA: return "CUDA runtime error";
        case FASTPFP_ERR_TIMEOUT: return "device barrier wait ran out of its time budget";
        case FASTPFP_ERR_NONFINITE: return "non-finite value in the iterate";
        case FASTPFP_ERR_UNSUPPORTED: return "option not supported";
        default: return "unknown error";
    }
}

int fastpfp_create(fastpfp_t* out, int device, int max_n, int max_batch) {
    if (!out) return FASTPFP_ERR_ARG;
    *out = nullptr;
    if (max_n < 1 || max_batch < 1) return FASTPFP_ERR_ARG;
    if (max_n > kMaxN) return FASTPFP_ERR_SIZE;
    if (cudaSetDevice(device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    fastpfp_s* h = new (std::nothrow) fastpfp_s();
    if (!h) return FASTPFP_ERR_CUDA;
    h->device = device;
    h->max_n = max_n;
    h->max_batch = max_batch;
    h->ld = round4(max_n);
    h->nslots = max_batch;   // one slot per pair of a batch: a batch streams inside one graph
    for (int c = 0; c < FASTPFP_TUNE_SIZES; ++c)
        for (int k = 0; k < FASTPFP_TUNE_COUNTS; ++k) {
            h->tile_f32[c][k] = 128;
            h->tile_tc[c][k] = 256;
        }
    if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        pd_configure() != cudaSuccess || pdb_configure() != cudaSuccess || tc_configure() != cudaSuccess ||
        ga_configure() != cudaSuccess ||
        gemm_f32t_configure() != cudaSuccess ||
        disc_configure() != cudaSuccess) {
        delete h;
        return FASTPFP_ERR_CUDA;
    }
    const size_t n = (size_t)max_n, ld = (size_t)h->ld;
    const size_t f32mat = align256(n * ld * sizeof(float));
    const size_t b16mat = align256(n * (size_t)round8(max_n) * sizeof(__nv_bfloat16));
    const size_t f8mat = align256(n * (size_t)round16(max_n));
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    struct SlotOff {
        size_t Y, X, T, K, A16, A216, Xt16, T16, col, s, d, ctrl, rm, cm, rb, cb, sA, sA2, sB, sB2, sX0,
            sXo, sp, A32, A232, qA, qA2, qXt, qT, scA, scA2, scX, scT, Ahi, Alo, A2hi, A2lo, Xthi, Xtlo, Thi,
            Tlo;
    };
    std::vector<SlotOff> so(h->nslots);
    for (auto& o : so) {
        o.Y = take(f32mat); o.X = take(f32mat); o.T = take(f32mat); o.K = take(f32mat);
        o.A16 = take(b16mat); o.A216 = take(b16mat); o.Xt16 = take(b16mat); o.T16 = take(b16mat);
        o.col = take(colbuf_bytes((int)ld)); o.s = take(3 * sizeof(double));
        o.d = take(kDbufWords * sizeof(unsigned)); o.ctrl = take(sizeof(Ctrl));
        o.rm = take(n * 4); o.cm = take(n * 4); o.rb = take(n * 8); o.cb = take(2 * n * 8);
        o.sA = take(n * n * 4); o.sA2 = take(n * n * 4); o.sB = take(n * kMaxK * 4);
        o.sB2 = take(n * kMaxK * 4); o.sX0 = take(n * n * 4); o.sXo = take(n * n * 4); o.sp = take(n * 4);
        o.A32 = take(f32mat); o.A232 = take(f32mat);
        o.qA = take(f8mat); o.qA2 = take(f8mat); o.qXt = take(f8mat); o.qT = take(f8mat);
        o.scA = take(n * 4); o.scA2 = take(n * 4); o.scX = take(n * 4); o.scT = take(n * 4);
        o.Ahi = take(f32mat); o.Alo = take(f32mat); o.A2hi = take(f32mat); o.A2lo = take(f32mat);
        o.Xthi = take(f32mat); o.Xtlo = take(f32mat); o.Thi = take(f32mat); o.Tlo = take(f32mat);
    }
    const size_t opairs = take(sizeof(PairDesc) * kMaxWavePairs);
    const size_t otmpl = take(sizeof(PairDesc) * (size_t)max_batch);
    const size_t ostream = take(sizeof(StreamState));
    const size_t oband = take(sizeof(int) * 2 * (h->num_sms + 1));
    const size_t owave = take(sizeof(WaveCtrl));
    const size_t oloop = take(sizeof(int));
    const size_t oflags = take(sizeof(int) * (kMaxWavePairs + 1));
    const size_t otrace = take((size_t)max_batch * kTraceBytes);
    const size_t nch = (n + 63) / 64;
    const size_t wFb = take(n * kMlpIn * 4), wFs = take(n * kMlpIn * 4), wHb = take(n * kMlpHidden * 4),
                 wHs = take(n * kMlpHidden * 4), wEb = take(n * kMlpOut * 4), wEs = take(n * kMlpOut * 4),
                 wEb8 = take(n * kMlpOut * 4), wEs8 = take(n * kMlpOut * 4), wEsT = take(kMlpOut * ld * 4),
                 wdEb = take(n * kMlpOut * 4), wdEs = take(n * kMlpOut * 4), wdH = take(n * kMlpHidden * 4),
                 wgrad = take(kMlpParams * 4), wscal = take(16), wlc = take(n * 4), wlr = take(n * 4),
                 wpart = take(nch * n * 8), wt = take(n * 4), wtinv = take(n * 4), wloss = take(16);
    h->pool_bytes = off;
    auto fail = [&](int code) {
        for (int e = 0; e < kProfEvents; ++e)
            if (h->ev[e]) cudaEventDestroy(h->ev[e]);
        for (int e = 0; e < 2; ++e)
            if (h->chunk_ev[e]) cudaEventDestroy(h->chunk_ev[e]);
        if (h->host_ctrl) cudaFreeHost(h->host_ctrl);
        if (h->h_pairs) cudaFreeHost(h->h_pairs);
        if (h->h_band) cudaFreeHost(h->h_band);
        if (h->h_done) cudaFreeHost(h->h_done);
        if (h->h_flags) cudaFreeHost(h->h_flags);
        if (h->h_tmpl) cudaFreeHost(h->h_tmpl);
        if (h->h_stream) cudaFreeHost(h->h_stream);
        if (h->cap) cudaStreamDestroy(h->cap);
        if (h->pool) cudaFree(h->pool);
        delete h;
        return code;
    };
    if (cudaMalloc(&h->pool, off) != cudaSuccess) return fail(FASTPFP_ERR_CUDA);
    if (cudaMallocHost(&h->host_ctrl, sizeof(Ctrl) * (size_t)max_batch) != cudaSuccess ||
        cudaMallocHost(&h->h_pairs, sizeof(PairDesc) * kMaxWavePairs) != cudaSuccess ||
        cudaMallocHost(&h->h_band, sizeof(int) * 2 * (h->num_sms + 1)) != cudaSuccess ||
        cudaMallocHost(&h->h_done, sizeof(int) * 8) != cudaSuccess ||
        cudaMallocHost(&h->h_flags, sizeof(int) * (kMaxWavePairs + 1)) != cudaSuccess ||
        cudaMallocHost(&h->h_tmpl, sizeof(PairDesc) * (size_t)max_batch) != cudaSuccess ||
        cudaMallocHost(&h->h_stream, sizeof(StreamState)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess)
        return fail(FASTPFP_ERR_CUDA);
    char* b = h->pool;
    h->slots.resize(h->nslots);
    for (int i = 0; i < h->nslots; ++i) {
        const SlotOff& o = so[i];
        Slot& sl = h->slots[i];
        sl.Y = (float*)(b + o.Y);
        sl.X = (float*)(b + o.X);
        sl.T = (float*)(b + o.T);
        sl.K = (float*)(b + o.K);
        sl.A16 = (__nv_bfloat16*)(b + o.A16);
        sl.A216 = (__nv_bfloat16*)(b + o.A216);
        sl.Xt16 = (__nv_bfloat16*)(b + o.Xt16);
        sl.T16 = (__nv_bfloat16*)(b + o.T16);
        sl.colbuf = (float*)(b + o.col);
        sl.sbuf = (double*)(b + o.s);
        sl.dbuf = (unsigned*)(b + o.d);
        sl.ctrl = (Ctrl*)(b + o.ctrl);
        sl.disc.row_match = (int32_t*)(b + o.rm);
        sl.disc.col_match = (int32_t*)(b + o.cm);
        sl.disc.row_best = (unsigned long long*)(b + o.rb);
        sl.disc.col_best = (unsigned long long*)(b + o.cb);
        sl.sA = (float*)(b + o.sA);
        sl.sA2 = (float*)(b + o.sA2);
        sl.sB = (float*)(b + o.sB);
        sl.sB2 = (float*)(b + o.sB2);
        sl.sX0 = (float*)(b + o.sX0);
        sl.sXout = (float*)(b + o.sXo);
        sl.A32 = (float*)(b + o.A32);
        sl.A232 = (float*)(b + o.A232);
        sl.qA = (uint8_t*)(b + o.qA);
        sl.qA2 = (uint8_t*)(b + o.qA2);
        sl.qXt = (uint8_t*)(b + o.qXt);
        sl.qT = (uint8_t*)(b + o.qT);
        sl.scA = (float*)(b + o.scA);
        sl.scA2 = (float*)(b + o.scA2);
        sl.scX = (float*)(b + o.scX);
        sl.scT = (float*)(b + o.scT);
        sl.sperm = (int32_t*)(b + o.sp);
        sl.Ahi = (float*)(b + o.Ahi);
        sl.Alo = (float*)(b + o.Alo);
        sl.A2hi = (float*)(b + o.A2hi);
        sl.A2lo = (float*)(b + o.A2lo);
        sl.Xthi = (float*)(b + o.Xthi);
        sl.Xtlo = (float*)(b + o.Xtlo);
        sl.Thi = (float*)(b + o.Thi);
        sl.Tlo = (float*)(b + o.Tlo);
    }
    h->d_pairs = (PairDesc*)(b + opairs);
    h->d_tmpl = (PairDesc*)(b + otmpl);
    h->d_stream = (StreamState*)(b + ostream);
    h->d_band = (int*)(b + oband);
    h->d_wave = (WaveCtrl*)(b + owave);
    h->d_loop = (int*)(b + oloop);
    h->d_flags = (int*)(b + oflags);
    h->trace_store = b + otrace;
    h->ws.Fb = (float*)(b + wFb);
    h->ws.Fs = (float*)(b + wFs);
    h->ws.Hb = (float*)(b + wHb);
    h->ws.Hs = (float*)(b + wHs);
    h->ws.Eb = (float*)(b + wEb);
    h->ws.Es = (float*)(b + wEs);
    h->ws.Eb8 = (float*)(b + wEb8);
    h->ws.Es8 = (float*)(b + wEs8);
    h->ws.EsT = (float*)(b + wEsT);
    h->ws.dEb = (float*)(b + wdEb);
    h->ws.dEs = (float*)(b + wdEs);
    h->ws.dH = (float*)(b + wdH);
    h->ws.grad = (float*)(b + wgrad);
    h->ws.scalar = (float*)(b + wscal);
    h->ws.lse_c = (float*)(b + wlc);
    h->ws.lse_r = (float*)(b + wlr);
    h->ws.part = (float2*)(b + wpart);
    h->ws.t = (int32_t*)(b + wt);
    h->ws.tinv = (int32_t*)(b + wtinv);
    h->ws.loss = (double*)(b + wloss);
    for (int e = 0; e < kProfEvents; ++e)
        if (cudaEventCreate(&h->ev[e]) != cudaSuccess) return fail(FASTPFP_ERR_CUDA);
    for (int e = 0; e < 2; ++e)
        if (cudaEventCreateWithFlags(&h->chunk_ev[e], cudaEventDisableTiming) != cudaSuccess)
            return fail(FASTPFP_ERR_CUDA);
    if (cudaMemset(h->pool, 0, off) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess)
        return fail(FASTPFP_ERR_CUDA);
    *out = h;
    return FASTPFP_OK;
}

void fastpfp_destroy(fastpfp_t h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    release_graphs(h);
    for (int e = 0; e < kProfEvents; ++e)
        if (h->ev[e]) cudaEventDestroy(h->ev[e]);
    for (int e = 0; e < 2; ++e)
        if (h->chunk_ev[e]) cudaEventDestroy(h->chunk_ev[e]);
    if (h->host_ctrl) cudaFreeHost(h->host_ctrl);
    if (h->h_pairs) cudaFreeHost(h->h_pairs);
    if (h->h_band) cudaFreeHost(h->h_band);
    if (h->h_done) cudaFreeHost(h->h_done);
    if (h->h_flags) cudaFreeHost(h->h_flags);
    if (h->h_tmpl) cudaFreeHost(h->h_tmpl);
    if (h->h_stream) cudaFreeHost(h->h_stream);
    if (h->ga_z) cudaFree(h->ga_z);
    if (h->cap) cudaStreamDestroy(h->cap);
    if (h->pool) cudaFree(h->pool);
    delete h;
}

int fastpfp_match(fastpfp_t h, void* stream, const float* A, int n_a, const float* A2, int n_b,
                  const float* B, const float* B2, int k, const fastpfp_params* p, const float* X0,
                  int32_t* perm_out, float* X_out, fastpfp_stats* st) {
    int rc = check_pair(h, A, n_a, A2, n_b, B, B2, k, p, perm_out);
    if (rc != FASTPFP_OK) return rc;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    fastpfp_pair x{A, A2, B, B2, n_a, n_b, k, X0, perm_out, X_out};
    return solve_batch(h, (cudaStream_t)stream, 1, &x, p, st, false);
}

int fastpfp_match_host(fastpfp_t h, void* stream, const float* A, int n_a, const float* A2, int n_b,
                       const float* B, const float* B2, int k, const fastpfp_params* p,
                       const float* X0, int32_t* perm_out, float* X_out, fastpfp_stats* st) {
    int rc = check_pair(h, A, n_a, A2, n_b, B, B2, k, p, perm_out);
    if (rc != FASTPFP_OK) return rc;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const fastpfp_pair pr{A, A2, B, B2, n_a, n_b, k, X0, perm_out, X_out};
    rc = solve_batch(h, s, 1, &pr, p, st, true);
    return rc;
}

int fastpfp_match_batched(fastpfp_t h, void* stream, int count, const fastpfp_pair* pairs,
                          const fastpfp_params* p, fastpfp_stats* st) {
    if (!h || count < 0 || (count > 0 && !pairs)) return FASTPFP_ERR_ARG;
    if (count > h->max_batch) return FASTPFP_ERR_ARG;
    for (int b = 0; b < count; ++b) {
        const fastpfp_pair& q = pairs[b];
        int rc = check_pair(h, q.A, q.n_a, q.A2, q.n_b, q.B, q.B2, q.k, p, q.perm_out);
        if (rc != FASTPFP_OK) return rc;
    }
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    return solve_batch(h, (cudaStream_t)stream, count, pairs, p, st, false);
}

int fastpfp_match_batched_host(fastpfp_t h, void* stream, int count, const fastpfp_pair* pairs,
                               const fastpfp_params* p, fastpfp_stats* st) {
    if (!h || count < 0 || (count > 0 && !pairs)) return FASTPFP_ERR_ARG;
    if (count > h->max_batch) return FASTPFP_ERR_ARG;
    for (int b = 0; b < count; ++b) {
        const fastpfp_pair& q = pairs[b];
        int rc = check_pair(h, q.A, q.n_a, q.A2, q.n_b, q.B, q.B2, q.k, p, q.perm_out);
        if (rc != FASTPFP_OK) return rc;
    }
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    return solve_batch(h, (cudaStream_t)stream, count, pairs, p, st, true);
}

}  // extern "C"

namespace {

// The batch driver of fastpfp_match_batched (device memory) and of the
// *_host calls (host memory: each wave's inputs are staged into its slots
// and the outputs copied back before the next wave).
// Host-memory inputs of pair x staged into `slot`; *q is rewritten to
// point at the staged copies (caller orientation preserved).
// One host input buffer into the device: appended to `L` (copied later by
// one gather kernel, see gather_copy) when the GPU can read it in place --
// pinned host memory with a device address, 16-byte aligned, the list not
// full -- otherwise an ordinary copy on the stream (pageable memory).
int stage_copy(CopyList* L, void* dst, const void* src, size_t bytes, cudaStream_t s) {
    if (L && L->count < kMaxCopySegs && bytes % 4 == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, src) == cudaSuccess && a.type == cudaMemoryTypeHost &&
            a.devicePointer && (reinterpret_cast<uintptr_t>(a.devicePointer) & 15) == 0) {
            L->seg[L->count++] = CopySeg{a.devicePointer, dst, (unsigned long long)bytes};
            return 0;
        }
        cudaGetLastError();   // a pageable pointer is not an error
    }
    FP_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
    return 0;
}

// The pair's host inputs into its slot's staging buffers (through `L` when
// given: the caller launches gather_copy before anything reads them).
int stage_in(fastpfp_t h, cudaStream_t s, const fastpfp_pair& x, const fastpfp_params* p, int slot,
             Problem* q, CopyList* L = nullptr) {
    const Slot& sl = h->slots[slot];
    const int kk = (x.k > 0 && p->lambda != 0.f) ? x.k : 0;
    if (stage_copy(L, sl.sA, x.A, (size_t)x.n_a * x.n_a * 4, s) < 0 ||
        stage_copy(L, sl.sA2, x.A2, (size_t)x.n_b * x.n_b * 4, s) < 0)
        return FASTPFP_ERR_CUDA;
    if (kk && (stage_copy(L, sl.sB, x.B, (size_t)x.n_a * kk * 4, s) < 0 ||
               stage_copy(L, sl.sB2, x.B2, (size_t)x.n_b * kk * 4, s) < 0))
        return FASTPFP_ERR_CUDA;
    if (x.X0 && stage_copy(L, sl.sX0, x.X0, (size_t)x.n_a * x.n_b * 4, s) < 0) return FASTPFP_ERR_CUDA;
    *q = canonical(sl.sA, x.n_a, sl.sA2, x.n_b, kk ? sl.sB : nullptr, kk ? sl.sB2 : nullptr, kk, p->lambda,
                   x.X0 ? sl.sX0 : nullptr, sl.sperm, x.X_out ? sl.sXout : nullptr);
    return 0;
}

// Staged outputs of the pair in `slot` copied back to host memory.
int stage_out(fastpfp_t h, cudaStream_t s, const fastpfp_pair& x, int slot) {
    const Slot& sl = h->slots[slot];
    FP_CUDA(cudaMemcpyAsync(x.perm_out, sl.sperm, (size_t)x.n_a * 4, cudaMemcpyDeviceToHost, s));
    if (x.X_out)
        FP_CUDA(cudaMemcpyAsync(x.X_out, sl.sXout, (size_t)x.n_a * x.n_b * 4, cudaMemcpyDeviceToHost, s));
    return 0;
}

// A batch larger than one wave, streamed inside one CUDA graph.  Every pair
// is set up in its own slot; the planner kernel (wave_stream.cu) chooses each
// outer iteration's wave on the device (stopped pairs leave, waiting pairs
// join while the band plan fits, the same plans the host would make), the
// grouped products run over every pair of the batch and skip the idle ones,
// and the projection launch takes the wave the planner wrote.  The while
// node ends once every pair has stopped; then every pair is discretised and
// its outputs written.  One graph launch and one host synchronisation per
// call.  Returns the worst status.
int solve_graph_stream(fastpfp_t h, cudaStream_t s, std::vector<Problem>& qs, const fastpfp_pair* pairs,
                       const fastpfp_params* p, fastpfp_stats* st, bool host) {
    const int count = (int)qs.size();
    const bool lowp = lowp_of(p);   // a BF16 or FP8 phase
    int nl = 0;
    auto fail = [&](int code) {
        cudaStreamSynchronize(s);
        release_graphs(h);
        return code;
    };
    if (host) {   // every pair's inputs, pinned ones by one gather launch
        CopyList L;
        L.count = 0;
        for (int i = 0; i < count; ++i) {
            if (L.count + 5 > kMaxCopySegs) {
                FP_CUDA(gather_copy(L, s));
                L.count = 0;
            }
            const int r = stage_in(h, s, pairs[i], p, i, &qs[i], &L);
            if (r < 0) return fail(r);
        }
        FP_CUDA(gather_copy(L, s));
    }
    for (int i = 0; i < count; ++i) {
        const int r = enqueue_setup(h->slots[i], s, qs[i], p, h->ld);
        if (r < 0) return fail(r);
        nl += r;
        h->h_tmpl[i] = pair_desc(h->slots[i], qs[i], lowp);
    }
    StreamState init{};
    init.count = count;
    init.first = 1;
    init.num_sms = h->num_sms;
    *h->h_stream = init;
    if (cudaMemcpyAsync(h->d_tmpl, h->h_tmpl, sizeof(PairDesc) * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(h->d_stream, h->h_stream, sizeof(StreamState), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(h->d_wave, 0, sizeof(WaveCtrl), s) != cudaSuccess ||
        cudaMemsetAsync(h->d_band, 0, sizeof(int) * (h->num_sms + 1), s) != cudaSuccess)
        return fail(FASTPFP_ERR_CUDA);
    // the products of every pair (idle and stopped pairs skip theirs)
    std::vector<Member> all(count);
    for (int i = 0; i < count; ++i) all[i] = Member{i, i};
    std::vector<GemmF32TGroup> f32a, f32b;
    f32_groups(h, qs, all, p, f32a, f32b);
    TcPlan tc;
    if (lowp && !plan_tc(h, qs.data(), count, p, &tc)) return fail(FASTPFP_ERR_UNSUPPORTED);
    if (!simt_of(p) && !plan_split(h, qs.data(), count, p, &tc)) return fail(FASTPFP_ERR_UNSUPPORTED);
    Wave none;
    PdbParams P = wave_params(h, none, 0, p);
    P.dyn = 1;
    // the first wave, then the loop: products, projection, next wave
    if (wave_plan(h->d_stream, h->d_tmpl, h->d_pairs, h->d_band, h->d_wave, s) != cudaSuccess)
        return fail(FASTPFP_ERR_CUDA);
    nl += 1;
    const int cap = count * std::max(1, p->max_outer);   // each iteration advances every pair of a wave
    static_assert(offsetof(StreamState, done) == 0 && offsetof(StreamState, error) == 4, "StreamState head");
    const int r = run_outer_graph(h, s, reinterpret_cast<const int*>(h->d_stream), 0, 1, cap,
                                  [&](int, cudaStream_t cs) -> int {
        int n = 0;
        if (lowp) {
            n = enqueue_tc(tc, cs);
            if (n < 0) return n;
        }
        const int f = enqueue_fp32(tc, cs);   // split-TF32 FP32 products (none with SIMT)
        if (f < 0) return f;
        n += f;
        for (const GemmF32TGroup& g : f32a) FP_CUDA(gemm_f32t_group(g, cs));   // T^T = X^T A
        for (const GemmF32TGroup& g : f32b) FP_CUDA(gemm_f32t_group(g, cs));   // Y = T A' + lambda K
        n += (int)(f32a.size() + f32b.size());
        FP_CUDA(pdb_launch(P, h->num_sms, (size_t)kPdMaxSmem, cs));
        FP_CUDA(wave_plan(h->d_stream, h->d_tmpl, h->d_pairs, h->d_band, h->d_wave, cs));
        return n + 2;
    });
    if (r < 0) return fail(r);
    for (int i = 0; i < count; ++i) {
        const int f = enqueue_finish(h->slots[i], s, qs[i], p, h->num_sms, &h->host_ctrl[i]);
        if (f < 0) return fail(f);
        nl += f;
        if (save_trace(h, s, i, i, p->max_outer) < 0) return fail(FASTPFP_ERR_CUDA);
        if (host && stage_out(h, s, pairs[i], i) < 0) return fail(FASTPFP_ERR_CUDA);
    }
    const cudaError_t es = cudaStreamSynchronize(s);
    h->host_syncs += 1;
    int loop_iters = 0;
    StreamState fin{};
    if (es == cudaSuccess) {
        FP_CUDA(cudaMemcpy(&loop_iters, h->d_loop, sizeof(int), cudaMemcpyDeviceToHost));
        FP_CUDA(cudaMemcpy(&fin, h->d_stream, offsetof(StreamState, act), cudaMemcpyDeviceToHost));
    }
    release_graphs(h);
    if (es != cudaSuccess) return FASTPFP_ERR_CUDA;
    nl += 1 + h->loop_body * loop_iters;   // loop_init + iterations
    int worst = FASTPFP_OK;
    for (int i = 0; i < count; ++i) {
        Ctrl& c = h->host_ctrl[i];
        // an error of a shared launch belongs to every pair it left unfinished
        if (fin.error != 0 && c.error == 0 && !c.done) c.error = fin.error;
        const int rc = fill_stats(c, qs[i].transposed, nl / count + (i < nl % count ? 1 : 0), c.wave_pairs,
                                  st ? &st[i] : nullptr, h->host_syncs);
        if (rc != FASTPFP_OK && worst == FASTPFP_OK) worst = rc;
    }
    h->last_count = count;
    return worst;
}

// True when a batch can stream inside one graph: the graph loop is asked
// for, every pair has its own slot, and every pair fits in a wave alone.
bool graph_streamable(fastpfp_t h, const std::vector<Problem>& qs, const fastpfp_params* p) {
    if (p->loop_mode != 0 || p->profile || (int)qs.size() > h->nslots) return false;
    std::vector<int> seen;
    for (const Problem& q : qs) {
        if (q.N > kPdbMaxN) return false;
        if (std::find(seen.begin(), seen.end(), q.N) != seen.end()) continue;
        Wave w;
        if (!plan_bands(qs, (int)(&q - qs.data()), 1, h->num_sms, &w)) return false;
        seen.push_back(q.N);
    }
    return true;
}

// Continuous batching for batches that do not fit in one wave.  A wave is
// kept full: after every outer iteration (one pdb_kernel launch over the
// wave's active pairs and their grouped products) the host reads the pairs'
// stop words, finishes the pairs that stopped (discretisation, objective,
// outputs) and admits waiting pairs into the freed slots while the wave's
// band plan still fits on chip.  Each pair's iterations are independent of
// its wave-mates, so the result of a pair does not depend on the schedule
// beyond FP32 summation order.  Returns the worst status.
int solve_stream(fastpfp_t h, cudaStream_t s, std::vector<Problem>& qs, const fastpfp_pair* pairs,
                 const fastpfp_params* p, fastpfp_stats* st, bool host) {
    const int count = (int)qs.size();
    const bool lowp = lowp_of(p);   // a BF16 or FP8 phase
    const bool prof = p->profile != 0;
    std::vector<int> free_slots;
    for (int i = h->nslots - 1; i >= 0; --i) free_slots.push_back(i);
    std::vector<Member> act;
    std::vector<int> nl(count, 0), wave_of(count, 0), werr_of(count, 0);
    std::vector<float> ms_g(count, 0.f), ms_p(count, 0.f);
    int next = 0;
    auto fail = [&](int code) {
        cudaStreamSynchronize(s);
        return code;
    };
    auto problems_of = [&](const std::vector<Member>& m, std::vector<Problem>& out, std::vector<int>& slots) {
        out.clear();
        slots.clear();
        for (const Member& x : m) {
            out.push_back(qs[x.pair]);
            slots.push_back(x.slot);
        }
    };
    std::vector<Problem> cand;
    std::vector<int> cand_slots;
    std::vector<GemmF32TGroup> f32a, f32b;
    int launch_no = 0;
    while (true) {
        // admit waiting pairs while the wave still fits on chip
        Wave w;
        bool planned = false;
        while (next < count && !free_slots.empty() && (int)act.size() < kMaxWavePairs &&
               qs[next].N <= kPdbMaxN) {
            problems_of(act, cand, cand_slots);
            cand.push_back(qs[next]);
            Wave cw;
            if (!plan_bands(cand, 0, (int)cand.size(), h->num_sms, &cw, act.empty() ? 3 : kAdmitLevel)) break;
            const int slot = free_slots.back();
            free_slots.pop_back();
            if (host) {
                const int r = stage_in(h, s, pairs[next], p, slot, &qs[next]);
                if (r < 0) return fail(r);
            }
            const int r = enqueue_setup(h->slots[slot], s, qs[next], p, h->ld);
            if (r < 0) return fail(r);
            nl[next] += r;
            act.push_back(Member{next, slot, -1});
            ++next;
            w = cw;
            planned = true;
        }
        if (act.empty()) {
            if (next >= count) break;
            // a pair that fits in no wave runs alone through pd_kernel
            const int slot = free_slots.back();
            if (host) {
                const int r = stage_in(h, s, pairs[next], p, slot, &qs[next]);
                if (r < 0) return fail(r);
            }
            const int r = enqueue_single(h, s, h->slots[slot], qs[next], p, &h->host_ctrl[next]);
            if (r < 0) return fail(r);
            nl[next] += r;
            if (save_trace(h, s, slot, next, p->max_outer) < 0) return fail(FASTPFP_ERR_CUDA);
            if (host && stage_out(h, s, pairs[next], slot) < 0) return fail(FASTPFP_ERR_CUDA);
            if (cudaStreamSynchronize(s) != cudaSuccess) return FASTPFP_ERR_CUDA;
            h->host_syncs += 1;
            if (h->loop_body > 0) {
                int it = 0;
                FP_CUDA(cudaMemcpy(&it, h->d_loop, sizeof(int), cudaMemcpyDeviceToHost));
                nl[next] += 1 + h->loop_body * it;
            }
            release_graphs(h);
            ++next;
            continue;
        }
        // the pairs of this launch: every active pair when they fit on chip
        // together, else as many as fit, least recently run first (a pair
        // left out simply waits: its state is in its slot)
        std::vector<Member> run;
        problems_of(act, cand, cand_slots);
        if (planned || plan_bands(cand, 0, (int)cand.size(), h->num_sms, &w)) {
            run = act;
        } else {
            std::vector<Member> order = act;
            std::stable_sort(order.begin(), order.end(),
                             [](const Member& a, const Member& b) { return a.last < b.last; });
            std::vector<Member> trial;
            for (const Member& m : order) {
                trial = run;
                trial.push_back(m);
                problems_of(trial, cand, cand_slots);
                Wave tw;
                if (!plan_bands(cand, 0, (int)cand.size(), h->num_sms, &tw)) continue;
                run = trial;
                w = tw;
            }
            if (run.empty()) return fail(FASTPFP_ERR_UNSUPPORTED);
            problems_of(run, cand, cand_slots);
        }
        ++launch_no;
        // one outer iteration of the wave
        const int n = (int)run.size();
        if (write_wave_tables(h, s, qs, run, w, lowp) < 0) return fail(FASTPFP_ERR_CUDA);
        const PdbParams P = wave_params(h, w, n, p);
        TcPlan tc;
        if (lowp && !plan_tc(h, cand.data(), n, p, &tc, cand_slots.data())) return fail(FASTPFP_ERR_UNSUPPORTED);
        if (!simt_of(p) && !plan_split(h, cand.data(), n, p, &tc, cand_slots.data()))
            return fail(FASTPFP_ERR_UNSUPPORTED);
        f32_groups(h, qs, run, p, f32a, f32b);
        int kl = 0;
        if (prof && cudaEventRecord(h->ev[0], s) != cudaSuccess) return fail(FASTPFP_ERR_CUDA);
        if (lowp) {
            const int r = enqueue_tc(tc, s);
            if (r < 0) return fail(r);
            kl += r;
        }
        {
            const int r = enqueue_fp32(tc, s);   // split-TF32 FP32 products (none with SIMT)
            if (r < 0) return fail(r);
            kl += r;
        }
        for (const GemmF32TGroup& g : f32a)
            if (gemm_f32t_group(g, s) != cudaSuccess) return fail(FASTPFP_ERR_CUDA);
        for (const GemmF32TGroup& g : f32b)
            if (gemm_f32t_group(g, s) != cudaSuccess) return fail(FASTPFP_ERR_CUDA);
        kl += (int)(f32a.size() + f32b.size());
        if (prof && cudaEventRecord(h->ev[1], s) != cudaSuccess) return fail(FASTPFP_ERR_CUDA);
        if (pdb_launch(P, w.grid, w.smem, s) != cudaSuccess) return fail(FASTPFP_ERR_CUDA);
        if (prof && cudaEventRecord(h->ev[2], s) != cudaSuccess) return fail(FASTPFP_ERR_CUDA);
        FlagList fl{};
        for (int i = 0; i < n; ++i) fl.ctrl[i] = h->slots[run[i].slot].ctrl;
        fl.wave = h->d_wave;
        fl.n = n;
        if (gather_flags(fl, h->d_flags, s) != cudaSuccess ||
            cudaMemcpyAsync(h->h_flags, h->d_flags, sizeof(int) * (kMaxWavePairs + 1), cudaMemcpyDeviceToHost,
                            s) != cudaSuccess)
            return fail(FASTPFP_ERR_CUDA);
        kl += 2;   // the flag gather and the pdb launch
        if (cudaStreamSynchronize(s) != cudaSuccess) return FASTPFP_ERR_CUDA;
        h->host_syncs += 1;
        float tg = 0.f, tp = 0.f;
        if (prof) {
            cudaEventElapsedTime(&tg, h->ev[0], h->ev[1]);
            cudaEventElapsedTime(&tp, h->ev[1], h->ev[2]);
        }
        const int werr = h->h_flags[kMaxWavePairs];
        std::vector<int> stopped(count, 0);
        for (int i = 0; i < n; ++i) {
            const Member& m = run[i];
            nl[m.pair] += kl / n + (i < kl % n ? 1 : 0);
            ms_g[m.pair] += tg / (float)n;
            ms_p[m.pair] += tp / (float)n;
            wave_of[m.pair] = std::max(wave_of[m.pair], n);
            if ((h->h_flags[i] & 3) == 0 && werr == 0) continue;
            stopped[m.pair] = 1;
            // an error of the shared launch belongs to every pair of the wave
            if (werr != 0) werr_of[m.pair] = werr;
            const int f = enqueue_finish(h->slots[m.slot], s, qs[m.pair], p, h->num_sms, &h->host_ctrl[m.pair]);
            if (f < 0) return fail(f);
            nl[m.pair] += f;
            if (save_trace(h, s, m.slot, m.pair, p->max_outer) < 0) return fail(FASTPFP_ERR_CUDA);
            if (host && stage_out(h, s, pairs[m.pair], m.slot) < 0) return fail(FASTPFP_ERR_CUDA);
            free_slots.push_back(m.slot);
        }
        std::vector<Member> keep;
        for (Member m : act) {
            if (stopped[m.pair]) continue;
            for (const Member& r : run)
                if (r.pair == m.pair) m.last = launch_no;
            keep.push_back(m);
        }
        act.swap(keep);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return FASTPFP_ERR_CUDA;
    h->host_syncs += 1;
    int worst = FASTPFP_OK;
    for (int b = 0; b < count; ++b) {
        if (werr_of[b] != 0 && h->host_ctrl[b].error == 0) h->host_ctrl[b].error = werr_of[b];
        fastpfp_stats* sb = st ? &st[b] : nullptr;
        const int rc = fill_stats(h->host_ctrl[b], qs[b].transposed, nl[b], wave_of[b], sb, h->host_syncs);
        if (sb && prof) {
            sb->ms_gemm = ms_g[b];
            sb->ms_proj = ms_p[b];
            sb->ms_disc = 0.f;
        }
        if (rc != FASTPFP_OK && worst == FASTPFP_OK) worst = rc;
    }
    h->last_count = count;
    return worst;
}

// FastGA over a batch: the pairs one after another on the stream (slot i
// for pair i), one synchronisation at the end.
int solve_ga(fastpfp_t h, cudaStream_t s, std::vector<Problem>& qs, const fastpfp_pair* pairs,
             const fastpfp_params* p, fastpfp_stats* st, bool host) {
    const int count = (int)qs.size();
    std::vector<int> nl(count, 0), body(count, 0);
    for (int i = 0; i < count; ++i) {
        if (host) {
            const int r = stage_in(h, s, pairs[i], p, i, &qs[i]);
            if (r < 0) return r;
        }
        int r = enqueue_ga(h, s, h->slots[i], qs[i], p, &h->host_ctrl[i]);
        if (r >= 0 && save_trace(h, s, i, i, p->max_outer) < 0) r = FASTPFP_ERR_CUDA;
        if (r >= 0 && host && stage_out(h, s, pairs[i], i) < 0) r = FASTPFP_ERR_CUDA;
        if (r < 0) {
            cudaStreamSynchronize(s);
            release_graphs(h);
            return r;
        }
        nl[i] = r;
        body[i] = h->loop_body;
    }
    const cudaError_t es = cudaStreamSynchronize(s);
    h->host_syncs += 1;
    release_graphs(h);
    if (es != cudaSuccess) return FASTPFP_ERR_CUDA;
    int worst = FASTPFP_OK;
    for (int i = 0; i < count; ++i) {
        // graph mode: a loop-init kernel plus one body per outer iteration run
        const int launches = nl[i] + (body[i] > 0 ? 1 + body[i] * h->host_ctrl[i].outer : 0);
        const int rc = fill_stats(h->host_ctrl[i], qs[i].transposed, launches, 0, st ? &st[i] : nullptr,
                                  h->host_syncs);
        if (rc != FASTPFP_OK && worst == FASTPFP_OK) worst = rc;
    }
    h->last_count = count;
    return worst;
}

int solve_batch(fastpfp_t h, cudaStream_t s, int count, const fastpfp_pair* pairs,
                const fastpfp_params* p, fastpfp_stats* st, bool host) {
    h->host_syncs = 0;
    std::vector<Problem> qs(count);
    for (int b = 0; b < count; ++b) {
        const fastpfp_pair& x = pairs[b];
        qs[b] = canonical(x.A, x.n_a, x.A2, x.n_b, x.B, x.B2, x.k, p->lambda, x.X0, x.perm_out, x.X_out);
    }
    if (p->algorithm == FASTPFP_ALG_FASTGA) return solve_ga(h, s, qs, pairs, p, st, host);
    // a batch that fits in one wave runs as one wave (its loop on the
    // device), a lone pair included: its slacked matrix then stays on chip
    // (TMEM + shared memory) instead of streaming through L2; a larger batch
    // is streamed through waves kept full by the host; a pair that fits in
    // no wave runs through pd_kernel
    Wave w;
    const bool batched = plan_wave(qs, 0, h->nslots, h->num_sms, &w);
    if (count > 1 && (!batched || w.count < count))
        return graph_streamable(h, qs, p) ? solve_graph_stream(h, s, qs, pairs, p, st, host)
                                          : solve_stream(h, s, qs, pairs, p, st, host);
    const int cnt = batched ? w.count : 1;
    if (host) {   // pinned inputs by one gather launch
        CopyList L;
        L.count = 0;
        for (int i = 0; i < cnt; ++i) {
            if (L.count + 5 > kMaxCopySegs) {
                FP_CUDA(gather_copy(L, s));
                L.count = 0;
            }
            const int r = stage_in(h, s, pairs[i], p, i, &qs[i], &L);
            if (r < 0) return r;
        }
        FP_CUDA(gather_copy(L, s));
    }
    int nl = batched ? enqueue_wave(h, s, qs, w, p, h->host_ctrl)
                     : enqueue_single(h, s, h->slots[0], qs[0], p, &h->host_ctrl[0]);
    if (nl >= 0 && !batched) {
        const int r = save_trace(h, s, 0, 0, p->max_outer);
        if (r < 0) nl = r;
    }
    if (nl < 0) {
        cudaStreamSynchronize(s);
        release_graphs(h);
        return nl;
    }
    if (host)
        for (int i = 0; i < cnt; ++i)
            if (stage_out(h, s, pairs[i], i) < 0) return FASTPFP_ERR_CUDA;
    const cudaError_t es = cudaStreamSynchronize(s);
    h->host_syncs += 1;
    int loop_iters = 0;
    if (es == cudaSuccess && h->loop_body > 0)
        FP_CUDA(cudaMemcpy(&loop_iters, h->d_loop, sizeof(int), cudaMemcpyDeviceToHost));
    release_graphs(h);
    if (es != cudaSuccess) return FASTPFP_ERR_CUDA;
    if (h->loop_body > 0) nl += 1 + h->loop_body * loop_iters;   // loop_init + iterations
    if (batched) {
        // an error of the shared projection launch belongs to every pair of the wave
        WaveCtrl wc{};
        FP_CUDA(cudaMemcpy(&wc, h->d_wave, sizeof(WaveCtrl), cudaMemcpyDeviceToHost));
        if (wc.error != 0)
            for (int i = 0; i < cnt; ++i)
                if (h->host_ctrl[i].error == 0) h->host_ctrl[i].error = wc.error;
    }
    int worst = FASTPFP_OK;
    int outer = 0;
    for (int j = 0; j < cnt; ++j) outer = std::max(outer, h->host_ctrl[j].outer);
    for (int i = 0; i < cnt; ++i) {
        const int launches = nl / cnt + (i == 0 ? nl % cnt : 0);
        const int rc = fill_stats(h->host_ctrl[i], qs[i].transposed, launches, batched ? cnt : 0,
                                  st ? &st[i] : nullptr, h->host_syncs);
        if (st && p->profile) read_profile(h, outer, 1.0f / (float)cnt, &st[i]);
        if (rc != FASTPFP_OK && worst == FASTPFP_OK) worst = rc;
    }
    h->last_count = cnt;
    return worst;
}

}  // namespace

extern "C" {

int fastpfp_bandwidth_probe(int device, int level, int sweeps, double* gbs) {
    if (!gbs || sweeps < 1 || level < 0 || level > 3) return FASTPFP_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return FASTPFP_ERR_CUDA;
    float ms = 0.f;
    double bytes = 0.0;
    cudaError_t e;
    if (level == 0) e = probe_smem(num_sms, sweeps, 0, &ms, &bytes);
    else if (level == 3) e = probe_tmem(num_sms, sweeps, 0, &ms, &bytes);
    else e = probe_gmem(level == 1 ? (size_t)64 << 20 : (size_t)2 << 30, num_sms, sweeps, 0, &ms, &bytes);
    if (e != cudaSuccess || ms <= 0.f) return FASTPFP_ERR_CUDA;
    *gbs = bytes / ((double)ms * 1e-3) / 1e9;
    return FASTPFP_OK;
}

int fastpfp_gemm_probe(int device, int precision, int n, int reps, double* tflops) {
    if (!tflops || reps < 1 || reps > 1000 || n < 256 || n > 16384 || (n % 16) != 0) return FASTPFP_ERR_ARG;
    if (precision != FASTPFP_FP32 && precision != FASTPFP_BF16 && precision != FASTPFP_FP8 &&
        precision != FASTPFP_FP32_SIMT)
        return FASTPFP_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    if (tc_configure() != cudaSuccess || gemm_f32t_configure() != cudaSuccess) return FASTPFP_ERR_CUDA;
    float ms = 0.f;
    if (probe_gemm(precision, n, reps, 0, &ms) != cudaSuccess || ms <= 0.f) return FASTPFP_ERR_CUDA;
    *tflops = 2.0 * (double)n * n * n / ((double)ms * 1e-3) / 1e12;
    return FASTPFP_OK;
}

int fastpfp_autotune(fastpfp_t h, void* stream, int reps, double* times_ms) {
    if (!h || reps < 1 || reps > 100) return FASTPFP_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    constexpr int kSlotsPerClass = 4;
    if (times_ms)
        for (int i = 0; i < FASTPFP_TUNE_SIZES * FASTPFP_TUNE_COUNTS * kSlotsPerClass; ++i) times_ms[i] = 0.0;
    int* d_err = h->d_flags;   // free between solves; receives a tensor-core timeout
    FP_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    cudaEvent_t e0 = h->ev[0], e1 = h->ev[1];
    // best time of `launch` (one product pair) over reps, after one untimed run
    auto best_of = [&](auto&& launch, double* out) -> int {
        FP_CUDA(launch());
        float best = 0.f;
        for (int r = 0; r < reps; ++r) {
            FP_CUDA(cudaEventRecord(e0, s));
            FP_CUDA(launch());
            FP_CUDA(cudaEventRecord(e1, s));
            FP_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            FP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (r == 0 || ms < best) best = ms;
        }
        *out = best;
        return 0;
    };
    for (int sc = 0; sc < FASTPFP_TUNE_SIZES; ++sc) {
        const int lo = sc == 0 ? 1 : (64 << sc) + 1;
        if (lo > h->max_n) break;
        const int N = std::min(128 << sc, h->max_n), m = N;
        const int ld4 = round4(N), ld8 = round8(N);
        for (int cc = 0; cc < FASTPFP_TUNE_COUNTS; ++cc) {
            const int clo = cc == 0 ? 1 : kCountClassHi[cc - 1] + 1;
            if (clo > h->nslots) break;
            // a class whose smallest group already fills every SM four times
            // over with the large tiles of both products keeps them unmeasured
            const int tiles32 = ((N + 127) / 128) * ((m + 127) / 128);
            const int tiles16 = ((N + kTcTileM - 1) / kTcTileM) * ((m + 255) / 256);
            if ((long long)clo * std::min(tiles32, tiles16) >= 4ll * h->num_sms) continue;
            const int cnt = std::min(kCountClassHi[cc], h->nslots);
            double t[kSlotsPerClass] = {0, 0, 0, 0};
            // FP32 products T^T = X^T A, Y = T A' in the slots' scratch
            for (int v = 0; v < 2; ++v) {
                GemmF32TGroup g1{}, g2{};
                g1.count = g2.count = cnt;
                g1.tile_m = g2.tile_m = v == 0 ? 128 : 64;
                for (int i = 0; i < cnt; ++i) {
                    const Slot& sl = h->slots[i];
                    g1.a[i] = GemmF32TArgs{sl.X, ld4, sl.A32, ld4, sl.T, ld4, nullptr, 0, 0.f, m, N, N, nullptr};
                    g2.a[i] = GemmF32TArgs{sl.T, ld4, sl.A232, ld4, sl.Y, ld4, nullptr, 0, 0.f, N, m, m, nullptr};
                }
                const int r = best_of([&]() {
                    cudaError_t e = gemm_f32t_group(g1, s);
                    return e == cudaSuccess ? gemm_f32t_group(g2, s) : e;
                }, &t[v]);
                if (r < 0) return r;
            }
            // BF16 products T = A X, Y = T A' on the tensor cores
            for (int v = 0; v < 2; ++v) {
                const int bn = v == 0 ? 256 : 128;
                TcGroup a{}, c{};
                a.count = c.count = cnt;
                a.mode = kTcOutBf16;
                c.mode = kTcOutF32;
                a.bn = c.bn = bn;
                for (int i = 0; i < cnt; ++i) {
                    const Slot& sl = h->slots[i];
                    if (!tc_make_map(&a.map_a[i], sl.A16, N, N, ld8, kTcTileM) ||
                        !tc_make_map(&a.map_b[i], sl.Xt16, m, N, ld8, bn) ||
                        !tc_make_map(&c.map_a[i], sl.T16, N, m, ld8, kTcTileM) ||
                        !tc_make_map(&c.map_b[i], sl.A216, m, m, ld8, bn))
                        return FASTPFP_ERR_UNSUPPORTED;
                    a.prob[i] = TcProblem{N, m, N, sl.T16, ld8, nullptr, 0, 0.f, nullptr, d_err};
                    c.prob[i] = TcProblem{N, m, m, sl.Y, ld4, nullptr, 0, 0.f, nullptr, d_err};
                }
                const int r = best_of([&]() {
                    cudaError_t e = tc_gemm(a, s);
                    return e == cudaSuccess ? tc_gemm(c, s) : e;
                }, &t[2 + v]);
                if (r < 0) return r;
            }
            int err = 0;
            FP_CUDA(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
            FP_CUDA(cudaStreamSynchronize(s));
            if (err != 0) return err;
            h->tile_f32[sc][cc] = t[1] < t[0] ? 64 : 128;
            h->tile_tc[sc][cc] = t[3] < t[2] ? 128 : 256;
            if (times_ms)
                for (int k = 0; k < kSlotsPerClass; ++k)
                    times_ms[(sc * FASTPFP_TUNE_COUNTS + cc) * kSlotsPerClass + k] = t[k];
        }
    }
    return FASTPFP_OK;
}

int fastpfp_get_tiles(fastpfp_t h, int n, int count, int* f32_tile_m, int* tc_tile_n) {
    if (!h || n < 1 || count < 1) return FASTPFP_ERR_ARG;
    if (f32_tile_m) *f32_tile_m = f32_tile(h, n, count);
    if (tc_tile_n) *tc_tile_n = tc_tile(h, n, count);
    return FASTPFP_OK;
}

int fastpfp_set_tiles(fastpfp_t h, int n, int count, int f32_tile_m, int tc_tile_n) {
    if (!h || (f32_tile_m != 128 && f32_tile_m != 64) || (tc_tile_n != 256 && tc_tile_n != 128))
        return FASTPFP_ERR_ARG;
    for (int c = 0; c < FASTPFP_TUNE_SIZES; ++c)
        for (int k = 0; k < FASTPFP_TUNE_COUNTS; ++k)
            if ((n <= 0 || c == size_class(n)) && (count <= 0 || k == count_class(count))) {
                h->tile_f32[c][k] = f32_tile_m;
                h->tile_tc[c][k] = tc_tile_n;
            }
    return FASTPFP_OK;
}

int fastpfp_last_trace(fastpfp_t h, int pair, int* inner_counts, double* deltas, int cap) {
    if (!h || cap < 0) return FASTPFP_ERR_ARG;
    if (pair < 0 || pair >= h->last_count) return FASTPFP_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    const int outer = h->host_ctrl[pair].outer;
    const int n = std::min(std::min(outer, cap), kMaxOuterTrace);
    const char* src = h->trace_store + (size_t)pair * kTraceBytes;
    if (n > 0 && inner_counts)
        FP_CUDA(cudaMemcpy(inner_counts, src, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost));
    if (n > 0 && deltas)
        FP_CUDA(cudaMemcpy(deltas, src + (size_t)kMaxOuterTrace * sizeof(int), (size_t)n * sizeof(double),
                           cudaMemcpyDeviceToHost));
    return outer;
}

int fastpfp_gradient(fastpfp_t h, void* stream, const float* A, const float* X, const float* A2,
                     const float* K, float lambda, int N, int m, float* Y, int ldy, int precision) {
    if (!h || !A || !X || !A2 || !Y || N < 1 || m < 1 || m > N || ldy < m) return FASTPFP_ERR_ARG;
    if (lambda != 0.f && !K) return FASTPFP_ERR_ARG;
    if (N > h->max_n) return FASTPFP_ERR_SIZE;
    if (precision != FASTPFP_FP32 && precision != FASTPFP_BF16 && precision != FASTPFP_FP8 &&
        precision != FASTPFP_FP32_SIMT)
        return FASTPFP_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const Slot& sl = h->slots[0];
    if (precision == FASTPFP_FP32) {
        // split-TF32 products on the tensor cores: A, A' and X^T split into
        // TF32 parts and remainders in the slot, T written split, Y and K
        // through the slot's padded FP32 buffers (16-byte aligned rows)
        const int l4N = round4(N), l4m = round4(m);
        SplitGroup g{};
        g.count = 3;
        g.q[0] = SplitRows{A, N, N, N, sl.Ahi, sl.Alo, l4N, 0, nullptr};
        g.q[1] = SplitRows{A2, m, m, m, sl.A2hi, sl.A2lo, l4m, 0, nullptr};
        g.q[2] = SplitRows{X, N, m, m, sl.Xthi, sl.Xtlo, l4N, 1, nullptr};
        FP_CUDA(split_tf32_group(g, s));
        if (lambda != 0.f)
            FP_CUDA(cudaMemcpy2DAsync(sl.K, (size_t)l4m * 4, K, (size_t)m * 4, (size_t)m * 4, N,
                                      cudaMemcpyDeviceToDevice, s));
        TcGroup a{}, c{};
        a.count = c.count = 1;
        a.mode = kTcOutSplit;
        c.mode = kTcOutF32;
        a.kind = c.kind = kTcTf32x3;
        a.phase = c.phase = 1;
        const int bn = kTcSplitBN;
        a.bn = c.bn = bn;
        if (!tc_make_map(&a.map_a[0], sl.Ahi, N, N, l4N, kTcTileM, kTcTf32x3) ||
            !tc_make_map(&a.map_a_lo[0], sl.Alo, N, N, l4N, kTcTileM, kTcTf32x3) ||
            !tc_make_map(&a.map_b[0], sl.Xthi, m, N, l4N, bn, kTcTf32x3) ||
            !tc_make_map(&a.map_b_lo[0], sl.Xtlo, m, N, l4N, bn, kTcTf32x3) ||
            !tc_make_map(&c.map_a[0], sl.Thi, N, m, l4m, kTcTileM, kTcTf32x3) ||
            !tc_make_map(&c.map_a_lo[0], sl.Tlo, N, m, l4m, kTcTileM, kTcTf32x3) ||
            !tc_make_map(&c.map_b[0], sl.A2hi, m, m, l4m, bn, kTcTf32x3) ||
            !tc_make_map(&c.map_b_lo[0], sl.A2lo, m, m, l4m, bn, kTcTf32x3))
            return FASTPFP_ERR_UNSUPPORTED;
        a.prob[0] = TcProblem{N, m, N, sl.Thi, l4m, nullptr, 0, 0.f, nullptr, nullptr};
        a.prob[0].out_lo = sl.Tlo;
        c.prob[0] = TcProblem{N, m, m, sl.Y, l4m, lambda != 0.f ? sl.K : nullptr, l4m, lambda, nullptr, nullptr};
        FP_CUDA(tc_gemm(a, s));
        FP_CUDA(tc_gemm(c, s));
        FP_CUDA(cudaMemcpy2DAsync(Y, (size_t)ldy * 4, sl.Y, (size_t)l4m * 4, (size_t)m * 4, N,
                                  cudaMemcpyDeviceToDevice, s));
        return FASTPFP_OK;
    }
    if (precision == FASTPFP_FP8) {
        // E4M3 copies with per-row scales: A, A' and X^T (through the BF16
        // transpose the solve's blend writes), then T between the products
        const int l16N = round8(N), l16m = round8(m), l8N = round16(N), l8m = round16(m), l4m = round4(m);
        FP_CUDA(transpose_to_bf16(X, N, m, m, sl.Xt16, l16N, s));
        QuantGroup q1{};
        q1.count = 3;
        q1.q[0] = QuantRows{A, 0, N, N, N, sl.qA, l8N, sl.scA, nullptr};
        q1.q[1] = QuantRows{A2, 0, m, m, m, sl.qA2, l8m, sl.scA2, nullptr};
        q1.q[2] = QuantRows{sl.Xt16, 1, m, N, l16N, sl.qXt, l8N, sl.scX, nullptr};
        FP_CUDA(quant_fp8_group(q1, s));
        if (lambda != 0.f)
            FP_CUDA(cudaMemcpy2DAsync(sl.K, (size_t)l4m * 4, K, (size_t)m * 4, (size_t)m * 4, N,
                                      cudaMemcpyDeviceToDevice, s));
        TcGroup a{}, c{};
        a.count = c.count = 1;
        a.mode = kTcOutBf16;
        c.mode = kTcOutF32;
        a.kind = c.kind = kTcE4m3;
        const int bn = tc_tile(h, N, 1);
        a.bn = c.bn = bn;
        if (!tc_make_map(&a.map_a[0], sl.qA, N, N, l8N, kTcTileM, kTcE4m3) ||
            !tc_make_map(&a.map_b[0], sl.qXt, m, N, l8N, bn, kTcE4m3) ||
            !tc_make_map(&c.map_a[0], sl.qT, N, m, l8m, kTcTileM, kTcE4m3) ||
            !tc_make_map(&c.map_b[0], sl.qA2, m, m, l8m, bn, kTcE4m3))
            return FASTPFP_ERR_UNSUPPORTED;
        a.prob[0] = TcProblem{N, m, N, sl.T16, l16m, nullptr, 0, 0.f, nullptr, nullptr, sl.scA, sl.scX};
        c.prob[0] = TcProblem{N, m, m, sl.Y, l4m, lambda != 0.f ? sl.K : nullptr, l4m, lambda, nullptr, nullptr,
                              sl.scT, sl.scA2};
        QuantGroup q2{};
        q2.count = 1;
        q2.q[0] = QuantRows{sl.T16, 1, N, m, l16m, sl.qT, l8m, sl.scT, nullptr};
        FP_CUDA(tc_gemm(a, s));
        FP_CUDA(quant_fp8_group(q2, s));
        FP_CUDA(tc_gemm(c, s));
        FP_CUDA(cudaMemcpy2DAsync(Y, (size_t)ldy * 4, sl.Y, (size_t)l4m * 4, (size_t)m * 4, N,
                                  cudaMemcpyDeviceToDevice, s));
        return FASTPFP_OK;
    }
    if (precision == FASTPFP_BF16) {
        // BF16 operand copies in the slot, products on the tensor cores; Y and
        // K go through the slot's padded FP32 buffers (16-byte aligned rows)
        const int l16N = round8(N), l16m = round8(m), l4m = round4(m);
        FP_CUDA(to_bf16(A, N, N, N, sl.A16, l16N, s));
        FP_CUDA(to_bf16(A2, m, m, m, sl.A216, l16m, s));
        FP_CUDA(transpose_to_bf16(X, N, m, m, sl.Xt16, l16N, s));
        if (lambda != 0.f)
            FP_CUDA(cudaMemcpy2DAsync(sl.K, (size_t)l4m * 4, K, (size_t)m * 4, (size_t)m * 4, N,
                                      cudaMemcpyDeviceToDevice, s));
        TcGroup a{}, c{};
        a.count = c.count = 1;
        a.mode = kTcOutBf16;
        c.mode = kTcOutF32;
        const int bn = tc_tile(h, N, 1);
        a.bn = c.bn = bn;
        if (!tc_make_map(&a.map_a[0], sl.A16, N, N, l16N, kTcTileM) || !tc_make_map(&a.map_b[0], sl.Xt16, m, N, l16N, bn) ||
            !tc_make_map(&c.map_a[0], sl.T16, N, m, l16m, kTcTileM) || !tc_make_map(&c.map_b[0], sl.A216, m, m, l16m, bn))
            return FASTPFP_ERR_UNSUPPORTED;
        a.prob[0] = TcProblem{N, m, N, sl.T16, l16m, nullptr, 0, 0.f, nullptr, nullptr};
        c.prob[0] = TcProblem{N, m, m, sl.Y, l4m, lambda != 0.f ? sl.K : nullptr, l4m, lambda, nullptr, nullptr};
        FP_CUDA(tc_gemm(a, s));
        FP_CUDA(tc_gemm(c, s));
        FP_CUDA(cudaMemcpy2DAsync(Y, (size_t)ldy * 4, sl.Y, (size_t)l4m * 4, (size_t)m * 4, N,
                                  cudaMemcpyDeviceToDevice, s));
        return FASTPFP_OK;
    }
    // the solve's FP32 products: X staged with 16-byte rows, A and A' used
    // in place when their rows are 16-byte aligned
    const int ldx = round4(m), ldt = round4(N);
    FP_CUDA(cudaMemcpy2DAsync(sl.X, (size_t)ldx * 4, X, (size_t)m * 4, (size_t)m * 4, N, cudaMemcpyDeviceToDevice, s));
    if (!rows16(A, N))
        FP_CUDA(cudaMemcpy2DAsync(sl.A32, (size_t)ldt * 4, A, (size_t)N * 4, (size_t)N * 4, N,
                                  cudaMemcpyDeviceToDevice, s));
    if (!rows16(A2, m))
        FP_CUDA(cudaMemcpy2DAsync(sl.A232, (size_t)ldx * 4, A2, (size_t)m * 4, (size_t)m * 4, m,
                                  cudaMemcpyDeviceToDevice, s));
    int lda = 0, lda2 = 0;
    const float* Aop = f32_operand(A, N, sl.A32, &lda);
    const float* A2op = f32_operand(A2, m, sl.A232, &lda2);
    GemmF32TGroup g1{}, g2{};
    g1.count = g2.count = 1;
    g1.tile_m = g2.tile_m = f32_tile(h, N, 1);
    g1.a[0] = GemmF32TArgs{sl.X, ldx, Aop, lda, sl.T, ldt, nullptr, 0, 0.f, m, N, N, nullptr};
    g2.a[0] = GemmF32TArgs{sl.T, ldt, A2op, lda2, Y, ldy, lambda != 0.f ? K : nullptr, m, lambda, N, m, m, nullptr};
    FP_CUDA(gemm_f32t_group(g1, s));
    FP_CUDA(gemm_f32t_group(g2, s));
    return FASTPFP_OK;
}

int fastpfp_affinity(fastpfp_t h, void* stream, const float* B, const float* B2, int N, int m,
                     int k, float* K) {
    if (!h || !B || !B2 || !K || N < 1 || m < 1 || k < 1 || k > kMaxK) return FASTPFP_ERR_ARG;
    if (N > h->max_n || m > h->max_n) return FASTPFP_ERR_SIZE;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    FP_CUDA(affinity(B, B2, N, m, k, K, m, (cudaStream_t)stream));
    return FASTPFP_OK;
}

int fastpfp_project(fastpfp_t h, void* stream, float* Y, int N, double tol, int max_iter, int* iters,
                    double* last_delta) {
    if (!h || !Y || N < 1 || max_iter < 1 || !(tol >= 0.0)) return FASTPFP_ERR_ARG;
    if (N > h->max_n) return FASTPFP_ERR_SIZE;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const Slot& sl = h->slots[0];
    const int ldy = round4(N);
    FP_CUDA(cudaMemsetAsync(sl.ctrl, 0, kCtrlHeader, s));
    FP_CUDA(cudaMemsetAsync(sl.colbuf, 0, colbuf_bytes(h->ld), s));
    FP_CUDA(cudaMemsetAsync(sl.sbuf, 0, 3 * sizeof(double), s));
    FP_CUDA(cudaMemsetAsync(sl.dbuf, 0, kDbufWords * sizeof(unsigned), s));
    FP_CUDA(cudaMemsetAsync(sl.Y, 0, (size_t)N * ldy * sizeof(float), s));
    FP_CUDA(cudaMemcpy2DAsync(sl.Y, (size_t)ldy * 4, Y, (size_t)N * 4, (size_t)N * 4, N,
                              cudaMemcpyDeviceToDevice, s));
    PdLaunch L;
    pd_plan(N, h->num_sms, &L);
    PdParams P{};
    P.Y = sl.Y;
    P.N = N;
    P.ldy = ldy;
    P.m = N;
    P.tol_inner = tol;
    P.max_inner = max_iter;
    P.colbuf = sl.colbuf;
    P.sbuf = sl.sbuf;
    P.dbuf = sl.dbuf;
    P.ctrl = sl.ctrl;
    P.timeout_ns = 2000ll * 1000000ll;
    P.rpc = L.rpc;
    P.mode = kPdProjectOnly;
    FP_CUDA(pd_launch(L, P, s));
    FP_CUDA(cudaMemcpy2DAsync(Y, (size_t)N * 4, sl.Y, (size_t)ldy * 4, (size_t)N * 4, N,
                              cudaMemcpyDeviceToDevice, s));
    FP_CUDA(cudaMemcpyAsync(&h->host_ctrl[0], sl.ctrl, kCtrlHeader, cudaMemcpyDeviceToHost, s));
    if (cudaStreamSynchronize(s) != cudaSuccess) return FASTPFP_ERR_CUDA;
    const Ctrl& c = h->host_ctrl[0];
    if (iters) *iters = c.last_inner;
    if (last_delta) *last_delta = c.last_delta;
    return c.error != 0 ? c.error : FASTPFP_OK;
}

int fastpfp_discretize(fastpfp_t h, void* stream, const float* X, int N, int m,
                       int32_t* row_of_col) {
    if (!h || !X || !row_of_col || N < 1 || m < 1 || m > N) return FASTPFP_ERR_ARG;
    if (N > h->max_n) return FASTPFP_ERR_SIZE;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const Slot& sl = h->slots[0];
    FP_CUDA(cudaMemsetAsync(sl.ctrl, 0, kCtrlHeader, s));
    FP_CUDA(discretize(X, N, m, m, sl.disc, sl.ctrl, 2000ll * 1000000ll, h->num_sms, s));
    FP_CUDA(cudaMemcpyAsync(row_of_col, sl.disc.col_match, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
    return FASTPFP_OK;
}

}  // extern "C"

namespace {

// Features, MLP and S = E_big E_small^T / 8 of a canonical pair into slot 0's
// Y (leading dimension round4(m)); keeps the activations for the backward.
int ws_forward(fastpfp_t h, cudaStream_t s, const Problem& q, int kk, const float* params) {
    const Slot& sl = h->slots[0];
    const int N = q.N, m = q.m, ldS = round4(m);
    auto& w = h->ws;
    FP_CUDA(ws_features(q.A, N, kk ? q.B : nullptr, kk, w.Fb, s));
    FP_CUDA(ws_features(q.A2, m, kk ? q.B2 : nullptr, kk, w.Fs, s));
    FP_CUDA(ws_mlp_forward(w.Fb, N, params, w.Hb, w.Eb, 1.0f, s));
    FP_CUDA(ws_mlp_forward(w.Fs, m, params, w.Hs, w.Es, 1.0f, s));
    // E_big / 8 (exact) so that the product is S; E_small / 8 for dE_big
    FP_CUDA(cudaMemcpyAsync(w.Eb8, w.Eb, (size_t)N * kMlpOut * 4, cudaMemcpyDeviceToDevice, s));
    FP_CUDA(ws_scale(w.Eb8, (size_t)N * kMlpOut, 0.125f, s));
    FP_CUDA(cudaMemcpyAsync(w.Es8, w.Es, (size_t)m * kMlpOut * 4, cudaMemcpyDeviceToDevice, s));
    FP_CUDA(ws_scale(w.Es8, (size_t)m * kMlpOut, 0.125f, s));
    FP_CUDA(ws_transpose(w.Es, m, kMlpOut, kMlpOut, w.EsT, ldS, s));
    GemmF32Args g{w.Eb8, kMlpOut, w.EsT, ldS, sl.Y, ldS, nullptr, 0, 0.f, N, m, kMlpOut, nullptr};
    FP_CUDA(gemm_f32(g, s));
    return FASTPFP_OK;
}

int ws_check(fastpfp_t h, const float* A, int n_a, const float* A2, int n_b, const float* B, const float* B2,
             int k, const float* params) {
    if (!h || !A || !A2 || !params || n_a < 1 || n_b < 1 || k < 0) return FASTPFP_ERR_ARG;
    if (k > 0 && (!B || !B2)) return FASTPFP_ERR_ARG;
    if (n_a > h->max_n || n_b > h->max_n) return FASTPFP_ERR_SIZE;
    return FASTPFP_OK;
}

}  // namespace

extern "C" {

int fastpfp_warmstart(fastpfp_t h, void* stream, const float* A, int n_a, const float* A2, int n_b,
                      const float* B, const float* B2, int k, const float* params, int sinkhorn_iters,
                      float* X0_out) {
    int rc = ws_check(h, A, n_a, A2, n_b, B, B2, k, params);
    if (rc != FASTPFP_OK) return rc;
    if (!X0_out || sinkhorn_iters < 0) return FASTPFP_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int kk = k < 15 ? k : 15;
    const Problem q = canonical(A, n_a, A2, n_b, B, B2, kk, 1.0f, nullptr, nullptr, X0_out);
    rc = ws_forward(h, s, q, kk, params);
    if (rc != FASTPFP_OK) return rc;
    const Slot& sl = h->slots[0];
    const int ldS = round4(q.m);
    FP_CUDA(ws_sinkhorn(sl.Y, q.N, q.m, ldS, sinkhorn_iters, reinterpret_cast<float*>(h->ws.part),
                        h->ws.scalar, s));
    FP_CUDA(write_outputs(nullptr, q.N, q.m, q.transposed, nullptr, sl.Y, ldS, X0_out, s));
    return FASTPFP_OK;
}

int fastpfp_warmstart_train_step(fastpfp_t h, void* stream, const float* A, int n_a, const float* A2,
                                 int n_b, const float* B, const float* B2, int k, const int32_t* perm,
                                 float* params, float* adam_m, float* adam_v, int step, float lr,
                                 double* loss_out, float* grad_out) {
    int rc = ws_check(h, A, n_a, A2, n_b, B, B2, k, params);
    if (rc != FASTPFP_OK) return rc;
    if (!perm || step < 0 || (step > 0 && (!adam_m || !adam_v)) || !(lr >= 0.f)) return FASTPFP_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int kk = k < 15 ? k : 15;
    const Problem q = canonical(A, n_a, A2, n_b, B, B2, kk, 1.0f, nullptr, nullptr, nullptr);
    const int N = q.N, m = q.m, ldS = round4(m);
    auto& w = h->ws;
    const Slot& sl = h->slots[0];
    rc = ws_forward(h, s, q, kk, params);
    if (rc != FASTPFP_OK) return rc;
    FP_CUDA(ws_targets(perm, n_a, q.transposed, N, m, w.t, w.tinv, s));
    // dL/dS into slot 0's T (N x ldS), its transpose into slot 0's K (m x round4(N))
    FP_CUDA(ws_loss_grad_S(sl.Y, N, m, ldS, w.t, w.tinv, w.lse_c, w.lse_r, w.part, sl.T, ldS, w.loss, s));
    FP_CUDA(ws_transpose(sl.T, N, m, ldS, sl.K, round4(N), s));
    GemmF32Args gb{sl.T, ldS, w.Es8, kMlpOut, w.dEb, kMlpOut, nullptr, 0, 0.f, N, kMlpOut, m, nullptr};
    GemmF32Args gs{sl.K, round4(N), w.Eb8, kMlpOut, w.dEs, kMlpOut, nullptr, 0, 0.f, m, kMlpOut, N, nullptr};
    FP_CUDA(gemm_f32(gb, s));   // dE_big = dS E_small / 8
    FP_CUDA(gemm_f32(gs, s));   // dE_small = dS^T E_big / 8
    FP_CUDA(ws_mlp_backward(w.Fb, w.Hb, w.dEb, N, params, w.dH, w.grad, 0, s));
    FP_CUDA(ws_mlp_backward(w.Fs, w.Hs, w.dEs, m, params, w.dH, w.grad, 1, s));
    if (grad_out)
        FP_CUDA(cudaMemcpyAsync(grad_out, w.grad, kMlpParams * 4, cudaMemcpyDeviceToDevice, s));
    if (step > 0) FP_CUDA(ws_adam(params, adam_m, adam_v, w.grad, step, lr, s));
    if (loss_out) {
        FP_CUDA(cudaMemcpyAsync(loss_out, w.loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        if (cudaStreamSynchronize(s) != cudaSuccess) return FASTPFP_ERR_CUDA;
    }
    return FASTPFP_OK;
}

}  // extern "C"
