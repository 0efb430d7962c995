// fastpfp_api.cu -- the C ABI declared in include/fastpfp.h.
//
// A handle owns every device buffer the solver touches, allocated once in
// fastpfp_create for graphs of up to max_n nodes.  A solve enqueues, on the
// caller's stream, the whole of Algorithm 1 without host round trips: for
// every outer iteration the two products of the gradient and one cooperative
// launch of the projection kernel, which also blends, normalises and decides
// (on the device) whether the loop continues.  Launches after the decision
// to stop return at once.  The greedy discretisation and the objective
// follow, and the control block is copied back once at the end.
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "common.cuh"
#include "internal.h"

using namespace fpfp;

namespace {

constexpr int kMaxN = 16384;     // four float4 column quads per thread of a 1024-thread CTA
constexpr int kMaxK = 256;       // attribute dimension staged by fastpfp_match_host
constexpr size_t kCtrlHeader = offsetof(Ctrl, inner_trace);
constexpr int kProfIters = 128;                   // outer iterations timed when profile = 1
constexpr int kProfEvents = 2 * kProfIters + 3;   // iteration boundaries + discretisation

inline int round4(int x) { return (x + 3) & ~3; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

struct fastpfp_s {
    int device = 0, max_n = 0, max_batch = 0, num_sms = 0, ld = 0;
    char* pool = nullptr;
    size_t pool_bytes = 0;
    float *Y = nullptr, *X = nullptr, *T = nullptr, *K = nullptr;
    __nv_bfloat16 *A16 = nullptr, *A216 = nullptr, *Xt16 = nullptr, *T16 = nullptr;
    float* colbuf = nullptr;
    double* sbuf = nullptr;
    unsigned* dbuf = nullptr;
    Ctrl* ctrl = nullptr;
    DiscBuffers disc{};
    // staging for fastpfp_match_host
    float *sA = nullptr, *sA2 = nullptr, *sB = nullptr, *sB2 = nullptr, *sX0 = nullptr, *sXout = nullptr;
    int32_t* sperm = nullptr;
    Ctrl* host_ctrl = nullptr;   // pinned, max_batch control-block headers
    int last_outer = 0;
    cudaEvent_t ev[kProfEvents] = {};
};

namespace {

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
    if (p->precision != FASTPFP_FP32 && p->precision != FASTPFP_BF16) return false;
    if (p->refine_iters < 0) return false;
    return true;
}

long long timeout_ns(const fastpfp_params* p) {
    const int ms = (p && p->timeout_ms > 0) ? p->timeout_ms : 2000;
    return (long long)ms * 1000000ll;
}

// The projection kernel leaves its rotating accumulators zero when it
// completes; a launch that stopped on an error may not.  Every solve
// therefore starts from cleared accumulators.
cudaError_t clear_accumulators(fastpfp_t h, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(h->colbuf, 0, 3 * (size_t)h->ld * sizeof(float), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(h->sbuf, 0, 3 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(h->dbuf, 0, 3 * sizeof(unsigned), s);
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

// Enqueues one whole solve on stream s.  The control-block header lands in
// *host_slot (pinned) once the stream reaches the end of the solve.  With
// p->profile the handle's events bracket every phase; *launches receives the
// number of kernels enqueued.
int enqueue_solve(fastpfp_t h, cudaStream_t s, const Problem& q, const fastpfp_params* p,
                  Ctrl* host_slot, int* launches) {
    const int N = q.N, m = q.m;
    const int ldy = round4(N), ldx = round4(m);
    const bool bf16 = p->precision == FASTPFP_BF16;
    if (bf16) return FASTPFP_ERR_UNSUPPORTED;

    FP_CUDA(cudaMemsetAsync(h->ctrl, 0, kCtrlHeader, s));
    FP_CUDA(clear_accumulators(h, s));
    FP_CUDA(cudaMemsetAsync(h->Y, 0, (size_t)N * ldy * sizeof(float), s));
    FP_CUDA(init_ctrl(h->ctrl, bf16 ? 1 : 0, s));
    const float* Kp = nullptr;
    if (q.k > 0) {
        FP_CUDA(affinity(q.B, q.B2, N, m, q.k, h->K, ldx, s));
        Kp = h->K;
    }
    FP_CUDA(init_x(h->X, N, m, ldx, q.X0, q.transposed, bf16 ? h->Xt16 : nullptr, ldy, s));

    PdLaunch L;
    pd_plan(N, h->num_sms, &L);
    PdParams P{};
    P.Y = h->Y;
    P.N = N;
    P.ldy = ldy;
    P.m = m;
    P.X = h->X;
    P.ldx = ldx;
    P.Xt16 = bf16 ? h->Xt16 : nullptr;
    P.ldxt = ldy;
    P.alpha = p->alpha;
    P.normalize = p->normalize_max ? 1 : 0;
    P.slack_reset = p->slack_policy == 1 ? 1 : 0;
    P.tol_inner = p->tol_inner;
    P.max_inner = p->max_inner;
    P.tol_outer = p->tol_outer;
    P.max_outer = p->max_outer;
    P.refine_iters = p->refine_iters;
    P.switch_tol = p->switch_tol;
    P.colbuf = h->colbuf;
    P.sbuf = h->sbuf;
    P.dbuf = h->dbuf;
    P.ctrl = h->ctrl;
    P.timeout_ns = timeout_ns(p);
    P.rpc = L.rpc;
    P.mode = kPdOuterStep;
    P.skip_arrive = (p->debug_flags & 1) ? 1 : 0;

    GemmF32Args g1{q.A, N, h->X, ldx, h->T, ldx, nullptr, 0, 0.f, N, m, N, h->ctrl};
    GemmF32Args g2{h->T, ldx, q.A2, m, h->Y, ldy, Kp, ldx, q.k ? (float)p->lambda : 0.f, N, m, m,
                   h->ctrl};
    const bool prof = p->profile != 0;
    int nl = 2 + (q.k > 0 ? 1 : 0);   // init_ctrl, init_x, affinity
    for (int t = 0; t < p->max_outer; ++t) {
        const bool pt = prof && t < kProfIters;
        if (pt && t == 0) FP_CUDA(cudaEventRecord(h->ev[0], s));
        FP_CUDA(gemm_f32(g1, s));   // T = A X
        FP_CUDA(gemm_f32(g2, s));   // Y[:, :m] = T A' + lambda K
        if (pt) FP_CUDA(cudaEventRecord(h->ev[2 * t + 1], s));
        FP_CUDA(pd_launch(L, P, s));
        if (pt) FP_CUDA(cudaEventRecord(h->ev[2 * t + 2], s));
        nl += 3;
    }
    if (prof) FP_CUDA(cudaEventRecord(h->ev[kProfEvents - 2], s));
    FP_CUDA(discretize(h->X, N, m, ldx, h->disc, h->ctrl, timeout_ns(p), h->num_sms, s));
    if (prof) FP_CUDA(cudaEventRecord(h->ev[kProfEvents - 1], s));
    FP_CUDA(objective(q.A, N, q.A2, m, Kp, ldx, q.k ? (float)p->lambda : 0.f, h->disc.col_match,
                      h->ctrl, s));
    FP_CUDA(write_outputs(h->disc.col_match, N, m, q.transposed, q.perm_out, h->X, ldx, q.X_out, s));
    nl += 2 + (q.perm_out ? (q.transposed ? 1 : 2) : 0) + (q.X_out ? 1 : 0);
    FP_CUDA(cudaMemcpyAsync(host_slot, h->ctrl, kCtrlHeader, cudaMemcpyDeviceToHost, s));
    if (launches) *launches = nl;
    return FASTPFP_OK;
}

// Per-phase times of the last profiled solve (call after the stream synced).
void read_profile(fastpfp_t h, int outer, int max_outer, fastpfp_stats* st) {
    if (!st) return;
    float g = 0.f, pr = 0.f, d = 0.f, x = 0.f;
    const int T = outer < kProfIters ? outer : kProfIters;
    (void)max_outer;
    for (int t = 0; t < T; ++t) {
        if (cudaEventElapsedTime(&x, h->ev[2 * t], h->ev[2 * t + 1]) == cudaSuccess) g += x;
        if (cudaEventElapsedTime(&x, h->ev[2 * t + 1], h->ev[2 * t + 2]) == cudaSuccess) pr += x;
    }
    if (cudaEventElapsedTime(&x, h->ev[kProfEvents - 2], h->ev[kProfEvents - 1]) == cudaSuccess) d = x;
    st->ms_gemm = g;
    st->ms_proj = pr;
    st->ms_disc = d;
}

int fill_stats(const Ctrl& c, int transposed, int launches, fastpfp_stats* st) {
    const int status = c.error != 0 ? c.error : FASTPFP_OK;
    if (st) {
        st->launches = launches;
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
    p->debug_flags = 0;
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
    if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
        pd_configure() != cudaSuccess || disc_configure() != cudaSuccess) {
        delete h;
        return FASTPFP_ERR_CUDA;
    }
    const size_t n = (size_t)max_n, ld = (size_t)h->ld;
    const size_t f32mat = align256(n * ld * sizeof(float));
    const size_t b16mat = align256(n * ld * sizeof(__nv_bfloat16));
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    const size_t oY = take(f32mat), oX = take(f32mat), oT = take(f32mat), oK = take(f32mat);
    const size_t oA16 = take(b16mat), oA216 = take(b16mat), oXt16 = take(b16mat), oT16 = take(b16mat);
    const size_t ocol = take(3 * ld * sizeof(float)), os = take(3 * sizeof(double)),
                 od = take(3 * sizeof(unsigned)), octrl = take(sizeof(Ctrl));
    const size_t orm = take(n * 4), ocm = take(n * 4), orb = take(n * 8), ocb = take(2 * n * 8);
    const size_t osA = take(n * n * 4), osA2 = take(n * n * 4), osB = take(n * kMaxK * 4),
                 osB2 = take(n * kMaxK * 4), osX0 = take(n * n * 4), osXo = take(n * n * 4),
                 osp = take(n * 4);
    h->pool_bytes = off;
    if (cudaMalloc(&h->pool, off) != cudaSuccess) {
        delete h;
        return FASTPFP_ERR_CUDA;
    }
    if (cudaMallocHost(&h->host_ctrl, sizeof(Ctrl) * (size_t)max_batch) != cudaSuccess) {
        cudaFree(h->pool);
        delete h;
        return FASTPFP_ERR_CUDA;
    }
    char* b = h->pool;
    h->Y = (float*)(b + oY);
    h->X = (float*)(b + oX);
    h->T = (float*)(b + oT);
    h->K = (float*)(b + oK);
    h->A16 = (__nv_bfloat16*)(b + oA16);
    h->A216 = (__nv_bfloat16*)(b + oA216);
    h->Xt16 = (__nv_bfloat16*)(b + oXt16);
    h->T16 = (__nv_bfloat16*)(b + oT16);
    h->colbuf = (float*)(b + ocol);
    h->sbuf = (double*)(b + os);
    h->dbuf = (unsigned*)(b + od);
    h->ctrl = (Ctrl*)(b + octrl);
    h->disc.row_match = (int32_t*)(b + orm);
    h->disc.col_match = (int32_t*)(b + ocm);
    h->disc.row_best = (unsigned long long*)(b + orb);
    h->disc.col_best = (unsigned long long*)(b + ocb);
    h->sA = (float*)(b + osA);
    h->sA2 = (float*)(b + osA2);
    h->sB = (float*)(b + osB);
    h->sB2 = (float*)(b + osB2);
    h->sX0 = (float*)(b + osX0);
    h->sXout = (float*)(b + osXo);
    h->sperm = (int32_t*)(b + osp);
    for (int e = 0; e < kProfEvents; ++e) {
        if (cudaEventCreate(&h->ev[e]) != cudaSuccess) {
            for (int f = 0; f < e; ++f) cudaEventDestroy(h->ev[f]);
            cudaFreeHost(h->host_ctrl);
            cudaFree(h->pool);
            delete h;
            return FASTPFP_ERR_CUDA;
        }
    }
    if (cudaMemset(h->pool, 0, off) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        for (int e = 0; e < kProfEvents; ++e) cudaEventDestroy(h->ev[e]);
        cudaFreeHost(h->host_ctrl);
        cudaFree(h->pool);
        delete h;
        return FASTPFP_ERR_CUDA;
    }
    *out = h;
    return FASTPFP_OK;
}

void fastpfp_destroy(fastpfp_t h) {
    if (!h) return;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (int e = 0; e < kProfEvents; ++e)
        if (h->ev[e]) cudaEventDestroy(h->ev[e]);
    if (h->host_ctrl) cudaFreeHost(h->host_ctrl);
    if (h->pool) cudaFree(h->pool);
    delete h;
}

int fastpfp_match(fastpfp_t h, void* stream, const float* A, int n_a, const float* A2, int n_b,
                  const float* B, const float* B2, int k, const fastpfp_params* p, const float* X0,
                  int32_t* perm_out, float* X_out, fastpfp_stats* st) {
    int rc = check_pair(h, A, n_a, A2, n_b, B, B2, k, p, perm_out);
    if (rc != FASTPFP_OK) return rc;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const Problem q = canonical(A, n_a, A2, n_b, B, B2, k, p->lambda, X0, perm_out, X_out);
    int nl = 0;
    rc = enqueue_solve(h, s, q, p, &h->host_ctrl[0], &nl);
    if (rc != FASTPFP_OK) return rc;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FASTPFP_ERR_CUDA;
    h->last_outer = h->host_ctrl[0].outer;
    rc = fill_stats(h->host_ctrl[0], q.transposed, nl, st);
    if (p->profile) read_profile(h, h->host_ctrl[0].outer, p->max_outer, st);
    return rc;
}

int fastpfp_match_host(fastpfp_t h, void* stream, const float* A, int n_a, const float* A2, int n_b,
                       const float* B, const float* B2, int k, const fastpfp_params* p,
                       const float* X0, int32_t* perm_out, float* X_out, fastpfp_stats* st) {
    int rc = check_pair(h, A, n_a, A2, n_b, B, B2, k, p, perm_out);
    if (rc != FASTPFP_OK) return rc;
    const int kk = (k > 0 && p->lambda != 0.f) ? k : 0;
    if (kk > kMaxK) return FASTPFP_ERR_SIZE;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    FP_CUDA(cudaMemcpyAsync(h->sA, A, (size_t)n_a * n_a * 4, cudaMemcpyHostToDevice, s));
    FP_CUDA(cudaMemcpyAsync(h->sA2, A2, (size_t)n_b * n_b * 4, cudaMemcpyHostToDevice, s));
    if (kk) {
        FP_CUDA(cudaMemcpyAsync(h->sB, B, (size_t)n_a * kk * 4, cudaMemcpyHostToDevice, s));
        FP_CUDA(cudaMemcpyAsync(h->sB2, B2, (size_t)n_b * kk * 4, cudaMemcpyHostToDevice, s));
    }
    if (X0) FP_CUDA(cudaMemcpyAsync(h->sX0, X0, (size_t)n_a * n_b * 4, cudaMemcpyHostToDevice, s));
    const Problem q = canonical(h->sA, n_a, h->sA2, n_b, kk ? h->sB : nullptr, kk ? h->sB2 : nullptr,
                                kk, p->lambda, X0 ? h->sX0 : nullptr, h->sperm,
                                X_out ? h->sXout : nullptr);
    int nl = 0;
    rc = enqueue_solve(h, s, q, p, &h->host_ctrl[0], &nl);
    if (rc != FASTPFP_OK) return rc;
    FP_CUDA(cudaMemcpyAsync(perm_out, h->sperm, (size_t)n_a * 4, cudaMemcpyDeviceToHost, s));
    if (X_out)
        FP_CUDA(cudaMemcpyAsync(X_out, h->sXout, (size_t)n_a * n_b * 4, cudaMemcpyDeviceToHost, s));
    if (cudaStreamSynchronize(s) != cudaSuccess) return FASTPFP_ERR_CUDA;
    h->last_outer = h->host_ctrl[0].outer;
    rc = fill_stats(h->host_ctrl[0], q.transposed, nl, st);
    if (p->profile) read_profile(h, h->host_ctrl[0].outer, p->max_outer, st);
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
    cudaStream_t s = (cudaStream_t)stream;
    int worst = FASTPFP_OK;
    for (int b = 0; b < count; ++b) {
        const fastpfp_pair& x = pairs[b];
        const Problem q = canonical(x.A, x.n_a, x.A2, x.n_b, x.B, x.B2, x.k, p->lambda, x.X0,
                                    x.perm_out, x.X_out);
        int nl = 0;
        int rc = enqueue_solve(h, s, q, p, &h->host_ctrl[b], &nl);
        if (rc != FASTPFP_OK) return rc;
        if (p->profile || b + 1 == count) {
            // profiled batches read each pair's events before they are reused
            if (cudaStreamSynchronize(s) != cudaSuccess) return FASTPFP_ERR_CUDA;
        }
        if (p->profile) {
            rc = fill_stats(h->host_ctrl[b], q.transposed, nl, st ? &st[b] : nullptr);
            if (st) read_profile(h, h->host_ctrl[b].outer, p->max_outer, &st[b]);
            if (rc != FASTPFP_OK && worst == FASTPFP_OK) worst = rc;
        } else if (st) {
            st[b].launches = nl;
        }
    }
    if (!p->profile) {
        for (int b = 0; b < count; ++b) {
            const int tr = pairs[b].n_a < pairs[b].n_b;
            const int nl = st ? st[b].launches : 0;
            int rc = fill_stats(h->host_ctrl[b], tr, nl, st ? &st[b] : nullptr);
            if (rc != FASTPFP_OK && worst == FASTPFP_OK) worst = rc;
        }
    }
    if (count > 0) h->last_outer = h->host_ctrl[count - 1].outer;
    return worst;
}

int fastpfp_last_trace(fastpfp_t h, int* inner_counts, double* deltas, int cap) {
    if (!h || cap < 0) return FASTPFP_ERR_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    const int n = h->last_outer < cap ? h->last_outer : cap;
    if (n > 0 && inner_counts)
        FP_CUDA(cudaMemcpy(inner_counts, h->ctrl->inner_trace, (size_t)n * sizeof(int),
                           cudaMemcpyDeviceToHost));
    if (n > 0 && deltas)
        FP_CUDA(cudaMemcpy(deltas, h->ctrl->delta_trace, (size_t)n * sizeof(double),
                           cudaMemcpyDeviceToHost));
    return h->last_outer;
}

int fastpfp_gradient(fastpfp_t h, void* stream, const float* A, const float* X, const float* A2,
                     const float* K, float lambda, int N, int m, float* Y, int ldy, int precision) {
    if (!h || !A || !X || !A2 || !Y || N < 1 || m < 1 || m > N || ldy < m) return FASTPFP_ERR_ARG;
    if (lambda != 0.f && !K) return FASTPFP_ERR_ARG;
    if (N > h->max_n) return FASTPFP_ERR_SIZE;
    if (precision != FASTPFP_FP32) return FASTPFP_ERR_UNSUPPORTED;
    if (cudaSetDevice(h->device) != cudaSuccess) return FASTPFP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    GemmF32Args g1{A, N, X, m, h->T, m, nullptr, 0, 0.f, N, m, N, nullptr};
    GemmF32Args g2{h->T, m, A2, m, Y, ldy, lambda != 0.f ? K : nullptr, m, lambda, N, m, m, nullptr};
    FP_CUDA(gemm_f32(g1, s));
    FP_CUDA(gemm_f32(g2, s));
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
    const int ldy = round4(N);
    FP_CUDA(cudaMemsetAsync(h->ctrl, 0, kCtrlHeader, s));
    FP_CUDA(clear_accumulators(h, s));
    FP_CUDA(cudaMemsetAsync(h->Y, 0, (size_t)N * ldy * sizeof(float), s));
    FP_CUDA(cudaMemcpy2DAsync(h->Y, (size_t)ldy * 4, Y, (size_t)N * 4, (size_t)N * 4, N,
                              cudaMemcpyDeviceToDevice, s));
    PdLaunch L;
    pd_plan(N, h->num_sms, &L);
    PdParams P{};
    P.Y = h->Y;
    P.N = N;
    P.ldy = ldy;
    P.m = N;
    P.tol_inner = tol;
    P.max_inner = max_iter;
    P.colbuf = h->colbuf;
    P.sbuf = h->sbuf;
    P.dbuf = h->dbuf;
    P.ctrl = h->ctrl;
    P.timeout_ns = 2000ll * 1000000ll;
    P.rpc = L.rpc;
    P.mode = kPdProjectOnly;
    FP_CUDA(pd_launch(L, P, s));
    FP_CUDA(cudaMemcpy2DAsync(Y, (size_t)N * 4, h->Y, (size_t)ldy * 4, (size_t)N * 4, N,
                              cudaMemcpyDeviceToDevice, s));
    FP_CUDA(cudaMemcpyAsync(&h->host_ctrl[0], h->ctrl, kCtrlHeader, cudaMemcpyDeviceToHost, s));
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
    FP_CUDA(cudaMemsetAsync(h->ctrl, 0, kCtrlHeader, s));
    FP_CUDA(discretize(X, N, m, m, h->disc, h->ctrl, 2000ll * 1000000ll, h->num_sms, s));
    FP_CUDA(cudaMemcpyAsync(row_of_col, h->disc.col_match, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
    return FASTPFP_OK;
}

}  // extern "C"
