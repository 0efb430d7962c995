// wave_stream.cu -- the planner of a batch streamed through waves inside one
// CUDA graph.
//
// A batch larger than one wave keeps a wave full: pairs that stopped leave,
// waiting pairs join while the wave's band plan still fits on chip.  This
// kernel takes those decisions on the device after every outer iteration
// (one CTA): it reads the stop words of the wave's pairs, admits waiting
// pairs in batch order, cuts the new wave into bands with the shared band
// planner (band_plan.cuh; its binary search on the band cost bound runs as
// rounds of candidate bounds evaluated by all threads at once, and finds the
// same bound as the host's search), and writes the wave tables pdb_kernel
// reads.  The products run over every pair of the batch and skip the pairs
// that are idle (not in the wave), so no launch depends on host decisions
// and the whole repeat loop is one graph launch.
#include "band_plan.cuh"
#include "common.cuh"
#include "internal.h"

namespace fpfp {
namespace {

constexpr int kPlanThreads = 512;

struct PlanShared {
    int list[kMaxWavePairs + 1];   // pair indices of the wave being planned, in admission order
    int Ns[kMaxWavePairs + 1];     // their canonical row counts
    int n;                         // pairs in list
    int best;                      // smallest candidate index whose cut fits
    long long lo, hi;              // search interval of the band cost bound
    int Gmax, t2, ok;
    int G;                         // bands of the cut being finished
    int pre[kMaxWavePairs + 2];    // prefix sums of Ns: pair p holds rows [pre[p], pre[p + 1])
    int mx[4];                     // maxima over the bands: rows, columns, shared-memory floats, segments
    int rp;                        // the most row-partial slots a pair needs
    WavePlan plan;                 // the last plan that fit
    WavePlan trial;
};

// The smallest band cost bound whose greedy cut needs at most Gmax bands, for
// the pairs Ns[0..n): rounds in which every thread tests one of kPlanThreads
// bounds spread over the interval; the interval shrinks to the step between
// the last bound that did not fit and the first that did.  Block-wide.
__device__ long long search_bound(PlanShared& S, const int* Ns, int n, long long seg_cost, int Gmax) {
    const int tid = threadIdx.x;
    constexpr int nthr = kPlanThreads;   // the launch's block size (a power of two: shifts, not divisions)
    if (tid == 0) cut_interval(Ns, n, seg_cost, Gmax, &S.lo, &S.hi);
    __syncthreads();
    while (true) {
        const long long lo = S.lo, hi = S.hi;
        if (lo >= hi) break;   // every thread reads the same interval
        __syncthreads();
        if (tid == 0) S.best = nthr;
        __syncthreads();
        const long long C = lo + ((hi - lo) * (long long)(tid + 1)) / nthr;   // thread nthr - 1 tests hi
        if (cut_rows(Ns, n, C, seg_cost, Gmax, nullptr) <= Gmax) atomicMin(&S.best, tid);
        __syncthreads();
        if (tid == 0) {
            const int t = S.best < nthr ? S.best : nthr - 1;   // hi always fits (one band holds all)
            S.hi = lo + ((hi - lo) * (long long)(t + 1)) / nthr;
            S.lo = t == 0 ? lo : lo + ((hi - lo) * (long long)t) / nthr + 1;
        }
        __syncthreads();
    }
    return S.lo;
}

// finish_plan of band_plan.cuh with the bands' statistics spread over the
// block (one band per thread; the maxima are order-free, so the layout is
// the same).  Block-wide; returns S.ok.
__device__ bool finish_plan_par(PlanShared& S, const int* Ns, int n, long long C, long long seg_cost, int Gmax,
                                int t2, WavePlan* w) {
    const int tid = threadIdx.x;
    constexpr int nthr = kPlanThreads;
    if (tid == 0) {
        S.pre[0] = 0;
        for (int i = 0; i < n; ++i) S.pre[i + 1] = S.pre[i] + Ns[i];
        const int used = cut_rows(Ns, n, C, seg_cost, Gmax, w->band);
        for (int c = used; c <= Gmax; ++c) w->band[c] = S.pre[n];
        S.G = used > 1 ? used : 1;
        S.mx[0] = S.mx[1] = S.mx[2] = S.mx[3] = 0;
        S.rp = 1;
    }
    __syncthreads();
    for (int b = tid; b < S.G; b += nthr) {
        const int lo = w->band[b], hi = w->band[b + 1];
        int a = 0, z = n - 1;   // the first pair whose rows end after lo
        while (a < z) {
            const int mid = (a + z) >> 1;
            if (S.pre[mid + 1] > lo) z = mid; else a = mid + 1;
        }
        const BandStat st = band_stat(Ns, n, a, S.pre[a], lo, hi, t2);
        atomicMax(&S.mx[0], st.rows);
        atomicMax(&S.mx[1], st.cols);
        atomicMax(&S.mx[2], st.elems);
        atomicMax(&S.mx[3], st.segs);
    }
    for (int i = tid; i < n; i += nthr) atomicMax(&S.rp, pdb_row_warps(bp_round4(Ns[i]), kPdbThreads, t2));
    __syncthreads();
    if (tid == 0) {
        PdbLayout L{S.mx[0], S.mx[1], S.mx[2], S.rp, t2, S.mx[3] > 1 ? S.mx[3] : 1, n};
        S.ok = layout_fits(&L, &w->smem) ? 1 : 0;
        if (S.ok) {
            w->grid = S.G;
            w->layout = L;
        }
    }
    __syncthreads();
    return S.ok != 0;
}

// plan_bands_seq of band_plan.cuh with the bound search and the bands'
// statistics spread over the block; the result (into *w) is the same.
// Block-wide; returns S.ok.
__device__ bool plan_bands_par(PlanShared& S, const int* Ns, int n, int num_sms, int max_level, WavePlan* w) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        wave_shape(Ns, n, num_sms, &S.Gmax, &S.t2);
        S.ok = 0;
    }
    __syncthreads();
    for (int lv = 0; lv <= max_level && lv < 4; ++lv) {
        const long long seg_cost = seg_cost_of_level(lv);
        const long long C = search_bound(S, Ns, n, seg_cost, S.Gmax);
        if (finish_plan_par(S, Ns, n, C, seg_cost, S.Gmax, S.t2, w)) break;
    }
    return S.ok != 0;
}

// Admission candidates planned side by side: group g of kAdmitGroups (each
// kPlanThreads / kAdmitGroups threads) plans the wave of the first n + g + 1
// pairs of the list at the admission level -- the plans the sequential
// admission loop would make one after another, so the first that does not
// fit decides the same admissions.  Each group's search and finish are those
// of plan_bands_par with fewer candidate bounds per round (the same
// smallest bound: the band count never grows with the bound).
constexpr int kAdmitGroups = 8;
constexpr int kGroupThreads = kPlanThreads / kAdmitGroups;
struct GroupPlan {
    long long lo, hi;
    int best, Gmax, t2, ok, G, live;
    int mx[4];
    int rp;
    WavePlan w;
};

// Block-wide: groups 0..K-1 plan n + 1 .. n + K pairs at segment cost
// seg_cost (S.pre must hold the prefix sums of S.Ns up to n + K).
__device__ void plan_candidates(PlanShared& S, GroupPlan* gp, int n, int K, int num_sms, long long seg_cost) {
    const int tid = threadIdx.x, g = tid / kGroupThreads, t = tid % kGroupThreads;
    GroupPlan& P = gp[g];
    const int cnt = n + g + 1;
    if (t == 0) {
        P.live = g < K;
        P.ok = 0;
        if (P.live) {
            wave_shape(S.Ns, cnt, num_sms, &P.Gmax, &P.t2);
            cut_interval(S.Ns, cnt, seg_cost, P.Gmax, &P.lo, &P.hi);
        }
    }
    __syncthreads();
    // the bound searches, all groups in step
    while (__syncthreads_or(P.live && P.lo < P.hi)) {
        const bool go = P.live && P.lo < P.hi;
        const long long lo = P.lo, hi = P.hi;
        if (go && t == 0) P.best = kGroupThreads;
        __syncthreads();
        if (go) {
            const long long C = lo + ((hi - lo) * (long long)(t + 1)) / kGroupThreads;
            if (cut_rows(S.Ns, cnt, C, seg_cost, P.Gmax, nullptr) <= P.Gmax) atomicMin(&P.best, t);
        }
        __syncthreads();
        if (go && t == 0) {
            const int b = P.best < kGroupThreads ? P.best : kGroupThreads - 1;   // hi always fits
            P.hi = lo + ((hi - lo) * (long long)(b + 1)) / kGroupThreads;
            P.lo = b == 0 ? lo : lo + ((hi - lo) * (long long)b) / kGroupThreads + 1;
        }
        __syncthreads();
    }
    // the cuts at the bounds found and their bands' statistics
    if (P.live && t == 0) {
        const int used = cut_rows(S.Ns, cnt, P.lo, seg_cost, P.Gmax, P.w.band);
        for (int c = used; c <= P.Gmax; ++c) P.w.band[c] = S.pre[cnt];
        P.G = used > 1 ? used : 1;
        P.mx[0] = P.mx[1] = P.mx[2] = P.mx[3] = 0;
        P.rp = 1;
    }
    __syncthreads();
    if (P.live) {
        for (int b = t; b < P.G; b += kGroupThreads) {
            const int lo = P.w.band[b], hi = P.w.band[b + 1];
            int a = 0, z = cnt - 1;   // the first pair whose rows end after lo
            while (a < z) {
                const int mid = (a + z) >> 1;
                if (S.pre[mid + 1] > lo) z = mid; else a = mid + 1;
            }
            const BandStat st = band_stat(S.Ns, cnt, a, S.pre[a], lo, hi, P.t2);
            atomicMax(&P.mx[0], st.rows);
            atomicMax(&P.mx[1], st.cols);
            atomicMax(&P.mx[2], st.elems);
            atomicMax(&P.mx[3], st.segs);
        }
        for (int i = t; i < cnt; i += kGroupThreads)
            atomicMax(&P.rp, pdb_row_warps(bp_round4(S.Ns[i]), kPdbThreads, P.t2));
    }
    __syncthreads();
    if (P.live && t == 0) {
        PdbLayout L{P.mx[0], P.mx[1], P.mx[2], P.rp, P.t2, P.mx[3] > 1 ? P.mx[3] : 1, cnt};
        P.ok = layout_fits(&L, &P.w.smem) ? 1 : 0;
        if (P.ok) {
            P.w.grid = P.G;
            P.w.layout = L;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kPlanThreads, 1)
    wave_plan_kernel(StreamState* st, const PairDesc* tmpl, PairDesc* wave, int* band, WaveCtrl* W) {
    __shared__ PlanShared S;
    __shared__ GroupPlan gp[kAdmitGroups];
    __shared__ int s_first, s_err, s_nact, s_count, s_next, s_try, s_left, s_more;
    __shared__ int s_warp[kMaxWavePairs / 32];
    __shared__ int s_row0[kMaxWavePairs + 1];
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_first = st->first;
        s_err = ld_relaxed_i32(&W->error);
        s_nact = st->nact;
        s_count = st->count;
        st->error = s_err;
        if (s_err != 0) st->done = 1;
    }
    __syncthreads();
    if (s_err != 0) return;
    // the wave's pairs that are still running stay, in order (one thread per
    // pair reads its stop words; a ballot per warp keeps the order)
    const int nact = s_nact;
    int keep = 0, p = 0, N = 0;
    unsigned bal = 0;
    if (tid < nact) {
        p = st->act[tid];
        const Ctrl* c = tmpl[p].ctrl;
        N = tmpl[p].N;
        keep = ld_relaxed_i32(&c->done) == 0 && ld_relaxed_i32(&c->error) == 0;
    }
    if (warp < kMaxWavePairs / 32) {   // warp-uniform
        bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) s_warp[warp] = __popc(bal);
    }
    __syncthreads();
    if (keep) {
        int pos = __popc(bal & ((1u << lane) - 1u));
        for (int w = 0; w < warp; ++w) pos += s_warp[w];
        S.list[pos] = p;
        S.Ns[pos] = N;
    }
    __syncthreads();
    if (tid == 0) {
        int kept = 0;
        for (int w = 0; w < kMaxWavePairs / 32; ++w) kept += s_warp[w];
        S.n = kept;
        s_left = nact - kept;
    }
    __syncthreads();
    // nothing changes until a pair stops (the wave and its plan stay)
    if (!s_first && s_left == 0) return;
    if (s_first) {   // every pair of the batch waits until it is admitted
        for (int p = tid; p < s_count; p += nthr) tmpl[p].ctrl->idle = 1;
        __syncthreads();
    }
    // admit waiting pairs in batch order while the plan with the next one
    // still fits: at the admission level once the wave has pairs (up to
    // kAdmitGroups candidates planned at once), at any level for its first
    // pair
    bool have = false;
    if (tid == 0) s_next = st->next;
    __syncthreads();
    while (true) {
        if (tid == 0) {
            int K = 0;
            while (K < kAdmitGroups) {
                const int j = s_next + K;
                if (j >= s_count || S.n + K >= kMaxWavePairs || tmpl[j].N > kPdbMaxN) break;
                S.list[S.n + K] = j;
                S.Ns[S.n + K] = tmpl[j].N;
                ++K;
            }
            if (S.n == 0 && K > 1) K = 1;   // a wave's first pair alone (any level)
            s_try = K;
            S.pre[0] = 0;
            for (int i = 0; i < S.n + K; ++i) S.pre[i + 1] = S.pre[i] + S.Ns[i];
        }
        __syncthreads();
        const int K = s_try;
        if (K == 0) break;
        if (S.n == 0) {
            if (!plan_bands_par(S, S.Ns, 1, st->num_sms, 3, &S.trial)) break;
            if (tid == 0) {
                S.plan = S.trial;
                S.n = 1;
                s_next += 1;
            }
            have = true;
            __syncthreads();
            continue;
        }
        plan_candidates(S, gp, S.n, K, st->num_sms, seg_cost_of_level(kAdmitLevel));
        if (tid == 0) {
            int f = 0;   // candidates that fit before the first that does not
            while (f < K && gp[f].ok) ++f;
            if (f > 0) {
                S.plan = gp[f - 1].w;
                S.n += f;
                s_next += f;
            }
            s_more = f == K;
            s_try = f;
        }
        __syncthreads();
        const int admitted = s_try;
        const bool more = s_more != 0;
        __syncthreads();   // read by every thread before the next round writes them
        if (admitted > 0) have = true;
        if (!more) break;
    }
    // no admission: the remaining pairs, at any level; if even that does not
    // fit, the longest prefix of them that does (the others wait)
    if (!have) {
        while (S.n > 0 && !plan_bands_par(S, S.Ns, S.n, st->num_sms, 3, &S.plan)) {
            if (tid == 0) S.n -= 1;
            __syncthreads();
        }
    }
    __syncthreads();
    // the wave tables: pairs (rows numbered through the wave), bands (the
    // launch's extra CTAs get empty bands), layout and the idle words
    const int n = S.n;
    for (int i = tid; i < nact; i += nthr) tmpl[st->act[i]].ctrl->idle = 1;
    if (tid == 0) {
        s_row0[0] = 0;
        for (int i = 0; i < n; ++i) s_row0[i + 1] = s_row0[i] + S.Ns[i];
    }
    __syncthreads();
    for (int i = tid; i < n; i += nthr) {
        PairDesc d = tmpl[S.list[i]];
        d.row0 = s_row0[i];
        wave[i] = d;
        Ctrl* c = d.ctrl;
        c->idle = 0;
        if (n > c->wave_pairs) c->wave_pairs = n;
        st->act[i] = S.list[i];
    }
    const int G = n > 0 ? S.plan.grid : 0, rows = s_row0[n];
    for (int c = tid; c <= st->num_sms; c += nthr) band[c] = c <= G && n > 0 ? S.plan.band[c] : rows;
    if (tid == 0) {
        st->nact = n;
        st->next = s_next;
        W->npairs = n;
        W->layout = S.plan.layout;
        W->all_done = n == 0 ? 1 : 0;
        st->first = 0;
        st->done = (n == 0 && s_next >= s_count) ? 1 : 0;
        st->waves += 1;
        if (n == 0 && s_next < s_count) {   // a waiting pair fits in no wave
            atomicCAS(&W->error, 0, FASTPFP_ERR_UNSUPPORTED);
            st->error = FASTPFP_ERR_UNSUPPORTED;
            st->done = 1;
        }
    }
}

}  // namespace

cudaError_t wave_plan(StreamState* st, const PairDesc* tmpl, PairDesc* wave, int* band, WaveCtrl* W,
                      cudaStream_t s) {
    wave_plan_kernel<<<1, kPlanThreads, 0, s>>>(st, tmpl, wave, band, W);
    return cudaGetLastError();
}

}  // namespace fpfp
