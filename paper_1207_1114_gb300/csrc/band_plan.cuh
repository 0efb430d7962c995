// band_plan.cuh -- the band planner of the wave kernel (pdb_kernel).
//
// A wave's pairs have their slacked rows concatenated and cut into one
// band per CTA, each kept on chip (tensor memory + shared memory) for every
// P1/P2 round of an outer iteration.  The same code plans a wave on the host
// (between launches) and on the device (the planner kernel of a batch
// streamed inside one CUDA graph), so a wave is cut identically on either
// side and the two give bit-identical results.
#pragma once

#include "internal.h"

namespace fpfp {

// Band cost model of pdb_kernel, in entry equivalents: a band costs its
// entries plus kSegCost for every pair it spans (a segment brings its own
// loop tails, reductions and read-back; measured on GB300 by clock stamps
// at 2500-2750 cycles against 0.07-0.09 cycles per entry of a pass).
constexpr long long kSegCost = 32768;
constexpr long long kMinElemsPerCta = 8192;   // smallest band worth a CTA of its own
// Waves with at least this many rows per CTA lay out tied pairs with two
// column quads per thread (pdb_shape): measured +7 % at 112 rows per CTA
// (17 pairs of n = 1000), -25 % at 7 (one pair of n = 1000).
constexpr int kTwoQuadRowsPerCta = 32;
// Pairs join a streamed wave only while its bands can still be cut with at
// least this segment-cost level (0 = kSegCost, 1 = half of it, ...): a wave
// filled until only pure entry balance fits leaves the CTAs that span
// several pairs slower than the rest, and every grid barrier waits for them.
// Measured: level 0 gives the 512-pair mixed batch 451 pair-solves/s against
// 405 with no limit, and streamed n = 1000 batches 153 against 148.  A batch
// that fits in one wave as a whole takes any plan instead: splitting it
// would leave a tail wave of a few pairs (17 pairs of n = 1000: 117 against
// 146 pair-solves/s).
constexpr int kAdmitLevel = 0;
constexpr int kMaxBands = 256;   // CTAs of one wave (one per SM)
constexpr int kSegBytes = 44;    // a segment record of pdb_kernel's shared-memory tables
constexpr int kPairBytes = 80;   // a pair record of the same

__host__ __device__ inline int bp_round4(int x) { return (x + 3) & ~3; }

// Shared memory pdb_kernel carves for a wave with layout L (its tables, then
// the band storage), 16-byte aligned pieces.
__host__ __device__ inline size_t pdb_smem_bytes(const PdbLayout& L, int nthr) {
    (void)nthr;
    size_t off = 0;
    auto take = [&off](size_t bytes) { off = (off + bytes + 15) & ~size_t(15); };
    take((size_t)kSegBytes * L.max_segs);
    take((size_t)kPairBytes * L.npairs);
    take(4 * (size_t)L.npairs);
    take(4 * (size_t)L.npairs);
    take(4 * 8);
    take(4 * ((size_t)L.npairs + 1));
    take(4 * (size_t)L.max_segs * 32);
    take(4 * (size_t)L.max_band_rows);
    take(4 * (size_t)L.max_band_rows * L.rp_stride);
    take(4 * (size_t)L.max_band_cols);
    take(4 * (size_t)L.max_band_elems);
    return off;
}

// Greedy cut of the concatenated rows of pairs with row counts Ns[0..count)
// into consecutive bands of cost at most C: row by row, a row joins the open
// band while the band's cost stays within C (a row of pair i costs its row
// length, plus the segment cost when the band holds no row of pair i yet),
// else it opens the next band (alone when even that exceeds C).  Writes the
// boundaries to band[0..] (when band != nullptr) and returns the number of
// bands, or max_bands + 1 as soon as more would be needed.  For a cost that
// only grows as rows are added, the greedy uses the fewest bands, and the
// count never grows with C.
//
// Within one pair every fresh band takes the same number of rows, so the
// cut is taken a pair at a time: the rows that still fit in the open band,
// then whole fresh bands of that many rows, the last one left open -- O(count)
// steps to count the bands (the bound search runs this for hundreds of
// candidate bounds), O(bands) more to write their boundaries.
__host__ __device__ inline long long bp_div(long long a, long long b) {
    return a <= 0x7fffffffll ? (long long)((unsigned)a / (unsigned)b) : a / b;   // 32-bit division when it fits
}
__host__ __device__ inline int cut_rows(const int* Ns, int count, long long C, long long seg_cost, int max_bands,
                                        int* band) {
    int b = 0, gr = 0, rows_in = 0;   // the open band b, the rows before it or in it, its rows
    long long cur = 0;                // the open band's cost
    if (band) band[0] = 0;
    const long long room = C - seg_cost;   // a fresh band's budget for its rows of one pair
    for (int i = 0; i < count; ++i) {
        const int N = Ns[i];
        if (N <= 0) continue;
        const long long ldy = bp_round4(N);
        int r = 0;
        if (rows_in > 0) {   // rows of pair i that still fit in the open band (a new segment of it)
            const long long avail = C - cur - seg_cost;
            if (avail >= ldy) {
                const long long fit = bp_div(avail, ldy);
                r = fit < (long long)N ? (int)fit : N;
                cur += seg_cost + r * ldy;
                rows_in += r;
                gr += r;
                if (r == N) continue;
            }
            if (++b >= max_bands) return max_bands + 1;   // the band is closed
            if (band) band[b] = gr;
            rows_in = 0;
        }
        // the rest in fresh bands of kk rows each (one row when a row alone exceeds C)
        const int rest = N - r;
        const long long kk = room >= ldy ? bp_div(room, ldy) : 1;
        const long long nb = kk >= rest ? 1 : (long long)(((unsigned)rest + (unsigned)kk - 1u) / (unsigned)kk);
        if ((long long)b + nb - 1 >= (long long)max_bands) return max_bands + 1;
        for (long long t = 1; band && t < nb; ++t) band[b + t] = gr + (int)(t * kk);
        b += (int)(nb - 1);
        rows_in = rest - (int)((nb - 1) * kk);
        gr += rest;
        cur = seg_cost + rows_in * ldy;
    }
    return rows_in > 0 || b == 0 ? b + 1 : b;
}

// The search interval [lo, hi] of the smallest band cost bound that fits
// Gmax bands.  lo: every row fits in a band alone (seg + its row length),
// and no bound below (E + count seg) / Gmax fits -- with no row costing more
// than the bound every band costs at most it, and the bands together cost at
// least the entries E plus one segment cost per pair.  hi: one band holding
// everything, or, if smaller, (E + (count + Gmax) seg) / Gmax + seg + the
// longest row, which always fits -- every band the greedy closes costs more
// than the bound less one row and its segment, and Gmax such bands would
// cost more than the cut's at most E + (count + Gmax) seg.  Since the band
// count never grows with the bound, the smallest fitting bound in [lo, hi]
// is the smallest at or above the row lower bound: the interval only saves
// search rounds.
__host__ __device__ inline void cut_interval(const int* Ns, int count, long long seg_cost, int Gmax, long long* lo,
                                             long long* hi) {
    long long rowmax = 1, E = 0, ldymax = 0;
    for (int i = 0; i < count; ++i) {
        const long long ldy = bp_round4(Ns[i]);
        if (seg_cost + ldy > rowmax) rowmax = seg_cost + ldy;
        if (ldy > ldymax) ldymax = ldy;
        E += (long long)Ns[i] * ldy;
    }
    const long long g = Gmax > 0 ? Gmax : 1;
    const long long all = E + (long long)count * seg_cost;   // one band holds everything
    const long long avg = (E + (long long)count * seg_cost + g - 1) / g;
    *lo = rowmax > avg ? rowmax : avg;
    long long h = (E + ((long long)count + g) * seg_cost + g - 1) / g + seg_cost + ldymax;
    if (h > all) h = all;
    *hi = h > *lo ? h : *lo;
}

// A planned wave: `grid` CTAs (bands), their row boundaries (band[grid] =
// the wave's rows; a launch on more CTAs gives the extra ones empty bands)
// and the shared-memory layout.
struct WavePlan {
    int grid;
    int band[kMaxBands + 1];
    PdbLayout layout;
    unsigned smem;
};

// Wave-level choices before the cut: the largest CTA count worth using and
// the thread-layout tie rule.
__host__ __device__ inline void wave_shape(const int* Ns, int count, int num_sms, int* Gmax, int* t2) {
    long long E = 0, rows = 0;
    for (int i = 0; i < count; ++i) {
        E += (long long)Ns[i] * bp_round4(Ns[i]);
        rows += Ns[i];
    }
    long long g = (E + kMinElemsPerCta - 1) / kMinElemsPerCta;
    if (g < 1) g = 1;
    if (g > num_sms) g = num_sms;
    if (g > kMaxBands) g = kMaxBands;
    *Gmax = (int)g;
    *t2 = rows >= (long long)kTwoQuadRowsPerCta * g ? 1 : 0;
}

__host__ __device__ inline long long seg_cost_of_level(int lv) {
    return lv == 0 ? kSegCost : lv == 1 ? kSegCost / 2 : lv == 2 ? kSegCost / 4 : 0ll;
}

// Statistics of band [lo, hi) of the concatenated rows (pair p holds rows
// [p0, p0 + Ns[p]) and is the pair holding row lo): its rows, columns (the
// sum of its segments' row lengths), floats kept in shared memory and
// segments.  The first rows of every row group of a segment go to tensor
// memory (pdb_tmem_rows, the band's segments in pair order as the kernel
// places them), the rest to shared memory.
struct BandStat {
    int rows, cols, elems, segs;
};
__host__ __device__ inline BandStat band_stat(const int* Ns, int count, int p, int p0, int lo, int hi, int t2) {
    BandStat st{0, 0, 0, 0};
    int tcol = 0;
    for (int q = p, q0 = p0; q < count && q0 < hi; q0 += Ns[q++]) {
        const int s0 = lo > q0 ? lo : q0, s1 = hi < q0 + Ns[q] ? hi : q0 + Ns[q];
        if (s0 >= s1) continue;
        const int nr = s1 - s0, ldy = bp_round4(Ns[q]);
        int ntm = 0, next = 0;
        pdb_tmem_rows(nr, ldy, kPdbThreads, tcol, &ntm, &next, t2);
        tcol = next;
        st.rows += nr;
        st.cols += ldy;
        st.elems += (nr - ntm) * ldy;
        ++st.segs;
    }
    return st;
}

// The wave's layout from its bands' statistics (maxima over the bands, the
// pairs' row-partial stride); false when a CTA's band would not fit (more
// than kMaxSeg segments, or more shared memory than a CTA has).
__host__ __device__ inline bool layout_fits(PdbLayout* L, unsigned* smem) {
    if (L->max_segs > kMaxSeg) return false;
    const size_t b = pdb_smem_bytes(*L, kPdbThreads);
    if (b > (size_t)kPdMaxSmem) return false;
    *smem = (unsigned)b;
    return true;
}

// Per-band statistics of the cut at bound C into w->band / w->grid, and the
// wave's layout (band_stat per band, layout_fits).
__host__ __device__ inline bool finish_plan(const int* Ns, int count, long long C, long long seg_cost, int Gmax,
                                            int t2, WavePlan* w) {
    int rows = 0;
    for (int i = 0; i < count; ++i) rows += Ns[i];
    const int used = cut_rows(Ns, count, C, seg_cost, Gmax, w->band);
    for (int c = used; c <= Gmax; ++c) w->band[c] = rows;
    const int G = used > 1 ? used : 1;
    PdbLayout L{0, 0, 0, 1, t2, 0, count};
    for (int i = 0; i < count; ++i) {
        const int rw = pdb_row_warps(bp_round4(Ns[i]), kPdbThreads, t2);
        if (rw > L.rp_stride) L.rp_stride = rw;
    }
    int p = 0, p0 = 0;   // the pair holding row band[b], and its first row
    for (int b = 0; b < G; ++b) {
        const int lo = w->band[b], hi = w->band[b + 1];
        while (p < count && p0 + Ns[p] <= lo) p0 += Ns[p++];
        const BandStat st = band_stat(Ns, count, p, p0, lo, hi, t2);
        if (st.rows > L.max_band_rows) L.max_band_rows = st.rows;
        if (st.cols > L.max_band_cols) L.max_band_cols = st.cols;
        if (st.elems > L.max_band_elems) L.max_band_elems = st.elems;
        if (st.segs > L.max_segs) L.max_segs = st.segs;
    }
    if (L.max_segs < 1) L.max_segs = 1;
    if (!layout_fits(&L, &w->smem)) return false;
    w->grid = G;
    w->layout = L;
    return true;
}

// Plans a wave of pairs with row counts Ns[0..count) on at most num_sms
// CTAs: for the measured segment cost first, then cheaper ones (levels up to
// max_level) when that plan does not fit on chip (pair-aligned bands hold
// more entries), finally pure entry balance; at each level the smallest
// bound whose greedy cut needs at most Gmax bands (binary search).  False
// when no level fits.  Sequential: the host's planner.
inline bool plan_bands_seq(const int* Ns, int count, int num_sms, int max_level, WavePlan* w) {
    int Gmax = 1, t2 = 0;
    wave_shape(Ns, count, num_sms, &Gmax, &t2);
    for (int lv = 0; lv <= max_level && lv < 4; ++lv) {
        const long long seg_cost = seg_cost_of_level(lv);
        long long lo, hi;
        cut_interval(Ns, count, seg_cost, Gmax, &lo, &hi);
        while (lo < hi) {
            const long long mid = lo + (hi - lo) / 2;
            if (cut_rows(Ns, count, mid, seg_cost, Gmax, nullptr) <= Gmax) hi = mid;
            else lo = mid + 1;
        }
        if (finish_plan(Ns, count, lo, seg_cost, Gmax, t2, w)) return true;
    }
    return false;
}

}  // namespace fpfp
