"""The wave kernel's band planner (band_plan.cuh), compiled for the host
with g++ and checked against what its definition fixes, on the wave shapes
the solver meets (equal pairs of 1000 and 4000 nodes, mixed small pairs):

  * the bands cut the concatenated rows into consecutive pieces that cover
    every row once (band[0] = 0, band[grid] = all rows);
  * every band's cost (entries plus one segment cost per pair it touches)
    is within the planned bound, and the bound is the smallest for which the
    greedy cut needs no more bands than the wave may use (the cut one below
    it needs more);
  * the layout's maxima are those of the bands, and the shared memory it
    needs fits a CTA.
The same header plans waves on the device; the GPU tests check that a
batch planned there gives the bits the host-planned batch gives."""
import json
import os
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1207_1114_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

DRIVER = r'''
#include <cstdio>
#include <vector>
#include "band_plan.cuh"
using namespace fpfp;
int main(int argc, char** argv) {
    int mode = 0;
    if (scanf("%d", &mode) != 1) return 1;
    if (mode == 2) {   // smallest fitting bound: from the row bound up to one band, and in cut_interval's interval
        long long seg = 0;
        int Gmax = 0, count = 0;
        if (scanf("%lld %d %d", &seg, &Gmax, &count) != 3) return 1;
        std::vector<int> Ns(count);
        for (int& n : Ns) if (scanf("%d", &n) != 1) return 1;
        long long lo = 1, hi = 0;
        for (int i = 0; i < count; ++i) {
            const long long ldy = bp_round4(Ns[i]);
            if (seg + ldy > lo) lo = seg + ldy;
            hi += (long long)Ns[i] * ldy + seg;
        }
        while (lo < hi) {
            const long long mid = lo + (hi - lo) / 2;
            if (cut_rows(Ns.data(), count, mid, seg, Gmax, nullptr) <= Gmax) hi = mid; else lo = mid + 1;
        }
        long long l2 = 0, h2 = 0;
        cut_interval(Ns.data(), count, seg, Gmax, &l2, &h2);
        const int hi_fits = cut_rows(Ns.data(), count, h2, seg, Gmax, nullptr) <= Gmax;
        while (l2 < h2) {
            const long long mid = l2 + (h2 - l2) / 2;
            if (cut_rows(Ns.data(), count, mid, seg, Gmax, nullptr) <= Gmax) h2 = mid; else l2 = mid + 1;
        }
        printf("{\"wide\": %lld, \"narrow\": %lld, \"hi_fits\": %d}\n", lo, l2, hi_fits);
        return 0;
    }
    if (mode == 1) {   // one greedy cut: C seg max_bands count Ns...
        long long C = 0, seg = 0;
        int max_bands = 0, count = 0;
        if (scanf("%lld %lld %d %d", &C, &seg, &max_bands, &count) != 4) return 1;
        std::vector<int> Ns(count);
        for (int& n : Ns) if (scanf("%d", &n) != 1) return 1;
        std::vector<int> band(max_bands + 2, -1);
        const int used = cut_rows(Ns.data(), count, C, seg, max_bands, band.data());
        const int counted = cut_rows(Ns.data(), count, C, seg, max_bands, nullptr);
        printf("{\"used\": %d, \"counted\": %d, \"band\": [", used, counted);
        for (int b = 0; b < used && b <= max_bands; ++b) printf("%s%d", b ? ", " : "", band[b]);
        printf("]}\n");
        return 0;
    }
    int num_sms = 0, count = 0, level = 3;
    if (scanf("%d %d %d", &num_sms, &level, &count) != 3) return 1;
    std::vector<int> Ns(count);
    for (int& n : Ns) if (scanf("%d", &n) != 1) return 1;
    WavePlan w;
    const bool ok = plan_bands_seq(Ns.data(), count, num_sms, level, &w);
    int Gmax = 0, t2 = 0;
    wave_shape(Ns.data(), count, num_sms, &Gmax, &t2);
    printf("{\"ok\": %d, \"Gmax\": %d, \"t2\": %d", ok ? 1 : 0, Gmax, t2);
    if (ok) {
        printf(", \"grid\": %d, \"smem\": %u, \"band\": [", w.grid, w.smem);
        for (int b = 0; b <= w.grid; ++b) printf("%s%d", b ? ", " : "", w.band[b]);
        const PdbLayout& L = w.layout;
        printf("], \"layout\": [%d, %d, %d, %d, %d, %d, %d]", L.max_band_rows, L.max_band_cols,
               L.max_band_elems, L.rp_stride, L.two_quad_ties, L.max_segs, L.npairs);
        // the cost bound the bands were cut with, and the cut one below it
        for (int lv = 0; lv < 4; ++lv) {
            const long long seg = seg_cost_of_level(lv);
            long long lo, hi;
            cut_interval(Ns.data(), count, seg, Gmax, &lo, &hi);
            while (lo < hi) {
                const long long mid = lo + (hi - lo) / 2;
                if (cut_rows(Ns.data(), count, mid, seg, Gmax, nullptr) <= Gmax) hi = mid; else lo = mid + 1;
            }
            WavePlan t;
            if (finish_plan(Ns.data(), count, lo, seg, Gmax, t2, &t)) {
                printf(", \"level\": %d, \"seg_cost\": %lld, \"bound\": %lld, \"below\": %d", lv, seg, lo,
                       cut_rows(Ns.data(), count, lo - 1, seg, Gmax, nullptr));
                break;
            }
        }
    }
    printf("}\n");
    return 0;
}
'''


@pytest.fixture(scope="module")
def planner():
    if not os.path.isdir(CUDA_INC):
        pytest.skip("CUDA headers not installed")
    d = tempfile.mkdtemp()
    src, exe = os.path.join(d, "plan.cpp"), os.path.join(d, "plan")
    open(src, "w").write(DRIVER)
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, "-I", CUDA_INC, "-I", os.path.join(ROOT, "include"),
                    src, "-o", exe], check=True)

    def run(Ns, num_sms=152, level=3, cut=None, bound=None):
        if bound is not None:   # (seg_cost, Gmax): the smallest fitting bound two ways
            inp = "2 {} {} {} ".format(*bound, len(Ns)) + " ".join(map(str, Ns))
        elif cut is not None:   # (C, seg_cost, max_bands): one greedy cut
            inp = "1 {} {} {} {} ".format(*cut, len(Ns)) + " ".join(map(str, Ns))
        else:
            inp = f"0 {num_sms} {level} {len(Ns)} " + " ".join(map(str, Ns))
        out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
        return json.loads(out)
    return run


def _greedy_by_rows(Ns, C, seg_cost, max_bands):
    """The greedy cut by its definition, one row at a time: a row of pair i
    costs its row length plus the segment cost when the open band holds no
    row of pair i; it joins the open band while the band stays within C,
    else opens the next band (alone when even that exceeds C).  Returns
    (bands, starts) or (max_bands + 1, None) once more bands are needed."""
    starts, cur, pairs_in, rows_in, g = [0], 0, set(), 0, 0
    for i, n in enumerate(Ns):
        ldy = (n + 3) & ~3
        for _ in range(n):
            cost = ldy + (seg_cost if i not in pairs_in else 0)
            if rows_in > 0 and cur + cost > C:
                if len(starts) >= max_bands:
                    return max_bands + 1, None
                starts.append(g)
                cur, pairs_in, rows_in = 0, set(), 0
                cost = ldy + seg_cost
            cur += cost
            pairs_in.add(i)
            rows_in += 1
            g += 1
    return len(starts), starts


def _band_costs(Ns, band, seg_cost):
    """Entries plus one segment cost per pair touched, per band."""
    starts = np.concatenate([[0], np.cumsum(Ns)])
    ldy = [(n + 3) & ~3 for n in Ns]
    out = []
    for b in range(len(band) - 1):
        lo, hi = band[b], band[b + 1]
        c = 0
        for i in range(len(Ns)):
            s0, s1 = max(lo, starts[i]), min(hi, starts[i + 1])
            if s0 < s1:
                c += (s1 - s0) * ldy[i] + seg_cost
        out.append(c)
    return out


@pytest.mark.parametrize("Ns", [[1000] * 17, [1000] * 18, [4000], [1200] * 9, [64, 700, 33, 1000, 5, 250] * 4,
                                [100] * 128, [7]])
def test_plan_covers_rows_within_a_minimal_bound(planner, Ns):
    r = planner(Ns)
    if not r["ok"]:
        # only a wave too large for the chip may fail: more than 152 SMs' worth
        assert sum(4 * n * ((n + 3) & ~3) for n in Ns) > 152 * 256 * 1024
        return
    band = r["band"]
    assert band[0] == 0 and band[-1] == sum(Ns) and all(a < b for a, b in zip(band, band[1:]))
    assert 1 <= r["grid"] <= r["Gmax"] <= 152
    costs = _band_costs(Ns, band, r["seg_cost"])
    assert max(costs) <= r["bound"]
    assert r["below"] > r["Gmax"]          # the bound is the smallest that fits Gmax bands
    rows, cols, elems, rp, t2, segs, npairs = r["layout"]
    assert npairs == len(Ns) and t2 == r["t2"]
    assert rows == max(b - a for a, b in zip(band, band[1:]))
    assert 1 <= segs <= 32 and r["smem"] <= 226 * 1024


def test_a_wave_of_seventeen_pairs_of_1000_fits_and_eighteen_at_level_0_does_not(planner):
    """The admission rule's boundary at n = 1000: 17 pairs fit on chip with
    the full segment cost (the measured wave size), 18 do not."""
    assert planner([1000] * 17, level=0)["ok"] == 1
    assert planner([1000] * 18, level=0)["ok"] == 0


def test_cut_matches_the_row_by_row_greedy(planner):
    """The planner's cut takes a pair at a time (whole fresh bands in closed
    form); on random waves and bounds it gives the row-by-row greedy's bands
    exactly, including the bound where a row alone exceeds C and the early
    stop once more than max_bands bands would be needed."""
    rng = np.random.default_rng(11)
    cases = [([1000] * 17, 111_000, 32768, 152), ([1000] * 17, 1000 + 32768, 32768, 152),
             ([7], 10, 32768, 4), ([5, 9, 1, 13], 40, 8, 3), ([4000], 2_000_000, 0, 152)]
    for _ in range(300):
        Ns = list(rng.integers(1, 300, size=rng.integers(1, 9)))
        seg = int(rng.choice([0, 16, 256, 4096]))
        tot = sum(n * ((n + 3) & ~3) for n in Ns) + seg * len(Ns)
        C = int(rng.integers(1, tot + 2))
        cases.append((Ns, C, seg, int(rng.integers(1, 40))))
    for Ns, C, seg, mb in cases:
        want, starts = _greedy_by_rows(Ns, C, seg, mb)
        got = planner(Ns, cut=(C, seg, mb))
        assert got["used"] == want and got["counted"] == want, (Ns, C, seg, mb, got, want)
        if starts is not None:
            assert got["band"] == starts, (Ns, C, seg, mb)


def test_search_interval_keeps_the_smallest_fitting_bound(planner):
    """cut_interval's interval (a provable lower bound from the total cost, a
    provable upper bound that always fits) gives the same smallest fitting
    bound as the search from one row up to one band holding everything."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        Ns = list(rng.integers(1, 1100 if rng.random() < 0.5 else 300, size=rng.integers(1, 60)))
        seg = int(rng.choice([0, 8192, 32768]))
        r = planner(Ns, bound=(seg, int(rng.integers(1, 153))))
        assert r["hi_fits"] == 1 and r["narrow"] == r["wide"], (Ns, seg, r)
