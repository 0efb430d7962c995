// discretize.cu -- greedy discretisation of Section 4.5 as rounds of
// locally dominant entries.
//
// Section 4.5 takes, one at a time, the largest entry of X among the rows and
// columns still free, ties to the lowest row-major index.  Under that strict
// total order the sequence of picks is the same as repeating, until every
// column is matched:
//   accept every free entry (i, j) that is the largest of its free row AND of
//   its free column,
// because such an entry can only be removed by a larger entry in its row or
// column, and there is none.  Each round is data parallel: a warp per free
// row finds the row maxima, column maxima are folded with 64-bit atomicMax
// over row chunks, and a bounded grid barrier separates the phases.  Entries
// are compared as 64-bit keys (order-preserving float bits, then the
// complement of the flat index), so the result is bit-exact with the
// sequential definition.
#include "common.cuh"
#include "internal.h"

namespace fpfp {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 32;   // rows per column-maximum work item

__device__ __forceinline__ unsigned long long make_key(float v, unsigned idx) {
    return ((unsigned long long)float_to_ordered(v) << 32) | (unsigned long long)(0xffffffffu - idx);
}
__device__ __forceinline__ unsigned key_index(unsigned long long key) {
    return 0xffffffffu - (unsigned)(key & 0xffffffffull);
}

struct DiscArgs {
    const float* X;
    int N, m, ldx;
    DiscBuffers b;
    Ctrl* ctrl;
    long long timeout_ns;
};

__global__ void __launch_bounds__(kThreads) disc_kernel(const DiscArgs a) {
    Ctrl* C = a.ctrl;
    int* err = &C->error;
    const unsigned G = gridDim.x;
    const unsigned bar_base = C->bar_base;
    unsigned gen = 0;
    const int N = a.N, m = a.m;
    const size_t gtid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t gthreads = (size_t)G * blockDim.x;
    const int lane = threadIdx.x & 31;
    const size_t gwarp = gtid >> 5, gwarps = gthreads >> 5;
    int32_t* rowm = a.b.row_match;
    int32_t* colm = a.b.col_match;

    for (size_t i = gtid; i < (size_t)N; i += gthreads) {
        rowm[i] = -1;
        a.b.row_best[i] = 0ull;
    }
    for (size_t j = gtid; j < (size_t)m; j += gthreads) {
        colm[j] = -1;
        a.b.col_best[j] = 0ull;
        a.b.col_best[m + j] = 0ull;
    }
    if (gtid == 0) C->matched = 0;
    if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, a.timeout_ns)) return;
    ++gen;

    const int nchunks = (N + kChunk - 1) / kChunk;
    for (int round = 0;; ++round) {
        unsigned long long* cb = a.b.col_best + (size_t)(round & 1) * m;
        unsigned long long* cbn = a.b.col_best + (size_t)((round + 1) & 1) * m;
        // row maxima over free columns: one warp per free row
        for (size_t i = gwarp; i < (size_t)N; i += gwarps) {
            if (__ldcg(rowm + i) >= 0) continue;
            unsigned long long best = 0ull;
            const float* xr = a.X + i * (size_t)a.ldx;
            for (int j = lane; j < m; j += 32) {
                if (__ldcg(colm + j) >= 0) continue;
                const unsigned long long k = make_key(__ldg(xr + j), (unsigned)(i * m + j));
                best = k > best ? k : best;
            }
            best = warp_max_u64(best);
            if (lane == 0) a.b.row_best[i] = best;
        }
        // column maxima over free rows: one item per (column, chunk of rows)
        for (size_t it = gtid; it < (size_t)m * nchunks; it += gthreads) {
            const int j = (int)(it % m), ch = (int)(it / m);
            if (__ldcg(colm + j) >= 0) continue;
            unsigned long long best = 0ull;
            const int i1 = min(N, (ch + 1) * kChunk);
            for (int i = ch * kChunk; i < i1; ++i) {
                if (__ldcg(rowm + i) >= 0) continue;
                const unsigned long long k =
                    make_key(__ldg(a.X + (size_t)i * a.ldx + j), (unsigned)((size_t)i * m + j));
                best = k > best ? k : best;
            }
            if (best) atomicMax(cb + j, best);
        }
        if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, a.timeout_ns)) return;
        ++gen;
        // accept mutual maxima; clear the other column-maximum buffer
        for (size_t i = gtid; i < (size_t)N; i += gthreads) {
            if (__ldcg(rowm + i) >= 0) continue;
            const unsigned long long k = __ldcg(a.b.row_best + i);
            if (k == 0ull) continue;
            const int j = (int)(key_index(k) % (unsigned)m);
            if (__ldcg(cb + j) == k) {
                rowm[i] = j;
                colm[j] = (int32_t)i;
                atomicAdd(&C->matched, 1);
            }
        }
        for (size_t j = gtid; j < (size_t)m; j += gthreads) cbn[j] = 0ull;
        if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, a.timeout_ns)) return;
        ++gen;
        if (__ldcg(&C->matched) >= m || round >= m) break;
    }
    if (!grid_barrier(&C->bar, bar_base + G * (gen + 1), err, a.timeout_ns)) return;
    ++gen;
    if (gtid == 0) C->bar_base = bar_base + G * gen;
}

}  // namespace

cudaError_t disc_configure() { return cudaSuccess; }

cudaError_t discretize(const float* X, int N, int m, int ldx, const DiscBuffers& b, Ctrl* ctrl,
                       long long timeout_ns, int num_sms, cudaStream_t s) {
    DiscArgs a{X, N, m, ldx, b, ctrl, timeout_ns};
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, disc_kernel, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorLaunchOutOfResources;
    int G = num_sms * (per_sm < 2 ? per_sm : 2);
    const size_t work = (size_t)m * ((N + kChunk - 1) / kChunk);
    const int want = (int)((work + kThreads - 1) / kThreads);
    if (want < G) G = want < 1 ? 1 : want;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)disc_kernel, dim3(G), dim3(kThreads), args, 0, s);
}

}  // namespace fpfp
