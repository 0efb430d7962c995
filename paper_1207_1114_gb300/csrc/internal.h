// internal.h -- launch interfaces between the C ABI (fastpfp_api.cu) and the
// kernels.  Not installed; not part of the public ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace fpfp {

struct Ctrl;

// ------------------------------------------------------------ projection
// Column-sum scratch of one pair whose slacked rows hold ldy floats: three
// rotating FP32 accumulators of the rounds (3 x ldy floats), then the FP64
// column sums of the launch's input (ldy doubles, 16-byte aligned since ldy
// is a multiple of 4).  The round maxima take kDbufWords words: three
// rotating max|dY|, then max|y| of the launch's input.
constexpr int kDbufWords = 4;
__host__ __device__ inline size_t colbuf_bytes(int ldy) {
    return (size_t)ldy * (3 * sizeof(float) + sizeof(double));
}
__host__ __device__ inline double* colbuf64(float* colbuf, int ldy) {
    return reinterpret_cast<double*>(colbuf + 3 * (size_t)ldy);
}

constexpr int kPdOuterStep = 1;     // P_D rounds + blend/normalise + loop control
constexpr int kPdProjectOnly = 0;   // P_D rounds only (fastpfp_project)
constexpr int kPdMaxSmem = 226 * 1024;   // dynamic shared memory per CTA (the opt-in limit is 227 KB)
constexpr long long kPdElemsPerCta = 8192;  // target band size of one CTA

struct PdParams {
    float* Y;           // N x ldy slacked matrix, ldy = round_up(N, 4), pad columns zero
    int N, ldy;
    int m;              // columns of X (outer step); m <= N
    float* X;           // N x ldx master X, ldx = round_up(m, 4), pad columns zero
    int ldx;
    __nv_bfloat16* Xt16;  // nullable: BF16 copy of X^T (m x ldxt) for the BF16 products
    int ldxt;
    float alpha;
    int normalize, slack_reset;
    double tol_inner;
    int max_inner;
    double tol_outer;
    int max_outer;
    int refine_iters;
    double switch_tol;
    float* colbuf;      // colbuf_bytes(ldy) of column sums, zero between launches
    double* sbuf;       // 3 rotating totals
    unsigned* dbuf;     // kDbufWords words: 3 rotating max|dY|, max|y| of the input (float bits)
    Ctrl* ctrl;
    long long timeout_ns;
    int rpc;            // rows per CTA
    int mode;           // kPdOuterStep or kPdProjectOnly
    int skip_arrive;    // testing only: CTA 0 does not arrive at the first barrier of outer step 0
};

struct PdLaunch {
    int grid, block, rpc, ldy;
    size_t smem;
    bool resident;
};

cudaError_t pd_configure();
void pd_plan(int N, int num_sms, PdLaunch* L);
size_t pd_smem_bytes(int rpc, int Q, bool res);
cudaError_t pd_launch(const PdLaunch& L, const PdParams& P, cudaStream_t s);

// -------------------------------------------------- batched projection
constexpr int kPdbThreads = 512;     // CTA size of the batched kernel
constexpr int kMaxSeg = 32;          // pairs one CTA band may span
constexpr int kMaxWavePairs = 128;   // pairs of one cooperative launch
constexpr int kPdbMaxN = 4096;       // widest pair (two column quads per thread)

// One pair of a wave (device-resident table, read-only in the kernel).
struct PairDesc {
    float* Y;             // N x ldy slacked matrix
    float* X;             // N x ldx master X
    __nv_bfloat16* Xt16;  // nullable BF16 copy of X^T (m x ldxt)
    float* colbuf;        // colbuf_bytes(ldy) of column sums
    double* sbuf;         // 3 totals
    unsigned* dbuf;       // kDbufWords round maxima
    Ctrl* ctrl;           // the pair's control block
    int N, ldy, m, ldx, ldxt;
    int row0;             // first row of the pair in the wave's concatenated rows
};

// Shared-memory sizing of the batched kernel (maxima over the CTAs' bands).
struct PdbLayout {
    int max_band_rows;    // rows of the largest band
    int max_band_cols;    // sum of ldy over the segments of one band
    int max_band_elems;   // floats of the largest band kept in shared memory (the rest is in TMEM)
    int rp_stride;        // row-partial slots per row: the most warps sharing one row, <= 16
    int two_quad_ties;    // pdb_shape's tie rule for this wave (1: two quads per thread)
    int max_segs;         // segments of the band that spans the most pairs (<= kMaxSeg)
    int npairs;           // pairs of the wave: the per-pair tables are sized for this many
};

// Wave-level state: error word, "every pair done", the grid-barrier counter
// (it only grows within a call) and its value when the next launch starts.
// A wave planned on the device (dyn launches) also finds its pair count and
// layout here.
struct WaveCtrl {
    int error;
    int all_done;
    unsigned bar;
    unsigned bar_base;
    int npairs;
    PdbLayout layout;
};

// Warps sharing one row of a pair whose slacked rows hold ldy floats, in a
// CTA of nthr threads (one column quad per thread, or two when a row has
// more quads than threads).
// Thread layout of one pair's rows in a CTA of nthr threads: qpg threads (a
// multiple of 32) cover a row, each owning kq column quads (kq = 1 or 2,
// qpg apart), and rp = nthr / qpg row groups work on different rows.  kq
// maximises rp / kq, the rows a pass advances per quad a thread handles
// (a 1200-node row, 300 quads, takes 3 groups of 160 threads with two quads
// each rather than one group of 320).  On a tie, two_quad_ties picks two
// quads per thread: the per-row work (row offset, row-sum shuffles) then
// serves twice the entries, which pays when a CTA's band has many rows; a
// band of a few rows is better spread over more row groups.
struct PdbShape {
    int kq, qpg, rp;
};
__host__ __device__ inline PdbShape pdb_shape(int ldy, int nthr, int two_quad_ties) {
    const int Q = ldy >> 2;
    PdbShape best{0, 0, 0};
    for (int kq = 1; kq <= 2; ++kq) {
        const int qpg = ((Q + kq - 1) / kq + 31) & ~31;
        if (qpg > nthr) continue;
        const int rp = nthr / qpg;
        // the layout that keeps more threads busy; ties as the wave says
        if (best.kq == 0 || rp * best.kq > best.rp * kq || (two_quad_ties && rp * best.kq == best.rp * kq))
            best = PdbShape{kq, qpg, rp};
    }
    return best;   // kq == 0: rows too wide for one CTA (more than 2 * nthr quads)
}
__host__ __device__ inline int pdb_row_warps(int ldy, int nthr, int two_quad_ties) {
    return pdb_shape(ldy, nthr, two_quad_ties).qpg >> 5;
}

// Tensor memory as band storage: a CTA of kPdbThreads threads allocates all
// 512 TMEM columns; the four warps sharing a 32-lane quarter split them, so
// every thread owns kTmemColsPerThread 32-bit columns of its lane.
constexpr int kTmemCols = 512;
constexpr int kTmemColsPerThread = kTmemCols * 128 / kPdbThreads;

// Placement of one segment of a band (nrows rows of a pair with row length
// ldy) after col_used of the thread's TMEM columns are taken by earlier
// segments: the first `tm` rows of every row group (band rows 0 ..
// rp * tm - 1 of the segment) live in TMEM columns col_used + 4 kq k (the
// thread's kq quads of its k-th row); the rest in shared memory.  Returns tm
// and sets *tm_band_rows (band rows in TMEM) and *col_next.
__host__ __device__ inline int pdb_tmem_rows(int nrows, int ldy, int nthr, int col_used, int* tm_band_rows,
                                             int* col_next, int two_quad_ties) {
    const PdbShape sh = pdb_shape(ldy, nthr, two_quad_ties);
    *col_next = col_used;
    *tm_band_rows = 0;
    if (sh.kq == 0) return 0;
    const int nk = (nrows + sh.rp - 1) / sh.rp;
    int avail = (kTmemColsPerThread - col_used) / (4 * sh.kq);
    if (avail < 0) avail = 0;
    const int tm = nk < avail ? nk : avail;
    *col_next = col_used + 4 * sh.kq * tm;
    *tm_band_rows = sh.rp * tm < nrows ? sh.rp * tm : nrows;
    return tm;
}

struct PdbParams {
    const PairDesc* pairs;
    int npairs;
    const int* band_row;  // grid + 1 row boundaries in the wave's concatenated rows
    WaveCtrl* wave;
    PdbLayout layout;
    float alpha;
    int normalize, slack_reset;
    double tol_inner;
    float tol_inner_f;    // the least float >= tol_inner: for a float d, d < tol_inner_f iff d < tol_inner
    int max_inner;
    double tol_outer;
    int max_outer;
    int refine_iters;
    double switch_tol;
    long long timeout_ns;
    int skip_arrive;      // testing only: CTA 0 does not arrive at the first barrier of a solve's first launch
    int dyn;              // 1: npairs and layout come from the wave control block (a device-planned wave)
};

cudaError_t pdb_configure();
cudaError_t pdb_launch(const PdbParams& P, int grid, size_t smem, cudaStream_t s);

// A batch streamed through waves inside one CUDA graph (wave_stream.cu):
// pair p of the batch has the wave-table template tmpl[p] (row0 unset); the
// planner kernel keeps the current wave in act[0..nact) and admits pairs
// from `next` on.  Words 0 and 1 are the loop's stop and error words.
struct StreamState {
    int done;      // 1 once every pair of the batch has stopped, or after an error
    int error;     // the wave's error word, copied by the planner
    int count;     // pairs of the batch
    int next;      // first pair not yet admitted
    int nact;      // pairs of the current wave
    int first;     // 1 until the first plan
    int num_sms;   // CTAs of a wave launch (bands past the plan's are empty)
    int waves;     // plans made
    int act[kMaxWavePairs];
};
// One planning step (after an outer iteration, or before the first): the
// wave's stopped pairs leave, waiting pairs join while the band plan fits;
// writes wave[0..n) and band[0..num_sms], W->npairs / layout / all_done and
// every pair's idle word.
cudaError_t wave_plan(StreamState* st, const PairDesc* tmpl, PairDesc* wave, int* band, WaveCtrl* W,
                      cudaStream_t s);

// ------------------------------------------------- tensor-core products
constexpr int kTcMaxGroup = 32;      // problems of one grouped launch (a whole wave)
constexpr int kTcOutBf16 = 0;        // epilogue writes BF16 (T = A X)
constexpr int kTcOutF32 = 1;         // epilogue writes FP32 + lambda K (Y = T A' + lambda K)
constexpr int kTcOutSplit = 2;       // epilogue writes T as its TF32 part and the FP32 remainder
// Operand kinds: BF16 (kind::f16), E4M3 with per-row scales (kind::f8f6f4),
// or FP32 split into a TF32 part and its FP32 remainder, multiplied as
// hi*hi + hi*lo + lo*hi (three kind::tf32 MMAs; the FP32 products).
constexpr int kTcBf16 = 0, kTcE4m3 = 1, kTcTf32x3 = 2;

// C[M x N] = A[M x K] B[N x K]^T, both operands K-major (tensor maps),
// both BF16 or both E4M3 (the group's fp8 flag).  With rs / cs set the
// accumulator is scaled by rs[i] * cs[j] before the epilogue adds lambda K:
// the dequantisation of operands stored as E4M3 with one scale per row.
struct TcProblem {
    int M, N, K;
    void* out;            // BF16 or FP32 row-major, leading dimension ldo
    int ldo;
    const float* Kmat;    // FP32 mode: nullable lambda * K addend, leading dimension ldk
    int ldk;
    float lambda;
    const Ctrl* ctrl;     // nullable: skip unless the solve runs (not stopped, no error, not idle)
                          // in its low-precision phase
    int* err;             // nullable: receives FASTPFP_ERR_TIMEOUT
    const float* rs;      // nullable: per-row output scale (M entries)
    const float* cs;      // nullable: per-column output scale (N entries)
    // FP32 mode, nullable: out = addend + scale * acc + lambda K (the step of
    // the projected gradient method); leading dimension ld_add
    const float* addend;
    int ld_add;
    float scale;
    float* out_lo;        // split mode: the FP32 remainder of the output (out holds its TF32 part)
};
struct TcGroup {
    CUtensorMap map_a[kTcMaxGroup];
    CUtensorMap map_b[kTcMaxGroup];
    CUtensorMap map_a_lo[kTcMaxGroup];   // kTcTf32x3: the FP32 remainders of A and B
    CUtensorMap map_b_lo[kTcMaxGroup];
    TcProblem prob[kTcMaxGroup];
    int count;
    int mode;
    int bn;    // output tile columns: 256 (0 reads as 256) or 128; map_b's box has bn rows
    int kind;  // kTcBf16, kTcE4m3 (128-element K stages) or kTcTf32x3 (32-element K stages)
    int phase; // problems with ctrl run while their solve is in its low-precision phase (0) or
               // in its FP32 phase (1)
    // filled by tc_gemm: output tiles of problems before i (tile0[count] =
    // all tiles) and tiles per row of tiles of problem i
    int tile0[kTcMaxGroup + 1];
    int ntn[kTcMaxGroup];
};
// FastGA (fastga.cu): one cooperative launch per outer iteration over one
// pair's slacked matrix, after the gradient products.
constexpr int kGaThreads = 512;
struct GaParams {
    float* Y;                 // N x ldy: the products in columns 0..m-1, then Y of the normalisation
    float* Z;                 // N x ldy scratch (rows normalised)
    float* X;                 // N x ldx master X
    float* part;              // (grid) x ldy scratch: the CTAs' column partials
    float* csum;              // ldy scratch: column sums
    unsigned* dbuf;           // 3 words: a step's max|dY| by parity, max|Q| (zero between launches)
    Ctrl* ctrl;
    int N, m, ldy, ldx, rpc;
    float beta;
    double tol_inner, tol_outer;
    int max_inner, max_outer;
    long long timeout_ns;
};
int ga_rows_per_cta(int N, int num_sms);
cudaError_t ga_configure();
cudaError_t ga_launch(const GaParams& P, cudaStream_t s);

constexpr int kTcTileM = 128;   // output tile rows of tc_gemm (the A operand's box)
// Output tile columns of the split FP32 products (kTcTf32x3): each tile keeps
// two FP32 accumulators in tensor memory, so only 128-column tiles fit two
// tiles' worth (double buffering) in its 512 columns.
constexpr int kTcSplitBN = 128;
size_t tc_smem_bytes(int bn, int kind);
cudaError_t tc_configure();
// TMA map of a rows x cols operand for tc_gemm of operand kind `kind`: BF16
// (ld elements, a multiple of 8), E4M3 bytes (ld a multiple of 16) or FP32
// (either part of a split operand; ld a multiple of 4), read in boxes of 128
// bytes along K by box_rows rows: kTcTileM for an A operand, the group's bn
// for a B operand.  False if the layout does not suit TMA.
bool tc_make_map(CUtensorMap* map, const void* ptr, int rows, int cols, int ld, int box_rows, int kind = kTcBf16);
cudaError_t tc_gemm(const TcGroup& G, cudaStream_t s);

// ----------------------------------------------------------------- GEMM
// C[M x Nc] = Aop[M x K] * Bop[K x Nc] (+ lambda * Kmat), row-major FP32.
// When ctrl is set the kernel does nothing unless the solve is running (not
// stopped, no error, not idle) and its precision phase is FP32.
struct GemmF32Args {
    const float* A; int lda;
    const float* B; int ldb;
    float* C; int ldc;
    const float* Kmat; int ldk; float lambda;
    int M, Nc, K;
    const Ctrl* ctrl;
};
cudaError_t gemm_f32(const GemmF32Args& a, cudaStream_t s);

// Up to kF32MaxGroup independent products in one launch (blockIdx.z).
constexpr int kF32MaxGroup = 32;   // a whole wave in one launch per product
struct GemmF32Group {
    GemmF32Args a[kF32MaxGroup];
    int count;
};
cudaError_t gemm_f32_group(const GemmF32Group& g, cudaStream_t s);

// C[M x Nc] = AT^T B (+ lambda * Kmat): the left operand supplied transposed
// (AT is K x M row-major), B is K x Nc row-major.  AT, B 16-byte aligned,
// lda, ldb multiples of 4.  Same control gating as GemmF32Args.
struct GemmF32TArgs {
    const float* AT; int lda;
    const float* B; int ldb;
    float* C; int ldc;
    const float* Kmat; int ldk; float lambda;
    int M, Nc, K;
    const Ctrl* ctrl;
    // nullable: C = addend + scale * (AT^T B) + lambda * Kmat (the step of
    // the projected gradient method); leading dimension ld_add
    const float* addend; int ld_add; float scale;
};
struct GemmF32TGroup {
    GemmF32TArgs a[kF32MaxGroup];
    int count;
    int tile_m;   // output rows per CTA tile: 128 (0 reads as 128) or 64
};
cudaError_t gemm_f32t_configure();
cudaError_t gemm_f32t_group(const GemmF32TGroup& g, cudaStream_t s);

// ------------------------------------------------------ bandwidth probes
// Read + write sweeps of shared memory (all SMs) or of one global buffer;
// *ms = elapsed time of the timed sweeps, *bytes = bytes they moved.
cudaError_t probe_smem(int num_sms, int sweeps, cudaStream_t s, float* ms, double* bytes);
cudaError_t probe_gmem(size_t buf_bytes, int num_sms, int sweeps, cudaStream_t s, float* ms, double* bytes);
// Read + write sweeps of every SM's tensor memory (all 512 columns) with
// the wave kernel's 16-column tcgen05.ld / tcgen05.st accesses.
cudaError_t probe_tmem(int num_sms, int sweeps, cudaStream_t s, float* ms, double* bytes);
// Best time of one n x n x n product C = A B^T on the solver's kernels
// (FP32 SIMT, BF16 or E4M3 tensor cores) over reps timed launches.
cudaError_t probe_gemm(int precision, int n, int reps, cudaStream_t s, float* best_ms);

// ----------------------------------------------------------- misc kernels
cudaError_t init_ctrl(Ctrl* c, int lowp, cudaStream_t s);

// Condition kernel of the outer loop's graph while node: sets `handle` to
// continue while words[done_idx] == 0, words[err_idx] == 0 and the count in
// *iter (incremented here) is below max_iter.
cudaError_t loop_cond(const int* words, int done_idx, int err_idx, int* iter, int max_iter,
                      cudaGraphConditionalHandle handle, cudaStream_t s);
// Clears *iter and sets `handle` to 1; runs before the while node.
cudaError_t loop_init(int* iter, cudaGraphConditionalHandle handle, cudaStream_t s);

// Stop/error words of the pairs of a streamed wave: out[i] = 1 (done) | 2
// (error) for ctrl[i], out[kMaxWavePairs] = the wave's error word.
struct FlagList {
    const Ctrl* ctrl[kMaxWavePairs];
    const WaveCtrl* wave;
    int n;
};
cudaError_t gather_flags(const FlagList& f, int* out, cudaStream_t s);

// K[i, j] = sum_c B[i, c] * B2[j, c]   (N x m, leading dimension ldk)
cudaError_t affinity(const float* B, const float* B2, int N, int m, int k, float* K, int ldk,
                     cudaStream_t s);

// X (N x ldx) = uniform 1/(N m), or X0 (caller orientation; transposed when
// `transposed`), pad columns zero.  Also writes the BF16 X^T copy if Xt16.
cudaError_t init_x(float* X, int N, int m, int ldx, const float* X0, int transposed,
                   __nv_bfloat16* Xt16, int ldxt, cudaStream_t s);

// FP32 -> BF16 copy of an r x c matrix (leading dimensions lds, ldd); the
// pad columns c..ldd-1 are written as zero.
cudaError_t to_bf16(const float* src, int r, int c, int lds, __nv_bfloat16* dst, int ldd,
                    cudaStream_t s);

// dst (c x ldd, BF16) = src^T for an r x c FP32 src with leading dimension lds.
// E4M3 copies with one power-of-two scale per row, for the FP8 products:
// row r of src (BF16 or FP32, rows x cols, leading dimension lds) becomes
// dst[r] = E4M3(src[r] * 2^e_r) (round to nearest even, saturating) with the
// largest e_r that keeps max |src[r]| * 2^e_r <= 448 (e_r = 0 for a zero
// row), and scale[r] = 2^-e_r.  Up to kTcMaxGroup matrices per launch; an
// entry with ctrl set does nothing unless that solve is running its
// low-precision phase.
struct QuantRows {
    const void* src;
    int src_bf16;
    int rows, cols, lds;
    uint8_t* dst;
    int ldd;
    float* scale;
    const Ctrl* ctrl;
};
struct QuantGroup {
    QuantRows q[kTcMaxGroup];
    int count;
};
cudaError_t quant_fp8_group(const QuantGroup& g, cudaStream_t s);

cudaError_t transpose_to_bf16(const float* src, int r, int c, int lds, __nv_bfloat16* dst, int ldd,
                              cudaStream_t s);

// The split operands of the FP32 products (kTcTf32x3): dst = src (rows x
// cols, leading dimension lds) or its transpose, every value as its TF32
// part in hi and FP32 remainder in lo (leading dimension ldd, pad columns
// zero).  Up to kTcMaxGroup matrices per launch; an entry with ctrl set
// does nothing unless that solve runs (not stopped, no error, not idle) in
// its FP32 phase.
struct SplitRows {
    const float* src;
    int rows, cols, lds;
    float* hi;
    float* lo;
    int ldd;
    int transpose;
    const Ctrl* ctrl;
};
struct SplitGroup {
    SplitRows q[kTcMaxGroup];
    int count;
};
cudaError_t split_tf32_group(const SplitGroup& g, cudaStream_t s);

// Host-to-device staging of a batch by one kernel: pinned host memory is
// addressable by the GPU (over NVLink-C2C on this part), and one launch
// reading every input buffer of a batch runs at the link's rate, where a
// separate DMA copy per buffer of a few MB pays a fixed cost apiece (measured
// on GB300: 520 MB in 256 copies 30.5 ms, one 512 MB copy 2.6 ms).  Every
// segment's source and destination are 16-byte aligned device addresses and
// its size a multiple of 4 bytes.
constexpr int kMaxCopySegs = 640;
struct CopySeg {
    const void* src;
    void* dst;
    unsigned long long bytes;
};
struct CopyList {
    CopySeg seg[kMaxCopySegs];
    int count;
};
cudaError_t gather_copy(const CopyList& L, cudaStream_t s);

// Caller-orientation outputs from the canonical result.
cudaError_t write_outputs(const int32_t* row_of_col, int N, int m, int transposed, int32_t* perm_out,
                          const float* X, int ldx, float* X_out, cudaStream_t s);

// Eq. (3) at the discrete result, FP64, into ctrl->objective.
cudaError_t objective(const float* A, int N, const float* A2, int m, const float* K, int ldk,
                      float lambda, const int32_t* row_of_col, Ctrl* ctrl, cudaStream_t s);

// ------------------------------------------------------- learned warm start
constexpr int kMlpIn = 32, kMlpHidden = 128, kMlpOut = 64;
constexpr int kMlpParams = kMlpIn * kMlpHidden + kMlpHidden + kMlpHidden * kMlpOut + kMlpOut;

cudaError_t ws_features(const float* W, int n, const float* B, int k, float* F, cudaStream_t s);
// E = (relu(F W1 + b1) W2 + b2) * escale; H keeps the hidden activations.
cudaError_t ws_mlp_forward(const float* F, int n, const float* params, float* H, float* E, float escale,
                           cudaStream_t s);
cudaError_t ws_transpose(const float* src, int r, int c, int lds, float* dst, int ldd, cudaStream_t s);
cudaError_t ws_scale(float* x, size_t n, float v, cudaStream_t s);
// In place: S <- exp(S - max S), then `iters` row and column normalisations.
cudaError_t ws_sinkhorn(float* S, int r, int c, int ld, int iters, float* part, float* scalar,
                        cudaStream_t s);
// Loss of Section "learned warm start" and dL/dS (ld ldd); part holds
// ceil(r / 64) x c float2 partials.
cudaError_t ws_loss_grad_S(const float* S, int r, int c, int ld, const int32_t* t, const int32_t* tinv,
                           float* lse_c, float* lse_r, float2* part, float* dS, int ldd, double* loss,
                           cudaStream_t s);
// Parameter gradient of one graph's MLP pass, written or accumulated into grad.
cudaError_t ws_mlp_backward(const float* F, const float* H, const float* dE, int n, const float* params,
                            float* dH, float* grad, int accumulate, cudaStream_t s);
cudaError_t ws_adam(float* p, float* m, float* v, const float* g, int step, float lr, cudaStream_t s);
// t[j] = canonical row matched to column j, tinv[i] = column of row i or -1.
cudaError_t ws_targets(const int32_t* perm, int n_a, int transposed, int N, int m, int32_t* t,
                       int32_t* tinv, cudaStream_t s);

// ------------------------------------------------------- discretisation
struct DiscBuffers {
    int32_t* row_match;           // N
    int32_t* col_match;           // m (the output row_of_col)
    unsigned long long* row_best; // N
    unsigned long long* col_best; // 2 x m
};
cudaError_t disc_configure();
cudaError_t discretize(const float* X, int N, int m, int ldx, const DiscBuffers& b, Ctrl* ctrl,
                       long long timeout_ns, int num_sms, cudaStream_t s);

}  // namespace fpfp
