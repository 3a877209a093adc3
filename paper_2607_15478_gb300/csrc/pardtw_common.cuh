// Internal declarations shared by the CUDA translation units of libpardtw.
// Not part of the public C-ABI (include/pardtw.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "pardtw.h"

namespace pardtw {

// Launch facts of a kernel that are per device: its dynamic shared memory
// limit (cudaFuncSetAttribute applies to the current device) and the CTAs of
// it resident per SM.  Each launcher keeps one DeviceSlots per kernel
// instantiation (static storage: zero-initialised, 0 = not looked up yet).
constexpr int kMaxDevices = 64;
struct DeviceSlots {
    std::atomic<int> v[kMaxDevices];
};

// Raise `kern`'s dynamic shared memory limit to `smem` bytes on the current
// device, once per device.
template <class K>
cudaError_t raise_smem_once(K* kern, int smem, DeviceSlots& done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool slot = dev >= 0 && dev < kMaxDevices;
    if (slot && done.v[dev].load(std::memory_order_acquire) != 0) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    if (slot) done.v[dev].store(1, std::memory_order_release);
    return cudaSuccess;
}

// CTAs of `kern` (threads a CTA, smem bytes of dynamic shared memory)
// resident per SM of the current device, at least 1; raises the kernel's
// shared memory limit there first.  Looked up once per device.
template <class K>
cudaError_t blocks_per_sm_once(K* kern, int threads, int smem, DeviceSlots& cache, int* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool slot = dev >= 0 && dev < kMaxDevices;
    if (slot) {
        const int n = cache.v[dev].load(std::memory_order_acquire);
        if (n > 0) {
            *out = n;
            return cudaSuccess;
        }
    }
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (n < 1) n = 1;
    if (slot) cache.v[dev].store(n, std::memory_order_release);
    *out = n;
    return cudaSuccess;
}

constexpr int kWarp = 32;
constexpr long long kDefaultTimeoutNs = 2000000000LL;  // bounded device waits: 2 s
constexpr int kRowsPerStrip = 30;   // rows of A per warp: lanes 0..29 (lanes 30, 31 carry
                                    // the two bottom rows of the strip above)
constexpr int kColsPerWord = 16;    // 2-bit codes per uint32 backpointer word
constexpr int kWarpsPerGroup = 4;   // strips per CTA ("strip group") of the one-warp kernels
constexpr int kSplitStrips = 2;     // strips per CTA of the cost/DP warp-pair kernel
// CTAs of the warp-pair DP kernel resident per SM for one pair: two where the
// DP's registers allow it (two strips per CTA, up to 3 rows per lane and
// R x dp <= 36: at most 168 registers a thread, which the kernel's launch
// bounds then enforce), else one.
__host__ __device__ constexpr int split_ctas_per_sm(int R, int ns, int dp, bool bf16) {
    return (ns == 2 && !bf16 && R <= 3 && R * dp <= 36) ? 2 : 1;
}
// BF16 cost (tensor cores): a frame of B (or row of A) takes kBfStride bf16
// in memory, 128 features and 8 of padding, so that the 8 rows an ldmatrix
// reads start 272 bytes apart, in 8 different bank groups.
constexpr int kBfStride = 136;

// Device status words (workspace).  [0] first error (DTW_* code), [1] detail,
// [2] ticket counter of the persistent DP kernel, [3] spare.
struct DevCtl {
    int status;
    int detail;
    int ticket;
    int spare;
};

// Arguments of the column-sweep DP kernel.
struct DpArgs {
    const float* Ahat;              // nstrips*30 x dp, row-normalised, rows >= La are zero
    const float* Bhat;              // row-normalised B, chunk-transposed (see bt_index)
    const void* Bbf;                // BF16 cost only: normalised B as bf16, frame-major,
                                    // kBfStride elements per frame (else null)
    uint32_t* bp;                   // nstrips * nchunk * 32 words (strip, chunk, row in strip)
    unsigned long long* gborder;    // ngroups * Lb * 2 tagged values (group bottom rows)
    DevCtl* ctl;
    float* e_final;                 // shifted cumulative cost at (La-1, Lb-1)
    int La, Lb;
    int nstrips, nchunk, ngroups;
    int rps;                        // rows of A per strip (warp)
    int wpb;                        // backpointer words per (strip, 16 columns)
    float kcost;                    // 1 - cost_shift
    float mu;                       // cost_shift
    unsigned epoch;                 // call tag for global border entries
    long long timeout_ns;
    int skip_publish;               // group that never publishes (fault injection), -1 off
    const int2* ranges;             // banded DP (warp-pair kernel): per strip the sub-chunks
                                    // [x, y) of 8 columns it sweeps (x even; x and y
                                    // non-decreasing in the strip); null = every column
    float* lastrow;                 // subsequence DP (WSDTW): the cumulative cost of row
                                    // La-1 at every column (nchunk * 16 floats), else null
};

// Backpointer word address of cell (i, j): strip-major, then 16-column chunk,
// then row within the strip.  A strip of rps rows stores wpb >= rps words
// per chunk (32 per warp and row of a lane: the ghost lane's words are
// unused), so one warp store covers wpb consecutive words.
__host__ __device__ inline size_t bp_word_index(int i, int j, int nchunk, int rps, int wpb) {
    const int strip = i / rps;
    return ((size_t)strip * (size_t)nchunk + (size_t)(j >> 4)) * (size_t)wpb +
           (size_t)(i - strip * rps);
}

// Backpointer field of cell (i, j): 2 bits at bit 2 * (j % 16) of its word.
// Bit 0 is set when the (1,1) candidate attains the cell's minimum, bit 1
// when the (1,2) candidate does.  The step taken is the first attaining
// candidate in the order (1,1), (1,2), (2,1) (a later candidate must be
// strictly smaller), so: bit 0 set -> (1,1); field 2 -> (1,2); field 0 ->
// (2,1).  Returns the step code 0 = (1,1), 1 = (1,2), 2 = (2,1).
__host__ __device__ inline int step_of_field(uint32_t field) {
    return (field & 1u) ? 0 : (field == 2u ? 1 : 2);
}

// Strip geometry of the DP kernels: R rows per lane.  R = 1: lanes 0..29
// are rows, lanes 30, 31 carry the strip above (30 rows, 32 words).  R >= 2:
// lanes 0..30 hold R rows each, lane 31 carries the strip above (31 R rows,
// 32 R words).
__host__ __device__ inline int strip_rows(int R) { return R == 1 ? 30 : 31 * R; }
__host__ __device__ inline int strip_words(int R) { return 32 * R; }

// Normalised frames of B are stored chunk-transposed: 16 consecutive frames
// (one backpointer chunk) form a feature-major block of 16 * dp floats, so
// value d of frame f sits at ((f / 16) * dp + d) * 16 + f % 16.  A partial
// last chunk is zero-padded.  The DP kernel reads these blocks feature by
// feature to spread the 16 cost computations of a chunk over its steps.
__host__ __device__ inline size_t bt_index(int f, int d, int dp) {
    return ((size_t)(f >> 4) * (size_t)dp + (size_t)d) * 16u + (size_t)(f & 15);
}

// Normalisation of one pair of a batch (k_normalise_many).
struct NormArgs {
    const float* A;
    int La, La_pad;
    const float* B;
    int Lb, Lb_pad;
    float* Ahat;
    float* Bt;
    DevCtl* ctl;
};

// Launchers (each returns a cudaError_t from the launch).
cudaError_t launch_normalise(const float* A, int La, int La_pad, const float* B, int Lb,
                             int Lb_pad, int D, int dp, float* Ahat, float* Bt, DevCtl* ctl,
                             cudaStream_t s);
cudaError_t launch_cost(const float* Ahat, int La, const float* Bt, int Lb, int dp, float* C,
                        cudaStream_t s);
// n pairs at once (`many`: device array); max_frames = largest La_pad + Lb_pad;
// also zeroes *ticket, the work queue of launch_dp_split_many.
cudaError_t launch_normalise_many(const NormArgs* many, int n, int max_frames, int D, int dp,
                                  int* ticket, cudaStream_t s);
// Every DpArgs::epoch of a batch in device memory += 1 (0 skipped).
cudaError_t launch_bump_epoch(DpArgs* many, int n, cudaStream_t s);
cudaError_t launch_dp(const DpArgs& a, int dp, int num_sms, cudaStream_t s);           // R = 1
cudaError_t launch_dp_multirow(const DpArgs& a, int dp, int R, int num_sms, cudaStream_t s);
// Rows per lane the fused DP supports for a padded dimension (0 = none).
bool multirow_supported(int dp, int R);
// Warp-specialised DP (dp_split.cu, dp_split4.cu): a cost warp and a DP warp
// per strip, ns = 2 or 4 strips per CTA; R = 2, 3 or 4 rows per lane.
// transposed: the pair is swept with A and B swapped (rows of the kernel =
// frames of B), with the tie order mapped back (R = 3, one pair).
cudaError_t launch_dp_split(const DpArgs& a, int dp, int R, int ns, int num_sms, cudaStream_t s,
                            bool transposed = false);
bool split4_supported(int dp, int R);
cudaError_t launch_dp_split4(const DpArgs& a, const DpArgs* many, const int* item0, int n,
                             int items, int* ticket, int dp, int R, int num_sms, cudaStream_t s,
                             bool transposed);
// The subsequence DP of WSDTW over a batch (R = 3, dp <= 32): weights 1, 1, 2,
// free start in row 0, row La-1 of every pair into its DpArgs::lastrow.
cudaError_t launch_dp_subseq_many(const DpArgs* many, const int* item0, int n, int total_items,
                                  int* ticket, int dp, int num_sms, cudaStream_t s);
// ns strips per CTA: 2 (every dp <= 32) or 4 (dp <= 16, R = 2, 3).
bool split_supported(int dp, int R, int ns = 2);
// The same DP with the cost from BF16 features and FP32 accumulation on the
// tensor cores (mma.sync m16n8k16): D padded to 64 or 128, R = 3.
cudaError_t launch_dp_split_bf16(const DpArgs& a, int dp, int num_sms, cudaStream_t s,
                                 bool transposed = false);
// The warp-pair DP of one pair at 3 rows per lane and two strips per CTA,
// run in thread-block clusters whose CTAs pass the strip border through
// distributed shared memory (dp_split_cl.cu; dp <= 32, or 64 / 128 with
// bf16).  *used = false (and nothing launched) when no cluster
// configuration fits this device.
cudaError_t launch_dp_split_cl(const DpArgs& a, int dp, bool bf16, bool transposed,
                               cudaStream_t s, bool* used);
// The warp-pair DP with the FP32 cost at D = 64, 128 (dp_split_wide.cu): two
// cost warps per strip, 3 rows per lane, two strips per CTA; the same in
// thread-block clusters.
bool split_wide_supported(int dp);
cudaError_t launch_dp_split_wide(const DpArgs& a, int dp, int num_sms, cudaStream_t s,
                                 bool transposed = false);
cudaError_t launch_dp_split_wide_cl(const DpArgs& a, int dp, bool transposed, cudaStream_t s,
                                    bool* used);
bool split_bf16_supported(int dp);
// B normalised and stored as bf16 for the BF16 cost: Lb_pad frames of
// kBfStride elements (features beyond D and frames beyond Lb are zero).
cudaError_t launch_pack_b_bf16(const float* B, int Lb, int Lb_pad, int D, void* Bbf,
                               cudaStream_t s);
// Many pairs in one persistent launch: `many` (device) holds n DpArgs, item0
// (device, n + 1 ints) the prefix sums of their strip-group counts; CTAs take
// (pair, group) items from *ticket in that order, so a group only waits on
// groups of its own pair that were taken earlier.  Each pair's failures stay
// in its own control block.
cudaError_t launch_dp_split_many(const DpArgs* many, const int* item0, int n, int total_items,
                                 int* ticket, int dp, int R, int ns, int num_sms, cudaStream_t s);

// Which DP kernel runs a problem: kind 0 = one row per lane (dp_kernel.cu),
// 1 = fused multi-row (dp_multirow.cu), 2 = cost/DP warp pairs (dp_split.cu);
// R rows per lane, spg strips per CTA (strip group).
struct DpPlan {
    int kind, R, spg;
    int bf16;  // kind 2 only: the cost on the tensor cores from BF16 features
    int no_clusters;  // kind 2, R = 3, two strips: 1 = never run in thread-block clusters
};
DpPlan choose_plan(int La, int dp, const dtw_options& o, int num_sms);
// Whether a pair is swept transposed (B's frames as rows): B longer than A
// (or forced by the options) and the transposed pair's plan is the warp-pair
// DP at 3 rows per lane.
bool transpose_pair(int La, int Lb, int dp, const dtw_options& o, int num_sms);
cudaError_t launch_plan(const DpPlan& plan, const DpArgs& a, int dp, int num_sms,
                        cudaStream_t s, bool transposed = false);

// Parallel backtrace through per-band entry maps (bandmap.cu) of one pair:
// its backpointers and layout, its control block and end cell, the outputs,
// and caller-provided scratch of bandmap_scratch_bytes(La, Lb) bytes.
struct BtArgs {
    const uint32_t* bp;
    int La, Lb, nchunk, rps, wpb;
    DevCtl* ctl;
    const float* e_final;
    float mu;
    int32_t* path;
    int* path_len;
    float* total;
    void* scratch;
    const int2* ranges;  // banded DP: the strips' sub-chunk ranges (cells outside have no
                         // path), else null
    int transposed;      // the matrix is the transposed problem's: emit (column, row)
};
// The band map inside the DP kernel (one pair): after the strip groups, nbm
// band-map items (band, column segment) of bt's backtrace run on the same
// CTAs, each once the strips covering its band have set their flag in
// done[strip] to the call's epoch.
struct MapArgs {
    BtArgs bt;
    unsigned* done;  // nstrips flags (own zeroed allocation, written only with epochs)
    int nbm;
};
size_t bandmap_scratch_bytes(int La, int Lb);
// Band-map items (bands x column segments) of a pair when CTAs of `threads`
// threads run them inside the DP kernel.
int bandmap_items(int La, int Lb, int threads);
// with_map = false: the band map already ran inside the DP kernel.
cudaError_t launch_backtrace_bands(const BtArgs& a, cudaStream_t s, bool with_map = true);
// The warp-pair DP of one pair with its band map inside (dp_split_map.cu):
// m.nbm = bandmap_items(La, Lb, 192); the backtrace then runs with
// with_map = false.  R = 3, two strips per CTA, FP32 cost, dp <= 32.
bool split_map_supported(int dp, int R, int ns, bool bf16);
cudaError_t launch_dp_split_map(const DpArgs& a, const MapArgs& m, int dp, int num_sms,
                                cudaStream_t s, bool transposed);
// n pairs at once; `many` is a device array of n BtArgs, maxLa / maxLb the
// largest sizes among them.
cudaError_t launch_backtrace_bands_many(const BtArgs* many, int n, int maxLa, int maxLb,
                                        cudaStream_t s);

// Padded feature width used by the kernels for a given D (0 = unsupported).
int padded_dim(int D);

// Multiscale band (band.cu): Y (ceil(L/ds) x D) = averages of ds frames of X;
// per strip of rps fine rows the 8-column blocks within w columns of the
// coarse path (cpath, *clen cells) scaled by ds, widened to monotone; *touch
// = 1 if the banded path (path, *plen cells) comes within one block of a
// side of the band that is not the side of the matrix.
// wrow (may be null): per coarse row of A a half-width in fine frames that
// replaces w (the largest over the coarse rows next to a strip is used).
cudaError_t launch_pool(const float* X, int L, int D, int ds, float* Y, cudaStream_t s);
// swap: the fine DP sweeps the transposed pair (paths are read as (j, i);
// La, Lb, Lac are the swept pair's rows, columns, coarse rows).
cudaError_t launch_band_ranges(const int32_t* cpath, const int* clen, int ds, int w,
                               const float* wrow, int Lac, int La, int Lb, int nstrips, int rps,
                               int swap, int2* ranges, cudaStream_t s);
cudaError_t launch_band_touch(const int32_t* path, const int* plen, int cap, int Lb, int rps,
                              const int2* ranges, int swap, int* touch, cudaStream_t s);

// WSDTW (wsdtw.cu): one fragment of A, its backtrace matrix from the batched
// subsequence DP and the control block of its DP.
struct WsFrag {
    const uint32_t* bp;
    const DevCtl* pctl;
    int row0, len;          // first row of A, rows
    int nchunk, rps, wpb;   // backtrace matrix geometry (see bp_word_index)
};
// Segment-level DP over the fragments' last rows (stride floats apart) with
// shortest matches delta[k]; end frames, total (D_seg[N-1][Lb-1]) and status.
// agg: seg_dp_scratch_bytes(Lb) bytes; done: two counters (zeroed here);
// timeout_ns bounds each wait of the one-launch form.
cudaError_t launch_seg_dp(const WsFrag* fr, const float* lastrow, size_t stride, int N, int Lb,
                          const int* delta, float* Dseg, int* arg, void* agg, unsigned* done,
                          int* ends, float* total, DevCtl* ctl, long long timeout_ns,
                          cudaStream_t s);
size_t seg_dp_scratch_bytes(int Lb);
// Fragment backtraces from their end frames into `scratch` (2 La ints), then
// the concatenated path into `path` and its length (or -status) into path_len.
cudaError_t launch_bt_subseq(const WsFrag* fr, int N, const int* ends, int32_t* scratch,
                             int* count, int32_t* path, int* path_len, DevCtl* ctl,
                             cudaStream_t s);

// Band encoder (encoder.cu).  Parameter offsets (floats) of the flat
// parameter array for input dimension D; see pardtw.h for the layout.
constexpr int kEncChannels = 64;
constexpr int kEncEmbed = 16;
constexpr int kEncKernel = 5;
struct EncLayout {
    size_t W1, b1, W2, b2, W3, b3, W4, b4, W5, b5, count;
};
EncLayout enc_layout(int D);
cudaError_t launch_pool_norm(const float* X, int L, int D, int ds, float* Y, cudaStream_t s);
// conv5 of L rows: forward (bwd = 0: W [64][Cin][5], bias, relu) or the
// backward-data pass (bwd = 1: W the forward weight [64][64][5] read
// transposed and flipped, X masked by mask > 0); bf16 rounds inputs and
// weights (forward only).
cudaError_t launch_conv(const float* X, const float* mask, int L, int Cin, const float* W,
                        const float* b, int relu, int bwd, int bf16, float* Y, cudaStream_t s);
cudaError_t launch_conv_wgrad(const float* X, int L, int Cin, const float* dY, const float* Yout,
                              float* dW, float* db, cudaStream_t s);
cudaError_t launch_embed(const float* H, int L, const float* params, const EncLayout& p, int bf16,
                         float wmin, float wmax, float* Emb, float* invn, float* S, float* HW,
                         cudaStream_t s);
cudaError_t launch_embed_bwd(const float* Emb, const float* invn, int L, const float* W4,
                             float* G, float* dH, cudaStream_t s);
cudaError_t launch_outer(const float* U, int na, const float* V, int nb, int L, float* out,
                         cudaStream_t s);
cudaError_t launch_targets(const int32_t* path, const int* plen, int cap, int ds, int Lac, int Lbc,
                           unsigned long long* jsum, int* cnt, int* tgt, cudaStream_t s);
cudaError_t launch_loss_emb(const float* eA, int Lac, const float* eB, int Lbc, const int* tgt,
                            float* gA, float* gB, float* loss, cudaStream_t s);
cudaError_t launch_width_target(const int32_t* cpath, const int* clen, const int32_t* path,
                                const int* plen, int ds, int Lac, float wmin, float wmax,
                                float* wt, cudaStream_t s);
cudaError_t launch_loss_width(const float* S, const float* wt, int Lac, float* dS, float* loss,
                              cudaStream_t s);
cudaError_t launch_adam(int n, float* P, float* G, float* M, float* V, int step, float lr,
                        float b1, float b2, float eps, cudaStream_t s);

}  // namespace pardtw
