/*
 * pardtw.h — C-ABI of the GB300-native exact DTW (ParDTW) library.
 *
 * The library aligns two feature sequences A (La x D) and B (Lb x D) with
 * exact dynamic time warping:
 *
 *   C[i][j] = 1 - cos(a_i, b_j)                       cosine cost (Sec. IV)
 *   D[0][0] = C[0][0]
 *   D[i][j] = min( D[i-1][j-1] + 2 C[i][j],           step (1,1)
 *                  D[i-1][j-2] + 3 C[i][j],           step (1,2)
 *                  D[i-2][j-1] + 3 C[i][j] )          step (2,1)
 *
 * with the step set and multiplicative weights of the DTW baseline of
 * Sec. V ((di, dj) = (advance in A, advance in B)); ParDTW computes exactly
 * this alignment with the cost formed on the fly, the cumulative cost kept
 * only in a few live buffers, and a 2-bit backtrace matrix (Sec. II-D,
 * Sec. III-B, Sec. VI-D).  Ties between candidates are broken in the order
 * (1,1), (1,2), (2,1): a later candidate wins only when strictly smaller.
 * A zero frame has cosine cost 1 against every frame.
 *
 * Arithmetic: FP32 cost and FP32 cumulative cost on the GPU; no FP64 and no
 * CPU fallback.  Every call runs on the CUDA stream bound to the handle.
 *
 * Pointers.  Feature, path and result pointers may point to device memory
 * or to host memory; the library detects which (cudaPointerGetAttributes).
 * Host inputs are copied into the handle's workspace and host outputs are
 * copied back; a call with any host output synchronises the stream before
 * it returns.  With device-only arguments a call is asynchronous: it
 * returns DTW_OK once the work is enqueued, and device-side failures are
 * reported through the outputs (path_len < 0, see dtw_align).
 *
 * Layouts.  Features are row-major float32, frame k at X + k*D.  A path is
 * an array of int32 (i, j) pairs, ascending from (0, 0) to (La-1, Lb-1):
 * path[2k] = i_k, path[2k+1] = j_k.
 *
 * Thread safety: a handle may be used by one host thread at a time.
 */
#ifndef PARDTW_H
#define PARDTW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define DTW_OK 0
#define DTW_ERR_INVALID 1      /* null pointer, length < 1, D < 1, cap too small */
#define DTW_ERR_UNREACHABLE 2  /* (La-1, Lb-1) cannot be reached: Lb-1 > 2(La-1) or La-1 > 2(Lb-1) */
#define DTW_ERR_OOM 3          /* device allocation of the workspace failed */
#define DTW_ERR_CUDA 4         /* a CUDA runtime call failed */
#define DTW_ERR_TIMEOUT 5      /* a bounded device-side wait expired (the result is void) */
#define DTW_ERR_UNSUPPORTED 6  /* option or size outside what this build supports */
#define DTW_ERR_SCRATCH_LIMIT 7 /* dtw_align_static: the problem needs more than its fixed scratch */

/* ---- options -------------------------------------------------------------- */
#define DTW_COST_FP32 0        /* cost from FP32 features with FP32 accumulation */
#define DTW_COST_BF16 1        /* cost from BF16-rounded normalised features with FP32
                                  accumulation on the tensor cores (D <= 128); the DP
                                  stays FP32.  Approximate: costs differ from the FP32
                                  ones by up to ~1e-2, so paths may differ where
                                  alternatives are that close. */

typedef struct dtw_options {
    int cost_precision;    /* DTW_COST_FP32 (default) or DTW_COST_BF16 */
    /* The DP runs on C - cost_shift and adds cost_shift * (La + Lb - 2) to the
     * total at the end.  Every path weighs exactly (La-1) + (Lb-1) (Sec. V),
     * so the optimal path is unchanged in exact arithmetic; a shift near the
     * per-step cost along the path keeps FP32 partial sums small and cuts
     * their rounding.  0 = no shift. */
    float cost_shift;
    /* Deadline, in microseconds, of every device-side wait (for the border
     * of the strip above, or for a staged block of B); 0 = library default
     * (2 s).  On expiry the call fails with DTW_ERR_TIMEOUT. */
    int wait_limit;
    /* Fault injection for tests, -1 = off: the strip group with this index
     * never publishes its bottom border, so the group below it waits until
     * wait_limit and the call reports DTW_ERR_TIMEOUT. */
    int debug_skip_publish;
    /* Rows of A each GPU lane sweeps (1, 2, 3 or 4); 0 = chosen from La, D
     * and the SM count.  Results do not depend on it (it only changes the
     * work decomposition); 32 < D <= 128 runs with 3 (two cost warps per
     * strip) or 1, and a value the chosen schedule does not support falls
     * back to 1. */
    int rows_per_lane;
    /* Division of labour of the DP for rows_per_lane >= 2: DTW_SCHEDULE_AUTO
     * (0, the default: cost/DP warp pairs), DTW_SCHEDULE_FUSED (1: one warp
     * per strip computes the costs and the recurrence; rows_per_lane 2 or 4)
     * or DTW_SCHEDULE_SPLIT (2: a cost warp and a DP warp per strip;
     * rows_per_lane 2, 3 or 4).  Results do not depend on it. */
    int dp_schedule;
    /* Strips per CTA of the cost/DP warp-pair DP: 0 (default: four when a
     * pair has more two-strip groups than the GPU has SMs and the kernel has
     * the four-strip form for D and rows_per_lane, else two), 2 or 4 (D <= 16,
     * rows_per_lane 2 or 3; else two).  Results do not depend on it. */
    int strips_per_cta;
    /* DTW_TRANSPOSE_AUTO (0, default): the DP sweeps the transposed pair
     * (B's frames as rows) when a model of the sweep's time (waves of strip
     * groups x columns + the chain of strips) says it is faster, e.g. a pair
     * with B longer that fits one wave of strip groups; DTW_TRANSPOSE_NEVER
     * (1); DTW_TRANSPOSE_ALWAYS (2).
     * Applies to the default warp-pair DP at 3 rows per lane (FP32 or BF16
     * cost); the tie order is mapped so that results do not depend on it. */
    int transpose;
    /* DTW_CLUSTERS_AUTO (0, default): the default DP of one pair (warp pairs
     * at 3 rows per lane, two strips per CTA) runs in thread-block clusters
     * of up to 8 CTAs, which hand the strip border from CTA to CTA through
     * distributed shared memory instead of global memory, when the device
     * has room for them; DTW_CLUSTERS_NEVER (1): never.  Results do not
     * depend on it. */
    int clusters;
} dtw_options;

#define DTW_CLUSTERS_AUTO 0
#define DTW_CLUSTERS_NEVER 1

#define DTW_TRANSPOSE_AUTO 0
#define DTW_TRANSPOSE_NEVER 1
#define DTW_TRANSPOSE_ALWAYS 2

#define DTW_SCHEDULE_AUTO 0
#define DTW_SCHEDULE_FUSED 1
#define DTW_SCHEDULE_SPLIT 2

/* Fill *opt with the defaults: FP32 cost, no shift, default wait limit,
 * no fault injection. */
void dtw_default_options(dtw_options* opt);

/* Human-readable name of a status code (static string). */
const char* dtw_status_string(int status);

/* ---- handle --------------------------------------------------------------- */
typedef struct dtw_handle dtw_handle;

/* Create a handle on CUDA device `device`, bound to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The handle owns a
 * device workspace that grows on demand and is freed by dtw_destroy.
 * Errors: DTW_ERR_INVALID (h == NULL, bad device), DTW_ERR_CUDA. */
int dtw_create(dtw_handle** h, int device, void* cuda_stream);

/* Synchronise the handle's stream, free its workspace and the handle. */
int dtw_destroy(dtw_handle* h);

/* Rebind the handle to another stream (later calls are ordered on it). */
int dtw_set_stream(dtw_handle* h, void* cuda_stream);

/* Bytes of device workspace dtw_align needs for (La, Lb, D) with the
 * options `opt` (NULL = defaults), for either orientation of the sweep
 * (Sec. VI-D's memory model: the 2-bit backtrace matrix dominates, La*Lb/4
 * bytes plus 3% padding at 3 rows per lane (7% at 1); plus the tagged
 * border rows between strip groups, 16 bytes per column and group of two
 * 93-row strips (La*Lb/11.6 bytes; La*Lb/7.5 at 1 row per lane); plus the
 * parallel backtrace's band maps, 14 bytes per column and 128 rows
 * (La*Lb/9.1 bytes: each band's exits, and the maps two and four bands up);
 * plus O((La+Lb)*D)).  About 0.46 bytes per cell with the default options.
 * Errors: DTW_ERR_INVALID, DTW_ERR_UNSUPPORTED. */
int dtw_workspace_size(int La, int Lb, int D, const dtw_options* opt, size_t* bytes);

/* ---- cost matrix (Sec. IV cosine distance; Sec. VI-B explicit matrix) ---- */
/* Write the La x Lb row-major FP32 cost matrix C[i*Lb + j] = 1 - cos(a_i, b_j).
 * A, B: La x D and Lb x D float32 (device or host).  C: La*Lb float32,
 * caller-owned (device or host).  The exact aligner never materialises
 * this matrix (Sec. II-D); this entry point exists for inspection and tests.
 * Every value is the FP32 cost the aligner's DP uses for that cell, bit for
 * bit (one FMA per feature in feature order, from 1).  Host buffers are
 * staged through the workspace and the call then synchronises.
 * Errors: DTW_ERR_INVALID (NULL pointer, La, Lb or D < 1), DTW_ERR_UNSUPPORTED
 * (D > 128), DTW_ERR_OOM, DTW_ERR_CUDA. */
int dtw_cost(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D, float* C);

/* ---- exact alignment of one pair (Sec. II-D ParDTW, Sec. III-B) ----------- */
/* Align A (La x D) with B (Lb x D).
 *   opt         options, or NULL for the defaults
 *   path        caller-owned int32 buffer of 2*cap entries (device or host); a
 *               host buffer receives min(La, Lb) pairs in one copy, those past
 *               *path_len unspecified
 *   cap         capacity in (i, j) pairs; must be >= min(La, Lb)
 *   path_len    receives the number of pairs written (device or host int)
 *   total_cost  receives D[La-1][Lb-1] in FP32 (device or host float); may be NULL
 * Returns DTW_OK, DTW_ERR_INVALID, DTW_ERR_UNREACHABLE (checked on the host
 * before any launch), DTW_ERR_OOM, DTW_ERR_CUDA, or, when the call
 * synchronises (any host output), DTW_ERR_TIMEOUT.  When the call runs
 * asynchronously, a device-side failure sets *path_len to -status
 * (e.g. -DTW_ERR_TIMEOUT) and leaves path undefined. */
int dtw_align(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D,
              const dtw_options* opt, int32_t* path, int cap, int* path_len,
              float* total_cost);

/* ---- batch of independent pairs ------------------------------------------- */
/* Align n independent pairs (A[k], B[k]) of a common dimension D.
 *   A, B, La, Lb, path_off : HOST arrays of n entries; A[k], B[k] point to
 *                            device or host features
 *   paths      one int32 buffer (device or host); pair k writes its path at
 *              paths + 2*path_off[k], with room for min(La[k], Lb[k]) pairs
 *   path_len, cost, status : arrays of n entries (device or host)
 * A pair that fails (unreachable, timeout) gets its own status and
 * path_len = -status; the other pairs are still aligned.  Returns the first
 * argument or runtime error that prevented the batch from running. */
int dtw_align_many(dtw_handle* h, int n, const float* const* A, const int* La,
                   const float* const* B, const int* Lb, int D, const dtw_options* opt,
                   int32_t* paths, const int64_t* path_off, int* path_len, float* cost,
                   int* status);

/* ---- banded alignment ------------------------------------------------------ */
/* Exact DTW inside a band found at a coarser scale.  The paper notes that
 * bands and multiscale DTW cut the quadratic cost (Sec. II); this entry
 * point builds the band from the exact alignment of A and B averaged over
 * `downsample` frames: every row i of the fine problem keeps the columns
 * within `halfwidth` of the coarse path scaled by `downsample` (rounded out
 * to whole strips of rows and 8-column blocks), and the exact DP (Sec. V
 * recurrence, steps, weights and tie order) runs inside that band.  If the
 * best path inside the band comes within one block of a side of the band
 * (other than the matrix's own sides), the band may have cut off a better
 * path, and the full exact DTW runs instead; *fell_back then reads 1.
 *
 *   A, B, path, path_len, total_cost : device pointers (total_cost may be
 *       NULL), as in dtw_align; D <= 32 and FP32 cost
 *   downsample >= 1, halfwidth >= 0 (in fine frames)
 *   fell_back : host int (may be NULL)
 * The call synchronises the handle's stream (to read the band-side test).
 * Returns DTW_ERR_UNSUPPORTED for D > 32 or a BF16 cost. */
int dtw_align_banded(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D,
                     const dtw_options* opt, int downsample, int halfwidth, int32_t* path,
                     int cap, int* path_len, float* total_cost, int* fell_back);

/* ---- planned batch (CUDA graph, autotuned schedule) ------------------------- */
/* A batch that is aligned again and again with the same shapes and buffers
 * (a serving loop refilling fixed staging buffers): dtw_batch_create lays out
 * the batch once (its own workspace and border buffer), picks the DP schedule
 * with an autotuner when flags has DTW_BATCH_AUTOTUNE (it aligns the batch with
 * 2, 3 and 4 rows per lane and two or four strips per CTA, where D allows
 * them, and keeps the fastest; every schedule gives the same result, bit for
 * bit), and captures the whole batch
 * (a new tag for the border entries, the batched normalisation, the
 * persistent DP over the (pair, strip group) work queue, the batched
 * backtrace) into one CUDA graph.  dtw_batch_run launches that graph on the
 * handle's stream: it reads whatever A[k], B[k] hold at that time and writes
 * the outputs as dtw_align_many does.  Creation itself aligns the batch (the
 * outputs then hold its result) and synchronises the stream.
 *   A[k], B[k], paths, path_len, cost (may be NULL): device memory that must
 *     stay valid for the plan's life; path_off, lengths and D as in
 *     dtw_align_many; every pair must be valid (else its status is returned)
 *   D <= 32, FP32 cost, default options.
 * A device-side failure of a pair (bounded wait) shows as path_len[k] < 0. */
typedef struct dtw_batch dtw_batch;
#define DTW_BATCH_AUTOTUNE 1
int dtw_batch_create(dtw_handle* h, int n, const float* const* A, const int* La,
                     const float* const* B, const int* Lb, int D, int32_t* paths,
                     const int64_t* path_off, int* path_len, float* cost, int flags,
                     dtw_batch** out);
/* One replay of the plan's graph on the handle's stream (asynchronous). */
int dtw_batch_run(dtw_batch* b);
/* The chosen schedule (rows per lane, strips per CTA) and the autotuner's
 * times in ms: tuned_ms[0..2] for 2, 3, 4 rows per lane with two strips per
 * CTA, tuned_ms[3..5] with four (-1 where not tried or not supported); any
 * pointer may be NULL. */
int dtw_batch_info(const dtw_batch* b, int* rows_per_lane, int* strips_per_cta,
                   float* tuned_ms);
/* Waits for the plan's last replay and frees it; needs only the plan (it may
 * run after its handle was destroyed).  dtw_batch_run needs the handle alive. */
int dtw_batch_destroy(dtw_batch* b);

/* ---- weakly-ordered Segmental DTW (Sec. II-C) ------------------------------ */
/* WSDTW of the query A (La x D) against the reference B (Lb x D) with nfrag
 * fragments of A:
 *   1. fragment k holds rows floor(k La / nfrag) .. floor((k+1) La / nfrag) - 1;
 *   2. subsequence DTW of every fragment against all of B: steps (query,
 *      reference) (1,1), (1,2), (2,1) with weights 1, 1, 2, start anywhere in
 *      B (D_k[0][j] = C_k[0][j]), end anywhere; FP32, the same cost, tie order
 *      and kernels as dtw_align (the fragments run as one batch);
 *   3. C_seg[k][j] = D_k[last row][j];
 *   4. D_seg[k][j] = min(D_seg[k][j-1], D_seg[k-1][j - delta_k] + C_seg[k][j])
 *      with delta_k = floor(len_k / 2) (the shortest match of a fragment of
 *      len_k frames), D_seg[0][j] = min(D_seg[0][j-1], C_seg[0][j]); a match
 *      replaces the skip only when strictly smaller;
 *   5. every fragment's path from (last row, e_k) back to its first row.
 *   path       : device int32 pairs (row of A, frame of B), cap >= La; the
 *                fragments' paths one after another (each ascending), so the
 *                frame may step back at a fragment boundary (Sec. II-C)
 *   path_len   : device int; the number of pairs, or -status on a device-side
 *                failure (DTW_ERR_UNREACHABLE when B is too short to place the
 *                fragments in order)
 *   ends       : device int32[nfrag], end frame e_k of every fragment (may be NULL)
 *   total_cost : device float, D_seg[nfrag-1][Lb-1] (may be NULL)
 * D <= 32, 1 <= nfrag <= La.  Asynchronous on the handle's stream. */
int dtw_wsdtw(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D, int nfrag,
              int32_t* path, int cap, int* path_len, int32_t* ends, float* total_cost);

/* C_seg of the last dtw_wsdtw call on this handle (nfrag x Lb floats, row-major,
 * device), for inspection and tests; nfrag and Lb must be those of that call. */
int dtw_wsdtw_cseg(dtw_handle* h, int nfrag, int Lb, float* cseg);

/* ---- learned band ---------------------------------------------------------- */
/* A band predicted by a small network instead of a fixed half-width.  The
 * paper names bands and multiscale DTW only as related ways to cut the
 * quadratic cost (Sec. II); the encoder, its training and its use are this
 * library's.  The encoder maps each sequence, averaged over `downsample`
 * frames and L2-normalised per frame, through three convolutions of width 5
 * (64 channels, zero padding 2, ReLU) to a 16-dimensional unit embedding per
 * coarse frame, and for A to a half-width per coarse frame
 *   hw = DTW_BAND_WMIN * (DTW_BAND_WMAX / DTW_BAND_WMIN)^sigmoid(s)   (fine frames).
 * dtw_align_learned aligns the embeddings exactly (cosine cost), takes per
 * strip of the fine DP the band of the widest predicted half-width around
 * the upsampled coarse path, runs the exact DP inside it, and falls back to
 * the full exact DP when the banded path comes within one 8-column block of
 * a side of the band (as dtw_align_banded).
 *
 * Parameters: one float32 array of dtw_encoder_param_count(D) values (device
 * memory), in this order (weights of a convolution [out][in][5], row-major):
 *   W1 [64][D][5], b1 [64], W2 [64][64][5], b2 [64], W3 [64][64][5], b3 [64],
 *   W4 [16][64], b4 [16] (embedding), W5 [64], b5 [1] (half-width logit). */
#define DTW_BAND_WMIN 256
#define DTW_BAND_WMAX 2048
#define DTW_ENC_CHANNELS 64
#define DTW_ENC_EMBED 16
#define DTW_ENC_KERNEL 5

/* Number of parameters for input dimension D (1 <= D <= 64), else 0.  Host
 * function; needs no device. */
size_t dtw_encoder_param_count(int D);

/* Encoder forward of one sequence X (L x D, device) at `downsample`:
 * emb (ceil(L/downsample) x 16, device) and, if not NULL, halfwidth
 * (ceil(L/downsample), device, fine frames).  bf16 != 0 rounds the inputs
 * and weights of the convolutions and of the embedding head to bfloat16
 * (FP32 accumulation). */
int dtw_encode(dtw_handle* h, const float* params, int D, const float* X, int L, int downsample,
               int bf16, float* emb, float* halfwidth);

/* Training: adds to grad (device, dtw_encoder_param_count(D) floats) the
 * gradient of the loss of one pair and adds the loss to *loss (device).
 * path / path_len (device) is the exact alignment of (A, B) (as dtw_align
 * writes it).  Per coarse row i of A the exact path matches coarse column
 * c_i (its mean column in the row's frames / downsample).
 *   mode 0: embedding loss, mean over i of -log softmax_j(eA_i . eB_j / 0.1)
 *           at j = c_i, j over the coarse columns within 16 of c_i; gradient
 *           of the trunk and the embedding head.
 *   mode 1: half-width loss, mean over i of the pinball loss at quantile 0.9
 *           of sigmoid(s_i) against the log-scale half-width (in [0, 1]) the
 *           band of the coarse alignment of the current embeddings needs at
 *           row i to hold the exact path, plus 64 frames; gradient of W5, b5.
 * FP32 throughout; downsample >= 2.  Asynchronous. */
int dtw_encoder_grad(dtw_handle* h, const float* params, int D, int downsample, const float* A,
                     int La, const float* B, int Lb, const int32_t* path, const int* path_len,
                     int mode, float* grad, float* loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; `step`
 * counts from 1) over n parameters, all device arrays; grad is zeroed. */
int dtw_encoder_adam(dtw_handle* h, int n, float* params, float* grad, float* m, float* v,
                     int step, float lr);

/* Exact DTW inside the learned band, with the same arguments, device-only
 * rule, synchronisation and fallback as dtw_align_banded; params (device)
 * as above for this D (D <= 32, FP32 cost). */
int dtw_align_learned(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D,
                      const dtw_options* opt, const float* params, int downsample, int bf16,
                      int32_t* path, int cap, int* path_len, float* total_cost, int* fell_back);

/* Cells of the band the last dtw_align_banded / dtw_align_learned call on
 * this handle swept (rows x columns of every strip's range); 0 if it fell
 * back or no band was run.  Synchronises the handle's stream. */
int dtw_band_cells(dtw_handle* h, long long* cells);

/* ---- alignment without device allocation ---------------------------------- */
/* The paper has no counterpart of this entry point; it is a service of this
 * library.  Some callers cannot allocate device memory while they align: a
 * real-time loop (live score following) that must not block in the driver's
 * allocator, or a process whose device memory is already reserved by
 * another allocator (a framework's caching allocator, a plugin host with a
 * fixed budget).  dtw_align_static returns what dtw_align returns (the same
 * path and the same total, bit for bit) but allocates nothing: all of its
 * scratch lives in one fixed device array of dtw_static_scratch_bytes()
 * bytes (64 MiB) that every GPU loading the library holds until the process
 * exits.  It runs dtw_align's DP kernel and parallel backtrace on the pair as
 * given (A's frames as rows; it never takes the transposed sweep, which
 * yields the same cells).
 *
 *   A, B, path, path_len, total_cost : device pointers (total_cost may be
 *       NULL); a host pointer is rejected with DTW_ERR_INVALID
 *   cuda_stream : stream the work is ordered on (NULL = legacy default)
 *   opt : as in dtw_align, except that only the FP32 cost is offered
 *       (cost_precision = DTW_COST_BF16 returns DTW_ERR_UNSUPPORTED) and
 *       opt->transpose has no effect
 *   other arguments as in dtw_align; the call is asynchronous and reports
 *       device-side failures (a bounded wait that expired) through
 *       *path_len = -status
 * Sizes whose scratch (backpointers La*Lb/4 bytes plus padding, border rows,
 * the backtrace's band maps, normalised features) exceeds the array return
 * DTW_ERR_SCRATCH_LIMIT before any work is queued; about 1.44e8 cells fit
 * (2.15 cells per byte at D = 12, e.g. 12000 x 12000).
 * The first call on a device looks up the array's device address (a one-time
 * set-up per device, made with that device current); make that first call
 * before any stream capture.  Every call shares the array and leaves its
 * contents behind: calls whose work overlaps on the GPU (other streams,
 * other host threads) race on it and must be serialised by the caller. */
int dtw_align_static(const float* A, int La, const float* B, int Lb, int D,
                     const dtw_options* opt, void* cuda_stream, int32_t* path, int cap,
                     int* path_len, float* total_cost);
/* Size in bytes of the fixed scratch array used by dtw_align_static. */
size_t dtw_static_scratch_bytes(void);

/* ---- profiling ------------------------------------------------------------ */
/* Device time in ms of the stages of the last dtw_align on this handle,
 * measured with CUDA events on the handle's stream: ms[0] normalise,
 * ms[1] DP, ms[2] backtrace.  n = entries available in ms (<= 3).
 * Synchronises on the last call's events.  Returns DTW_ERR_INVALID if no
 * call has been timed (timing is enabled by dtw_enable_timing). */
int dtw_enable_timing(dtw_handle* h, int on);
int dtw_stage_times(dtw_handle* h, float* ms, int n);

/* Measured FP32 fused multiply-add throughput of `device`, in FFMA per
 * second over all SMs (best of three timed launches of a kernel that keeps
 * every SM sub-partition issuing independent FFMAs; `iters` loop trips of
 * 128 FFMA per thread, ~20 ms at 4096).  The paper has no counterpart: this
 * is the measured denominator of the roofline that the DP (bound by FP32
 * lane arithmetic, Sec. VI-C reports it compute-bound: 99.85% of ParDTW's
 * GPU time is the DP) is reported against.  Allocates and frees a small
 * device buffer; synchronises the device's legacy stream. */
int dtw_fp32_peak(int device, int iters, double* ffma_per_s);

#ifdef __cplusplus
}
#endif
#endif /* PARDTW_H */
