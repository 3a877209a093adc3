// C-ABI of libpardtw (declarations and contracts in include/pardtw.h).
//
// Host-side work only: argument checks, the reachability test, workspace
// management, pointer-kind detection, and the launch sequence
//   normalise -> column-sweep DP (cost on the fly) -> band map -> backtrace
// on the handle's stream.  Every step of the alignment runs in the kernels;
// there is no CPU fallback.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "pardtw_common.cuh"

using namespace pardtw;

struct dtw_handle {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    char* ws = nullptr;          // main workspace
    size_t ws_cap = 0;
    unsigned long long* border = nullptr;  // tagged border entries (own allocation, zeroed)
    size_t border_cap = 0;                 // bytes
    unsigned* done = nullptr;              // per-strip flags of the DP (own allocation, zeroed)
    size_t done_cap = 0;                   // flags
    unsigned epoch = 0;
    bool timing = false;
    bool timed = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int* h_small = nullptr;      // pinned host: [0] path_len, [1] total bits
    char* band = nullptr;        // banded calls: pooled inputs, coarse path, ranges, flag
    size_t band_cap = 0;
    int band_nstrips = 0;        // strips, rows per strip and columns of the last band
    int band_rps = 0;
    int band_Lb = 0;
    const int2* band_ranges = nullptr;
    char* enc = nullptr;         // band encoder activations and gradients
    size_t enc_cap = 0;
    char* wsd = nullptr;         // WSDTW: last rows, segment DP, fragment paths
    size_t wsd_cap = 0;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

#define CU(call)                                  \
    do {                                          \
        cudaError_t e_ = (call);                  \
        if (e_ != cudaSuccess) {                  \
            (void)cudaGetLastError();             \
            return DTW_ERR_CUDA;                  \
        }                                         \
    } while (0)

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool reachable(int La, int Lb) {
    long long i = La - 1, j = Lb - 1;
    return La >= 1 && Lb >= 1 && j <= 2 * i && i <= 2 * j;
}

struct Layout {
    DpPlan plan;
    int dp, R, rps, wpb, nstrips, nchunk, ngroups, La_pad, cap;
    size_t off_ctl, off_ahat, off_bhat, off_bbf, off_bp, off_bt, off_stage_a, off_stage_b,
        total;
    size_t border_bytes;
};

}  // namespace

// The DP kernel for a problem.  Explicit requests are honoured where the
// kernel supports them (else one row per lane); the default is the cost/DP
// warp pair with 3 rows per lane for D <= 32, one row per lane above.
DpPlan pardtw::choose_plan(int La, int dp, const dtw_options& o, int num_sms) {
    const DpPlan one = {0, 1, kWarpsPerGroup};
    const int nocl = o.clusters == DTW_CLUSTERS_NEVER ? 1 : 0;
    if (o.cost_precision == DTW_COST_BF16) return {2, 3, kSplitStrips, 1, nocl};
    const int req = o.rows_per_lane;
    if (req == 1) return one;
    if (o.dp_schedule == DTW_SCHEDULE_FUSED) {
        const int R = req == 0 ? 2 : req;
        if (multirow_supported(dp, R)) return {1, R, kWarpsPerGroup};
        return one;
    }
    const int R = req == 0 ? 3 : req;
    // D = 64, 128: the warp pairs with two cost warps per strip, 3 rows per lane
    if (split_wide_supported(dp)) return R == 3 ? DpPlan{2, 3, kSplitStrips, 0, nocl} : one;
    if (!split_supported(dp, R)) return one;
    // two strips per CTA unless asked for four: with the DP warp's costs
    // loaded at the start of each sub-chunk, two beat four on single pairs
    // of every size measured (1e5 x 1.26e5: 30.3 vs 31.5 ms; 5e4 x 6.25e4:
    // 8.32 vs 8.45 ms); batches pick theirs with the autotuner
    if (o.strips_per_cta == 4 && split_supported(dp, R, 4)) return {2, R, 4};
    return {2, R, kSplitStrips, 0, nocl};
}

cudaError_t pardtw::launch_plan(const DpPlan& plan, const DpArgs& a, int dp, int num_sms,
                        cudaStream_t s, bool transposed) {
    if (transposed && (plan.kind != 2 || plan.R != 3)) return cudaErrorInvalidValue;
    switch (plan.kind) {
        case 0: return launch_dp(a, dp, num_sms, s);
        case 1: return launch_dp_multirow(a, dp, plan.R, num_sms, s);
        case 2:
            if (!plan.no_clusters && plan.R == 3 && plan.spg == kSplitStrips) {
                bool used = false;
                const cudaError_t e = launch_dp_split_cl(a, dp, plan.bf16 != 0, transposed, s, &used);
                if (e != cudaSuccess || used) return e;
            }
            if (plan.bf16) return launch_dp_split_bf16(a, dp, num_sms, s, transposed);
            if (split_wide_supported(dp)) return launch_dp_split_wide(a, dp, num_sms, s, transposed);
            return launch_dp_split(a, dp, plan.R, plan.spg, num_sms, s, transposed);
        default: return cudaErrorInvalidValue;
    }
}

// Which way to sweep a pair.  The persistent warp-pair DP runs its strip
// groups in waves of one group per SM: a CTA sweeps all columns of a group
// before it takes the next, and the next group in the chain starts a few
// blocks behind the one above.  So the time is about
//   ceil(groups / SMs) x columns  +  strips x (lag of one strip, ~18 columns)
// column steps; the transposed sweep (B's frames as rows) wins when that is
// smaller for (Lb rows, La columns), e.g. a pair that fits one wave with B
// longer: its chain then runs over La columns instead of Lb.  Only the
// warp-pair DP at 3 rows per lane has the transposed tie order.
namespace {
double sweep_estimate(int rows, int cols, int dp, const dtw_options& o, int num_sms) {
    const DpPlan p = choose_plan(rows, dp, o, num_sms);
    const int rps = strip_rows(p.R);
    const long long strips = (rows + rps - 1) / rps;
    const long long groups = (strips + p.spg - 1) / p.spg;
    const long long waves = num_sms > 0 ? (groups + num_sms - 1) / num_sms : 1;
    return (double)waves * cols + 18.0 * (double)strips;
}
}  // namespace

bool pardtw::transpose_pair(int La, int Lb, int dp, const dtw_options& o, int num_sms) {
    if (o.transpose == DTW_TRANSPOSE_NEVER) return false;
    const DpPlan pt = choose_plan(Lb, dp, o, num_sms);  // the plan the transposed pair gets
    if (pt.kind != 2 || pt.R != 3) return false;
    if (o.transpose == DTW_TRANSPOSE_ALWAYS) return true;
    return sweep_estimate(Lb, La, dp, o, num_sms) < sweep_estimate(La, Lb, dp, o, num_sms);
}

namespace {

Layout make_layout(int La, int Lb, int D, const DpPlan& plan) {
    Layout L;
    L.plan = plan;
    // the BF16 cost runs its tensor-core products over 64 or 128 features
    L.dp = plan.bf16 ? (D <= 64 ? 64 : 128) : padded_dim(D);
    const int R = plan.R;
    L.R = R;
    L.rps = strip_rows(R);
    L.wpb = strip_words(R);
    L.nstrips = (La + L.rps - 1) / L.rps;
    L.nchunk = (Lb + kColsPerWord - 1) / kColsPerWord;
    L.ngroups = (L.nstrips + plan.spg - 1) / plan.spg;
    L.La_pad = L.nstrips * L.rps;
    L.cap = std::min(La, Lb);
    size_t o = 0;
    L.off_ctl = o;  // DevCtl, e_final, total, path_len
    o += 256;
    L.off_ahat = o;
    o = align256(o + (size_t)L.La_pad * L.dp * sizeof(float));
    L.off_bhat = o;
    o = align256(o + (size_t)L.nchunk * kColsPerWord * L.dp * sizeof(float));
    L.off_bbf = o;
    if (plan.bf16) o = align256(o + (size_t)L.nchunk * kColsPerWord * kBfStride * 2);
    L.off_bp = o;
    o = align256(o + (size_t)L.nstrips * L.nchunk * L.wpb * sizeof(uint32_t));
    L.off_bt = o;
    o = align256(o + bandmap_scratch_bytes(La, Lb));
    L.off_stage_a = o;
    o = align256(o + (size_t)La * D * sizeof(float));
    L.off_stage_b = o;
    o = align256(o + (size_t)Lb * D * sizeof(float));
    L.total = o;
    L.border_bytes = (size_t)L.ngroups * Lb * 2 * sizeof(unsigned long long);
    return L;
}

int ensure_workspace(dtw_handle* h, size_t bytes, size_t border_bytes) {
    if (bytes > h->ws_cap) {
        CU(cudaStreamSynchronize(h->stream));
        if (h->ws) cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_cap = 0;
        size_t want = bytes + bytes / 8;
        if (cudaMalloc(&h->ws, want) != cudaSuccess) {
            (void)cudaGetLastError();
            if (cudaMalloc(&h->ws, bytes) != cudaSuccess) {
                (void)cudaGetLastError();
                h->ws = nullptr;
                return DTW_ERR_OOM;
            }
            want = bytes;
        }
        h->ws_cap = want;
    }
    if (border_bytes > h->border_cap) {
        CU(cudaStreamSynchronize(h->stream));
        if (h->border) cudaFree(h->border);
        h->border = nullptr;
        h->border_cap = 0;
        size_t want = border_bytes + border_bytes / 8;
        if (cudaMalloc(&h->border, want) != cudaSuccess) {
            (void)cudaGetLastError();
            h->border = nullptr;
            return DTW_ERR_OOM;
        }
        // Entries are tagged with the call's epoch, which only grows; zeroed
        // memory can never carry the tag of a live call.
        CU(cudaMemsetAsync(h->border, 0, want, h->stream));
        h->border_cap = want;
    }
    return DTW_OK;
}

// The per-strip flags of a single-pair DP with its band map inside: a
// separate zeroed allocation, written only with call epochs (which only grow),
// so no flag can carry the tag of a live call before its strip is done.
int ensure_done(dtw_handle* h, int n) {
    if ((size_t)n <= h->done_cap) return DTW_OK;
    CU(cudaStreamSynchronize(h->stream));
    if (h->done) cudaFree(h->done);
    h->done = nullptr;
    h->done_cap = 0;
    const size_t want = (size_t)n + (size_t)n / 8;
    if (cudaMalloc(&h->done, want * sizeof(unsigned)) != cudaSuccess) {
        (void)cudaGetLastError();
        h->done = nullptr;
        return DTW_ERR_OOM;
    }
    CU(cudaMemsetAsync(h->done, 0, want * sizeof(unsigned), h->stream));
    h->done_cap = want;
    return DTW_OK;
}

dtw_options defaults() {
    dtw_options o;
    o.cost_precision = DTW_COST_FP32;
    o.cost_shift = 0.0f;
    o.wait_limit = 0;
    o.debug_skip_publish = -1;
    o.rows_per_lane = 0;
    o.dp_schedule = DTW_SCHEDULE_AUTO;
    o.strips_per_cta = 0;
    o.transpose = DTW_TRANSPOSE_AUTO;
    o.clusters = DTW_CLUSTERS_AUTO;
    return o;
}

// Rows per lane of a banded sweep: 3 unless the options ask for 2 or 4 (and
// the warp-pair kernel has it for this dimension).
int band_rows_per_lane(int dp, const dtw_options& o) {
    const int R = o.rows_per_lane;
    return ((R == 2 || R == 4) && split_supported(dp, R)) ? R : 3;
}

// One pair, all the way to device-resident outputs.  `out_path`,
// `out_len`, `out_total` are device pointers (out_total may be null).
int align_device(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D,
                 const dtw_options& o, int32_t* out_path, int* out_len, float* out_total,
                 const int2* ranges = nullptr, int transpose = -1) {
    // transpose < 0: decide here; a band's ranges come with the caller's
    // decision (they are per strip of the swept rows)
    const bool tr = transpose >= 0 ? transpose != 0
                                   : transpose_pair(La, Lb, padded_dim(D), o, h->num_sms);
    if (tr) {
        std::swap(A, B);
        std::swap(La, Lb);
    }
    // a band (per-strip column ranges) needs the warp-pair kernel at 3 rows
    // per lane, FP32 cost
    const DpPlan plan = ranges ? DpPlan{2, band_rows_per_lane(padded_dim(D), o), kSplitStrips, 0,
                                        o.clusters == DTW_CLUSTERS_NEVER ? 1 : 0}
                               : choose_plan(La, padded_dim(D), o, h->num_sms);
    const Layout L = make_layout(La, Lb, D, plan);
    int rc = ensure_workspace(h, L.total, L.border_bytes);
    if (rc != DTW_OK) return rc;
    // The warp-pair DP runs the backtrace's band map on its own CTAs when
    // its strip groups take more than one wave of resident CTAs: the CTAs
    // that find no group in the last wave map the bands above meanwhile
    // (1e5 x 1.26e5 frames: 28.9 ms against 30.1 ms with the band map
    // after the DP).  With one wave the first band is only ready when the
    // first strips end, near the end of the sweep, and six warps per SM map
    // more slowly than the separate kernel's sixteen (20000 x 25000: no
    // gain); a banded sweep's chain of strips is slowed by items beside it
    // (+5%).
    const bool fuse_map =
        plan.kind == 2 && !ranges && split_map_supported(L.dp, plan.R, plan.spg, plan.bf16 != 0) &&
        L.ngroups > split_ctas_per_sm(plan.R, plan.spg, L.dp, plan.bf16 != 0) * h->num_sms;
    if (fuse_map && (rc = ensure_done(h, L.nstrips)) != DTW_OK) return rc;
    cudaStream_t s = h->stream;
    char* ws = h->ws;
    DevCtl* ctl = reinterpret_cast<DevCtl*>(ws + L.off_ctl);
    float* e_final = reinterpret_cast<float*>(ws + L.off_ctl + 16);
    float* Ahat = reinterpret_cast<float*>(ws + L.off_ahat);
    float* Bhat = reinterpret_cast<float*>(ws + L.off_bhat);
    uint32_t* bp = reinterpret_cast<uint32_t*>(ws + L.off_bp);

    const float* dA = A;
    const float* dB = B;
    if (!is_device_ptr(A)) {
        float* st = reinterpret_cast<float*>(ws + L.off_stage_a);
        CU(cudaMemcpyAsync(st, A, (size_t)La * D * sizeof(float), cudaMemcpyHostToDevice, s));
        dA = st;
    }
    if (!is_device_ptr(B)) {
        float* st = reinterpret_cast<float*>(ws + L.off_stage_b);
        CU(cudaMemcpyAsync(st, B, (size_t)Lb * D * sizeof(float), cudaMemcpyHostToDevice, s));
        dB = st;
    }
    if (h->timing) CU(cudaEventRecord(h->ev[0], s));
    CU(launch_normalise(dA, La, L.La_pad, dB, Lb, L.nchunk * kColsPerWord, D, L.dp, Ahat, Bhat,
                        ctl, s));
    void* Bbf = L.plan.bf16 ? ws + L.off_bbf : nullptr;
    if (Bbf) CU(launch_pack_b_bf16(dB, Lb, L.nchunk * kColsPerWord, D, Bbf, s));
    if (h->timing) CU(cudaEventRecord(h->ev[1], s));

    DpArgs a;
    a.Ahat = Ahat;
    a.Bhat = Bhat;
    a.Bbf = Bbf;
    a.ranges = ranges;
    a.lastrow = nullptr;
    a.bp = bp;
    a.gborder = h->border;
    a.ctl = ctl;
    a.e_final = e_final;
    a.La = La;
    a.Lb = Lb;
    a.nstrips = L.nstrips;
    a.nchunk = L.nchunk;
    a.ngroups = L.ngroups;
    a.rps = L.rps;
    a.wpb = L.wpb;
    a.mu = o.cost_shift;
    a.kcost = 1.0f - o.cost_shift;
    a.epoch = ++h->epoch;
    if (a.epoch == 0) a.epoch = ++h->epoch;
    a.timeout_ns = o.wait_limit > 0 ? (long long)o.wait_limit * 1000LL : kDefaultTimeoutNs;
    a.skip_publish = o.debug_skip_publish;
    BtArgs bt;
    bt.bp = bp;
    bt.La = La;
    bt.Lb = Lb;
    bt.nchunk = L.nchunk;
    bt.rps = L.rps;
    bt.wpb = L.wpb;
    bt.ctl = ctl;
    bt.e_final = e_final;
    bt.mu = o.cost_shift;
    bt.path = out_path;
    bt.path_len = out_len;
    bt.total = out_total;
    bt.scratch = ws + L.off_bt;
    bt.ranges = ranges;
    bt.transposed = tr ? 1 : 0;
    if (fuse_map) {
        MapArgs m;
        m.bt = bt;
        m.done = h->done;
        m.nbm = bandmap_items(La, Lb, (2 * plan.spg + 2) * 32);
        CU(launch_dp_split_map(a, m, L.dp, h->num_sms, s, tr));
    } else {
        CU(launch_plan(L.plan, a, L.dp, h->num_sms, s, tr));
    }
    if (h->timing) CU(cudaEventRecord(h->ev[2], s));
    CU(launch_backtrace_bands(bt, s, !fuse_map));
    if (h->timing) {
        CU(cudaEventRecord(h->ev[3], s));
        h->timed = true;
    }
    return DTW_OK;
}

int validate(const float* A, int La, const float* B, int Lb, int D) {
    if (!A || !B || La < 1 || Lb < 1 || D < 1) return DTW_ERR_INVALID;
    if (!reachable(La, Lb)) return DTW_ERR_UNREACHABLE;
    if (padded_dim(D) == 0) return DTW_ERR_UNSUPPORTED;
    return DTW_OK;
}

// The batched path of dtw_align_many (device inputs and outputs, D <= 32):
// every pair of `idx` in one batched normalisation, one persistent DP launch
// over a (pair, strip group) work queue and one batched backtrace.
// Subsequence mode of align_batch (WSDTW): the DP of every pair in
// subsequence form, its last row into lastrow + k * stride, no backtrace;
// bts_out[k] receives pair k's backtrace geometry and control block.
struct SubseqBatch {
    float* lastrow;
    size_t stride;
    std::vector<BtArgs>* bts_out;
};

// Layout of a batch in one workspace: the descriptors, one control block per
// pair, then every pair's buffers; the border rows of all pairs in another.
// The work queue runs the pairs with the longest sweeps first, so that the
// last pairs to start are short and no long chain of strips is left alone at
// the end (the order does not change any result).
struct BatchSetup {
    int m = 0, D = 0, dp = 0, R = 3, NS = 2, maxLa = 0, maxLb = 0, max_frames = 0;
    std::vector<int> idx;  // pair indices in work-queue order
    std::vector<Layout> Ls;
    std::vector<size_t> off, boff;
    std::vector<int> item0;
    size_t off_dp = 0, off_norm = 0, off_bt = 0, off_item = 0, off_ctl = 0;
    size_t ws_bytes = 0, border_bytes = 0;
};

BatchSetup batch_setup(std::vector<int> idx, const int* La, const int* Lb, int D, int R, int NS) {
    BatchSetup b;
    b.m = (int)idx.size();
    b.R = R;
    b.NS = NS;
    b.D = D;
    b.dp = padded_dim(D);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        return (long long)Lb[x] * 256 + La[x] > (long long)Lb[y] * 256 + La[y];
    });
    b.idx = idx;
    const int m = b.m;
    const DpPlan plan = {2, R, NS};
    b.Ls.resize(m);
    b.off.resize(m);
    b.boff.resize(m);
    b.item0.assign(m + 1, 0);
    size_t o0 = 0;
    b.off_dp = o0;
    o0 = align256(o0 + sizeof(DpArgs) * m);
    b.off_norm = o0;
    o0 = align256(o0 + sizeof(NormArgs) * m);
    b.off_bt = o0;
    o0 = align256(o0 + sizeof(BtArgs) * m);
    b.off_item = o0;
    o0 = align256(o0 + sizeof(int) * (m + 1) + 16);  // + the work-queue ticket
    b.off_ctl = o0;
    o0 = align256(o0 + (size_t)256 * m);
    size_t border_total = 0;
    for (int q = 0; q < m; ++q) {
        const int k = idx[q];
        b.Ls[q] = make_layout(La[k], Lb[k], D, plan);
        const Layout& L = b.Ls[q];
        b.off[q] = o0;
        o0 = align256(o0 + (L.off_stage_a - L.off_ahat));  // Ahat, Bhat, bp, band maps
        b.boff[q] = border_total;
        border_total += L.border_bytes;
        b.item0[q + 1] = b.item0[q] + L.ngroups;
        b.maxLa = std::max(b.maxLa, La[k]);
        b.maxLb = std::max(b.maxLb, Lb[k]);
        b.max_frames = std::max(b.max_frames, L.La_pad + L.nchunk * kColsPerWord);
    }
    b.ws_bytes = o0;
    b.border_bytes = border_total;
    return b;
}

// Host copies of the descriptors of a batch laid out in `ws` and `border`.
struct BatchDesc {
    std::vector<DpArgs> dps;
    std::vector<NormArgs> nas;
    std::vector<BtArgs> bts;
};

BatchDesc batch_descriptors(const BatchSetup& b, char* ws, unsigned long long* border,
                            const float* const* A, const int* La, const float* const* B,
                            const int* Lb, const dtw_options& o, unsigned epoch, int32_t* paths,
                            const int64_t* path_off, int* path_len, float* cost,
                            const SubseqBatch* sub) {
    BatchDesc d;
    const int m = b.m;
    d.dps.resize(m);
    d.nas.resize(m);
    d.bts.resize(m);
    for (int q = 0; q < m; ++q) {
        const int k = b.idx[q];
        const Layout& L = b.Ls[q];
        char* base = ws + b.off[q] - L.off_ahat;  // so that base + L.off_* addresses this pair
        DevCtl* ctl = reinterpret_cast<DevCtl*>(ws + b.off_ctl + (size_t)256 * q);
        float* e_final = reinterpret_cast<float*>(ws + b.off_ctl + (size_t)256 * q + 16);
        float* Ahat = reinterpret_cast<float*>(base + L.off_ahat);
        float* Bhat = reinterpret_cast<float*>(base + L.off_bhat);
        uint32_t* bpw = reinterpret_cast<uint32_t*>(base + L.off_bp);
        NormArgs& na = d.nas[q];
        na.A = A[k];
        na.La = La[k];
        na.La_pad = L.La_pad;
        na.B = B[k];
        na.Lb = Lb[k];
        na.Lb_pad = L.nchunk * kColsPerWord;
        na.Ahat = Ahat;
        na.Bt = Bhat;
        na.ctl = ctl;
        DpArgs& a = d.dps[q];
        a.Ahat = Ahat;
        a.Bhat = Bhat;
        a.Bbf = nullptr;
        a.ranges = nullptr;
        a.bp = bpw;
        a.gborder = border + b.boff[q] / sizeof(unsigned long long);
        a.ctl = ctl;
        a.e_final = e_final;
        a.La = La[k];
        a.Lb = Lb[k];
        a.nstrips = L.nstrips;
        a.nchunk = L.nchunk;
        a.ngroups = L.ngroups;
        a.rps = L.rps;
        a.wpb = L.wpb;
        a.mu = o.cost_shift;
        a.kcost = 1.0f - o.cost_shift;
        a.epoch = epoch;
        a.timeout_ns = o.wait_limit > 0 ? (long long)o.wait_limit * 1000LL : kDefaultTimeoutNs;
        a.skip_publish = o.debug_skip_publish;
        a.lastrow = sub ? sub->lastrow + (size_t)k * sub->stride : nullptr;
        BtArgs& bt = d.bts[q];
        bt.bp = bpw;
        bt.La = La[k];
        bt.Lb = Lb[k];
        bt.nchunk = L.nchunk;
        bt.rps = L.rps;
        bt.wpb = L.wpb;
        bt.ctl = ctl;
        bt.e_final = e_final;
        bt.mu = o.cost_shift;
        bt.path = sub ? nullptr : paths + 2 * path_off[k];
        bt.path_len = sub ? nullptr : path_len + k;
        bt.total = (cost && !sub) ? cost + k : nullptr;
        bt.scratch = base + L.off_bt;
        bt.ranges = nullptr;
        if (sub) (*sub->bts_out)[k] = bt;
    }
    return d;
}

int batch_upload(const BatchSetup& b, const BatchDesc& d, char* ws, cudaStream_t s) {
    const int m = b.m;
    CU(cudaMemcpyAsync(ws + b.off_dp, d.dps.data(), sizeof(DpArgs) * m, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(ws + b.off_norm, d.nas.data(), sizeof(NormArgs) * m, cudaMemcpyHostToDevice,
                       s));
    CU(cudaMemcpyAsync(ws + b.off_bt, d.bts.data(), sizeof(BtArgs) * m, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(ws + b.off_item, b.item0.data(), sizeof(int) * (m + 1),
                       cudaMemcpyHostToDevice, s));
    return DTW_OK;
}

// The launches of a batch whose descriptors are in `ws`: normalisation, the
// persistent DP, and (unless subseq) the batched backtrace.  `ev` (4 events
// or null) brackets the stages.
int batch_launch(const BatchSetup& b, char* ws, bool subseq, int num_sms, cudaStream_t s,
                 cudaEvent_t* ev) {
    const int m = b.m;
    int* ticket = reinterpret_cast<int*>(ws + b.off_item + sizeof(int) * (m + 1));
    if (ev) CU(cudaEventRecord(ev[0], s));
    CU(launch_normalise_many(reinterpret_cast<const NormArgs*>(ws + b.off_norm), m, b.max_frames,
                             b.D, b.dp, ticket, s));
    if (ev) CU(cudaEventRecord(ev[1], s));
    const DpArgs* dps = reinterpret_cast<const DpArgs*>(ws + b.off_dp);
    const int* item0 = reinterpret_cast<const int*>(ws + b.off_item);
    if (subseq)
        CU(launch_dp_subseq_many(dps, item0, m, b.item0[m], ticket, b.dp, num_sms, s));
    else
        CU(launch_dp_split_many(dps, item0, m, b.item0[m], ticket, b.dp, b.R, b.NS, num_sms, s));
    if (ev) CU(cudaEventRecord(ev[2], s));
    if (!subseq)
        CU(launch_backtrace_bands_many(reinterpret_cast<const BtArgs*>(ws + b.off_bt), m, b.maxLa,
                                       b.maxLb, s));
    if (ev) CU(cudaEventRecord(ev[3], s));
    return DTW_OK;
}

int align_batch(dtw_handle* h, std::vector<int> idx, const float* const* A, const int* La,
                const float* const* B, const int* Lb, int D, const dtw_options& o, int R,
                int32_t* paths, const int64_t* path_off, int* path_len, float* cost,
                const SubseqBatch* sub = nullptr, int NS = 2) {
    if (idx.empty()) return DTW_OK;
    const BatchSetup b = batch_setup(std::move(idx), La, Lb, D, R, NS);
    int rc = ensure_workspace(h, b.ws_bytes, b.border_bytes);
    if (rc != DTW_OK) return rc;
    unsigned epoch = ++h->epoch;
    if (epoch == 0) epoch = ++h->epoch;
    const BatchDesc d = batch_descriptors(b, h->ws, h->border, A, La, B, Lb, o, epoch, paths,
                                          path_off, path_len, cost, sub);
    rc = batch_upload(b, d, h->ws, h->stream);
    if (rc != DTW_OK) return rc;
    rc = batch_launch(b, h->ws, sub != nullptr, h->num_sms, h->stream,
                      h->timing ? h->ev : nullptr);
    if (rc == DTW_OK && h->timing) h->timed = true;
    return rc;
}

}  // namespace

// A planned, graph-captured batch (dtw_batch_create).
struct dtw_batch {
    dtw_handle* h = nullptr;      // used by dtw_batch_run only
    int device = 0;
    cudaEvent_t done = nullptr;   // recorded after every replay (destroy waits on it)
    int n = 0, D = 0, R = 3, NS = 2;
    char* ws = nullptr;
    unsigned long long* border = nullptr;
    BatchSetup setup;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // R = 2, 3, 4 with two strips per CTA, then with four
    float tuned_ms[6] = {-1.f, -1.f, -1.f, -1.f, -1.f, -1.f};
};

extern "C" {

void dtw_default_options(dtw_options* opt) {
    if (opt) *opt = defaults();
}

const char* dtw_status_string(int status) {
    switch (status) {
        case DTW_OK: return "ok";
        case DTW_ERR_INVALID: return "invalid argument";
        case DTW_ERR_UNREACHABLE: return "end cell unreachable with steps (1,1),(1,2),(2,1)";
        case DTW_ERR_OOM: return "device workspace allocation failed";
        case DTW_ERR_CUDA: return "CUDA runtime error";
        case DTW_ERR_TIMEOUT: return "bounded device wait expired";
        case DTW_ERR_UNSUPPORTED: return "unsupported option or size";
        case DTW_ERR_SCRATCH_LIMIT: return "problem exceeds the fixed scratch of dtw_align_static";
        default: return "unknown status";
    }
}

int dtw_create(dtw_handle** out, int device, void* cuda_stream) {
    if (!out) return DTW_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess) {
        (void)cudaGetLastError();
        return DTW_ERR_CUDA;
    }
    if (device < 0 || device >= n) return DTW_ERR_INVALID;
    DeviceGuard g(device);
    if (!g.ok) return DTW_ERR_CUDA;
    dtw_handle* h = new (std::nothrow) dtw_handle();
    if (!h) return DTW_ERR_OOM;
    h->device = device;
    h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    if (cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device) !=
            cudaSuccess ||
        cudaMallocHost(&h->h_small, 64) != cudaSuccess) {
        (void)cudaGetLastError();
        delete h;
        return DTW_ERR_CUDA;
    }
    for (auto& e : h->ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            (void)cudaGetLastError();
            dtw_destroy(h);
            return DTW_ERR_CUDA;
        }
    *out = h;
    return DTW_OK;
}

int dtw_destroy(dtw_handle* h) {
    if (!h) return DTW_ERR_INVALID;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(h->stream);
    if (h->ws) cudaFree(h->ws);
    if (h->border) cudaFree(h->border);
    if (h->done) cudaFree(h->done);
    if (h->band) cudaFree(h->band);
    if (h->enc) cudaFree(h->enc);
    if (h->wsd) cudaFree(h->wsd);
    for (auto& e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->h_small) cudaFreeHost(h->h_small);
    (void)cudaGetLastError();
    delete h;
    return DTW_OK;
}

int dtw_set_stream(dtw_handle* h, void* cuda_stream) {
    if (!h) return DTW_ERR_INVALID;
    h->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    return DTW_OK;
}

int dtw_workspace_size(int La, int Lb, int D, const dtw_options* opt, size_t* bytes) {
    if (!bytes || La < 1 || Lb < 1 || D < 1) return DTW_ERR_INVALID;
    const int dp = padded_dim(D);
    if (dp == 0) return DTW_ERR_UNSUPPORTED;
    const dtw_options o = opt ? *opt : defaults();
    size_t most = 0;
    for (int t = 0; t < 2; ++t) {  // either orientation of the sweep
        const int rows = t ? Lb : La, cols = t ? La : Lb;
        // the plan dtw_align takes (the SM count only decides between plans
        // of the same layout)
        const DpPlan plan = choose_plan(rows, dp, o, 152);
        const Layout L = make_layout(rows, cols, D, plan);
        // a pair swept in several waves of CTAs also keeps one flag per strip
        most = std::max(most, L.total + L.border_bytes + align256((size_t)L.nstrips * 4));
    }
    // and a host path staged after the layout
    *bytes = most + align256((size_t)2 * std::min(La, Lb) * sizeof(int32_t));
    return DTW_OK;
}

int dtw_cost(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D, float* C) {
    if (!h || !A || !B || !C || La < 1 || Lb < 1 || D < 1) return DTW_ERR_INVALID;
    const int dp = padded_dim(D);
    if (dp == 0) return DTW_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    const Layout L = make_layout(La, Lb, D, DpPlan{0, 1, kWarpsPerGroup});
    const bool c_dev = is_device_ptr(C);
    const size_t cbytes = (size_t)La * Lb * sizeof(float);
    const size_t need = L.total + (c_dev ? 0 : align256(cbytes));
    int rc = ensure_workspace(h, need, 0);
    if (rc != DTW_OK) return rc;
    cudaStream_t s = h->stream;
    char* ws = h->ws;
    const float* dA = A;
    const float* dB = B;
    if (!is_device_ptr(A)) {
        float* st = reinterpret_cast<float*>(ws + L.off_stage_a);
        CU(cudaMemcpyAsync(st, A, (size_t)La * D * sizeof(float), cudaMemcpyHostToDevice, s));
        dA = st;
    }
    if (!is_device_ptr(B)) {
        float* st = reinterpret_cast<float*>(ws + L.off_stage_b);
        CU(cudaMemcpyAsync(st, B, (size_t)Lb * D * sizeof(float), cudaMemcpyHostToDevice, s));
        dB = st;
    }
    DevCtl* ctl = reinterpret_cast<DevCtl*>(ws + L.off_ctl);
    float* Ahat = reinterpret_cast<float*>(ws + L.off_ahat);
    float* Bhat = reinterpret_cast<float*>(ws + L.off_bhat);
    CU(launch_normalise(dA, La, L.La_pad, dB, Lb, L.nchunk * kColsPerWord, D, dp, Ahat, Bhat,
                        ctl, s));
    float* dC = c_dev ? C : reinterpret_cast<float*>(ws + L.total);
    CU(launch_cost(Ahat, La, Bhat, Lb, dp, dC, s));
    if (!c_dev) {
        CU(cudaMemcpyAsync(C, dC, cbytes, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    return DTW_OK;
}

int dtw_align(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D,
              const dtw_options* opt, int32_t* path, int cap, int* path_len,
              float* total_cost) {
    if (!h || !path || !path_len) return DTW_ERR_INVALID;
    int rc = validate(A, La, B, Lb, D);
    if (rc != DTW_OK) return rc;
    if (cap < std::min(La, Lb)) return DTW_ERR_INVALID;
    const dtw_options o = opt ? *opt : defaults();
    if (o.cost_precision != DTW_COST_FP32 &&
        (o.cost_precision != DTW_COST_BF16 || D > 128))
        return DTW_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;

    // The workspace holds either orientation's layout (align_device picks
    // one) with the staged path after both, so nothing moves or overlaps.
    const int dp = padded_dim(D);
    const Layout L1 = make_layout(La, Lb, D, choose_plan(La, dp, o, h->num_sms));
    const Layout L2 = make_layout(Lb, La, D, choose_plan(Lb, dp, o, h->num_sms));
    const int npairs = std::min(La, Lb);
    const size_t off_path = std::max(L1.total, L2.total);
    rc = ensure_workspace(h, off_path + align256((size_t)2 * npairs * sizeof(int32_t)),
                          std::max(L1.border_bytes, L2.border_bytes));
    if (rc != DTW_OK) return rc;
    const bool path_dev = is_device_ptr(path);
    const bool len_dev = is_device_ptr(path_len);
    const bool tot_dev = total_cost ? is_device_ptr(total_cost) : true;
    char* ws = h->ws;
    int32_t* dpath = path_dev ? path : reinterpret_cast<int32_t*>(ws + off_path);
    int* dlen = len_dev ? path_len : reinterpret_cast<int*>(ws + L1.off_ctl + 24);
    float* dtot = total_cost ? (tot_dev ? total_cost : reinterpret_cast<float*>(ws + L1.off_ctl + 20))
                             : nullptr;
    rc = align_device(h, A, La, B, Lb, D, o, dpath, dlen, dtot);
    if (rc != DTW_OK) return rc;
    cudaStream_t s = h->stream;
    const bool host_out = !path_dev || !len_dev || !tot_dev;
    if (!host_out) return DTW_OK;

    // host outputs: total, length and all min(La, Lb) path pairs the buffer
    // has room for, then one synchronisation
    CU(cudaMemcpyAsync(h->h_small, ws + L1.off_ctl + 20, 8, cudaMemcpyDeviceToHost, s));
    if (len_dev) CU(cudaMemcpyAsync(h->h_small + 1, path_len, 4, cudaMemcpyDeviceToHost, s));
    if (!path_dev)
        CU(cudaMemcpyAsync(path, dpath, (size_t)2 * npairs * sizeof(int32_t),
                           cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const int n = h->h_small[1];
    if (!len_dev) *path_len = n;
    if (total_cost && !tot_dev) memcpy(total_cost, &h->h_small[0], sizeof(float));
    if (n < 0) return -n;
    return DTW_OK;
}

int dtw_align_many(dtw_handle* h, int n, const float* const* A, const int* La,
                   const float* const* B, const int* Lb, int D, const dtw_options* opt,
                   int32_t* paths, const int64_t* path_off, int* path_len, float* cost,
                   int* status) {
    if (!h || n < 0 || (n > 0 && (!A || !La || !B || !Lb || !paths || !path_off || !path_len ||
                                  !status)))
        return DTW_ERR_INVALID;
    if (n == 0) return DTW_OK;
    const dtw_options o = opt ? *opt : defaults();
    if (o.cost_precision != DTW_COST_FP32 &&
        (o.cost_precision != DTW_COST_BF16 || D > 128))
        return DTW_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    const bool paths_dev = is_device_ptr(paths);
    const bool len_dev = is_device_ptr(path_len);
    const bool cost_dev = cost ? is_device_ptr(cost) : true;
    const bool st_dev = is_device_ptr(status);
    std::vector<int> hst(n, DTW_OK);
    std::vector<int> hlen(n, 0);
    std::vector<float> hcost(n, NAN);
    // One batched launch sequence when every buffer is on the device and the
    // warp-pair DP applies; otherwise one alignment after another.
    const int dp = padded_dim(D);
    const int Rb = (o.rows_per_lane >= 2 && o.rows_per_lane <= 4) ? o.rows_per_lane : 3;
    bool batched = paths_dev && len_dev && cost_dev && dp != 0 && split_supported(dp, Rb) &&
                   o.rows_per_lane != 1 && o.dp_schedule != DTW_SCHEDULE_FUSED &&
                   o.cost_precision == DTW_COST_FP32;
    std::vector<int> valid;
    for (int k = 0; k < n; ++k) {
        const int rc = validate(A[k], La[k], B[k], Lb[k], D);
        if (rc != DTW_OK) {
            hst[k] = rc;
            hlen[k] = -rc;
        } else {
            valid.push_back(k);
            if (!is_device_ptr(A[k]) || !is_device_ptr(B[k])) batched = false;
        }
    }
    if (batched) {
        // a batch fills the GPU: four strips per CTA where the kernel has them
        // (unless the options ask for two)
        const int NSb = (o.strips_per_cta != 2 && split_supported(dp, Rb, 4)) ? 4 : 2;
        const int rc = align_batch(h, valid, A, La, B, Lb, D, o, Rb, paths, path_off, path_len,
                                   cost, nullptr, NSb);
        if (rc != DTW_OK) return rc;
    }
    for (int k = 0; k < n && !batched; ++k) {
        int rc = hst[k];
        if (rc != DTW_OK) continue;
        int32_t* pk = paths + 2 * path_off[k];
        if (paths_dev && len_dev && cost_dev) {
            rc = align_device(h, A[k], La[k], B[k], Lb[k], D, o, pk, path_len + k,
                              cost ? cost + k : nullptr);
        } else {
            rc = dtw_align(h, A[k], La[k], B[k], Lb[k], D, &o, pk, std::min(La[k], Lb[k]),
                           len_dev ? path_len + k : &hlen[k],
                           cost ? (cost_dev ? cost + k : &hcost[k]) : nullptr);
            if (rc == DTW_ERR_TIMEOUT) {
                hst[k] = rc;
                hlen[k] = -rc;
                continue;
            }
        }
        if (rc != DTW_OK) return rc;
    }
    cudaStream_t s = h->stream;
    // host-side failures into device outputs
    for (int k = 0; k < n; ++k) {
        if (hst[k] == DTW_OK) continue;
        if (len_dev) CU(cudaMemcpyAsync(path_len + k, &hlen[k], 4, cudaMemcpyHostToDevice, s));
        if (cost && cost_dev) CU(cudaMemcpyAsync(cost + k, &hcost[k], 4, cudaMemcpyHostToDevice, s));
    }
    CU(cudaStreamSynchronize(s));
    if (!len_dev)
        for (int k = 0; k < n; ++k)
            if (hst[k] != DTW_OK) path_len[k] = hlen[k];
    if (cost && !cost_dev)
        for (int k = 0; k < n; ++k)
            if (hst[k] != DTW_OK) cost[k] = hcost[k];
    // statuses: host-side ones, or the sign of the device-side lengths
    std::vector<int> lens(n);
    if (len_dev) {
        CU(cudaMemcpyAsync(lens.data(), path_len, sizeof(int) * n, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    } else
        memcpy(lens.data(), path_len, sizeof(int) * n);
    for (int k = 0; k < n; ++k)
        if (hst[k] == DTW_OK && lens[k] < 0) hst[k] = -lens[k];
    if (st_dev) {
        CU(cudaMemcpyAsync(status, hst.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
        CU(cudaStreamSynchronize(s));  // hst is a local buffer
    } else
        memcpy(status, hst.data(), sizeof(int) * n);
    return DTW_OK;
}

}  // extern "C"

namespace {

// Grow a handle-owned device buffer (synchronising the stream first, since
// queued work may still use the old one).
int grow(dtw_handle* h, char** buf, size_t* cap, size_t need) {
    if (need <= *cap) return DTW_OK;
    CU(cudaStreamSynchronize(h->stream));
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    if (cudaMalloc(buf, need) != cudaSuccess) {
        (void)cudaGetLastError();
        *buf = nullptr;
        return DTW_ERR_OOM;
    }
    *cap = need;
    return DTW_OK;
}

// Offsets in the band buffer: pooled A and B (pooled = true), the coarse
// path and its length, the strip ranges and the band-side flag.
struct BandBuf {
    size_t pa, pb, cp, cl, rg, tc, total;
};
BandBuf band_buf(int Lac, int Lbc, int D, int nstrips, bool pooled) {
    BandBuf b;
    size_t o = 0;
    b.pa = o;
    if (pooled) o = align256(o + (size_t)Lac * D * sizeof(float));
    b.pb = o;
    if (pooled) o = align256(o + (size_t)Lbc * D * sizeof(float));
    b.cp = o;
    o = align256(o + (size_t)2 * std::min(Lac, Lbc) * sizeof(int32_t));
    b.cl = o;
    o = align256(o + 16);
    b.rg = o;
    o = align256(o + (size_t)nstrips * sizeof(int2));
    b.tc = o;
    b.total = o + 256;
    return b;
}

// The band pipeline after the coarse features: exact alignment of the
// coarse sequences cA (Lac x Dc) and cB (Lbc x Dc), per strip of the fine DP
// the blocks within the half-width (w, or wrow per coarse row) of the
// upsampled coarse path, the exact DP inside the band, and the full exact
// DP when the banded path meets a side of the band.
int band_align(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D,
               const dtw_options& o, int ds, const float* cA, int Lac, const float* cB, int Lbc,
               int Dc, int w, const float* wrowA, const float* wrowB, const BandBuf& bb,
               int32_t* path, int* path_len, float* total_cost, int* fell_back) {
    cudaStream_t s = h->stream;
    const int rps = strip_rows(band_rows_per_lane(padded_dim(D), o));
    // the fine DP may sweep the transposed pair (B's frames as rows): the
    // strips, their ranges and the band test are then over B.  A band is one
    // chain of strips over all columns whatever its size, so the sweep runs
    // over the shorter sequence's frames
    dtw_options ob = o;
    if (ob.transpose == DTW_TRANSPOSE_AUTO)
        ob.transpose = Lb > La ? DTW_TRANSPOSE_ALWAYS : DTW_TRANSPOSE_NEVER;
    const bool tr = transpose_pair(La, Lb, padded_dim(D), ob, h->num_sms);
    const int Lr = tr ? Lb : La, Lc = tr ? La : Lb, Lrc = tr ? Lbc : Lac;
    const float* wrow = tr ? wrowB : wrowA;
    const int nstrips = (Lr + rps - 1) / rps;
    int32_t* cpath = reinterpret_cast<int32_t*>(h->band + bb.cp);
    int* clen = reinterpret_cast<int*>(h->band + bb.cl);
    int2* ranges = reinterpret_cast<int2*>(h->band + bb.rg);
    int* touch = reinterpret_cast<int*>(h->band + bb.tc);
    dtw_options oc = o;
    oc.rows_per_lane = 0;
    oc.dp_schedule = DTW_SCHEDULE_AUTO;
    int rc = align_device(h, cA, Lac, cB, Lbc, Dc, oc, cpath, clen, nullptr);
    if (rc != DTW_OK) return rc;
    CU(launch_band_ranges(cpath, clen, ds, w, wrow, Lrc, Lr, Lc, nstrips, rps, tr ? 1 : 0,
                          ranges, s));
    h->band_nstrips = nstrips;
    h->band_rps = rps;
    h->band_Lb = Lc;
    h->band_ranges = ranges;
    rc = align_device(h, A, La, B, Lb, D, o, path, path_len, total_cost, ranges, tr ? 1 : 0);
    if (rc != DTW_OK) return rc;
    CU(launch_band_touch(path, path_len, std::min(La, Lb), Lc, rps, ranges, tr ? 1 : 0, touch,
                         s));
    CU(cudaMemcpyAsync(h->h_small + 2, touch, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (h->h_small[2]) {
        if (fell_back) *fell_back = 1;
        h->band_nstrips = 0;
        return align_device(h, A, La, B, Lb, D, o, path, path_len, total_cost);
    }
    return DTW_OK;
}

// Checks shared by the banded entry points; returns DTW_OK and the options.
int band_checks(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D,
                const dtw_options* opt, int ds, int32_t* path, int cap, int* path_len,
                float* total_cost, dtw_options* o) {
    if (!h || !path || !path_len || ds < 1) return DTW_ERR_INVALID;
    int rc = validate(A, La, B, Lb, D);
    if (rc != DTW_OK) return rc;
    if (cap < std::min(La, Lb)) return DTW_ERR_INVALID;
    *o = opt ? *opt : defaults();
    if (o->cost_precision != DTW_COST_FP32 || !split_supported(padded_dim(D), 3))
        return DTW_ERR_UNSUPPORTED;
    if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(path) ||
        !is_device_ptr(path_len) || (total_cost && !is_device_ptr(total_cost)))
        return DTW_ERR_INVALID;
    return DTW_OK;
}

// Encoder buffers of one sequence of Lc coarse frames in the handle's
// encoder buffer (floats unless noted).
struct EncSeq {
    size_t X, H1, H2, H3, E, invn, S, HW, G, dHa, dHb, total;
};
EncSeq enc_seq(size_t base, int Lc, int D) {
    EncSeq q;
    size_t o = base;
    auto take = [&](size_t n) { size_t at = o; o = align256(o + n * sizeof(float)); return at; };
    q.X = take((size_t)Lc * D);
    q.H1 = take((size_t)Lc * kEncChannels);
    q.H2 = take((size_t)Lc * kEncChannels);
    q.H3 = take((size_t)Lc * kEncChannels);
    q.E = take((size_t)Lc * kEncEmbed);
    q.invn = take(Lc);
    q.S = take(Lc);
    q.HW = take(Lc);
    q.G = take((size_t)Lc * kEncEmbed);
    q.dHa = take((size_t)Lc * kEncChannels);
    q.dHb = take((size_t)Lc * kEncChannels);
    q.total = o;
    return q;
}
// Both sequences, then the per-row training data of A: targets (int), the
// sums behind them (u64, int), width targets, width-logit gradients.
struct EncBuf {
    EncSeq a, b;
    size_t tgt, jsum, cnt, wt, dS, total;
};
EncBuf enc_buf(int Lac, int Lbc, int D) {
    EncBuf e;
    e.a = enc_seq(0, Lac, D);
    e.b = enc_seq(e.a.total, Lbc, D);
    size_t o = e.b.total;
    e.tgt = o; o = align256(o + (size_t)Lac * sizeof(int));
    e.jsum = o; o = align256(o + (size_t)Lac * sizeof(unsigned long long));
    e.cnt = o; o = align256(o + (size_t)Lac * sizeof(int));
    e.wt = o; o = align256(o + (size_t)Lac * sizeof(float));
    e.dS = o; o = align256(o + (size_t)Lac * sizeof(float));
    e.total = o;
    return e;
}

float* ef(dtw_handle* h, size_t off) { return reinterpret_cast<float*>(h->enc + off); }

// Encoder forward of one sequence X (L fine frames): pooled input, the three
// conv layers and the heads, into the buffers of q.
int enc_forward(dtw_handle* h, const float* P, const EncLayout& pl, int D, const float* X, int L,
                int ds, int bf16, const EncSeq& q) {
    cudaStream_t s = h->stream;
    const int Lc = (L + ds - 1) / ds;
    CU(launch_pool_norm(X, L, D, ds, ef(h, q.X), s));
    CU(launch_conv(ef(h, q.X), nullptr, Lc, D, P + pl.W1, P + pl.b1, 1, 0, bf16, ef(h, q.H1), s));
    CU(launch_conv(ef(h, q.H1), nullptr, Lc, kEncChannels, P + pl.W2, P + pl.b2, 1, 0, bf16,
                   ef(h, q.H2), s));
    CU(launch_conv(ef(h, q.H2), nullptr, Lc, kEncChannels, P + pl.W3, P + pl.b3, 1, 0, bf16,
                   ef(h, q.H3), s));
    CU(launch_embed(ef(h, q.H3), Lc, P, pl, bf16, (float)DTW_BAND_WMIN, (float)DTW_BAND_WMAX,
                    ef(h, q.E), ef(h, q.invn), ef(h, q.S), ef(h, q.HW), s));
    return DTW_OK;
}

// Backward of the trunk and the embedding head of one sequence, from the
// gradient of the loss with respect to its embeddings (in q.G).
int enc_backward(dtw_handle* h, const float* P, const EncLayout& pl, int D, int Lc,
                 const EncSeq& q, float* grad) {
    cudaStream_t s = h->stream;
    constexpr int C = kEncChannels;
    CU(launch_embed_bwd(ef(h, q.E), ef(h, q.invn), Lc, P + pl.W4, ef(h, q.G), ef(h, q.dHa), s));
    CU(launch_outer(ef(h, q.G), kEncEmbed, ef(h, q.H3), C, Lc, grad + pl.W4, s));
    CU(launch_outer(ef(h, q.G), kEncEmbed, nullptr, 1, Lc, grad + pl.b4, s));
    // layer 3: dH3 in dHa (masked by H3 inside)
    CU(launch_conv_wgrad(ef(h, q.H2), Lc, C, ef(h, q.dHa), ef(h, q.H3), grad + pl.W3,
                         grad + pl.b3, s));
    CU(launch_conv(ef(h, q.dHa), ef(h, q.H3), Lc, C, P + pl.W3, nullptr, 0, 1, 0, ef(h, q.dHb),
                   s));
    // layer 2: dH2 in dHb
    CU(launch_conv_wgrad(ef(h, q.H1), Lc, C, ef(h, q.dHb), ef(h, q.H2), grad + pl.W2,
                         grad + pl.b2, s));
    CU(launch_conv(ef(h, q.dHb), ef(h, q.H2), Lc, C, P + pl.W2, nullptr, 0, 1, 0, ef(h, q.dHa),
                   s));
    // layer 1: dH1 in dHa
    CU(launch_conv_wgrad(ef(h, q.X), Lc, D, ef(h, q.dHa), ef(h, q.H1), grad + pl.W1,
                         grad + pl.b1, s));
    return DTW_OK;
}

}  // namespace

extern "C" {

int dtw_align_banded(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D,
                     const dtw_options* opt, int downsample, int halfwidth, int32_t* path,
                     int cap, int* path_len, float* total_cost, int* fell_back) {
    if (halfwidth < 0) return DTW_ERR_INVALID;
    dtw_options o;
    int rc = band_checks(h, A, La, B, Lb, D, opt, downsample, path, cap, path_len, total_cost, &o);
    if (rc != DTW_OK) return rc;
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    if (fell_back) *fell_back = 0;
    h->band_nstrips = 0;
    const int Lac = (La + downsample - 1) / downsample, Lbc = (Lb + downsample - 1) / downsample;
    if (downsample == 1 || !reachable(Lac, Lbc)) {
        if (fell_back) *fell_back = 1;
        return align_device(h, A, La, B, Lb, D, o, path, path_len, total_cost);
    }
    // strips of the banded sweep at most (its shortest strips: 2 rows per lane)
    const int nstrips = (std::max(La, Lb) + strip_rows(2) - 1) / strip_rows(2);
    const BandBuf bb = band_buf(Lac, Lbc, D, nstrips, true);
    rc = grow(h, &h->band, &h->band_cap, bb.total);
    if (rc != DTW_OK) return rc;
    float* pa = reinterpret_cast<float*>(h->band + bb.pa);
    float* pb = reinterpret_cast<float*>(h->band + bb.pb);
    CU(launch_pool(A, La, D, downsample, pa, h->stream));
    CU(launch_pool(B, Lb, D, downsample, pb, h->stream));
    return band_align(h, A, La, B, Lb, D, o, downsample, pa, Lac, pb, Lbc, D, halfwidth, nullptr,
                      nullptr, bb, path, path_len, total_cost, fell_back);
}

size_t dtw_encoder_param_count(int D) {
    if (D < 1 || D > kEncChannels) return 0;
    return enc_layout(D).count;
}

int dtw_encode(dtw_handle* h, const float* params, int D, const float* X, int L, int downsample,
               int bf16, float* emb, float* halfwidth) {
    if (!h || !params || !X || !emb || L < 1 || D < 1 || D > kEncChannels || downsample < 1)
        return DTW_ERR_INVALID;
    if (!is_device_ptr(params) || !is_device_ptr(X) || !is_device_ptr(emb) ||
        (halfwidth && !is_device_ptr(halfwidth)))
        return DTW_ERR_INVALID;
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    const int Lc = (L + downsample - 1) / downsample;
    const EncSeq q = enc_seq(0, Lc, D);
    int rc = grow(h, &h->enc, &h->enc_cap, q.total);
    if (rc != DTW_OK) return rc;
    const EncLayout pl = enc_layout(D);
    rc = enc_forward(h, params, pl, D, X, L, downsample, bf16 != 0, q);
    if (rc != DTW_OK) return rc;
    CU(cudaMemcpyAsync(emb, ef(h, q.E), sizeof(float) * (size_t)Lc * kEncEmbed,
                       cudaMemcpyDeviceToDevice, h->stream));
    if (halfwidth)
        CU(cudaMemcpyAsync(halfwidth, ef(h, q.HW), sizeof(float) * (size_t)Lc,
                           cudaMemcpyDeviceToDevice, h->stream));
    return DTW_OK;
}

int dtw_encoder_grad(dtw_handle* h, const float* params, int D, int downsample, const float* A,
                     int La, const float* B, int Lb, const int32_t* path, const int* path_len,
                     int mode, float* grad, float* loss) {
    if (!h || !params || !A || !B || !path || !path_len || !grad || !loss || La < 1 || Lb < 1 ||
        D < 1 || D > kEncChannels || downsample < 2 || (mode != 0 && mode != 1))
        return DTW_ERR_INVALID;
    if (!is_device_ptr(params) || !is_device_ptr(A) || !is_device_ptr(B) ||
        !is_device_ptr(path) || !is_device_ptr(path_len) || !is_device_ptr(grad) ||
        !is_device_ptr(loss))
        return DTW_ERR_INVALID;
    const int Lac = (La + downsample - 1) / downsample, Lbc = (Lb + downsample - 1) / downsample;
    if (!reachable(La, Lb) || !reachable(Lac, Lbc)) return DTW_ERR_UNREACHABLE;
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    cudaStream_t s = h->stream;
    h->band_nstrips = 0;  // the band buffer may move
    const EncBuf eb = enc_buf(Lac, Lbc, D);
    int rc = grow(h, &h->enc, &h->enc_cap, eb.total);
    if (rc != DTW_OK) return rc;
    const EncLayout pl = enc_layout(D);
    rc = enc_forward(h, params, pl, D, A, La, downsample, 0, eb.a);
    if (rc == DTW_OK) rc = enc_forward(h, params, pl, D, B, Lb, downsample, 0, eb.b);
    if (rc != DTW_OK) return rc;
    if (mode == 0) {
        int* tgt = reinterpret_cast<int*>(h->enc + eb.tgt);
        CU(launch_targets(path, path_len, std::min(La, Lb), downsample, Lac, Lbc,
                          reinterpret_cast<unsigned long long*>(h->enc + eb.jsum),
                          reinterpret_cast<int*>(h->enc + eb.cnt), tgt, s));
        CU(launch_loss_emb(ef(h, eb.a.E), Lac, ef(h, eb.b.E), Lbc, tgt, ef(h, eb.a.G),
                           ef(h, eb.b.G), loss, s));
        rc = enc_backward(h, params, pl, D, Lac, eb.a, grad);
        if (rc == DTW_OK) rc = enc_backward(h, params, pl, D, Lbc, eb.b, grad);
        return rc;
    }
    // mode 1: the coarse path on the current embeddings, the half-width each
    // coarse row of A needs, and the width head's gradient (trunk frozen)
    const BandBuf bb = band_buf(Lac, Lbc, kEncEmbed, 1, false);
    rc = grow(h, &h->band, &h->band_cap, bb.total);
    if (rc != DTW_OK) return rc;
    int32_t* cpath = reinterpret_cast<int32_t*>(h->band + bb.cp);
    int* clen = reinterpret_cast<int*>(h->band + bb.cl);
    rc = align_device(h, ef(h, eb.a.E), Lac, ef(h, eb.b.E), Lbc, kEncEmbed, defaults(), cpath,
                      clen, nullptr);
    if (rc != DTW_OK) return rc;
    CU(launch_width_target(cpath, clen, path, path_len, downsample, Lac, (float)DTW_BAND_WMIN,
                           (float)DTW_BAND_WMAX, ef(h, eb.wt), s));
    CU(launch_loss_width(ef(h, eb.a.S), ef(h, eb.wt), Lac, ef(h, eb.dS), loss, s));
    CU(launch_outer(ef(h, eb.dS), 1, ef(h, eb.a.H3), kEncChannels, Lac, grad + pl.W5, s));
    CU(launch_outer(ef(h, eb.dS), 1, nullptr, 1, Lac, grad + pl.b5, s));
    return DTW_OK;
}

int dtw_encoder_adam(dtw_handle* h, int n, float* params, float* grad, float* m, float* v,
                     int step, float lr) {
    if (!h || n < 1 || !params || !grad || !m || !v || step < 1 || !(lr > 0.f))
        return DTW_ERR_INVALID;
    if (!is_device_ptr(params) || !is_device_ptr(grad) || !is_device_ptr(m) || !is_device_ptr(v))
        return DTW_ERR_INVALID;
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    CU(launch_adam(n, params, grad, m, v, step, lr, 0.9f, 0.999f, 1e-8f, h->stream));
    return DTW_OK;
}

int dtw_align_learned(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D,
                      const dtw_options* opt, const float* params, int downsample, int bf16,
                      int32_t* path, int cap, int* path_len, float* total_cost, int* fell_back) {
    dtw_options o;
    int rc = band_checks(h, A, La, B, Lb, D, opt, downsample, path, cap, path_len, total_cost, &o);
    if (rc != DTW_OK) return rc;
    if (!params || !is_device_ptr(params) || D > kEncChannels) return DTW_ERR_INVALID;
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    if (fell_back) *fell_back = 0;
    h->band_nstrips = 0;
    const int Lac = (La + downsample - 1) / downsample, Lbc = (Lb + downsample - 1) / downsample;
    if (downsample == 1 || !reachable(Lac, Lbc)) {
        if (fell_back) *fell_back = 1;
        return align_device(h, A, La, B, Lb, D, o, path, path_len, total_cost);
    }
    const EncBuf eb = enc_buf(Lac, Lbc, D);
    rc = grow(h, &h->enc, &h->enc_cap, eb.total);
    if (rc != DTW_OK) return rc;
    // strips of the banded sweep at most (its shortest strips: 2 rows per lane)
    const int nstrips = (std::max(La, Lb) + strip_rows(2) - 1) / strip_rows(2);
    const BandBuf bb = band_buf(Lac, Lbc, kEncEmbed, nstrips, false);
    rc = grow(h, &h->band, &h->band_cap, bb.total);
    if (rc != DTW_OK) return rc;
    const EncLayout pl = enc_layout(D);
    rc = enc_forward(h, params, pl, D, A, La, downsample, bf16 != 0, eb.a);
    if (rc == DTW_OK) rc = enc_forward(h, params, pl, D, B, Lb, downsample, bf16 != 0, eb.b);
    if (rc != DTW_OK) return rc;
    return band_align(h, A, La, B, Lb, D, o, downsample, ef(h, eb.a.E), Lac, ef(h, eb.b.E), Lbc,
                      kEncEmbed, 0, ef(h, eb.a.HW), ef(h, eb.b.HW), bb, path, path_len,
                      total_cost, fell_back);
}

int dtw_wsdtw(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D, int nfrag,
              int32_t* path, int cap, int* path_len, int32_t* ends, float* total_cost) {
    if (!h || !A || !B || !path || !path_len || La < 1 || Lb < 1 || D < 1 || nfrag < 1 ||
        nfrag > La || cap < La)
        return DTW_ERR_INVALID;
    const int dp = padded_dim(D);
    if (dp == 0 || !split_supported(dp, 3)) return DTW_ERR_UNSUPPORTED;
    if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(path) ||
        !is_device_ptr(path_len) || (ends && !is_device_ptr(ends)) ||
        (total_cost && !is_device_ptr(total_cost)))
        return DTW_ERR_INVALID;
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    cudaStream_t s = h->stream;
    const int N = nfrag;
    // step 1: fragments k of rows floor(k La / N) .. floor((k+1) La / N) - 1
    std::vector<const float*> Ap(N), Bp(N, B);
    std::vector<int> Lap(N), Lbp(N, Lb), delta(N), idx(N);
    std::vector<int> row0(N);
    for (int k = 0; k < N; ++k) {
        const int r0 = (int)((long long)k * La / N), r1 = (int)((long long)(k + 1) * La / N);
        row0[k] = r0;
        Ap[k] = A + (size_t)r0 * D;
        Lap[k] = r1 - r0;
        delta[k] = (r1 - r0) / 2;
        idx[k] = k;
    }
    // buffers: last rows, D_seg, arg, ends, deltas, fragments, counts, the
    // scratch path, total, control block
    const size_t stride = (size_t)((Lb + kColsPerWord - 1) / kColsPerWord) * kColsPerWord;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align256(o + bytes); return at; };
    const size_t o_last = take(sizeof(float) * stride * N);
    const size_t o_dseg = take(sizeof(float) * (size_t)Lb * N);
    const size_t o_arg = take(sizeof(int) * (size_t)Lb * N);
    const size_t o_ends = take(sizeof(int) * N);
    const size_t o_delta = take(sizeof(int) * N);
    const size_t o_frag = take(sizeof(WsFrag) * N);
    const size_t o_cnt = take(sizeof(int) * N);
    const size_t o_scr = take(sizeof(int32_t) * 2 * (size_t)La);
    const size_t o_tot = take(sizeof(float));
    const size_t o_ctl = take(sizeof(DevCtl));
    const size_t o_agg = take(seg_dp_scratch_bytes(Lb));
    const size_t o_done = take(2 * sizeof(unsigned));
    int rc = grow(h, &h->wsd, &h->wsd_cap, o);
    if (rc != DTW_OK) return rc;
    char* w = h->wsd;
    // step 2 (and the last rows of step 3): the batched subsequence DP
    dtw_options opt = defaults();
    std::vector<BtArgs> bts(N);
    SubseqBatch sb{reinterpret_cast<float*>(w + o_last), stride, &bts};
    rc = align_batch(h, idx, Ap.data(), Lap.data(), Bp.data(), Lbp.data(), D, opt, 3, nullptr,
                     nullptr, nullptr, nullptr, &sb);
    if (rc != DTW_OK) return rc;
    std::vector<WsFrag> fr(N);
    for (int k = 0; k < N; ++k) {
        fr[k].bp = bts[k].bp;
        fr[k].pctl = bts[k].ctl;
        fr[k].row0 = row0[k];
        fr[k].len = Lap[k];
        fr[k].nchunk = bts[k].nchunk;
        fr[k].rps = bts[k].rps;
        fr[k].wpb = bts[k].wpb;
    }
    DevCtl* ctl = reinterpret_cast<DevCtl*>(w + o_ctl);
    int* dends = reinterpret_cast<int*>(w + o_ends);
    float* dtot = reinterpret_cast<float*>(w + o_tot);
    CU(cudaMemcpyAsync(w + o_delta, delta.data(), sizeof(int) * N, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(w + o_frag, fr.data(), sizeof(WsFrag) * N, cudaMemcpyHostToDevice, s));
    CU(cudaMemsetAsync(ctl, 0, sizeof(DevCtl), s));
    // steps 3-4: the segment-level DP and the end frames; step 5: backtraces
    const WsFrag* dfr = reinterpret_cast<const WsFrag*>(w + o_frag);
    CU(launch_seg_dp(dfr, reinterpret_cast<const float*>(w + o_last), stride, N, Lb,
                     reinterpret_cast<const int*>(w + o_delta), reinterpret_cast<float*>(w + o_dseg),
                     reinterpret_cast<int*>(w + o_arg), w + o_agg,
                     reinterpret_cast<unsigned*>(w + o_done), dends, dtot, ctl,
                     kDefaultTimeoutNs, s));
    CU(launch_bt_subseq(dfr, N, dends, reinterpret_cast<int32_t*>(w + o_scr),
                        reinterpret_cast<int*>(w + o_cnt), path, path_len, ctl, s));
    if (ends) CU(cudaMemcpyAsync(ends, dends, sizeof(int) * N, cudaMemcpyDeviceToDevice, s));
    if (total_cost)
        CU(cudaMemcpyAsync(total_cost, dtot, sizeof(float), cudaMemcpyDeviceToDevice, s));
    return DTW_OK;
}

int dtw_wsdtw_cseg(dtw_handle* h, int nfrag, int Lb, float* cseg) {
    if (!h || !cseg || nfrag < 1 || Lb < 1 || !h->wsd || !is_device_ptr(cseg))
        return DTW_ERR_INVALID;
    const size_t stride = (size_t)((Lb + kColsPerWord - 1) / kColsPerWord) * kColsPerWord;
    if (sizeof(float) * stride * nfrag > h->wsd_cap) return DTW_ERR_INVALID;
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    CU(cudaMemcpy2DAsync(cseg, sizeof(float) * Lb, h->wsd, sizeof(float) * stride,
                         sizeof(float) * Lb, nfrag, cudaMemcpyDeviceToDevice, h->stream));
    return DTW_OK;
}

int dtw_batch_destroy(dtw_batch* b) {
    if (!b) return DTW_ERR_INVALID;
    // the plan's own device and event: the handle may already be gone
    DeviceGuard g(b->device);
    if (b->done) {
        cudaEventSynchronize(b->done);
        cudaEventDestroy(b->done);
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ws) cudaFree(b->ws);
    if (b->border) cudaFree(b->border);
    (void)cudaGetLastError();
    delete b;
    return DTW_OK;
}

int dtw_batch_create(dtw_handle* h, int n, const float* const* A, const int* La,
                     const float* const* B, const int* Lb, int D, int32_t* paths,
                     const int64_t* path_off, int* path_len, float* cost, int flags,
                     dtw_batch** out) {
    if (!out) return DTW_ERR_INVALID;
    *out = nullptr;
    if (!h || n < 1 || !A || !La || !B || !Lb || !paths || !path_off || !path_len)
        return DTW_ERR_INVALID;
    const int dp = padded_dim(D);
    if (dp == 0 || !split_supported(dp, 3)) return DTW_ERR_UNSUPPORTED;
    for (int k = 0; k < n; ++k) {
        const int rc = validate(A[k], La[k], B[k], Lb[k], D);
        if (rc != DTW_OK) return rc;
    }
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    if (!is_device_ptr(paths) || !is_device_ptr(path_len) || (cost && !is_device_ptr(cost)))
        return DTW_ERR_INVALID;
    for (int k = 0; k < n; ++k)
        if (!is_device_ptr(A[k]) || !is_device_ptr(B[k])) return DTW_ERR_INVALID;
    cudaStream_t s = h->stream;
    const dtw_options o = defaults();
    std::vector<int> idx(n);
    for (int k = 0; k < n; ++k) idx[k] = k;
    // candidate schedules: rows per lane and strips per CTA of the warp-pair DP
    std::vector<std::pair<int, int>> cands;
    if (flags & DTW_BATCH_AUTOTUNE) {
        for (int NS : {4, 2})
            for (int R = 2; R <= 4; ++R)
                if (split_supported(dp, R, NS)) cands.push_back({R, NS});
    } else {
        cands.push_back({3, split_supported(dp, 3, 4) ? 4 : 2});
    }
    std::vector<BatchSetup> setups;
    size_t ws_bytes = 0, border_bytes = 0;
    for (auto [R, NS] : cands) {
        setups.push_back(batch_setup(idx, La, Lb, D, R, NS));
        ws_bytes = std::max(ws_bytes, setups.back().ws_bytes);
        border_bytes = std::max(border_bytes, setups.back().border_bytes);
    }
    dtw_batch* b = new (std::nothrow) dtw_batch();
    if (!b) return DTW_ERR_OOM;
    b->h = h;
    b->device = h->device;
    b->n = n;
    b->D = D;
    if (cudaMalloc(&b->ws, ws_bytes) != cudaSuccess ||
        cudaMalloc(&b->border, border_bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        dtw_batch_destroy(b);
        return DTW_ERR_OOM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t cs = nullptr;
    int rc = DTW_OK;
    unsigned epoch = 0;
    auto fail = [&](int code) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (cs) cudaStreamDestroy(cs);
        (void)cudaGetLastError();
        dtw_batch_destroy(b);
        return code;
    };
    if (cudaMemsetAsync(b->border, 0, border_bytes, s) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess)
        return fail(DTW_ERR_CUDA);
    // the autotuner: every candidate twice, the second run timed (all
    // candidates compute the same result, bit for bit)
    int best = 0;
    float best_ms = 0.f;
    for (size_t c = 0; c < setups.size(); ++c) {
        float ms = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
            const BatchDesc d = batch_descriptors(setups[c], b->ws, b->border, A, La, B, Lb, o,
                                                  ++epoch, paths, path_off, path_len, cost,
                                                  nullptr);
            rc = batch_upload(setups[c], d, b->ws, s);
            if (rc != DTW_OK) return fail(rc);
            if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) return fail(DTW_ERR_CUDA);
            rc = batch_launch(setups[c], b->ws, false, h->num_sms, s, nullptr);
            if (rc != DTW_OK) return fail(rc);
            if (rep == 1 && (cudaEventRecord(e1, s) != cudaSuccess ||
                             cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                return fail(DTW_ERR_CUDA);
        }
        b->tuned_ms[(setups[c].NS == 4 ? 3 : 0) + setups[c].R - 2] = ms;
        if (c == 0 || ms < best_ms) {
            best = (int)c;
            best_ms = ms;
        }
    }
    b->setup = setups[best];
    b->R = b->setup.R;
    b->NS = b->setup.NS;
    // the chosen schedule's descriptors stay in the plan's workspace; the
    // graph bumps their epoch, then normalises, sweeps and backtraces
    const BatchDesc d = batch_descriptors(b->setup, b->ws, b->border, A, La, B, Lb, o, ++epoch,
                                          paths, path_off, path_len, cost, nullptr);
    rc = batch_upload(b->setup, d, b->ws, s);
    if (rc != DTW_OK) return fail(rc);
    if (cudaStreamSynchronize(s) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(DTW_ERR_CUDA);
    const bool ok_bump = launch_bump_epoch(reinterpret_cast<DpArgs*>(b->ws + b->setup.off_dp),
                                           n, cs) == cudaSuccess;
    const int rl = batch_launch(b->setup, b->ws, false, h->num_sms, cs, nullptr);
    cudaGraph_t graph = nullptr;
    const bool ok_end = cudaStreamEndCapture(cs, &graph) == cudaSuccess;
    b->graph = graph;
    if (!ok_bump || rl != DTW_OK || !ok_end ||
        cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess)
        return fail(DTW_ERR_CUDA);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(cs);
    *out = b;
    return DTW_OK;
}

int dtw_batch_run(dtw_batch* b) {
    if (!b || !b->exec) return DTW_ERR_INVALID;
    DeviceGuard g(b->h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    CU(cudaGraphLaunch(b->exec, b->h->stream));
    CU(cudaEventRecord(b->done, b->h->stream));
    return DTW_OK;
}

int dtw_batch_info(const dtw_batch* b, int* rows_per_lane, int* strips_per_cta,
                   float* tuned_ms) {
    if (!b) return DTW_ERR_INVALID;
    if (rows_per_lane) *rows_per_lane = b->R;
    if (strips_per_cta) *strips_per_cta = b->NS;
    if (tuned_ms)
        for (int k = 0; k < 6; ++k) tuned_ms[k] = b->tuned_ms[k];
    return DTW_OK;
}

int dtw_band_cells(dtw_handle* h, long long* cells) {
    if (!h || !cells) return DTW_ERR_INVALID;
    *cells = 0;
    if (h->band_nstrips <= 0) return DTW_OK;
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    std::vector<int2> r(h->band_nstrips);
    CU(cudaStreamSynchronize(h->stream));
    CU(cudaMemcpy(r.data(), h->band_ranges, sizeof(int2) * r.size(), cudaMemcpyDeviceToHost));
    long long c = 0;
    for (int q = 0; q < h->band_nstrips; ++q) {
        const int x = r[q].x * 8, y = std::min(r[q].y * 8, h->band_Lb);
        c += (long long)std::max(y - x, 0) * h->band_rps;
    }
    *cells = c;
    return DTW_OK;
}

int dtw_enable_timing(dtw_handle* h, int on) {
    if (!h) return DTW_ERR_INVALID;
    h->timing = on != 0;
    h->timed = false;
    return DTW_OK;
}

int dtw_stage_times(dtw_handle* h, float* ms, int n) {
    if (!h || !ms || n < 1 || !h->timed) return DTW_ERR_INVALID;
    DeviceGuard g(h->device);
    CU(cudaEventSynchronize(h->ev[3]));
    float t[3];
    for (int k = 0; k < 3; ++k) CU(cudaEventElapsedTime(&t[k], h->ev[k], h->ev[k + 1]));
    for (int k = 0; k < n && k < 3; ++k) ms[k] = t[k];
    return DTW_OK;
}

}  // extern "C"
