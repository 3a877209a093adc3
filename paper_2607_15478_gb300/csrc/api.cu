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
    unsigned epoch = 0;
    bool timing = false;
    bool timed = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int* h_small = nullptr;      // pinned host: [0] path_len, [1] total bits
    char* band = nullptr;        // dtw_align_banded: pooled inputs, coarse path, ranges
    size_t band_cap = 0;
};

namespace {

constexpr long long kDefaultTimeoutNs = 2000000000LL;  // 2 s

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
        off_stage_path, total;
    size_t border_bytes;
};

}  // namespace

// The DP kernel for a problem.  Explicit requests are honoured where the
// kernel supports them (else one row per lane); the default is the cost/DP
// warp pair with 3 rows per lane for D <= 32, one row per lane above.
DpPlan pardtw::choose_plan(int La, int dp, const dtw_options& o, int num_sms) {
    (void)La;
    (void)num_sms;
    const DpPlan one = {0, 1, kWarpsPerGroup};
    if (o.cost_precision == DTW_COST_BF16) return {2, 3, kSplitStrips, 1};
    const int req = o.rows_per_lane;
    if (req == 1) return one;
    if (o.dp_schedule == DTW_SCHEDULE_FUSED) {
        const int R = req == 0 ? 2 : req;
        if (multirow_supported(dp, R)) return {1, R, kWarpsPerGroup};
        return one;
    }
    const int R = req == 0 ? 3 : req;
    if (split_supported(dp, R)) return {2, R, kSplitStrips};
    return one;
}

cudaError_t pardtw::launch_plan(const DpPlan& plan, const DpArgs& a, int dp, int num_sms,
                        cudaStream_t s) {
    switch (plan.kind) {
        case 0: return launch_dp(a, dp, num_sms, s);
        case 1: return launch_dp_multirow(a, dp, plan.R, num_sms, s);
        case 2:
            return plan.bf16 ? launch_dp_split_bf16(a, dp, num_sms, s)
                             : launch_dp_split(a, dp, plan.R, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
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
    L.off_stage_path = o;
    o = align256(o + (size_t)2 * L.cap * sizeof(int32_t));
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

dtw_options defaults() {
    dtw_options o;
    o.cost_precision = DTW_COST_FP32;
    o.cost_shift = 0.0f;
    o.wait_limit = 0;
    o.debug_skip_publish = -1;
    o.rows_per_lane = 0;
    o.dp_schedule = DTW_SCHEDULE_AUTO;
    return o;
}

// One pair, all the way to device-resident outputs.  `out_path`,
// `out_len`, `out_total` are device pointers (out_total may be null).
int align_device(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D,
                 const dtw_options& o, int32_t* out_path, int* out_len, float* out_total,
                 const int2* ranges = nullptr) {
    // a band (per-strip column ranges) needs the warp-pair kernel at 3 rows
    // per lane, FP32 cost
    const DpPlan plan = ranges ? DpPlan{2, 3, kSplitStrips}
                               : choose_plan(La, padded_dim(D), o, h->num_sms);
    const Layout L = make_layout(La, Lb, D, plan);
    int rc = ensure_workspace(h, L.total, L.border_bytes);
    if (rc != DTW_OK) return rc;
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
    CU(launch_plan(L.plan, a, L.dp, h->num_sms, s));
    if (h->timing) CU(cudaEventRecord(h->ev[2], s));
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
    CU(launch_backtrace_bands(bt, s));
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
int align_batch(dtw_handle* h, std::vector<int> idx, const float* const* A, const int* La,
                const float* const* B, const int* Lb, int D, const dtw_options& o, int R,
                int32_t* paths, const int64_t* path_off, int* path_len, float* cost) {
    const int m = (int)idx.size();
    if (m == 0) return DTW_OK;
    // The work queue runs the pairs with the longest sweeps first, so that the
    // last pairs to start are short and no long chain of strips is left alone
    // at the end (the order does not change any result).
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
        return (long long)Lb[x] * 256 + La[x] > (long long)Lb[y] * 256 + La[y];
    });
    const int dp = padded_dim(D);
    const DpPlan plan = {2, R, kSplitStrips};
    std::vector<Layout> Ls(m);
    std::vector<size_t> off(m), boff(m);
    // descriptors, then one control block per pair, then every pair's buffers
    size_t o0 = 0;
    const size_t off_dp = o0;
    o0 = align256(o0 + sizeof(DpArgs) * m);
    const size_t off_norm = o0;
    o0 = align256(o0 + sizeof(NormArgs) * m);
    const size_t off_bt = o0;
    o0 = align256(o0 + sizeof(BtArgs) * m);
    const size_t off_item = o0;
    o0 = align256(o0 + sizeof(int) * (m + 1) + 16);  // + the work-queue ticket
    const size_t off_ctl = o0;
    o0 = align256(o0 + (size_t)256 * m);
    size_t border_total = 0;
    int maxLa = 0, maxLb = 0, max_frames = 0;
    std::vector<int> item0(m + 1, 0);
    for (int q = 0; q < m; ++q) {
        const int k = idx[q];
        Ls[q] = make_layout(La[k], Lb[k], D, plan);
        const Layout& L = Ls[q];
        off[q] = o0;
        o0 = align256(o0 + (L.off_stage_a - L.off_ahat));  // Ahat, Bhat, bp, band maps
        boff[q] = border_total;
        border_total += L.border_bytes;
        item0[q + 1] = item0[q] + L.ngroups;
        maxLa = std::max(maxLa, La[k]);
        maxLb = std::max(maxLb, Lb[k]);
        max_frames = std::max(max_frames, L.La_pad + L.nchunk * kColsPerWord);
    }
    int rc = ensure_workspace(h, o0, border_total);
    if (rc != DTW_OK) return rc;
    char* ws = h->ws;
    cudaStream_t s = h->stream;
    unsigned epoch = ++h->epoch;
    if (epoch == 0) epoch = ++h->epoch;
    std::vector<DpArgs> dps(m);
    std::vector<NormArgs> nas(m);
    std::vector<BtArgs> bts(m);
    for (int q = 0; q < m; ++q) {
        const int k = idx[q];
        const Layout& L = Ls[q];
        char* base = ws + off[q] - L.off_ahat;  // so that base + L.off_* addresses this pair
        DevCtl* ctl = reinterpret_cast<DevCtl*>(ws + off_ctl + (size_t)256 * q);
        float* e_final = reinterpret_cast<float*>(ws + off_ctl + (size_t)256 * q + 16);
        float* Ahat = reinterpret_cast<float*>(base + L.off_ahat);
        float* Bhat = reinterpret_cast<float*>(base + L.off_bhat);
        uint32_t* bpw = reinterpret_cast<uint32_t*>(base + L.off_bp);
        NormArgs& na = nas[q];
        na.A = A[k];
        na.La = La[k];
        na.La_pad = L.La_pad;
        na.B = B[k];
        na.Lb = Lb[k];
        na.Lb_pad = L.nchunk * kColsPerWord;
        na.Ahat = Ahat;
        na.Bt = Bhat;
        na.ctl = ctl;
        DpArgs& a = dps[q];
        a.Ahat = Ahat;
        a.Bhat = Bhat;
        a.Bbf = nullptr;
        a.ranges = nullptr;
        a.bp = bpw;
        a.gborder = h->border + boff[q] / sizeof(unsigned long long);
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
        BtArgs& bt = bts[q];
        bt.bp = bpw;
        bt.La = La[k];
        bt.Lb = Lb[k];
        bt.nchunk = L.nchunk;
        bt.rps = L.rps;
        bt.wpb = L.wpb;
        bt.ctl = ctl;
        bt.e_final = e_final;
        bt.mu = o.cost_shift;
        bt.path = paths + 2 * path_off[k];
        bt.path_len = path_len + k;
        bt.total = cost ? cost + k : nullptr;
        bt.scratch = base + L.off_bt;
        bt.ranges = nullptr;
    }
    CU(cudaMemcpyAsync(ws + off_dp, dps.data(), sizeof(DpArgs) * m, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(ws + off_norm, nas.data(), sizeof(NormArgs) * m, cudaMemcpyHostToDevice,
                       s));
    CU(cudaMemcpyAsync(ws + off_bt, bts.data(), sizeof(BtArgs) * m, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(ws + off_item, item0.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice,
                       s));
    int* ticket = reinterpret_cast<int*>(ws + off_item + sizeof(int) * (m + 1));
    if (h->timing) CU(cudaEventRecord(h->ev[0], s));
    CU(launch_normalise_many(reinterpret_cast<const NormArgs*>(ws + off_norm), m, max_frames, D,
                             dp, ticket, s));
    if (h->timing) CU(cudaEventRecord(h->ev[1], s));
    CU(launch_dp_split_many(reinterpret_cast<const DpArgs*>(ws + off_dp),
                            reinterpret_cast<const int*>(ws + off_item), m, item0[m], ticket, dp,
                            R, h->num_sms, s));
    if (h->timing) CU(cudaEventRecord(h->ev[2], s));
    CU(launch_backtrace_bands_many(reinterpret_cast<const BtArgs*>(ws + off_bt), m, maxLa, maxLb,
                                   s));
    if (h->timing) {
        CU(cudaEventRecord(h->ev[3], s));
        h->timed = true;
    }
    return DTW_OK;
}

}  // namespace

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
    if (h->band) cudaFree(h->band);
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
    (void)opt;
    if (!bytes || La < 1 || Lb < 1 || D < 1) return DTW_ERR_INVALID;
    if (padded_dim(D) == 0) return DTW_ERR_UNSUPPORTED;
    size_t most = 0;
    const DpPlan plans[] = {{0, 1, kWarpsPerGroup}, {1, 2, kWarpsPerGroup},
                            {1, 4, kWarpsPerGroup}, {2, 2, kSplitStrips},
                            {2, 3, kSplitStrips},   {2, 4, kSplitStrips},
                            {2, 3, kSplitStrips, 1}};
    for (const DpPlan& plan : plans) {
        const Layout L = make_layout(La, Lb, D, plan);
        most = std::max(most, L.total + L.border_bytes);
    }
    *bytes = most;
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

    const Layout L = make_layout(La, Lb, D, choose_plan(La, padded_dim(D), o, h->num_sms));
    rc = ensure_workspace(h, L.total, L.border_bytes);
    if (rc != DTW_OK) return rc;
    const bool path_dev = is_device_ptr(path);
    const bool len_dev = is_device_ptr(path_len);
    const bool tot_dev = total_cost ? is_device_ptr(total_cost) : true;
    char* ws = h->ws;
    int32_t* dpath = path_dev ? path : reinterpret_cast<int32_t*>(ws + L.off_stage_path);
    int* dlen = len_dev ? path_len : reinterpret_cast<int*>(ws + L.off_ctl + 24);
    float* dtot = total_cost ? (tot_dev ? total_cost : reinterpret_cast<float*>(ws + L.off_ctl + 20))
                             : nullptr;
    rc = align_device(h, A, La, B, Lb, D, o, dpath, dlen, dtot);
    if (rc != DTW_OK) return rc;
    cudaStream_t s = h->stream;
    const bool host_out = !path_dev || !len_dev || !tot_dev;
    if (!host_out) return DTW_OK;

    // host outputs: bring back length and total, then the path
    CU(cudaMemcpyAsync(h->h_small, ws + L.off_ctl + 20, 8, cudaMemcpyDeviceToHost, s));
    if (len_dev) CU(cudaMemcpyAsync(h->h_small + 1, path_len, 4, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const int n = h->h_small[1];
    if (!len_dev) *path_len = n;
    if (total_cost && !tot_dev) memcpy(total_cost, &h->h_small[0], sizeof(float));
    if (n < 0) return -n;
    if (!path_dev) {
        CU(cudaMemcpyAsync(path, dpath, (size_t)2 * n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
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
        const int rc = align_batch(h, valid, A, La, B, Lb, D, o, Rb, paths, path_off, path_len,
                                   cost);
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
    if (len_dev)
        CU(cudaMemcpy(lens.data(), path_len, sizeof(int) * n, cudaMemcpyDeviceToHost));
    else
        memcpy(lens.data(), path_len, sizeof(int) * n);
    for (int k = 0; k < n; ++k)
        if (hst[k] == DTW_OK && lens[k] < 0) hst[k] = -lens[k];
    if (st_dev)
        CU(cudaMemcpy(status, hst.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    else
        memcpy(status, hst.data(), sizeof(int) * n);
    return DTW_OK;
}

int dtw_align_banded(dtw_handle* h, const float* A, int La, const float* B, int Lb, int D,
                     const dtw_options* opt, int downsample, int halfwidth, int32_t* path,
                     int cap, int* path_len, float* total_cost, int* fell_back) {
    if (!h || !path || !path_len || downsample < 1 || halfwidth < 0) return DTW_ERR_INVALID;
    int rc = validate(A, La, B, Lb, D);
    if (rc != DTW_OK) return rc;
    if (cap < std::min(La, Lb)) return DTW_ERR_INVALID;
    const dtw_options o = opt ? *opt : defaults();
    if (o.cost_precision != DTW_COST_FP32 || !split_supported(padded_dim(D), 3))
        return DTW_ERR_UNSUPPORTED;
    DeviceGuard g(h->device);
    if (!g.ok) return DTW_ERR_CUDA;
    if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(path) ||
        !is_device_ptr(path_len) || (total_cost && !is_device_ptr(total_cost)))
        return DTW_ERR_INVALID;
    cudaStream_t s = h->stream;
    if (fell_back) *fell_back = 0;
    const int Lac = (La + downsample - 1) / downsample, Lbc = (Lb + downsample - 1) / downsample;
    if (downsample == 1 || !reachable(Lac, Lbc)) {
        if (fell_back) *fell_back = 1;
        return align_device(h, A, La, B, Lb, D, o, path, path_len, total_cost);
    }
    const int rps = strip_rows(3);
    const int nstrips = (La + rps - 1) / rps;
    const int capc = std::min(Lac, Lbc);
    // band buffer: pooled A and B, coarse path and length, ranges, touch flag
    const size_t off_pa = 0;
    const size_t off_pb = align256(off_pa + (size_t)Lac * D * sizeof(float));
    const size_t off_cp = align256(off_pb + (size_t)Lbc * D * sizeof(float));
    const size_t off_cl = align256(off_cp + (size_t)2 * capc * sizeof(int32_t));
    const size_t off_rg = align256(off_cl + 16);
    const size_t off_tc = align256(off_rg + (size_t)nstrips * sizeof(int2));
    const size_t need = off_tc + 256;
    if (need > h->band_cap) {
        CU(cudaStreamSynchronize(s));
        if (h->band) cudaFree(h->band);
        h->band = nullptr;
        h->band_cap = 0;
        if (cudaMalloc(&h->band, need) != cudaSuccess) {
            (void)cudaGetLastError();
            h->band = nullptr;
            return DTW_ERR_OOM;
        }
        h->band_cap = need;
    }
    float* pa = reinterpret_cast<float*>(h->band + off_pa);
    float* pb = reinterpret_cast<float*>(h->band + off_pb);
    int32_t* cpath = reinterpret_cast<int32_t*>(h->band + off_cp);
    int* clen = reinterpret_cast<int*>(h->band + off_cl);
    int2* ranges = reinterpret_cast<int2*>(h->band + off_rg);
    int* touch = reinterpret_cast<int*>(h->band + off_tc);
    // 1. the coarse pair and its exact alignment
    CU(launch_pool(A, La, D, downsample, pa, s));
    CU(launch_pool(B, Lb, D, downsample, pb, s));
    rc = align_device(h, pa, Lac, pb, Lbc, D, o, cpath, clen, nullptr);
    if (rc != DTW_OK) return rc;
    // 2. the band and the exact DP inside it
    CU(launch_band_ranges(cpath, clen, downsample, halfwidth, La, Lb, nstrips, rps, ranges, s));
    rc = align_device(h, A, La, B, Lb, D, o, path, path_len, total_cost, ranges);
    if (rc != DTW_OK) return rc;
    // 3. a path at the band's side: the full exact DP instead
    CU(launch_band_touch(path, path_len, std::min(La, Lb), Lb, rps, ranges, touch, s));
    CU(cudaMemcpyAsync(h->h_small + 2, touch, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (h->h_small[2]) {
        if (fell_back) *fell_back = 1;
        return align_device(h, A, La, B, Lb, D, o, path, path_len, total_cost);
    }
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
