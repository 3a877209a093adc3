// dtw_align_static: exact alignment without any device allocation.
//
// Some callers cannot allocate device memory when they align: a real-time
// loop (live score following, streaming alignment) that must not block in
// the driver's allocator, or a host process whose device memory is already
// fully reserved by another allocator (a framework's caching allocator, a
// plugin host with a fixed memory budget).  This entry point serves them: it
// runs the DP kernel and the parallel backtrace that dtw_align runs for the
// pair swept as given (A's frames as rows: it never takes the transposed
// sweep, whose cells, path and total are bit-identical), but every byte of
// scratch it needs (normalised features, the 2-bit backpointer matrix, the
// border rows between strip groups, control words, the backtrace's band
// maps) lives in one file-scope device array of fixed size, so a call
// allocates nothing.  Only the FP32 cost is offered.
//
// The array exists on every device that loads the library, for the life of
// the process.  In host code its name is only a stand-in for the symbol, not
// a device address, so the address is looked up once per device
// (cudaGetSymbolAddress, with that device current) and passed to the kernels.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "pardtw_common.cuh"

namespace pardtw {
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB
constexpr int kMaxDevices = 64;

// The scratch shared by every dtw_align_static call on a device.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

unsigned char* g_scratch_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

size_t align256s(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the array on `device` (current), looked up on first use.
int scratch_for(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return DTW_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return DTW_ERR_CUDA;
        }
        g_scratch_addr[device] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[device];
    return DTW_OK;
}

bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace pardtw

using namespace pardtw;

extern "C" size_t dtw_static_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" int dtw_align_static(const float* A, int La, const float* B, int Lb, int D,
                                const dtw_options* opt, void* cuda_stream, int32_t* path, int cap,
                                int* path_len, float* total_cost) {
    if (!A || !B || !path || !path_len || La < 1 || Lb < 1 || D < 1) return DTW_ERR_INVALID;
    {
        const long long i = La - 1, j = Lb - 1;
        if (j > 2 * i || i > 2 * j) return DTW_ERR_UNREACHABLE;
    }
    if (cap < std::min(La, Lb)) return DTW_ERR_INVALID;
    const int dp = padded_dim(D);
    if (dp == 0) return DTW_ERR_UNSUPPORTED;
    dtw_options o;
    dtw_default_options(&o);
    if (opt) o = *opt;
    if (o.cost_precision != DTW_COST_FP32) return DTW_ERR_UNSUPPORTED;
    // every argument must already be in device memory: staging a host buffer
    // would need scratch this call does not have
    if (!on_device(A) || !on_device(B) || !on_device(path) || !on_device(path_len) ||
        (total_cost && !on_device(total_cost)))
        return DTW_ERR_INVALID;

    int device = 0, num_sms = 0;
    if (cudaGetDevice(&device) != cudaSuccess ||
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        (void)cudaGetLastError();
        return DTW_ERR_CUDA;
    }

    // the DP kernel dtw_align would choose
    const DpPlan plan = choose_plan(La, dp, o, num_sms);
    const int R = plan.R;
    const int rps = strip_rows(R), wpb = strip_words(R);
    const int nstrips = (La + rps - 1) / rps;
    const int nchunk = (Lb + kColsPerWord - 1) / kColsPerWord;
    const int ngroups = (nstrips + plan.spg - 1) / plan.spg;
    const int La_pad = nstrips * rps;

    // scratch layout of this call
    size_t off = 0;
    const size_t off_ctl = off;
    off += 256;
    const size_t off_ahat = off;
    off = align256s(off + (size_t)La_pad * dp * sizeof(float));
    const size_t off_bt = off;
    off = align256s(off + (size_t)nchunk * kColsPerWord * dp * sizeof(float));
    const size_t off_bp = off;
    off = align256s(off + (size_t)nstrips * nchunk * wpb * sizeof(uint32_t));
    const size_t off_border = off;
    const size_t border_bytes = (size_t)ngroups * Lb * 2 * sizeof(unsigned long long);
    off = align256s(off + border_bytes);
    const size_t off_map = off;
    off = align256s(off + bandmap_scratch_bytes(La, Lb));
    if (off > kStaticScratchBytes) return DTW_ERR_SCRATCH_LIMIT;

    unsigned char* base = nullptr;
    int rc = scratch_for(device, &base);
    if (rc != DTW_OK) return rc;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    DevCtl* ctl = reinterpret_cast<DevCtl*>(base + off_ctl);
    float* e_final = reinterpret_cast<float*>(base + off_ctl + 16);
    float* Ahat = reinterpret_cast<float*>(base + off_ahat);
    float* Bt = reinterpret_cast<float*>(base + off_bt);
    uint32_t* bp = reinterpret_cast<uint32_t*>(base + off_bp);
    unsigned long long* border = reinterpret_cast<unsigned long long*>(base + off_border);

    // The array keeps the last call's contents.  Border entries must start
    // unmatched: clear them, and tag this call's entries with 1.
    if (cudaMemsetAsync(border, 0, border_bytes, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return DTW_ERR_CUDA;
    }
    if (launch_normalise(A, La, La_pad, B, Lb, nchunk * kColsPerWord, D, dp, Ahat, Bt, ctl, s) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return DTW_ERR_CUDA;
    }
    DpArgs a;
    a.Ahat = Ahat;
    a.Bhat = Bt;
    a.Bbf = nullptr;
    a.ranges = nullptr;
    a.lastrow = nullptr;
    a.bp = bp;
    a.gborder = border;
    a.ctl = ctl;
    a.e_final = e_final;
    a.La = La;
    a.Lb = Lb;
    a.nstrips = nstrips;
    a.nchunk = nchunk;
    a.ngroups = ngroups;
    a.rps = rps;
    a.wpb = wpb;
    a.mu = o.cost_shift;
    a.kcost = 1.0f - o.cost_shift;
    a.epoch = 1u;
    a.timeout_ns = o.wait_limit > 0 ? (long long)o.wait_limit * 1000LL : kDefaultTimeoutNs;
    a.skip_publish = o.debug_skip_publish;
    BtArgs bt;
    bt.bp = bp;
    bt.La = La;
    bt.Lb = Lb;
    bt.nchunk = nchunk;
    bt.rps = rps;
    bt.wpb = wpb;
    bt.ctl = ctl;
    bt.e_final = e_final;
    bt.mu = o.cost_shift;
    bt.path = path;
    bt.path_len = path_len;
    bt.total = total_cost;
    bt.scratch = base + off_map;
    bt.ranges = nullptr;
    bt.transposed = 0;
    const cudaError_t e = launch_plan(plan, a, dp, num_sms, s);
    if (e != cudaSuccess || launch_backtrace_bands(bt, s, true) != cudaSuccess) {
        (void)cudaGetLastError();
        return DTW_ERR_CUDA;
    }
    return DTW_OK;
}
