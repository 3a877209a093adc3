// Launch of the warp-pair DP of one pair in thread-block clusters
// (k_dp_split<..., kCl = true>, see dp_split.cuh), shared by the translation
// units that instantiate it (dp_split_cl.cu for D <= 32 and the BF16 cost,
// dp_split_wide.cu for the FP32 cost at D = 64, 128).
//
// Between two CTAs the strip border otherwise goes through global memory:
// the writer warp of the CTA above stores it, the reader warp of the CTA
// below polls it, and each hop costs about 3 us (measured on the 20000 x
// 25000 pair: 0.48 us from strip to strip inside a CTA, 3.0 us from CTA to
// CTA, 22% of the DP time).  In a cluster the writer warp of a CTA copies the
// border into a staging ring of the next CTA's shared memory and that CTA's
// reader warp forwards it (1.2 us a hop), so only one hop in cn stays global.
//
// Every CTA of a cluster sits on an SM of its own (the dynamic shared
// memory is raised so that two CTAs cannot share an SM, which would put two
// DP warps on one SM sub-partition).  The cluster size is the largest of 8
// down to 2 whose resident clusters hold every strip group of the pair at
// once (the 20000 x 25000 pair's 135 groups: 17 clusters of 8 do not fit at
// once, 23 of 6 do, and its DP takes 1.360 ms against 1.393 with clusters of
// 4, a third fewer hops through global memory); a band with more groups runs
// persistent clusters of 8, a full sweep with more groups no clusters.
#pragma once
#include <mutex>

#include "dp_split.cuh"

namespace pardtw {
namespace {

constexpr int kClSmemFloor = 120 * 1024;  // > half an SM's shared memory: one CTA per SM
constexpr int kClMaxDev = 64;
constexpr int kNClSizes = 7;
constexpr int kClSizes[kNClSizes] = {8, 7, 6, 5, 4, 3, 2};

template <int DP, bool kBF, bool kT>
struct ClKernel {
    static constexpr int R = 3, NS = 2;
    static constexpr int kThreads = split_threads<DP, NS, kBF>();
    static constexpr auto kern() { return k_dp_split<DP, R, NS, false, kBF, false, kT, false, true>; }
    static int smem() {
        return std::max(NS * SplitSmem<DP, R, kBF>::kStripBytes, kClSmemFloor);
    }
};

struct ClInfo {
    bool ready = false, ok = false;
    int max_clusters[kNClSizes] = {};  // resident clusters of size kClSizes[k]
};

cudaLaunchConfig_t cl_config(dim3 grid, int threads, int smem, cudaStream_t s,
                             cudaLaunchAttribute* at, int cn) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cn;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

// Attributes and cluster occupancy of one instantiation, once per device.
template <int DP, bool kBF, bool kT>
const ClInfo& cl_info(int dev) {
    static ClInfo info[kClMaxDev];
    static std::mutex mu;
    using K = ClKernel<DP, kBF, kT>;
    std::lock_guard<std::mutex> lock(mu);
    ClInfo& ci = info[dev];
    if (ci.ready) return ci;
    ci.ready = true;
    auto* kern = K::kern();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, K::smem()) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return ci;
    }
    for (int k = 0; k < kNClSizes; ++k) {
        cudaLaunchAttribute at[1];
        cudaLaunchConfig_t cfg =
            cl_config(dim3((unsigned)kClSizes[k]), K::kThreads, K::smem(), nullptr, at, kClSizes[k]);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            n = 0;
        }
        ci.max_clusters[k] = n;
    }
    ci.ok = true;
    return ci;
}

template <int DP, bool kBF, bool kT>
cudaError_t launch_cl(const DpArgs& a, cudaStream_t s, bool* used) {
    *used = false;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kClMaxDev) {
        (void)cudaGetLastError();
        return cudaSuccess;
    }
    const ClInfo& ci = cl_info<DP, kBF, kT>(dev);
    if (!ci.ok) return cudaSuccess;
    int cn = 0, nclusters = 0;
    // one wave: the largest cluster size whose resident clusters hold every group
    for (int k = 0; k < kNClSizes && cn == 0; ++k) {
        const int need = (a.ngroups + kClSizes[k] - 1) / kClSizes[k];
        if (ci.max_clusters[k] >= need) {
            cn = kClSizes[k];
            nclusters = need;
        }
    }
    // several waves: persistent clusters of 8 for a band (its strips are
    // short and start one after another along the band); a full sweep of
    // several waves runs faster without clusters (D = 128, 40000 x 48000:
    // 5.7 against 8.4 ms with the BF16 cost, 19.3 against 28.6 ms with FP32)
    if (cn == 0 && a.ranges && ci.max_clusters[0] > 0) {
        cn = kClSizes[0];
        nclusters = ci.max_clusters[0];
    }
    if (cn == 0) return cudaSuccess;
    using K = ClKernel<DP, kBF, kT>;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg =
        cl_config(dim3((unsigned)(nclusters * cn)), K::kThreads, K::smem(), s, at, cn);
    const cudaError_t e = cudaLaunchKernelEx(&cfg, K::kern(), a, MapArgs{},
                                             static_cast<const DpArgs*>(nullptr),
                                             static_cast<const int*>(nullptr), 1,
                                             static_cast<int*>(nullptr));
    if (e == cudaSuccess) *used = true;
    return e;
}

}  // namespace
}  // namespace pardtw
