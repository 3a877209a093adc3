// Warp-pair DP with the FP32 cost at D = 64 and 128 (k_dp_split with the
// wide cost warps of dp_split.cuh, run_cost_wide): per strip two cost warps
// (4 of the 8 columns of a sub-chunk each, the strip's rows of A^ in shared
// memory, B^ through L1) and the DP warp of the narrow kernels, so the FP32
// cost keeps one FMA per feature in feature order (the values of every other
// decomposition) while its 2 D FLOP per cell are spread over all four SM
// sub-partitions.  Eight warps a CTA: the four cost warps on four
// sub-partitions, the DP warps and the reader and writer beside them.
#include "dp_split_cl.cuh"

namespace pardtw {

bool split_wide_supported(int dp) { return dp == 64 || dp == 128; }

cudaError_t launch_dp_split_wide(const DpArgs& a, int dp, int num_sms, cudaStream_t s,
                                 bool transposed) {
    if (dp == 64)
        return transposed ? launch_t<64, 3, 2, false, false, false, true>(
                                a, nullptr, nullptr, 1, a.ngroups, nullptr, num_sms, s)
                          : launch_t<64, 3, 2, false>(a, nullptr, nullptr, 1, a.ngroups, nullptr,
                                                      num_sms, s);
    if (dp == 128)
        return transposed ? launch_t<128, 3, 2, false, false, false, true>(
                                a, nullptr, nullptr, 1, a.ngroups, nullptr, num_sms, s)
                          : launch_t<128, 3, 2, false>(a, nullptr, nullptr, 1, a.ngroups, nullptr,
                                                       num_sms, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_dp_split_wide_cl(const DpArgs& a, int dp, bool transposed, cudaStream_t s,
                                    bool* used) {
    *used = false;
    if (dp == 64)
        return transposed ? launch_cl<64, false, true>(a, s, used)
                          : launch_cl<64, false, false>(a, s, used);
    if (dp == 128)
        return transposed ? launch_cl<128, false, true>(a, s, used)
                          : launch_cl<128, false, false>(a, s, used);
    return cudaSuccess;
}

}  // namespace pardtw
