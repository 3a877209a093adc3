// Instantiations of the cluster DP (dp_split_cl.cuh) for the FP32 cost at
// D <= 32 and the BF16 cost at D = 64, 128; the FP32 cost at D = 64, 128 is
// in dp_split_wide.cu.
#include "dp_split_cl.cuh"

namespace pardtw {

cudaError_t launch_dp_split_cl(const DpArgs& a, int dp, bool bf16, bool transposed,
                               cudaStream_t s, bool* used) {
    *used = false;
    if (bf16) {
        switch (dp) {
            case 64: return transposed ? launch_cl<64, true, true>(a, s, used)
                                       : launch_cl<64, true, false>(a, s, used);
            case 128: return transposed ? launch_cl<128, true, true>(a, s, used)
                                        : launch_cl<128, true, false>(a, s, used);
            default: return cudaSuccess;
        }
    }
    switch (dp) {
        case 4: return transposed ? launch_cl<4, false, true>(a, s, used) : launch_cl<4, false, false>(a, s, used);
        case 8: return transposed ? launch_cl<8, false, true>(a, s, used) : launch_cl<8, false, false>(a, s, used);
        case 12: return transposed ? launch_cl<12, false, true>(a, s, used) : launch_cl<12, false, false>(a, s, used);
        case 16: return transposed ? launch_cl<16, false, true>(a, s, used) : launch_cl<16, false, false>(a, s, used);
        case 32: return transposed ? launch_cl<32, false, true>(a, s, used) : launch_cl<32, false, false>(a, s, used);
        case 64:
        case 128: return launch_dp_split_wide_cl(a, dp, transposed, s, used);
        default: return cudaSuccess;
    }
}

}  // namespace pardtw
