// Warp-pair DP of one pair with the backtrace's band map inside
// (k_dp_split<..., kMap = true>, see dp_split.cuh): two strips of 3 rows per
// lane per CTA, FP32 cost, either orientation.  For pairs whose strip groups
// outnumber the CTAs resident at once: the CTAs that find no group left in
// the last wave map the bands whose strips are done, while the last strips
// still sweep, instead of a separate band-map kernel after the DP.
#include "dp_split.cuh"

namespace pardtw {

bool split_map_supported(int dp, int R, int ns, bool bf16) {
    return R == 3 && ns == 2 && !bf16 && dp <= 32;
}

cudaError_t launch_dp_split_map(const DpArgs& a, const MapArgs& m, int dp, int num_sms,
                                cudaStream_t s, bool transposed) {
#define PARDTW_MAP_CASE(DD)                                                                      \
    case DD:                                                                                     \
        return transposed ? launch_t<DD, 3, 2, false, false, false, true, true>(                 \
                                a, nullptr, nullptr, 1, a.ngroups, nullptr, num_sms, s, &m)     \
                          : launch_t<DD, 3, 2, false, false, false, false, true>(                \
                                a, nullptr, nullptr, 1, a.ngroups, nullptr, num_sms, s, &m);
    switch (dp) {
        PARDTW_MAP_CASE(4)
        PARDTW_MAP_CASE(8)
        PARDTW_MAP_CASE(12)
        PARDTW_MAP_CASE(16)
        PARDTW_MAP_CASE(32)
        default: return cudaErrorInvalidValue;
    }
#undef PARDTW_MAP_CASE
}

}  // namespace pardtw
