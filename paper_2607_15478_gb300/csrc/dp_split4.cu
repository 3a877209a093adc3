// Warp-pair DP with four strips per CTA (k_dp_split<..., NS = 4, ...>, see
// dp_split.cuh): ten warps, one DP warp and one cost warp on every SM
// sub-partition, twice the DP warps of the two-strip CTA per SM.  The choice
// when there are more strip groups than SMs (a long pair, a batch): the
// per-column step of a strip is longer (the DP warp shares its
// sub-partition) but twice as many strips advance at once, and three of four
// strip-to-strip handoffs stay in shared memory.  Register budget: at ten
// warps a thread may hold 168 registers, which R = 2, 3 at D <= 16 fit.
#include "dp_split.cuh"

namespace pardtw {

bool split4_supported(int dp, int R) { return (R == 2 || R == 3) && dp <= 16; }

cudaError_t launch_dp_split4(const DpArgs& a, const DpArgs* many, const int* item0, int n,
                             int items, int* ticket, int dp, int R, int num_sms, cudaStream_t s,
                             bool transposed) {
    if (transposed) {  // one pair swept transposed (3 rows per lane)
        if (many || R != 3) return cudaErrorInvalidValue;
        switch (dp) {
            case 4: return launch_t<4, 3, 4, false, false, false, true>(a, many, item0, n, items, ticket, num_sms, s);
            case 8: return launch_t<8, 3, 4, false, false, false, true>(a, many, item0, n, items, ticket, num_sms, s);
            case 12: return launch_t<12, 3, 4, false, false, false, true>(a, many, item0, n, items, ticket, num_sms, s);
            case 16: return launch_t<16, 3, 4, false, false, false, true>(a, many, item0, n, items, ticket, num_sms, s);
            default: return cudaErrorInvalidValue;
        }
    }
#define PARDTW_SPLIT4_CASES(RR, MANY)                                                             \
    switch (dp) {                                                                                 \
        case 4: return launch_t<4, RR, 4, MANY>(a, many, item0, n, items, ticket, num_sms, s);     \
        case 8: return launch_t<8, RR, 4, MANY>(a, many, item0, n, items, ticket, num_sms, s);     \
        case 12: return launch_t<12, RR, 4, MANY>(a, many, item0, n, items, ticket, num_sms, s);   \
        case 16: return launch_t<16, RR, 4, MANY>(a, many, item0, n, items, ticket, num_sms, s);   \
        default: return cudaErrorInvalidValue;                                                    \
    }
    if (many) {
        if (R == 2) PARDTW_SPLIT4_CASES(2, true)
        if (R == 3) PARDTW_SPLIT4_CASES(3, true)
    } else {
        if (R == 2) PARDTW_SPLIT4_CASES(2, false)
        if (R == 3) PARDTW_SPLIT4_CASES(3, false)
    }
#undef PARDTW_SPLIT4_CASES
    return cudaErrorInvalidValue;
}

}  // namespace pardtw
