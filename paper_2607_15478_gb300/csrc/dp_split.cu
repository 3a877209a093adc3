// Warp-pair DP with two strips per CTA (k_dp_split<..., NS = 2, ...>, see
// dp_split.cuh): each DP warp has an SM sub-partition of its own, which keeps
// the per-column step of a strip short; the choice for a chain of strips
// that does not fill the GPU (one pair of up to ~2 x 152 strips, a band).
#include "dp_split.cuh"

namespace pardtw {
namespace {

template <bool kMany>
cudaError_t launch_any2(const DpArgs& a, const DpArgs* many, const int* item0, int n, int items,
                        int* ticket, int dp, int R, int num_sms, cudaStream_t s) {
#define PARDTW_SPLIT_CASES(RR)                                                                  \
    switch (dp) {                                                                               \
        case 4: return launch_t<4, RR, 2, kMany>(a, many, item0, n, items, ticket, num_sms, s);   \
        case 8: return launch_t<8, RR, 2, kMany>(a, many, item0, n, items, ticket, num_sms, s);   \
        case 12: return launch_t<12, RR, 2, kMany>(a, many, item0, n, items, ticket, num_sms, s); \
        case 16: return launch_t<16, RR, 2, kMany>(a, many, item0, n, items, ticket, num_sms, s); \
        default: break;                                                                         \
    }
    if (R == 2) {
        PARDTW_SPLIT_CASES(2)
        if (dp == 32) return launch_t<32, 2, 2, kMany>(a, many, item0, n, items, ticket, num_sms, s);
    } else if (R == 3) {
        PARDTW_SPLIT_CASES(3)
        if (dp == 32) return launch_t<32, 3, 2, kMany>(a, many, item0, n, items, ticket, num_sms, s);
    } else if (R == 4) {
        PARDTW_SPLIT_CASES(4)
    }
#undef PARDTW_SPLIT_CASES
    return cudaErrorInvalidValue;
}

}  // namespace

bool split_supported(int dp, int R, int ns) {
    if (ns == 4) return split4_supported(dp, R);
    if (ns != 2) return false;
    if (R == 2 || R == 3) return dp <= 32;
    if (R == 4) return dp <= 16;
    return false;
}

cudaError_t launch_dp_split(const DpArgs& a, int dp, int R, int ns, int num_sms, cudaStream_t s,
                            bool transposed) {
    if (ns == 4) return launch_dp_split4(a, nullptr, nullptr, 1, a.ngroups, nullptr, dp, R,
                                         num_sms, s, transposed);
    if (transposed) {
        if (R != 3) return cudaErrorInvalidValue;
        switch (dp) {
            case 4: return launch_t<4, 3, 2, false, false, false, true>(a, nullptr, nullptr, 1, a.ngroups, nullptr, num_sms, s);
            case 8: return launch_t<8, 3, 2, false, false, false, true>(a, nullptr, nullptr, 1, a.ngroups, nullptr, num_sms, s);
            case 12: return launch_t<12, 3, 2, false, false, false, true>(a, nullptr, nullptr, 1, a.ngroups, nullptr, num_sms, s);
            case 16: return launch_t<16, 3, 2, false, false, false, true>(a, nullptr, nullptr, 1, a.ngroups, nullptr, num_sms, s);
            case 32: return launch_t<32, 3, 2, false, false, false, true>(a, nullptr, nullptr, 1, a.ngroups, nullptr, num_sms, s);
            default: return cudaErrorInvalidValue;
        }
    }
    return launch_any2<false>(a, nullptr, nullptr, 1, a.ngroups, nullptr, dp, R, num_sms, s);
}

cudaError_t launch_dp_split_many(const DpArgs* many, const int* item0, int n, int total_items,
                                 int* ticket, int dp, int R, int ns, int num_sms, cudaStream_t s) {
    if (n <= 0 || total_items <= 0) return cudaSuccess;
    if (ns == 4) return launch_dp_split4(DpArgs{}, many, item0, n, total_items, ticket, dp, R,
                                         num_sms, s, false);
    return launch_any2<true>(DpArgs{}, many, item0, n, total_items, ticket, dp, R, num_sms, s);
}

cudaError_t launch_dp_subseq_many(const DpArgs* many, const int* item0, int n, int total_items,
                                  int* ticket, int dp, int num_sms, cudaStream_t s) {
    if (n <= 0 || total_items <= 0) return cudaSuccess;
    const DpArgs none{};
    switch (dp) {
        case 4: return launch_t<4, 3, 2, true, false, true>(none, many, item0, n, total_items, ticket, num_sms, s);
        case 8: return launch_t<8, 3, 2, true, false, true>(none, many, item0, n, total_items, ticket, num_sms, s);
        case 12: return launch_t<12, 3, 2, true, false, true>(none, many, item0, n, total_items, ticket, num_sms, s);
        case 16: return launch_t<16, 3, 2, true, false, true>(none, many, item0, n, total_items, ticket, num_sms, s);
        case 32: return launch_t<32, 3, 2, true, false, true>(none, many, item0, n, total_items, ticket, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

bool split_bf16_supported(int dp) { return dp == 64 || dp == 128; }

cudaError_t launch_dp_split_bf16(const DpArgs& a, int dp, int num_sms, cudaStream_t s,
                                 bool transposed) {
    if (dp == 64)
        return transposed ? launch_t<64, 3, 2, false, true, false, true>(
                                a, nullptr, nullptr, 1, a.ngroups, nullptr, num_sms, s)
                          : launch_t<64, 3, 2, false, true>(a, nullptr, nullptr, 1, a.ngroups,
                                                            nullptr, num_sms, s);
    if (dp == 128)
        return transposed ? launch_t<128, 3, 2, false, true, false, true>(
                                a, nullptr, nullptr, 1, a.ngroups, nullptr, num_sms, s)
                          : launch_t<128, 3, 2, false, true>(a, nullptr, nullptr, 1, a.ngroups,
                                                             nullptr, num_sms, s);
    return cudaErrorInvalidValue;
}

}  // namespace pardtw
