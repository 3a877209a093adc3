// Internal declarations shared by the CUDA translation units of libpardtw.
// Not part of the public C-ABI (include/pardtw.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pardtw.h"

namespace pardtw {

constexpr int kWarp = 32;
constexpr int kRowsPerStrip = 30;   // rows of A per warp: lanes 0..29 (lanes 30, 31 carry
                                    // the two bottom rows of the strip above)
constexpr int kColsPerWord = 16;    // 2-bit codes per uint32 backpointer word
constexpr int kWarpsPerGroup = 4;   // strips per CTA ("strip group")

// Device status words (workspace).  [0] first error (DTW_* code), [1] detail,
// [2] ticket counter of the persistent DP kernel, [3] spare.
struct DevCtl {
    int status;
    int detail;
    int ticket;
    int spare;
};

// Arguments of the column-sweep DP kernel.
struct DpArgs {
    const float* Ahat;              // nstrips*30 x dp, row-normalised, rows >= La are zero
    const float* Bhat;              // Lb x dp, row-normalised
    uint32_t* bp;                   // nstrips * nchunk * 32 words (strip, chunk, row in strip)
    unsigned long long* gborder;    // ngroups * Lb * 2 tagged values (group bottom rows)
    DevCtl* ctl;
    float* e_final;                 // shifted cumulative cost at (La-1, Lb-1)
    int La, Lb;
    int nstrips, nchunk, ngroups;
    float kcost;                    // 1 - cost_shift
    float mu;                       // cost_shift
    unsigned epoch;                 // call tag for global border entries
    long long timeout_ns;
    int skip_publish;               // group that never publishes (fault injection), -1 off
};

// Backpointer word address of cell (i, j): strip-major, then 16-column chunk,
// then row within the strip (32 words per strip and chunk, of which the
// first 30 hold rows).  One warp store covers 32 consecutive words (128 B).
__host__ __device__ inline size_t bp_word_index(int i, int j, int nchunk) {
    const int strip = i / kRowsPerStrip;
    return ((size_t)strip * (size_t)nchunk + (size_t)(j >> 4)) * 32u +
           (size_t)(i - strip * kRowsPerStrip);
}

// Launchers (each returns a cudaError_t from the launch).
cudaError_t launch_normalise(const float* A, int La, int La_pad, const float* B, int Lb, int D,
                             int dp, float* Ahat, float* Bhat, DevCtl* ctl, cudaStream_t s);
cudaError_t launch_cost(const float* Ahat, int La, const float* Bhat, int Lb, int dp,
                        float* C, cudaStream_t s);
cudaError_t launch_dp(const DpArgs& a, int dp, int num_sms, cudaStream_t s);
cudaError_t launch_backtrace(const uint32_t* bp, int La, int Lb, int nchunk, const DevCtl* ctl,
                             const float* e_final, float mu, int32_t* path, int32_t* scratch,
                             int* path_len, float* total, cudaStream_t s);

// Padded feature width used by the kernels for a given D (0 = unsupported).
int padded_dim(int D);

}  // namespace pardtw
