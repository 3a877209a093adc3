// Backtrace of the optimal path through the 2-bit backpointer matrix
// (Sec. II-D: the backtrace matrix is kept in memory and used to recover the
// path; Sec. VI-C: this stage is sequential).
//
// One CTA.  Thread 0 walks from (La-1, Lb-1) to (0, 0), following the step
// of each cell's backpointer field (step_of_field), and writes the cells into a scratch
// buffer from its end; then the whole CTA copies them in ascending order
// into the caller's path buffer.  The walk is bounded by min(La, Lb) cells
// and checks every index, so a damaged matrix yields an error, never an
// out-of-bounds access.
#include "pardtw_common.cuh"

namespace pardtw {

__global__ void k_backtrace(const uint32_t* __restrict__ bp, int La, int Lb, int nchunk, int rps,
                            int wpb, const DevCtl* __restrict__ ctl, const float* __restrict__ e_final,
                            float mu, int32_t* __restrict__ path, int32_t* __restrict__ scratch,
                            int* __restrict__ path_len, float* __restrict__ total) {
    __shared__ int s_len;
    __shared__ int s_err;
    const int cap = La < Lb ? La : Lb;
    if (threadIdx.x == 0) {
        int err = ctl->status;
        int n = 0;
        if (err == 0) {
            int i = La - 1, j = Lb - 1;
            // scratch[2*(cap-1-k)] holds the k-th cell from the end
            for (;;) {
                if (n >= cap || i < 0 || j < 0) {
                    err = DTW_ERR_CUDA;
                    break;
                }
                scratch[2 * (cap - 1 - n)] = i;
                scratch[2 * (cap - 1 - n) + 1] = j;
                ++n;
                if (i == 0 && j == 0) break;
                const uint32_t word = __ldg(bp + bp_word_index(i, j, nchunk, rps, wpb));
                const int step = step_of_field((word >> (2 * (j & 15))) & 3u);
                if (step == 0) {
                    i -= 1;
                    j -= 1;
                } else if (step == 1) {
                    i -= 1;
                    j -= 2;
                } else {
                    i -= 2;
                    j -= 1;
                }
            }
        }
        s_len = n;
        s_err = err;
        if (err != 0) {
            *path_len = -err;
            if (total) *total = NAN;
        } else {
            *path_len = n;
            // D = E + mu * (La - 1 + Lb - 1)
            if (total) *total = fmaf(mu, (float)(La + Lb - 2), *e_final);
        }
    }
    __syncthreads();
    if (s_err != 0) return;
    const int n = s_len;
    const int32_t* src = scratch + 2 * (cap - n);
    for (int k = threadIdx.x; k < 2 * n; k += blockDim.x) path[k] = src[k];
}

cudaError_t launch_backtrace(const uint32_t* bp, int La, int Lb, int nchunk, int rps, int wpb,
                             const DevCtl* ctl, const float* e_final, float mu, int32_t* path,
                             int32_t* scratch, int* path_len, float* total, cudaStream_t s) {
    k_backtrace<<<1, 256, 0, s>>>(bp, La, Lb, nchunk, rps, wpb, ctl, e_final, mu, path, scratch,
                                  path_len, total);
    return cudaGetLastError();
}

}  // namespace pardtw
