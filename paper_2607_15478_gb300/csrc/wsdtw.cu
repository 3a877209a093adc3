// Weakly-ordered Segmental DTW (WSDTW, Sec. II-C), steps 3 to 5 on the GPU.
// Steps 1 and 2 (the fragments of A and their subsequence DTW against all of
// B) run in the batched warp-pair DP (dp_split.cu, subsequence mode), which
// leaves every fragment's last row of cumulative costs (C_seg, step 3) and its
// 2-bit backtrace matrix.  Here:
//
//   k_seg_dp     step 4, one CTA: for fragment k = 0 .. N-1 in turn,
//                  match[j]   = D_seg[k-1][j - delta_k] + C_seg[k][j]
//                               (= C_seg[0][j] for k = 0; +inf for j < delta_k)
//                  D_seg[k][j] = running minimum of match over j' <= j,
//                  arg[k][j]   = the first j' attaining it,
//                as a block-wide prefix minimum (per-thread runs, a scan of
//                the run minima, a second pass); then the end frames
//                e_{N-1} = arg[N-1][Lb-1], e_{k-1} = arg[k-1][e_k - delta_k].
//   k_bt_subseq  step 5, one thread per fragment: the walk from (last row,
//                e_k) back to row 0 through the fragment's backtrace matrix,
//                written backwards into the fragment's slots of a scratch path.
//   k_compact    the fragment paths one after another into the caller's path.
#include "dp_device.cuh"

namespace pardtw {

namespace {

constexpr int kSegThreads = 1024;

// (value, index) minimum where the earlier index wins ties.
struct MinArg {
    float v;
    int j;
};
__device__ __forceinline__ MinArg better(MinArg a, MinArg b) {  // a is earlier
    return (b.v < a.v) ? b : a;
}

__global__ void __launch_bounds__(kSegThreads)
    k_seg_dp(const WsFrag* __restrict__ fr, const float* __restrict__ lastrow, size_t stride,
             int N, int Lb, const int* __restrict__ delta, float* __restrict__ Dseg, int* __restrict__ arg,
             int* __restrict__ ends, float* __restrict__ total, DevCtl* ctl) {
    __shared__ MinArg s_part[kSegThreads];
    __shared__ int s_fail;
    const int t = threadIdx.x;
    // a fragment whose DP failed (e.g. a bounded wait expired) fails the call
    if (t == 0) {
        s_fail = 0;
        for (int k = 0; k < N; ++k) {
            const int st = fr[k].pctl->status;
            if (st != 0) {
                raise_status(ctl, st, 20);
                s_fail = 1;
                break;
            }
        }
    }
    __syncthreads();
    if (s_fail) return;
    const int per = (Lb + kSegThreads - 1) / kSegThreads;
    const int j0 = min(t * per, Lb), j1 = min(j0 + per, Lb);
    for (int k = 0; k < N; ++k) {
        const float* cs = lastrow + (size_t)k * stride;
        const float* prev = k > 0 ? Dseg + (size_t)(k - 1) * Lb : nullptr;
        const int dk = k > 0 ? delta[k] : 0;
        // pass 1: the run minimum of match over this thread's columns
        MinArg m{INFINITY, -1};
        for (int j = j0; j < j1; ++j) {
            float mv;
            if (k == 0)
                mv = cs[j];
            else
                mv = (j - dk >= 0) ? prev[j - dk] + cs[j] : INFINITY;
            m = better(m, MinArg{mv, j});
        }
        s_part[t] = m;
        __syncthreads();
        // inclusive scan of the run minima (Hillis-Steele over the block)
        for (int off = 1; off < kSegThreads; off <<= 1) {
            const MinArg o = t >= off ? s_part[t - off] : MinArg{INFINITY, -1};
            __syncthreads();
            if (t >= off) s_part[t] = better(o, s_part[t]);
            __syncthreads();
        }
        MinArg run = t > 0 ? s_part[t - 1] : MinArg{INFINITY, -1};
        // pass 2: the running minimum from the carry-in
        float* drow = Dseg + (size_t)k * Lb;
        int* arow = arg + (size_t)k * Lb;
        for (int j = j0; j < j1; ++j) {
            float mv;
            if (k == 0)
                mv = cs[j];
            else
                mv = (j - dk >= 0) ? prev[j - dk] + cs[j] : INFINITY;
            run = better(run, MinArg{mv, j});
            drow[j] = run.v;
            arow[j] = run.j;
        }
        __syncthreads();  // row k is complete before row k+1 reads it
    }
    if (t == 0) {
        const float tot = Dseg[(size_t)(N - 1) * Lb + Lb - 1];
        if (!(tot < INFINITY)) {
            raise_status(ctl, DTW_ERR_UNREACHABLE, 21);
            return;
        }
        *total = tot;
        int e = arg[(size_t)(N - 1) * Lb + Lb - 1];
        ends[N - 1] = e;
        for (int k = N - 1; k > 0; --k) {
            e = arg[(size_t)(k - 1) * Lb + (e - delta[k])];
            ends[k - 1] = e;
        }
    }
}

// One thread per fragment: the subsequence path from (len-1, e_k) to row 0,
// stored backwards (ascending once read from slot row0 + len - n) as global
// (row of A, frame of B) pairs.  A step that leaves the fragment's cells
// raises DTW_ERR_CUDA (it cannot happen for a finite end cell).
__global__ void k_bt_subseq(const WsFrag* __restrict__ fr, int N, const int* __restrict__ ends,
                            int32_t* __restrict__ scratch, int* __restrict__ count,
                            DevCtl* ctl) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    if (ctl->status != 0) {
        count[k] = 0;
        return;
    }
    const WsFrag f = fr[k];
    int i = f.len - 1, j = ends[k];
    int n = 0;
    int32_t* out = scratch + 2 * (size_t)(f.row0 + f.len - 1);
    for (;;) {
        out[-2 * n] = f.row0 + i;
        out[-2 * n + 1] = j;
        ++n;
        if (i == 0) break;
        const uint32_t w = f.bp[bp_word_index(i, j, f.nchunk, f.rps, f.wpb)];
        const int st = step_of_field((w >> (2 * (j & 15))) & 3u);
        const int di = st == 2 ? 2 : 1, dj = st == 1 ? 2 : 1;
        i -= di;
        j -= dj;
        if (i < 0 || j < 0 || n >= f.len) {
            raise_status(ctl, DTW_ERR_CUDA, 22);
            count[k] = 0;
            return;
        }
    }
    count[k] = n;
}

// The fragment paths one after another: fragment k's n_k pairs sit at the
// end of its slots [row0, row0 + len); *path_len = sum n_k (or -status).
__global__ void __launch_bounds__(kSegThreads)
    k_compact(const WsFrag* __restrict__ fr, int N, const int* __restrict__ count,
              const int32_t* __restrict__ scratch, int32_t* __restrict__ path,
              int* __restrict__ path_len, const DevCtl* ctl) {
    const int st = ctl->status;
    if (st != 0) {
        if (threadIdx.x == 0) *path_len = -st;
        return;
    }
    int base = 0;
    for (int k = 0; k < N; ++k) {
        const int n = count[k];
        const WsFrag f = fr[k];
        const int32_t* src = scratch + 2 * (size_t)(f.row0 + f.len - n);
        for (int q = threadIdx.x; q < 2 * n; q += blockDim.x) path[2 * (size_t)base + q] = src[q];
        base += n;
    }
    if (threadIdx.x == 0) *path_len = base;
}

}  // namespace

cudaError_t launch_seg_dp(const WsFrag* fr, const float* lastrow, size_t stride, int N, int Lb,
                          const int* delta, float* Dseg, int* arg, int* ends, float* total,
                          DevCtl* ctl, cudaStream_t s) {
    k_seg_dp<<<1, kSegThreads, 0, s>>>(fr, lastrow, stride, N, Lb, delta, Dseg, arg, ends, total,
                                       ctl);
    return cudaGetLastError();
}

cudaError_t launch_bt_subseq(const WsFrag* fr, int N, const int* ends, int32_t* scratch,
                             int* count, int32_t* path, int* path_len, DevCtl* ctl,
                             cudaStream_t s) {
    k_bt_subseq<<<(N + 63) / 64, 64, 0, s>>>(fr, N, ends, scratch, count, ctl);
    k_compact<<<1, kSegThreads, 0, s>>>(fr, N, count, scratch, path, path_len, ctl);
    return cudaGetLastError();
}

}  // namespace pardtw
