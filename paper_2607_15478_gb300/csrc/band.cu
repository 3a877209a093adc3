// Band for the multiscale exact alignment (dtw_align_banded).  The paper
// mentions bands and multiscale DTW as ways to cut the quadratic cost
// (Sec. II); this library builds the band from an exact alignment of the two
// sequences averaged over `ds` frames, and the exact DP then runs inside it.
//
//   k_pool         average of each window of ds frames (the last window may
//                  be shorter)
//   k_band_ranges  per strip of the fine DP, the 8-column blocks within
//                  `w` columns (or the per-row predicted half-width of the
//                  learned band) of the upsampled coarse path over the strip's
//                  rows, widened to be monotone in the strip (the banded DP
//                  needs the start and the end of the ranges non-decreasing)
//   k_band_touch   whether the banded path comes within one block of a side
//                  of the band that is not the side of the matrix (the band
//                  may then have cut off a better path: the caller falls back
//                  to the full exact DP)
#include <climits>
#include "pardtw_common.cuh"

namespace pardtw {

namespace {

__global__ void k_pool(const float* __restrict__ X, int L, int D, int ds, float* __restrict__ Y) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int Lc = (L + ds - 1) / ds;
    if (t >= Lc * D) return;
    const int c = t / D, d = t - c * D;
    const int f0 = c * ds, f1 = min(f0 + ds, L);
    float acc = 0.f;
    for (int f = f0; f < f1; ++f) acc += X[(size_t)f * D + d];
    Y[(size_t)c * D + d] = acc / (float)(f1 - f0);
}

// One thread per strip (k_band_monotone then widens the ranges to monotone).
// swap: the fine DP sweeps the transposed pair, so a strip's rows are frames
// of B: the coarse path's entries are read as (column, row).  La, Lb, Lac are
// the swept pair's (rows, columns, coarse rows).
__global__ void k_band_ranges(const int32_t* __restrict__ cpath, const int* __restrict__ clen,
                              int ds, int w, const float* __restrict__ wrow, int Lac, int La,
                              int Lb, int nstrips, int rps, int swap,
                              int2* __restrict__ ranges) {
    const int ri = swap ? 1 : 0, ci = 1 - ri;
    const int n = *clen;
    const int nsub = (Lb + 7) / 8;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (n <= 0) {  // the coarse alignment failed: every strip sweeps all columns
        if (s < nstrips) ranges[s] = make_int2(0, nsub);
        return;
    }
    if (s < nstrips) {
        const int r0 = s * rps, r1 = min(r0 + rps, La) - 1;
        // coarse rows around the strip's rows (a (2,1) step may skip one)
        const int icl = r0 / ds - 1, ich = r1 / ds + 1;
        int lo = 0, hi = n;  // first path entry with row >= icl
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cpath[2 * mid + ri] < icl)
                lo = mid + 1;
            else
                hi = mid;
        }
        int jmin = 0x7fffffff, jmax = -1;
        for (int k = lo; k < n && cpath[2 * k + ri] <= ich; ++k) {
            jmin = min(jmin, cpath[2 * k + ci]);
            jmax = max(jmax, cpath[2 * k + ci]);
        }
        if (jmax < 0) {  // cannot happen for a path covering every coarse row
            jmin = 0;
            jmax = (Lb - 1) / ds;
        }
        if (wrow) {  // the widest predicted half-width of the coarse rows around the strip
            float wm = 0.f;
            for (int i = max(icl, 0); i <= min(ich, Lac - 1); ++i) wm = fmaxf(wm, wrow[i]);
            w = (int)ceilf(fminf(wm, (float)Lb));
        }
        const int jlo = max(jmin * ds - w, 0);
        const int jhi = min((jmax + 1) * ds - 1 + w, Lb - 1);
        int x = (jlo / 8) & ~1;           // even: whole 16-column words
        int y = min((jhi + 8) / 8, nsub);
        if (s == 0) x = 0;
        if (s == nstrips - 1) y = nsub;
        ranges[s] = make_int2(x, y);
    }
}

// Widen the ranges to monotone: starts by a suffix minimum, ends by a
// prefix maximum.  One block: thread t takes a run of consecutive strips,
// the runs' minima and maxima are scanned across the block (inclusive scans
// in shared memory, log2(kMonoThreads) rounds), and each thread rewrites its
// run from the carry of the runs after it (starts) and before it (ends).
// (A single thread took 125 us for 1075 strips.)
constexpr int kMonoThreads = 256;
__global__ void __launch_bounds__(kMonoThreads)
    k_band_monotone(int nstrips, int2* __restrict__ ranges) {
    __shared__ int s_min[kMonoThreads], s_max[kMonoThreads];
    const int t = threadIdx.x;
    const int per = (nstrips + kMonoThreads - 1) / kMonoThreads;
    const int lo = min(t * per, nstrips), hi = min(lo + per, nstrips);
    int mn = INT_MAX, mx = INT_MIN;
    for (int q = lo; q < hi; ++q) {
        const int2 r = ranges[q];
        mn = min(mn, r.x);
        mx = max(mx, r.y);
    }
    s_min[t] = mn;
    s_max[t] = mx;
    __syncthreads();
    for (int off = 1; off < kMonoThreads; off <<= 1) {
        const int a = t >= off ? s_max[t - off] : INT_MIN;               // runs before t
        const int b = t + off < kMonoThreads ? s_min[t + off] : INT_MAX;  // runs after t
        __syncthreads();
        s_max[t] = max(s_max[t], a);
        s_min[t] = min(s_min[t], b);
        __syncthreads();
    }
    int cmax = t > 0 ? s_max[t - 1] : INT_MIN;
    int cmin = t + 1 < kMonoThreads ? s_min[t + 1] : INT_MAX;
    for (int q = lo; q < hi; ++q) {
        cmax = max(cmax, ranges[q].y);
        ranges[q].y = cmax;
    }
    for (int q = hi - 1; q >= lo; --q) {
        cmin = min(cmin, ranges[q].x);
        ranges[q].x = cmin;
    }
}

__global__ void k_band_touch(const int32_t* __restrict__ path, const int* __restrict__ plen,
                             int Lb, int rps, const int2* __restrict__ ranges, int swap,
                             int* __restrict__ touch) {
    const int n = *plen;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k == 0 && n <= 0) atomicOr(touch, 1);  // no path inside the band
    if (k >= n) return;
    // (row, column) of the swept pair (the path is always the problem's (i, j))
    const int i = path[2 * k + (swap ? 1 : 0)], j = path[2 * k + (swap ? 0 : 1)];
    const int2 r = ranges[i / rps];
    const int x8 = r.x * 8, y8 = min(r.y * 8, Lb);
    if ((x8 > 0 && j < x8 + 8) || (y8 < Lb && j >= y8 - 8)) atomicOr(touch, 1);
}

}  // namespace

cudaError_t launch_pool(const float* X, int L, int D, int ds, float* Y, cudaStream_t s) {
    const int n = ((L + ds - 1) / ds) * D;
    k_pool<<<(n + 255) / 256, 256, 0, s>>>(X, L, D, ds, Y);
    return cudaGetLastError();
}

cudaError_t launch_band_ranges(const int32_t* cpath, const int* clen, int ds, int w,
                               const float* wrow, int Lac, int La, int Lb, int nstrips, int rps,
                               int swap, int2* ranges, cudaStream_t s) {
    const int threads = 256;
    const int blocks = (nstrips + threads - 1) / threads;
    k_band_ranges<<<blocks, threads, 0, s>>>(cpath, clen, ds, w, wrow, Lac, La, Lb, nstrips, rps,
                                             swap, ranges);
    k_band_monotone<<<1, kMonoThreads, 0, s>>>(nstrips, ranges);
    return cudaGetLastError();
}

cudaError_t launch_band_touch(const int32_t* path, const int* plen, int cap, int Lb, int rps,
                              const int2* ranges, int swap, int* touch, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(touch, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_band_touch<<<(cap + 255) / 256, 256, 0, s>>>(path, plen, Lb, rps, ranges, swap, touch);
    return cudaGetLastError();
}

}  // namespace pardtw
