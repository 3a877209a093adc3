// Parallel backtrace (Sec. II-D keeps the backtrace matrix and follows it
// back from the end cell; Sec. VI-C notes that this stage is sequential).
//
// A serial walk costs one dependent memory access per path cell (~2e4 for
// a 20000 x 25000 pair).  This file splits it:
//
//   1. k_bandmap: rows are cut into bands of 128 rows.  For every cell of
//      a band, "entry" = the cell of the band above where the optimal path
//      to this cell last sat before entering the band, encoded as
//      2 * column + (1 if that cell is in the band above's last row, 0 if in
//      its second-to-last; every step advances at most 2 rows).  It is
//      propagated forward row by row from the step codes:
//        entry(i, j) = entry(predecessor)       predecessor inside the band
//                    = encode(predecessor)      predecessor in the band above
//      All columns of a row are independent (the inputs are rows i-1, i-2),
//      so bands and column segments run in parallel.  A segment recomputes
//      2 * 128 columns to its left (dependencies move at most 2 columns
//      left per row, so those halo values are exact when they are used).
//      Only the entries of each band's last two rows are stored, and the
//      end cell's entry.
//   2. k_bt_compose composes the maps of bands b and b-1 (every other band),
//      k_bt_compose4 those of b and b-2 (every fourth band), and k_bt_chain
//      (one thread) follows the entries from the end cell up to band 0, four
//      bands per dependent load (with the two-band map of the same cell
//      loaded beside it): the path's last cell in every other band.
//   3. k_bt_walk (one warp per band): each band's piece of the path is
//      walked back from that cell (one lookup away for the bands the chain
//      stepped over) to the band's top, in parallel.
//   4. k_bt_emit: the pieces are concatenated in ascending order.
//
// Entry codes: -1 = the origin (0, 0); -2 = no path (unreachable cell).
#include "bandmap.cuh"
#include "block_walk.cuh"

namespace pardtw {
namespace {

constexpr int kSegCols = kSegThreads * kColsPerWord;  // 2048 columns computed per CTA

template <bool kMany, bool kBanded>
__global__ void __launch_bounds__(kSegThreads) k_bandmap(const BtArgs one,
                                                         const BtArgs* __restrict__ many) {
    const BtArgs& a = kMany ? many[blockIdx.z] : one;
    // left-neighbour exchange, double-buffered by row parity: columns 14, 15
    // of row i-1 and column 15 of row i-2 of every thread
    __shared__ int s_x[2][kSegThreads][3];
    // kMany: one pair per blockIdx.z (the grid covers the largest pair;
    // blocks beyond a pair's bands or columns leave at once)
    bandmap_segment<kSegThreads, kBanded>(a, blockIdx.y, blockIdx.x, s_x, [] { return 1; });
}

}  // namespace

// The cell named by entry e of a cell of band x: a cell of band x-1's last
// two rows.
__device__ __forceinline__ int2 entry_cell(int e, int x) {
    return make_int2((e & 1) ? x * kBand - 1 : x * kBand - 2, e >> 1);
}
// The entry of cell c of a band's last two rows from its exits word x (.x:
// second-to-last row, .y: last row); last = the band's last row.
__device__ __forceinline__ int pick_exit(int2 x, int ci, int last) { return ci == last ? x.y : x.x; }

// Two-band exit map: for band b = nbands-2-2m (m = blockIdx.y < n2) and
// column j, the entries of the cells of band b's last two rows two bands up,
// composed from band b's exits and band b-1's.  Only the columns a path can
// cross there are composed (the rest is never read).  Grid: (columns / 256,
// n2 of the largest pair, pairs).
template <bool kMany>
__global__ void __launch_bounds__(256) k_bt_compose(const BtArgs one,
                                                    const BtArgs* __restrict__ many) {
    const BtArgs& a = kMany ? many[blockIdx.z] : one;
    const int La = a.La, Lb = a.Lb;
    const BtScratch sc = bt_scratch(a.scratch, La, Lb);
    const int m = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= sc.n2 || j >= Lb) return;
    const int b = sc.nbands - 2 - 2 * m;
    const int r1 = (b + 1) * kBand;  // b <= nbands-2: a whole band
    // columns of rows r1-2, r1-1 that can lie on a path (see bandmap_segment)
    const int lo = max((r1 - 1) / 2, Lb - 1 - 2 * (La - 1 - (r1 - 2)));
    const int hi = min(2 * (r1 - 1), Lb - 1);
    if (j < lo || j > hi) return;
    const int2* __restrict__ exits = sc.exits;
    const int2 x = exits[(size_t)b * Lb + j];
    auto hop = [&](int e) -> int {
        if (e < 0) return kNoPath;
        const int2 c = entry_cell(e, b);
        if (c.y < 0 || c.y >= Lb) return kNoPath;
        return pick_exit(exits[(size_t)(b - 1) * Lb + c.y], c.x, b * kBand - 1);
    };
    sc.exits2[(size_t)m * Lb + j] = make_int2(hop(x.x), hop(x.y));
}

// Four-band exit map: for band b = nbands-2-4m (m = blockIdx.y < n4) and
// column j, the entries of the cells of band b's last two rows four bands
// up, composed from the two-band maps of bands b and b-2.  Same columns as
// k_bt_compose.
template <bool kMany>
__global__ void __launch_bounds__(256) k_bt_compose4(const BtArgs one,
                                                     const BtArgs* __restrict__ many) {
    const BtArgs& a = kMany ? many[blockIdx.z] : one;
    const int La = a.La, Lb = a.Lb;
    const BtScratch sc = bt_scratch(a.scratch, La, Lb);
    const int m = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= sc.n4 || j >= Lb) return;
    const int b = sc.nbands - 2 - 4 * m;
    const int r1 = (b + 1) * kBand;
    const int lo = max((r1 - 1) / 2, Lb - 1 - 2 * (La - 1 - (r1 - 2)));
    const int hi = min(2 * (r1 - 1), Lb - 1);
    if (j < lo || j > hi) return;
    const int2* __restrict__ exits2 = sc.exits2;
    const int2 x = exits2[(size_t)(2 * m) * Lb + j];  // into band b-2's last two rows
    auto hop = [&](int e) -> int {
        if (e < 0) return kNoPath;
        const int2 c = entry_cell(e, b - 1);
        if (c.y < 0 || c.y >= Lb) return kNoPath;
        return pick_exit(exits2[(size_t)(2 * m + 1) * Lb + c.y], c.x, (b - 1) * kBand - 1);
    };
    sc.exits4[(size_t)m * Lb + j] = make_int2(hop(x.x), hop(x.y));
}

// One thread: the path's last cell in bands nbands-1, nbands-2, nbands-4,
// ... and in band 0; the walks find the others.  Four bands per dependent
// load through the four-band exit map, the two-band map's entry of the same
// cell loaded beside it (it names the crossing in between); two at the end.
// cross[b] = (i, j) of that cell; status on failure.
template <bool kMany>
__global__ void k_bt_chain(const BtArgs one, const BtArgs* __restrict__ many) {
    if (threadIdx.x != 0) return;
    const BtArgs& a = kMany ? many[blockIdx.x] : one;
    const int La = a.La, Lb = a.Lb, band = kBand;
    DevCtl* ctl = a.ctl;
    const BtScratch sc = bt_scratch(a.scratch, La, Lb);
    const int2* __restrict__ exits = sc.exits;
    const int2* __restrict__ exits2 = sc.exits2;
    const int nbands = sc.nbands;
    int2* __restrict__ cross = sc.cross;
    if (ctl->status != 0) return;
    cross[nbands - 1] = make_int2(La - 1, Lb - 1);
    int e = *sc.end_entry;
    // c = the cell named by entry e of band x, checked to lie in band x-1
    int2 c;
    auto take = [&](int x) -> bool {
        if (e < 0) return false;  // an entry must name a cell of the band above
        c = entry_cell(e, x);
        return c.x >= (x - 1) * band && c.y >= 0 && c.y < Lb;
    };
    bool ok = true;
    int b = nbands - 1;
    if (b >= 1) {
        ok = take(b);
        if (ok) cross[--b] = c;
    }
    const int2* __restrict__ exits4 = sc.exits4;
    while (ok && b >= 4) {  // four bands at a time (b = nbands-2-4m, m < n4)
        const int m = (nbands - 2 - b) / 4;
        const int last = (b + 1) * band - 1;
        const int2 x2 = exits2[(size_t)(2 * m) * Lb + c.y];
        const int2 x4 = exits4[(size_t)m * Lb + c.y];
        const int e2 = pick_exit(x2, c.x, last), e4 = pick_exit(x4, c.x, last);
        e = e2;
        ok = take(b - 1);
        const int2 c2 = c;
        if (ok) {
            e = e4;
            ok = take(b - 3);
        }
        if (ok) {
            cross[b - 2] = c2;
            b -= 4;
            cross[b] = c;
        }
    }
    while (ok && b >= 2) {  // two bands at a time
        const int m = (nbands - 2 - b) / 2;
        e = pick_exit(exits2[(size_t)m * Lb + c.y], c.x, (b + 1) * band - 1);
        ok = take(b - 1);
        if (ok) {
            b -= 2;
            cross[b] = c;
        }
    }
    if (ok && b == 1) {
        e = pick_exit(exits[(size_t)Lb + c.y], c.x, 2 * band - 1);
        ok = take(1);
        if (ok) cross[b = 0] = c;
    }
    if (ok && nbands >= 2) e = pick_exit(exits[c.y], c.x, band - 1);
    if (!ok || e != kOrigin) atomicCAS(&ctl->status, 0, DTW_ERR_CUDA);
}

// One warp per band: walk back from the path's last cell in band b while
// inside the band (BlockWalker), writing the cells (descending) into
// seg + b * band; count[b] = cells written.
template <bool kMany>
__global__ void k_bt_walk(const BtArgs one, const BtArgs* __restrict__ many) {
    const BtArgs& a = kMany ? many[blockIdx.y] : one;
    const int band = kBand;
    DevCtl* ctl = a.ctl;
    const BtScratch sc = bt_scratch(a.scratch, a.La, a.Lb);
    const int nbands = sc.nbands;
    const int2* __restrict__ cross = sc.cross;
    int2* __restrict__ seg = sc.seg;
    int* __restrict__ count = sc.count;
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nbands) return;
    if (ctl->status != 0) {
        if (lane == 0) count[b] = 0;
        return;
    }
    const int r0 = b * band;
    const int2* __restrict__ exits = sc.exits;
    const int Lb = a.Lb;
    int bad = 0;
    // the walk's first cell: from the chain, or (for the bands it steps
    // over) the cell its band-below's crossing names; and the cell of the
    // band above where the walk must leave (the entry of the first cell)
    int2 c = cross[b];
    if (b < nbands - 1 && b > 0 && ((nbands - 2 - b) & 1)) {
        const int2 c1 = cross[b + 1];
        const int e = pick_exit(exits[(size_t)(b + 1) * Lb + c1.y], c1.x, (b + 2) * band - 1);
        c = entry_cell(e, b + 1);
        if (e < 0 || c.x < r0 || c.y < 0 || c.y >= Lb) bad = 1;
    }
    int2 target = make_int2(-1, -1);
    if (!bad && b > 0) {
        const int e = b == nbands - 1
                          ? *sc.end_entry
                          : pick_exit(exits[(size_t)b * Lb + c.y], c.x, (b + 1) * band - 1);
        target = e < 0 ? make_int2(-3, -3) : entry_cell(e, b);
    }
    if (bad) c = make_int2(r0, 0);  // no walk; reported below
    int i = c.x, j = c.y;
    BlockWalker w{a.bp, a.nchunk, a.rps, a.wpb, lane};
    w.start(i, j);
    int n = 0;
    int2* out = seg + (size_t)b * band;
    while (!bad && i >= r0) {
        if (n >= band || j < 0) {
            bad = 1;
            break;
        }
        if (lane == 0) out[n] = make_int2(i, j);
        ++n;
        if (i == 0 && j == 0) break;
        const uint32_t f = w.field(j);
        const int di = field_di(f);
        i -= di;
        j -= field_dj(f);
        w.step(di, j, i >= r0);
    }
    // the walk must leave the band exactly at the cell its first cell's entry names
    if (b > 0 && !bad && (i != target.x || j != target.y)) bad = 1;
    if (lane == 0) {
        if (bad) atomicCAS(&ctl->status, 0, DTW_ERR_CUDA);
        count[b] = n;
    }
}

// One CTA per band (grid.y: the pair): the band's offset (sum of the counts
// of the bands before it) and the total, each by a block-wide sum, then the
// band's cells in ascending order; the CTA of band 0 writes the length and
// the total (or -status).
template <bool kMany>
__global__ void __launch_bounds__(kBand) k_bt_emit(const BtArgs one, const BtArgs* __restrict__ many) {
    const BtArgs& a = kMany ? many[blockIdx.y] : one;
    const int La = a.La, Lb = a.Lb, band = kBand;
    const int cap = La < Lb ? La : Lb;
    const BtScratch sc = bt_scratch(a.scratch, La, Lb);
    const int nbands = sc.nbands;
    const int b = blockIdx.x;
    if (b >= nbands) return;  // CTA-uniform (the grid covers the largest pair)
    const int2* __restrict__ seg = sc.seg;
    const int* __restrict__ count = sc.count;
    __shared__ int s_red[2][kBand / 32];
    // this thread's share of the counts before band b and of all counts
    int before = 0, all = 0;
    for (int q = threadIdx.x; q < nbands; q += blockDim.x) {
        const int c = count[q];
        all += c;
        if (q < b) before += c;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        before += __shfl_xor_sync(0xffffffffu, before, off);
        all += __shfl_xor_sync(0xffffffffu, all, off);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        s_red[0][w] = before;
        s_red[1][w] = all;
    }
    __syncthreads();
    if (w == 0) {
        before = lane < (int)(blockDim.x >> 5) ? s_red[0][lane] : 0;
        all = lane < (int)(blockDim.x >> 5) ? s_red[1][lane] : 0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            before += __shfl_xor_sync(0xffffffffu, before, off);
            all += __shfl_xor_sync(0xffffffffu, all, off);
        }
        if (lane == 0) {
            s_red[0][0] = before;
            s_red[1][0] = all;
        }
    }
    __syncthreads();
    before = s_red[0][0];
    all = s_red[1][0];
    int err = a.ctl->status;
    if (err == 0 && (all < 1 || all > cap)) err = DTW_ERR_CUDA;
    if (b == 0 && threadIdx.x == 0) {
        if (err != 0) {
            *a.path_len = -err;
            if (a.total) *a.total = NAN;
        } else {
            *a.path_len = all;
            if (a.total) *a.total = fmaf(a.mu, (float)(La + Lb - 2), *a.e_final);
        }
    }
    if (err != 0) return;
    // band b's cells are stored descending; they go to before .. before+n-1 reversed
    const int n = count[b];
    int32_t* __restrict__ path = a.path;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int2 c = seg[(size_t)b * band + (n - 1 - k)];
        path[2 * (before + k)] = a.transposed ? c.y : c.x;
        path[2 * (before + k) + 1] = a.transposed ? c.x : c.y;
    }
}

int bandmap_band_rows() { return kBand; }

size_t bandmap_scratch_bytes(int La, int Lb) {
    const int nbands = (La + kBand - 1) / kBand;
    const int n2 = nbands >= 4 ? (nbands - 2) / 2 : 0;
    const int n4 = nbands >= 6 ? (nbands - 6) / 4 + 1 : 0;
    return (size_t)nbands * Lb * sizeof(int2)        // exits
           + (size_t)n2 * Lb * sizeof(int2)           // exits2
           + (size_t)n4 * Lb * sizeof(int2)           // exits4
           + (size_t)nbands * sizeof(int2)            // cross
           + (size_t)nbands * kBand * sizeof(int2)    // seg
           + (size_t)nbands * sizeof(int) + 64;       // count, end entry
}

int bandmap_items(int La, int Lb, int threads) {
    const int nbands = (La + kBand - 1) / kBand;
    const int width = threads * kColsPerWord - 2 * kBand;
    return nbands * ((Lb + width - 1) / width);
}

cudaError_t launch_backtrace_bands(const BtArgs& a, cudaStream_t s, bool with_map) {
    const int nbands = (a.La + kBand - 1) / kBand;
    const int width = kSegCols - 2 * kBand;
    dim3 grid((unsigned)((a.Lb + width - 1) / width), (unsigned)nbands, 1);
    if (with_map) {
        if (a.ranges)
            k_bandmap<false, true><<<grid, kSegThreads, 0, s>>>(a, nullptr);
        else
            k_bandmap<false, false><<<grid, kSegThreads, 0, s>>>(a, nullptr);
    }
    const int n2 = nbands >= 4 ? (nbands - 2) / 2 : 0;
    if (n2 > 0)
        k_bt_compose<false><<<dim3((unsigned)((a.Lb + 255) / 256), (unsigned)n2, 1), 256, 0, s>>>(
            a, nullptr);
    const int n4 = nbands >= 6 ? (nbands - 6) / 4 + 1 : 0;
    if (n4 > 0)
        k_bt_compose4<false><<<dim3((unsigned)((a.Lb + 255) / 256), (unsigned)n4, 1), 256, 0, s>>>(
            a, nullptr);
    k_bt_chain<false><<<1, 32, 0, s>>>(a, nullptr);
    k_bt_walk<false><<<(nbands + 3) / 4, 128, 0, s>>>(a, nullptr);
    k_bt_emit<false><<<dim3((unsigned)nbands, 1), kBand, 0, s>>>(a, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_backtrace_bands_many(const BtArgs* many, int n, int maxLa, int maxLb,
                                        cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int nbands = (maxLa + kBand - 1) / kBand;
    const int width = kSegCols - 2 * kBand;
    dim3 grid((unsigned)((maxLb + width - 1) / width), (unsigned)nbands, (unsigned)n);
    k_bandmap<true, false><<<grid, kSegThreads, 0, s>>>(BtArgs{}, many);
    const int n2 = nbands >= 4 ? (nbands - 2) / 2 : 0;
    if (n2 > 0)
        k_bt_compose<true><<<dim3((unsigned)((maxLb + 255) / 256), (unsigned)n2, (unsigned)n),
                             256, 0, s>>>(BtArgs{}, many);
    const int n4 = nbands >= 6 ? (nbands - 6) / 4 + 1 : 0;
    if (n4 > 0)
        k_bt_compose4<true><<<dim3((unsigned)((maxLb + 255) / 256), (unsigned)n4, (unsigned)n),
                              256, 0, s>>>(BtArgs{}, many);
    k_bt_chain<true><<<n, 32, 0, s>>>(BtArgs{}, many);
    k_bt_walk<true><<<dim3((unsigned)((nbands + 3) / 4), (unsigned)n), 128, 0, s>>>(BtArgs{},
                                                                                     many);
    k_bt_emit<true><<<dim3((unsigned)nbands, (unsigned)n), kBand, 0, s>>>(BtArgs{}, many);
    return cudaGetLastError();
}

}  // namespace pardtw
