// Band map of the parallel backtrace (see bandmap.cu for the whole scheme):
// the per-band, per-segment propagation of entries, shared by the standalone
// kernel (bandmap.cu) and the DP kernel, which runs band-map items on its CTAs
// as the strips they need complete (dp_split.cuh).
#pragma once
#include "pardtw_common.cuh"

namespace pardtw {

namespace {

constexpr int kSegThreads = 128;  // with 128-row bands: 64 +5%, 256 +5%, 512 +40% (backtrace time)
constexpr int kNoPath = -2;
constexpr int kOrigin = -1;
constexpr int kBand = 128;  // rows per band

// The backtrace scratch of one pair (bandmap_scratch_bytes(La, Lb) bytes).
struct BtScratch {
    int2* exits;     // nbands x Lb: entries of each band's last two rows
    int2* exits2;    // n2 x Lb: for band b = nbands-2-2m (m < n2, b >= 2), the entries two
                     // bands up (into band b-2's last two rows) of band b's last two rows
    int2* exits4;    // n4 x Lb: for band b = nbands-2-4m (m < n4, b >= 4), the entries four
                     // bands up (into band b-4's last two rows)
    int2* cross;     // nbands: the path's last cell in each band
    int2* seg;       // nbands x band: each band's piece of the path, descending
    int* count;      // nbands: cells in each piece
    int* end_entry;  // the end cell's entry
    int nbands, n2, n4;
};
__host__ __device__ inline BtScratch bt_scratch(void* scratch, int La, int Lb) {
    BtScratch r;
    r.nbands = (La + kBand - 1) / kBand;
    r.n2 = r.nbands >= 4 ? (r.nbands - 2) / 2 : 0;
    r.n4 = r.nbands >= 6 ? (r.nbands - 6) / 4 + 1 : 0;
    char* p = static_cast<char*>(scratch);
    r.exits = reinterpret_cast<int2*>(p);
    p += (size_t)r.nbands * Lb * sizeof(int2);
    r.exits2 = reinterpret_cast<int2*>(p);
    p += (size_t)r.n2 * Lb * sizeof(int2);
    r.exits4 = reinterpret_cast<int2*>(p);
    p += (size_t)r.n4 * Lb * sizeof(int2);
    r.cross = reinterpret_cast<int2*>(p);
    p += (size_t)r.nbands * sizeof(int2);
    r.seg = reinterpret_cast<int2*>(p);
    p += (size_t)r.nbands * kBand * sizeof(int2);
    r.count = reinterpret_cast<int*>(p);
    p += (size_t)r.nbands * sizeof(int);
    r.end_entry = reinterpret_cast<int*>(p);
    return r;
}


// A segment of a band is mapped by a block of NT threads: thread t owns the
// 16 columns s0 + 16 t .. + 15 of the segment's computed range, where
// s0 = c0 - halo; the segment stores columns c0 .. c0 + width - 1 with
// width = NT * 16 - 2 * band (segments are width apart).  Two row buffers of
// entries per thread live in registers; the left-neighbour columns a thread
// needs come through shared memory.
//
// One row of the band map for a thread's 16 columns.  kTop: the row is one
// of the band's first two rows, whose predecessors may lie in the band above.
template <int NT, bool kTop, bool kBanded>
__device__ __forceinline__ void bandmap_row(int i, int r0, int r1, int La, int Lb, int jb, int c0,
                                            int width, int b, uint32_t word, int t,
                                            int (*s_x)[NT][3], int* e1, int* e2,
                                            int2* __restrict__ exits, int* __restrict__ end_entry,
                                            const int2* __restrict__ ranges, int rps) {
    // banded DP: cells outside the row's strip range were never computed
    int cx = 0, cy = 0;
    if (kBanded) {
        const int2 r = __ldg(ranges + i / rps);
        cx = r.x * 8;
        cy = r.y * 8;
    }
    const int par = i & 1;
    s_x[par][t][0] = e1[kColsPerWord - 2];
    s_x[par][t][1] = e1[kColsPerWord - 1];
    s_x[par][t][2] = e2[kColsPerWord - 1];
    __syncthreads();
    // (i-1, jb-2), (i-1, jb-1), (i-2, jb-1) from the left neighbour
    const int l1m2 = t > 0 ? s_x[par][t - 1][0] : kNoPath;
    const int l1m1 = t > 0 ? s_x[par][t - 1][1] : kNoPath;
    const int l2m1 = t > 0 ? s_x[par][t - 1][2] : kNoPath;
    int en[kColsPerWord];
#pragma unroll
    for (int q = 0; q < kColsPerWord; ++q) {
        // field bits of column q (see step_of_field): bit 0 -> (1,1), else
        // bit 1 -> (1,2), else (2,1)
        int p11 = (q >= 1) ? e1[q - 1] : l1m1;                    // (i-1, j-1)
        int p12 = (q >= 2) ? e1[q - 2] : (q == 1 ? l1m1 : l1m2);  // (i-1, j-2)
        int p21 = (q >= 1) ? e2[q - 1] : l2m1;                    // (i-2, j-1)
        // the field's bits 0 and 1, each tested into a predicate
        if (kTop) {
            // predecessors in the band above are named 2 * column + (1 if in
            // its last row)
            const int j = jb + q;
            if (i == r0) {
                p11 = (i >= 1 && j >= 1) ? 2 * (j - 1) + 1 : kNoPath;
                p12 = (i >= 1 && j >= 2) ? 2 * (j - 2) + 1 : kNoPath;
                p21 = (i >= 2 && j >= 1) ? 2 * (j - 1) : kNoPath;
            } else {  // i == r0 + 1: only (i-2, j-1) is above
                p21 = (r0 >= 1 && j >= 1) ? 2 * (j - 1) + 1 : kNoPath;
            }
        }
        int v = (word & (2u << (2 * q))) ? p12 : p21;  // bit 1: (1,2), else (2,1)
        v = (word & (1u << (2 * q))) ? p11 : v;        // bit 0: (1,1)
        if (kTop && i == 0 && jb + q == 0) v = kOrigin;
        if (kBanded && (jb + q < cx || jb + q >= cy)) v = kNoPath;
        en[q] = v;
    }
    // the band's last two rows are kept for the band below
    if (i >= r1 - 2 && r1 < La) {
        const int which = (i == r1 - 1) ? 1 : 0;
#pragma unroll
        for (int q = 0; q < kColsPerWord; ++q) {
            const int j = jb + q;
            if (j >= c0 && j < c0 + width && j < Lb)
                reinterpret_cast<int*>(exits + (size_t)b * Lb + j)[which] = en[q];
        }
    }
    if (i == La - 1) {
        const int q = (Lb - 1) - jb;
        if (q >= 0 && q < kColsPerWord && Lb - 1 >= c0 && Lb - 1 < c0 + width) {
#pragma unroll
            for (int u = 0; u < kColsPerWord; ++u)
                if (u == q) *end_entry = en[u];
        }
    }
#pragma unroll
    for (int q = 0; q < kColsPerWord; ++q) {
        e2[q] = e1[q];
        e1[q] = en[q];
    }
}

constexpr int kRowsAhead = 8;  // backpointer rows loaded ahead of use

// The band map of band b over segment segx of its columns, by the NT threads
// of the calling block (all of them must call it; t = threadIdx.x < NT).
// s_x: the block's left-neighbour exchange buffer.
// kInKernel: the backpointers were written by the calling kernel itself (by
// other CTAs, released through flags), so they are read through L2 rather than
// the read-only path.  ready(): called by every thread once the segment is
// known to have work, before its first backpointer load (the DP kernel waits
// there for the strips that cover the band).
template <int NT, bool kBanded, bool kInKernel = false, class Ready>
__device__ __forceinline__ void bandmap_segment(const BtArgs& a, int b, int segx,
                                                int (*s_x)[NT][3], Ready ready) {
    const uint32_t* __restrict__ bp = a.bp;
    const int La = a.La, Lb = a.Lb, nchunk = a.nchunk, rps = a.rps, wpb = a.wpb;
    const int band = kBand;
    const BtScratch sc = bt_scratch(a.scratch, La, Lb);
    int2* __restrict__ exits = sc.exits;
    int* __restrict__ end_entry = sc.end_entry;
    const int width = NT * kColsPerWord - 2 * band;
    if (b >= sc.nbands) return;  // CTA-uniform
    const int r0 = b * band;
    const int r1 = min(r0 + band, La);
    int c0, halo;  // first stored column; columns recomputed to its left (multiple of 16)
    if (kBanded) {
        // segments start at the band's first column over these rows (the
        // ranges are monotone in the strip): every cell left of it has no
        // path, so the first segment needs no halo and the rest of the grid
        // covers only the band's columns
        const int xs = a.ranges[r0 / rps].x * 8, ys = a.ranges[(r1 - 1) / rps].y * 8;
        c0 = (xs & ~(kColsPerWord - 1)) + segx * width;
        if (c0 >= min(ys, Lb)) return;  // CTA-uniform
        halo = segx == 0 ? 0 : 2 * band;
    } else {
        // Only cells that can lie on a path: with steps of slope 1/2 to 2, row
        // i's cells reachable from (0, 0) that can still reach (La-1, Lb-1)
        // are the columns lo(i) = max(ceil(i/2), Lb-1 - 2(La-1-i)) through
        // hi(i) = min(2i, Lb-1 - ceil((La-1-i)/2)).  lo and hi grow with i,
        // so the band's are within [lo(r0), hi(r1-1)], and a path cell's
        // predecessors are path cells too: segments start at lo(r0) (the
        // first without a halo) and end at hi(r1-1); the cells left out
        // (two thirds of a square matrix) are never asked for.
        const int xs = max(0, max((r0 + 1) / 2, Lb - 1 - 2 * (La - 1 - r0)));
        const int ys = min(Lb, min(2 * (r1 - 1), Lb - 1 - (La - r1 + 1) / 2) + 1);
        c0 = (xs & ~(kColsPerWord - 1)) + segx * width;
        if (c0 >= ys) return;  // CTA-uniform
        halo = segx == 0 ? 0 : 2 * band;
    }
    const int s0 = c0 - halo;
    const int t = threadIdx.x;
    const int jb = s0 + kColsPerWord * t;  // first column of this thread
    const bool have = jb < nchunk * kColsPerWord;
    // rows are loaded in order r0, r0 + 1, ...: the word address of the next
    // one (see bp_word_index) advances by one, and by a strip's stride less
    // its rows where the next row starts a strip
    int lrow = r0 % rps;
    const uint32_t* lp =
        have ? bp + bp_word_index(r0, jb, nchunk, rps, wpb) : bp;
    const size_t wrap = (size_t)nchunk * wpb - rps;
    auto load = [&](int i) -> uint32_t {
        uint32_t w = 0u;
        if (have && i < r1) w = kInKernel ? __ldcg(lp) : __ldg(lp);
        ++lp;
        if (++lrow == rps) {
            lrow = 0;
            lp += wrap;
        }
        return w;
    };
    if (!ready()) return;  // CTA-uniform

    int e1[kColsPerWord], e2[kColsPerWord];  // entries of rows i-1 and i-2
#pragma unroll
    for (int q = 0; q < kColsPerWord; ++q) e1[q] = e2[q] = kNoPath;

    // the band's first two rows
    const uint32_t top0 = load(r0), top1 = load(r0 + 1);
    uint32_t wq[kRowsAhead];
#pragma unroll
    for (int u = 0; u < kRowsAhead; ++u) wq[u] = load(r0 + 2 + u);
    bandmap_row<NT, true, kBanded>(r0, r0, r1, La, Lb, jb, c0, width, b, top0, t, s_x, e1, e2,
                               exits, end_entry, a.ranges, rps);
    if (r0 + 1 < r1)
        bandmap_row<NT, true, kBanded>(r0 + 1, r0, r1, La, Lb, jb, c0, width, b, top1, t, s_x, e1,
                                   e2, exits, end_entry, a.ranges, rps);
    // the rest, kRowsAhead at a time, loading the next group meanwhile; whole
    // groups run without a per-row guard (so the two row buffers rotate by
    // renaming, not by moves: -15%), then the last rows of the band
    int i = r0 + 2;
    for (; i + kRowsAhead <= r1; i += kRowsAhead) {
        uint32_t wn[kRowsAhead];
#pragma unroll
        for (int u = 0; u < kRowsAhead; ++u) wn[u] = load(i + kRowsAhead + u);
#pragma unroll
        for (int u = 0; u < kRowsAhead; ++u)
            bandmap_row<NT, false, kBanded>(i + u, r0, r1, La, Lb, jb, c0, width, b, wq[u], t,
                                        s_x, e1, e2, exits, end_entry, a.ranges, rps);
#pragma unroll
        for (int u = 0; u < kRowsAhead; ++u) wq[u] = wn[u];
    }
#pragma unroll 1
    for (int u = 0; i + u < r1; ++u) {
        uint32_t w = 0;
#pragma unroll
        for (int v = 0; v < kRowsAhead; ++v)
            if (v == u) w = wq[v];
        bandmap_row<NT, false, kBanded>(i + u, r0, r1, La, Lb, jb, c0, width, b, w, t, s_x, e1, e2,
                                    exits, end_entry, a.ranges, rps);
    }
}

}  // namespace
}  // namespace pardtw
