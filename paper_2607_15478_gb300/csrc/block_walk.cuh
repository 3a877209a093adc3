// Walking a path back through a backtrace matrix with one warp (the band
// walks of the parallel backtrace, bandmap.cu; the fragment walks of WSDTW,
// wsdtw.cu).  Each step reads one 2-bit field (see step_of_field) whose
// address depends on the step before, so the warp keeps the backpointer
// block (one strip of rps rows x 16 columns, wpb words; see bp_word_index)
// of the current cell in registers, lane l holding words l, l+32, l+64,
// l+96, and reads a field with one shuffle.  A step moves at most two rows
// and two columns up and left and a strip has more than two rows, so the
// next block is the current one or its neighbour above, to the left or
// above-left: the three are loaded when the path enters a block, while it
// crosses it.  The row within the strip is tracked, not divided out.
#pragma once
#include "pardtw_common.cuh"

namespace pardtw {
namespace {

struct BlockWalker {
    const uint32_t* __restrict__ bp;
    int nchunk, rps, wpb, lane;
    int st, rr, ch;  // strip of the current row, row within it, chunk of the current column
    uint32_t cur[4], up[4], lf[4], ul[4];

    __device__ __forceinline__ void fetch(int bs, int bc, uint32_t (&w)[4]) const {
        const bool ok = bs >= 0 && bc >= 0;
        const uint32_t* src = bp + (ok ? ((size_t)bs * nchunk + bc) * wpb : 0);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            w[k] = (ok && lane + 32 * k < wpb) ? __ldg(src + lane + 32 * k) : 0u;
    }
    __device__ __forceinline__ void fetch_next() {
        fetch(st - 1, ch, up);
        fetch(st, ch - 1, lf);
        fetch(st - 1, ch - 1, ul);
    }
    // start at cell (i, j) (all lanes, warp-uniform arguments)
    __device__ __forceinline__ void start(int i, int j) {
        st = i / rps;
        rr = i - st * rps;
        ch = j >> 4;
        fetch(st, ch, cur);
        fetch_next();
    }
    // the 2-bit field of the current cell, whose column is j
    __device__ __forceinline__ uint32_t field(int j) const {
        const int slot = rr >> 5;
        const uint32_t mine =
            slot == 0 ? cur[0] : (slot == 1 ? cur[1] : (slot == 2 ? cur[2] : cur[3]));
        return (__shfl_sync(0xffffffffu, mine, rr & 31) >> (2 * (j & 15))) & 3u;
    }
    // the step to the cell di rows up whose column is j_new; the new
    // neighbours are loaded only if `more` (the walk goes on from there)
    __device__ __forceinline__ void step(int di, int j_new, bool more) {
        rr -= di;
        const bool su = rr < 0;               // into the strip above
        const bool sl = (j_new >> 4) != ch;   // into the chunk to the left
        if (su || sl) {                       // warp-uniform
#pragma unroll
            for (int k = 0; k < 4; ++k) cur[k] = su ? (sl ? ul[k] : up[k]) : lf[k];
            if (su) {
                rr += rps;
                --st;
            }
            if (sl) --ch;
            if (more) fetch_next();
        }
    }
};

// step_of_field as row and column moves: bit 0 -> (1,1); field 2 -> (1,2);
// field 0 -> (2,1).
__device__ __forceinline__ int field_di(uint32_t f) { return f == 0u ? 2 : 1; }
__device__ __forceinline__ int field_dj(uint32_t f) { return f == 2u ? 2 : 1; }

}  // namespace
}  // namespace pardtw
