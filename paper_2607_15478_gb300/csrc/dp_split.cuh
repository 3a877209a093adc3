// Exact DTW dynamic programming, warp-specialised: every strip of A has a
// DP warp and a cost warp, and every CTA of NS strips a reader and a writer
// warp for the border it shares with the neighbouring CTAs.  Same
// recurrence, step set, weights and tie order as the other DP kernels
// (Sec. V, Sec. II-D); only the division of labour differs.
//
//   - The strip geometry is that of the multi-row kernel: 31 R rows, lane t
//     (0..30) of the DP warp holds rows R t .. R t + R - 1 of the strip,
//     lane 31 is the ghost lane that carries the two bottom rows of the strip
//     above (cost 1e30, weight 0 on the (1,2) candidate fed the border value).
//   - The cost warp of the strip computes C' = (1 - mu) - a^_i . b^_j for the
//     same rows, 8 columns at a time (one FMA per feature, in feature order,
//     so the values are bit-identical to the other kernels'), reading the
//     frames of B from its TMA-fed ring, and hands them to the DP warp
//     through a ring of kCostSlots sub-chunks in shared memory with one
//     full and one empty mbarrier per slot.  The DP warp loads a
//     sub-chunk's costs at its start, before the eight steps.
//   - The DP warp runs only the recurrence: per column two shuffles, three
//     FMAs, a three-way minimum and two compares per cell.
//   - Every DP warp takes its top border from a ring of kRingBlk sub-chunks
//     in shared memory and writes its two bottom rows into the next ring,
//     with a full and an empty mbarrier per block.  The first strip's ring
//     is filled by the reader warp from the global border that the CTA
//     above publishes; the last strip's ring is drained by the writer warp
//     into this CTA's global border.  The L2 round trips of that exchange
//     thus never sit in a DP warp, and all DP warps do the same work per
//     sub-chunk (in a chain of strips the slowest one sets the pace).
//   - Every wait is bounded (DTW_ERR_TIMEOUT) and gives up when the call has
//     failed elsewhere.
#pragma once
#include "bandmap.cuh"
#include "dp_device.cuh"

// The kernel templates are included by dp_split.cu (two strips per CTA) and
// dp_split4.cu (four strips per CTA), which instantiate and launch them.
namespace pardtw {
namespace {

constexpr int kGhostLane = 31;
constexpr int kOutLane = 30;    // holds the strip's two bottom rows
constexpr int kCostSlots = 4;   // sub-chunks of costs in flight per strip
static_assert(kRingBlk >= 4, "the DP warp waits for output ring blocks four at a time");

// One slot holds the 8 costs of each of a lane's R rows: float4 q of lane l
// (q = 2 k + half) at [q][l], so a warp's 16-byte accesses are contiguous.
template <int R>
struct CostRing {
    static constexpr int kF4 = 2 * R;
    static constexpr int kSlotBytes = kF4 * kWarp * 16;
    static constexpr int kBytes = kCostSlots * kSlotBytes;
};

// BF16 cost: one cost slot holds the 8 costs of each of the 32 R rows of the
// strip row by row, kRowFloats floats per row (48-byte rows: the DP warp's
// 16-byte loads of rows 3l+k then fall in distinct bank groups).
constexpr int kRowFloats = 12;
template <int R>
struct CostRingRM {
    static constexpr int kSlotBytes = 32 * R * kRowFloats * 4;
    static constexpr int kBytes = kCostSlots * kSlotBytes;
};
// BF16 cost: the strip's rows of A as bf16 (32 R rows of kBfStride), and a
// ring of kBfSlots blocks of 16 frames of B (one chunk each) filled by TMA.
constexpr int kBfSlots = 4;
constexpr int kBfBlkBytes = kColsPerWord * kBfStride * 2;

// FP32 cost for D > 32 ("wide"): -a^ of the lane's R rows no longer fits in
// registers, so the strip's rows of A^ sit in shared memory (rows padded by 4
// floats: the 16-byte loads of rows 3l + k of a warp fall in distinct bank
// groups), and two cost warps share a strip, taking alternate sub-chunks
// (all 8 columns each).
template <int DP, bool kBF>
struct CostWide {
    static constexpr bool kOn = DP > 32 && !kBF;
    static constexpr int kNC = kOn ? 2 : 1;  // cost warps per strip
    static constexpr int kStride = DP + 4;   // floats per row of the A tile
    static constexpr int kBSlots = 2;        // chunks of B in each cost warp's ring
};
template <int DP, int R, bool kBF>
struct SplitSmem {
    // per strip slot: the cost warp's operands (B stage; A tile and B stage
    // for the BF16 cost; A tile for the wide FP32 cost), then the cost ring
    static constexpr int kOperandBytes =
        kBF ? 32 * R * kBfStride * 2 + kBfSlots * kBfBlkBytes
            : (CostWide<DP, kBF>::kOn
                   ? 32 * R * CostWide<DP, kBF>::kStride * 4 +
                         2 * BStage<DP, CostWide<DP, kBF>::kBSlots>::kWarpBytes
                   : BStage<DP>::kWarpBytes);
    static constexpr int kStripBytes =
        kOperandBytes + (kBF ? CostRingRM<R>::kBytes : CostRing<R>::kBytes);
};
// Threads of a CTA of NS strips: per strip the cost warp(s) and a DP warp,
// plus the reader and the writer.
template <int DP, int NS, bool kBF>
__host__ __device__ constexpr int split_threads() {
    return ((CostWide<DP, kBF>::kNC + 1) * NS + 2) * 32;
}

// Barrier `slot` of an array of 8-byte mbarriers, and the phase parity a
// waiter for the t-th (lifetime) use of a ring of n slots expects.
__device__ __forceinline__ unsigned bar_at(unsigned base, unsigned slot) { return base + 8 * slot; }
__device__ __forceinline__ unsigned use_parity(unsigned t, unsigned n) { return (t / n) & 1u; }

// Sub-chunks [x, y) (columns 8x .. 8y-1) that `strip` sweeps: all of them
// without a band, else the band's range of the strip.
__device__ __forceinline__ int2 strip_range(const DpArgs& p, int strip) {
    if (!p.ranges) return make_int2(0, (p.Lb + kSub - 1) / kSub);
    return p.ranges[strip];
}

// Cost warp of `strip`: all sub-chunks of the sweep, in order.
template <int DP, int R>
__device__ __forceinline__ void run_cost(const DpArgs& p, int strip, int lane, unsigned cring,
                                         unsigned cfull, unsigned cempty, unsigned csub,
                                         BRing<DP>& br) {
    using S = BStage<DP>;
    using CR = CostRing<R>;
    constexpr int kRows = 31 * R;
    constexpr int kFG = 4;            // features per group of loads
    constexpr int kNG = DP / kFG;     // DP is a multiple of 4
    const bool ghost = lane == kGhostLane;
    const int i0 = strip * kRows + lane * R;
    float na[R][DP];  // -a^_i of the lane's rows (0 in the ghost lane)
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const float4* s = reinterpret_cast<const float4*>(p.Ahat + (size_t)(i0 + k) * DP);
#pragma unroll
        for (int q = 0; q < DP / 4; ++q) {
            const float4 v = ghost ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldg(s + q);
            na[k][4 * q] = -v.x;
            na[k][4 * q + 1] = -v.y;
            na[k][4 * q + 2] = -v.z;
            na[k][4 * q + 3] = -v.w;
        }
    }
    const float kc = ghost ? kGhostCost : p.kcost;
    const int Lb_pad = p.nchunk * kColsPerWord;
    const int2 rg = strip_range(p, strip);  // sub-chunks rg.x .. rg.y-1
    const int q0 = rg.x * kSub / S::kBlk;
    br.begin(q0, min((rg.y * kSub + S::kBlk - 1) / S::kBlk, (Lb_pad + S::kBlk - 1) / S::kBlk));
    br.top_up(q0, p.Bhat, Lb_pad, lane);
    for (int n = rg.x; n < rg.y; ++n) {
        const int js = n * kSub;
        if (js % S::kBlk == 0 || n == rg.x) {
            const int q = js / S::kBlk;
            if (!br.wait(q, p.ctl, p.timeout_ns)) break;
            br.top_up(q, p.Bhat, Lb_pad, lane);
        }
        const unsigned t = csub + (unsigned)(n - rg.x);
        const unsigned slot = t % kCostSlots;
        // the DP warp has read this slot's previous contents
        if (!mbar_wait(bar_at(cempty, slot), use_parity(t, kCostSlots) ^ 1u, p.ctl, p.timeout_ns,
                       6))
            break;
        // the 8 frames of the sub-chunk, feature-major (16 floats per feature)
        const unsigned nb = br.chunk_s(js >> 4) + (unsigned)(js & kSub) * 4u;
        float c[R][kSub];
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int f = 0; f < kSub; ++f) c[k][f] = kc;
        // loads of the next feature group are issued before the FMAs of the
        // current one
        float4 bv[2][2 * kFG];
#pragma unroll
        for (int e = 0; e < kFG; ++e) {
            bv[0][2 * e] = lds128(nb + (unsigned)(e * kColsPerWord) * 4u);
            bv[0][2 * e + 1] = lds128(nb + (unsigned)(e * kColsPerWord + 4) * 4u);
        }
#pragma unroll
        for (int gi = 0; gi < kNG; ++gi) {
            if (gi + 1 < kNG) {
#pragma unroll
                for (int e = 0; e < kFG; ++e) {
                    const int d = (gi + 1) * kFG + e;
                    bv[(gi + 1) & 1][2 * e] = lds128(nb + (unsigned)(d * kColsPerWord) * 4u);
                    bv[(gi + 1) & 1][2 * e + 1] =
                        lds128(nb + (unsigned)(d * kColsPerWord + 4) * 4u);
                }
            }
#pragma unroll
            for (int e = 0; e < kFG; ++e) {
                const int d = gi * kFG + e;
                const float4 b0 = bv[gi & 1][2 * e], b1 = bv[gi & 1][2 * e + 1];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    c[k][0] = fmaf(na[k][d], b0.x, c[k][0]);
                    c[k][1] = fmaf(na[k][d], b0.y, c[k][1]);
                    c[k][2] = fmaf(na[k][d], b0.z, c[k][2]);
                    c[k][3] = fmaf(na[k][d], b0.w, c[k][3]);
                    c[k][4] = fmaf(na[k][d], b1.x, c[k][4]);
                    c[k][5] = fmaf(na[k][d], b1.y, c[k][5]);
                    c[k][6] = fmaf(na[k][d], b1.z, c[k][6]);
                    c[k][7] = fmaf(na[k][d], b1.w, c[k][7]);
                }
            }
        }
        const unsigned dst = cring + slot * CR::kSlotBytes + (unsigned)lane * 16u;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            sts128(dst + (unsigned)(2 * k) * (kWarp * 16),
                   make_float4(c[k][0], c[k][1], c[k][2], c[k][3]));
            sts128(dst + (unsigned)(2 * k + 1) * (kWarp * 16),
                   make_float4(c[k][4], c[k][5], c[k][6], c[k][7]));
        }
        mbar_arrive(bar_at(cfull, slot));
    }
    br.drain();
}

// Cost warp `half` (0 or 1) of `strip` for D > 32, FP32: every other
// sub-chunk of the strip (the (n - first)-th for n - first = half mod 2), all
// 8 columns, C' = (1 - mu) - a^_i . b^_j with one FMA per feature in feature
// order (the values of every other decomposition).  A^ of the strip comes
// from the A tile in shared memory (`tile`, 32 R rows of kStride floats),
// which the two cost warps of the strip load together at the strip's start
// (named barrier 1 + w), and is reused for 8 columns per load; B^ from the
// warp's own ring of two 16-frame chunks in shared memory, filled by bulk
// copies one chunk ahead (B^ through L1 instead ran at L2 latency, ~1100
// cycles per column; 4 columns per warp and sub-chunk, at 426).  A slot of
// the cost ring is written by one warp, as in the narrow kernel.
template <int DP, int R>
__device__ __forceinline__ void run_cost_wide(const DpArgs& p, int strip, int w, int half,
                                              int lane, float* tile, unsigned cring,
                                              unsigned cfull, unsigned cempty, unsigned csub,
                                              BRing<DP, CostWide<DP, false>::kBSlots>& br) {
    using W = CostWide<DP, false>;
    using S = BStage<DP, W::kBSlots>;
    using CR = CostRing<R>;
    constexpr int kRows = 31 * R;
    constexpr int kS = W::kStride;
    static_assert(S::kBlk == 2 * kSub, "one chunk of B per sub-chunk pair");
    const bool ghost = lane == kGhostLane;
    // the strip's rows of A^ (ghost rows zero) into the tile, 16 bytes a lane
    {
        const int tid = half * kWarp + lane;
        for (int e = tid; e < 32 * R * (DP / 4); e += 2 * kWarp) {
            const int r = e / (DP / 4), q = e - r * (DP / 4);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < kRows)
                v = __ldg(reinterpret_cast<const float4*>(p.Ahat + (size_t)(strip * kRows + r) * DP) + q);
            *reinterpret_cast<float4*>(tile + r * kS + 4 * q) = v;
        }
        asm volatile("bar.sync %0, %1;" ::"r"(1 + w), "r"(2 * kWarp) : "memory");
    }
    const float kc = ghost ? kGhostCost : p.kcost;
    const int Lb_pad = p.nchunk * kColsPerWord;
    const int2 rg = strip_range(p, strip);  // rg.x even: sub-chunk pairs are chunks
    const float* arow = tile + (lane * R) * kS;
    const int n0 = rg.x + half;
    const int q0 = n0 * kSub / S::kBlk;
    br.begin(q0, min((rg.y * kSub + S::kBlk - 1) / S::kBlk, (Lb_pad + S::kBlk - 1) / S::kBlk));
    br.top_up(q0, p.Bhat, Lb_pad, lane);
    for (int n = n0; n < rg.y; n += 2) {
        const int js = n * kSub;
        const int q = js / S::kBlk;
        if (!br.wait(q, p.ctl, p.timeout_ns)) break;
        br.top_up(q, p.Bhat, Lb_pad, lane);
        // feature d of the sub-chunk's 8 frames: 32 bytes at bsrc + 64 d
        const unsigned bsrc = br.chunk_s(js >> 4) + (unsigned)(js & 15) * 4u;
        const unsigned t = csub + (unsigned)(n - rg.x);
        const unsigned slot = t % kCostSlots;
        // the DP warp has read this slot's previous contents
        if (!mbar_wait(bar_at(cempty, slot), use_parity(t, kCostSlots) ^ 1u, p.ctl, p.timeout_ns,
                       6))
            break;
        // costs of columns 2q, 2q+1 of row k in c[k][q]: each paired FMA is
        // two FP32 FMAs, each rounded once (the values of one FMA per feature
        // in feature order), at half the instructions of scalar FMAs
        float2 c[R][kSub / 2];
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int q = 0; q < kSub / 2; ++q) c[k][q] = make_float2(kc, kc);
        // per group of 4 features: R rows of A^ (one 16-byte load each) and
        // the 8 frames of 4 features of B^ (two 16-byte loads each); two
        // buffers, the next group's loads issued before this group's FMAs
        float4 a0[R], b0[8], a1[R], b1[8];
        auto load = [&](int g, float4* a, float4* b) {
#pragma unroll
            for (int k = 0; k < R; ++k) a[k] = *reinterpret_cast<const float4*>(arow + k * kS + 4 * g);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                b[2 * e] = lds128(bsrc + (unsigned)(4 * g + e) * 64u);
                b[2 * e + 1] = lds128(bsrc + (unsigned)(4 * g + e) * 64u + 16u);
            }
        };
        auto fmas = [&](const float4* a, const float4* b) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float4 u = b[2 * e], v = b[2 * e + 1];
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    const float x = e == 0 ? a[k].x : (e == 1 ? a[k].y : (e == 2 ? a[k].z : a[k].w));
                    const float2 xx = make_float2(-x, -x);
                    c[k][0] = __ffma2_rn(xx, make_float2(u.x, u.y), c[k][0]);
                    c[k][1] = __ffma2_rn(xx, make_float2(u.z, u.w), c[k][1]);
                    c[k][2] = __ffma2_rn(xx, make_float2(v.x, v.y), c[k][2]);
                    c[k][3] = __ffma2_rn(xx, make_float2(v.z, v.w), c[k][3]);
                }
            }
        };
        // four groups a trip (measured on GB300, one warp alone: 4833 cycles
        // a sub-chunk at D = 128, against 5967 with scalar FMAs and two
        // groups a trip)
        static_assert((DP / 4) % 4 == 0, "whole trips of four feature groups");
        load(0, a0, b0);
#pragma unroll 1
        for (int g = 0; g < DP / 4; g += 4) {
            load(g + 1, a1, b1);
            fmas(a0, b0);
            load(g + 2, a0, b0);
            fmas(a1, b1);
            load(g + 3, a1, b1);
            fmas(a0, b0);
            if (g + 4 < DP / 4) load(g + 4, a0, b0);
            fmas(a1, b1);
        }
        const unsigned dst = cring + slot * CR::kSlotBytes + (unsigned)lane * 16u;
#pragma unroll
        for (int k = 0; k < R; ++k) {
            sts128(dst + (unsigned)(2 * k) * (kWarp * 16),
                   make_float4(c[k][0].x, c[k][0].y, c[k][1].x, c[k][1].y));
            sts128(dst + (unsigned)(2 * k + 1) * (kWarp * 16),
                   make_float4(c[k][2].x, c[k][2].y, c[k][3].x, c[k][3].y));
        }
        mbar_arrive(bar_at(cfull, slot));
    }
    br.drain();
}

__device__ __forceinline__ void ldsm_x4(unsigned addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                        uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr)
                 : "memory");
}
// d += a (16x16 bf16, row) * b (16x8 bf16, col), FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
        "{%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

// BF16 cost warp of `strip` (DP = K = 64 or 128, R = 3 rows per lane): per
// 16 columns one 96 x 16 x DP product on the tensor cores (6 x 2 tiles of
// m16n8k16 per 16 features), costs C' = (1 - mu) - dot written row-major into
// two cost slots; the ghost lane's rows get 1e30.  A's rows are converted to
// bf16 into shared memory once per strip; B's bf16 frames arrive by TMA, one
// chunk per block.
template <int DP, int R>
__device__ __forceinline__ void run_cost_bf16(const DpArgs& p, int strip, int lane, unsigned a_s,
                                              unsigned b_s, unsigned bbar_s, unsigned& bbase,
                                              unsigned cring, unsigned cfull, unsigned cempty,
                                              unsigned csub) {
    constexpr int kRows = 31 * R;       // real rows of the strip
    constexpr int kM = 32 * R;          // rows of the product (6 tiles of 16)
    constexpr int kMT = kM / 16;
    constexpr int kKS = DP / 16;        // k-steps of 16 features
    constexpr int kRowBytes = kBfStride * 2;
    const int2 rg = strip_range(p, strip);  // sub-chunks rg.x (even) .. rg.y-1
    const int c_lo = rg.x / 2, c_hi = (rg.y + 1) / 2;
    const int nsub = rg.y;
    // A: rows r = 0 .. kM-1 of the strip as bf16 (rows >= kRows are zero)
    for (int r = lane; r < kM; r += kWarp) {
        const float* src = p.Ahat + (size_t)(strip * kRows + r) * DP;
#pragma unroll 4
        for (int d = 0; d < DP; d += 8) {
            float4 v0 = make_float4(0.f, 0.f, 0.f, 0.f), v1 = v0;
            if (r < kRows) {
                v0 = __ldg(reinterpret_cast<const float4*>(src + d));
                v1 = __ldg(reinterpret_cast<const float4*>(src + d + 4));
            }
            const uint32_t w0 = pack_bf16x2(v0.x, v0.y), w1 = pack_bf16x2(v0.z, v0.w);
            const uint32_t w2 = pack_bf16x2(v1.x, v1.y), w3 = pack_bf16x2(v1.z, v1.w);
            asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(
                             a_s + (unsigned)(r * kRowBytes + d * 2)),
                         "r"(w0), "r"(w1), "r"(w2), "r"(w3)
                         : "memory");
        }
    }
    __syncwarp();
    const char* gb = static_cast<const char*>(p.Bbf);
    int issued = c_lo, waited = c_lo;
    auto issue = [&](int c) {  // lane 0: chunk c of B into slot (bbase + c - c_lo) % kBfSlots
        if (lane == 0) {
            const unsigned t = bbase + (unsigned)(c - c_lo);
            tma_load(b_s + (t % kBfSlots) * kBfBlkBytes, gb + (size_t)c * kBfBlkBytes,
                     (unsigned)kBfBlkBytes, bbar_s + 8 * (t % kBfSlots));
        }
    };
    while (issued < c_hi && issued < c_lo + kBfSlots - 1) issue(issued++);
    const float kc = p.kcost;
    const int g = lane >> 2, t4 = lane & 3;
    bool ok = true;
    for (int c = c_lo; c < c_hi && ok; ++c) {
        // chunk c of B is in its slot
        const unsigned tb = bbase + (unsigned)(c - c_lo);
        if (!mbar_wait(bbar_s + 8 * (tb % kBfSlots), (tb / kBfSlots) & 1u, p.ctl, p.timeout_ns,
                       4)) {
            ok = false;
            break;
        }
        waited = c + 1;
        if (issued < c_hi) issue(issued++);
        const int nj = (2 * c + 1 < nsub) ? 2 : 1;  // sub-chunks of this chunk
        const unsigned t0 = csub + (unsigned)(2 * c - rg.x);
        for (int j = 0; j < nj; ++j)
            if (!mbar_wait(bar_at(cempty, (t0 + j) % kCostSlots),
                           use_parity(t0 + j, kCostSlots) ^ 1u, p.ctl, p.timeout_ns, 6)) {
                ok = false;
                break;
            }
        if (!ok) break;
        // B fragments of the chunk's 16 frames: n-tile j = frames 8j .. 8j+7
        const unsigned bslot = b_s + (tb % kBfSlots) * kBfBlkBytes;
        uint32_t bf[2][kKS][2];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int kq = 0; kq < kKS / 2; ++kq)
                ldsm_x4(bslot + (unsigned)((8 * j + (lane & 7)) * kRowBytes +
                                           (32 * kq + 8 * (lane >> 3)) * 2),
                        bf[j][2 * kq][0], bf[j][2 * kq][1], bf[j][2 * kq + 1][0],
                        bf[j][2 * kq + 1][1]);
        float acc[kMT][2][4];
#pragma unroll
        for (int mt = 0; mt < kMT; ++mt)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mt][j][e] = 0.f;
#pragma unroll
        for (int mt = 0; mt < kMT; ++mt)
#pragma unroll
            for (int ks = 0; ks < kKS; ++ks) {
                uint32_t a[4];
                ldsm_x4(a_s + (unsigned)((16 * mt + (lane & 7) + 8 * ((lane >> 3) & 1)) *
                                             kRowBytes +
                                         (16 * ks + 8 * (lane >> 4)) * 2),
                        a[0], a[1], a[2], a[3]);
                mma_bf16(acc[mt][0], a, bf[0][ks]);
                mma_bf16(acc[mt][1], a, bf[1][ks]);
            }
        // costs into the two slots: rows 16 mt + g (+8), columns 2 t4, 2 t4 + 1
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (j >= nj) break;
            const unsigned slot = cring + ((t0 + j) % kCostSlots) * CostRingRM<R>::kSlotBytes;
#pragma unroll
            for (int mt = 0; mt < kMT; ++mt) {
                const int r0 = 16 * mt + g, r1 = r0 + 8;
                const float v00 = r0 < kRows ? kc - acc[mt][j][0] : kGhostCost;
                const float v01 = r0 < kRows ? kc - acc[mt][j][1] : kGhostCost;
                const float v10 = r1 < kRows ? kc - acc[mt][j][2] : kGhostCost;
                const float v11 = r1 < kRows ? kc - acc[mt][j][3] : kGhostCost;
                asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(
                                 slot + (unsigned)(r0 * kRowFloats * 4 + t4 * 8)),
                             "f"(v00), "f"(v01)
                             : "memory");
                asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(
                                 slot + (unsigned)(r1 * kRowFloats * 4 + t4 * 8)),
                             "f"(v10), "f"(v11)
                             : "memory");
            }
            mbar_arrive(bar_at(cfull, (t0 + j) % kCostSlots));
        }
    }
    // leave no copy in flight (bounded)
    for (int c = waited; c < issued; ++c) {
        const unsigned tb = bbase + (unsigned)(c - c_lo);
        const long long t0 = __shfl_sync(kFull, global_ns(), 0);
        while (!__all_sync(kFull, mbar_try_wait(bbar_s + 8 * (tb % kBfSlots),
                                                (tb / kBfSlots) & 1u))) {
            if (__shfl_sync(kFull, global_ns(), 0) - t0 > 1000000000LL) break;
        }
    }
    bbase += (unsigned)(issued - c_lo);
}

// The costs of lifetime sub-chunk t (its slot must be full) into c;
// kRM: the row-major slot of the BF16 cost.
template <int R, bool kRM>
__device__ __forceinline__ void load_costs(unsigned cring, unsigned t, int lane,
                                           float (*c)[kSub]) {
    if constexpr (kRM) {
        const unsigned src = cring + (t % kCostSlots) * CostRingRM<R>::kSlotBytes +
                             (unsigned)(lane * R) * (kRowFloats * 4);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const float4 v0 = lds128(src + (unsigned)k * (kRowFloats * 4));
            const float4 v1 = lds128(src + (unsigned)k * (kRowFloats * 4) + 16);
            c[k][0] = v0.x;
            c[k][1] = v0.y;
            c[k][2] = v0.z;
            c[k][3] = v0.w;
            c[k][4] = v1.x;
            c[k][5] = v1.y;
            c[k][6] = v1.z;
            c[k][7] = v1.w;
        }
        return;
    }
    using CR = CostRing<R>;
    const unsigned src = cring + (t % kCostSlots) * CR::kSlotBytes + (unsigned)lane * 16u;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const float4 v0 = lds128(src + (unsigned)(2 * k) * (kWarp * 16));
        const float4 v1 = lds128(src + (unsigned)(2 * k + 1) * (kWarp * 16));
        c[k][0] = v0.x;
        c[k][1] = v0.y;
        c[k][2] = v0.z;
        c[k][3] = v0.w;
        c[k][4] = v1.x;
        c[k][5] = v1.y;
        c[k][6] = v1.z;
        c[k][7] = v1.w;
    }
}

// Which rings of a CTA a strip group uses: ring w < NS feeds DP slot w (ring
// 0 from the reader warp, which has nothing to read in group 0; ring w >= 1
// from DP slot w-1, when strip w exists); ring NS takes the last DP slot's
// bottom rows to the writer warp, when a group below needs them.  Producer
// and consumer of a ring count its uses (in sub-chunks) the same way, which
// keeps every barrier's phase in step across groups.
struct GroupRoles {
    int g, nstrips_here;
    bool reader, writer;
};
template <int NS>
__device__ __forceinline__ GroupRoles group_roles(const DpArgs& p, int g) {
    GroupRoles r;
    r.g = g;
    r.nstrips_here = min(NS, p.nstrips - g * NS);
    r.reader = g > 0;
    r.writer = (g + 1 < p.ngroups) && (g != p.skip_publish);
    return r;
}
template <int NS>
__device__ __forceinline__ bool ring_used(const GroupRoles& r, int w) {
    if (w == 0) return r.reader;
    if (w < NS) return w < r.nstrips_here;
    return r.writer;
}

// cur[k] for a runtime k < R without indexing the register array.
template <int R>
__device__ __forceinline__ float pick_row(const float* cur, int k) {
    float v = cur[0];
#pragma unroll
    for (int q = 1; q < R; ++q) v = (k == q) ? cur[q] : v;
    return v;
}

// The two border rows of a ring block (8 columns each) into registers.
__device__ __forceinline__ void load_border(unsigned s, float* g0, float* g1) {
    const float4 a0 = lds128(s), a1 = lds128(s + 16);
    const float4 b0 = lds128(s + 32), b1 = lds128(s + 48);
    g0[0] = a0.x; g0[1] = a0.y; g0[2] = a0.z; g0[3] = a0.w;
    g0[4] = a1.x; g0[5] = a1.y; g0[6] = a1.z; g0[7] = a1.w;
    g1[0] = b0.x; g1[1] = b0.y; g1[2] = b0.z; g1[3] = b0.w;
    g1[4] = b1.x; g1[5] = b1.y; g1[6] = b1.z; g1[7] = b1.w;
}
// The strip's two bottom rows of a sub-chunk into a ring block.
__device__ __forceinline__ void store_border(unsigned d, const float* o0, const float* o1) {
    sts128(d, make_float4(o0[0], o0[1], o0[2], o0[3]));
    sts128(d + 16, make_float4(o0[4], o0[5], o0[6], o0[7]));
    sts128(d + 32, make_float4(o1[0], o1[1], o1[2], o1[3]));
    sts128(d + 48, make_float4(o1[4], o1[5], o1[6], o1[7]));
}
// Subsequence DP: row La-1 of the nsteps columns at dst.
__device__ __forceinline__ void store_lastrow(float* dst, int nsteps, const float* ol) {
    if (nsteps == kSub) {
        reinterpret_cast<float4*>(dst)[0] = make_float4(ol[0], ol[1], ol[2], ol[3]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(ol[4], ol[5], ol[6], ol[7]);
    } else {
#pragma unroll
        for (int u = 0; u < kSub; ++u)
            if (u < nsteps) dst[u] = ol[u];
    }
}
// The 8 DP steps of a full sub-chunk.
template <int R, bool kSubseq, bool kT>
__device__ __forceinline__ void sweep_full(const float (*c)[kSub], const float* g0, const float* g1,
                                           bool first_col, bool is_origin, int srcA,
                                           const float* w12, bool ghost, float mu, float* cur,
                                           float* prv, float& ylp, float* fw, float* o0, float* o1,
                                           float* ol, int kl) {
#pragma unroll
    for (int u = 0; u < kSub; ++u) {
        float cu[R];
#pragma unroll
        for (int k = 0; k < R; ++k) cu[k] = c[k][u];
        dp_step<R, kSubseq, kT>(cu, u, srcA, w12, ghost, g0[u], g1[u],
                                (kSubseq || (first_col && u == 0)) && is_origin, mu, cur, prv, ylp,
                                fw, o0[u], o1[u]);
        if constexpr (kSubseq) ol[u] = pick_row<R>(cur, kl);
    }
}

// The DP steps of one sub-chunk (nsteps <= 8 columns; the cell of the first
// column of the sweep is the origin when first_col and is_origin hold).
template <int R, bool kSubseq, bool kT>
__device__ __forceinline__ void sweep_sub(const float (*c)[kSub], const float* g0, const float* g1,
                                          int nsteps, bool first_col, bool is_origin, int srcA,
                                          const float* w12, bool ghost, float mu, float* cur,
                                          float* prv, float& ylp, float* fw, float* o0, float* o1,
                                          float* ol, int kl) {
    if (nsteps == kSub) {
#pragma unroll
        for (int u = 0; u < kSub; ++u) {
            float cu[R];
#pragma unroll
            for (int k = 0; k < R; ++k) cu[k] = c[k][u];
            dp_step<R, kSubseq, kT>(cu, u, srcA, w12, ghost, g0[u], g1[u],
                                    (kSubseq || (first_col && u == 0)) && is_origin, mu, cur, prv,
                                    ylp, fw, o0[u], o1[u]);
            if constexpr (kSubseq) ol[u] = pick_row<R>(cur, kl);
        }
    } else {
#pragma unroll
        for (int u = 0; u < kSub; ++u) {
            if (u >= nsteps) break;
            float cu[R];
#pragma unroll
            for (int k = 0; k < R; ++k) cu[k] = c[k][u];
            dp_step<R, kSubseq, kT>(cu, u, srcA, w12, ghost, g0[u], g1[u],
                                    (kSubseq || (first_col && u == 0)) && is_origin, mu, cur, prv,
                                    ylp, fw, o0[u], o1[u]);
            if constexpr (kSubseq) ol[u] = pick_row<R>(cur, kl);
        }
    }
}

// DP warp of `strip` (slot w of group g).  ring: the NS + 1 border rings;
// bfull / bempty: their mbarriers (kRingBlk per ring); rin / rout: lifetime
// sub-chunk counts of the input and output rings at the start of this
// group; csub: that of the cost ring.
// kFlag: the strip raises its flag in done[strip] when its words are stored
// (one pair with the band map inside the kernel).
// kWords: a trip of the sweep takes a whole backpointer word (two sub-chunks,
// one set of barrier tests, loads and arrivals for 16 columns) instead of
// one sub-chunk; kTwoCost: two cost warps fill alternate cost slots.  Taken
// where the DP warp alone sets the pace (BF16 cost: 12% faster at D = 128)
// and not for the FP32 cost at D <= 32, where the trip of a sub-chunk was
// faster on GB300 (the strip below waits for a whole word of the border, and
// the per-column work did not shrink).
template <int R, int NS, bool kRM, bool kSubseq = false, bool kT = false, bool kFlag = false,
          bool kWords = false, bool kTwoCost = false>
__device__ __forceinline__ void run_dp(const DpArgs& p, const GroupRoles& gr, int w, int strip,
                                       int lane, float (*ring)[kRingBlk][2][kSub], unsigned bfull,
                                       unsigned bempty, unsigned rin, unsigned rout,
                                       unsigned cring, unsigned cfull, unsigned cempty,
                                       unsigned csub,
                                       unsigned inf_blk, unsigned* done = nullptr) {
    constexpr int kRows = 31 * R;
    const bool ghost = lane == kGhostLane;
    const int i0 = strip * kRows + lane * R;
    const int Lb = p.Lb;
    const bool from_ring = ring_used<NS>(gr, w);
    const bool to_ring = ring_used<NS>(gr, w + 1);
    float (*myring)[2][kSub] = ring[w];
    float (*nextring)[2][kSub] = ring[w + 1];
    const unsigned bfull_in = bfull + 8 * kRingBlk * w;
    const unsigned bempty_in = bempty + 8 * kRingBlk * w;
    const unsigned bfull_out = bfull + 8 * kRingBlk * (w + 1);
    const unsigned bempty_out = bempty + 8 * kRingBlk * (w + 1);
    const float mu = p.mu;
    float w12[R];
#pragma unroll
    for (int k = 0; k < R; ++k) w12[k] = (ghost && k >= R - 2) ? 0.0f : (kSubseq ? 1.0f : 3.0f);
    const int srcA = (lane + 31) & 31;
    const bool is_origin = (i0 == 0) && !ghost;
    // subsequence DP: the lane and row slot of row La-1, if this strip holds it
    const int rl = p.La - 1 - strip * kRows;
    const bool has_last = kSubseq && rl >= 0 && rl < kRows && lane == rl / R;
    const int kl = kSubseq ? rl - (rl / R) * R : 0;
    // this strip's sub-chunks, and those its border ring's producer publishes
    // (the strip above; for the first strip of a group the reader, which
    // publishes exactly this strip's range)
    const int2 rg = strip_range(p, strip);
    const int2 rp = w > 0 ? strip_range(p, strip - 1) : rg;
    // blocks the strip above published before this strip's first column are
    // consumed unread, so that the ring's producer and consumer stay in step
    if (from_ring)
        for (int n = rp.x; n < rg.x; ++n) {
            const unsigned ti = rin + (unsigned)(n - rp.x);
            if (!mbar_wait(bar_at(bfull_in, ti % kRingBlk), use_parity(ti, kRingBlk), p.ctl,
                           p.timeout_ns, 1))
                return;
            mbar_arrive(bar_at(bempty_in, ti % kRingBlk));
        }

    float cur[R], prv[R];
#pragma unroll
    for (int k = 0; k < R; ++k) cur[k] = prv[k] = INFINITY;
    float ylp = INFINITY;
    // (no poll of the failure flag in the sweep: every wait checks it on its
    // slow path, and a warp that never waits ends with its strip)
    if constexpr (kWords) {
        const int jend = min(rg.y * kSub, Lb);
        // whole words first (16 full columns), then the last, ragged word
        uint32_t tailw[R];
        const int jfull = rg.x * kSub + ((jend - rg.x * kSub) / kColsPerWord) * kColsPerWord;
        for (int j0 = rg.x * kSub; j0 < jfull; j0 += kColsPerWord) {
            // One backpointer word per trip: sub-chunks n (even; ranges start on
            // whole words) and n + 1.
            const int n = j0 / kSub;
            const unsigned ti = rin + (unsigned)(n - rp.x), to = rout + (unsigned)(n - rg.x);
            const unsigned t = csub + (unsigned)(n - rg.x);
            const bool in0 = from_ring && n < rp.y;
            const bool in1 = from_ring && n + 1 < rp.y;

            // The waits of the word, first tested together without blocking: the
            // border blocks from the ring above (the producer publishes them in
            // order, so the second one's barrier implies the first's; columns the
            // strip above did not sweep are +inf), every other word the output
            // ring (its consumer empties it in order, so once the previous use of
            // block to+3 is consumed so are those of to .. to+2), and the cost
            // slots (filled in order by one cost warp; with two cost warps, which
            // take alternate slots, both are tested).
            const bool need_out = to_ring && ((n - rg.x) & 3) == 0;
            const unsigned tl = to + 3u, tb = in1 ? ti + 1u : ti, tc = t + 1u;
            const int rb = in0 ? mbar_test_wait(bar_at(bfull_in, tb % kRingBlk),
                                                 use_parity(tb, kRingBlk))
                               : 1;
            const int ro = need_out ? mbar_test_wait(bar_at(bempty_out, tl % kRingBlk),
                                                     use_parity(tl, kRingBlk) ^ 1u)
                                    : 1;
            const int rc = mbar_test_wait(bar_at(cfull, tc % kCostSlots), use_parity(tc, kCostSlots));
            const int rc0 = kTwoCost ? mbar_test_wait(bar_at(cfull, t % kCostSlots),
                                                      use_parity(t, kCostSlots))
                                     : 1;
            if (!__all_sync(kFull, rb) &&
                !mbar_wait_slow(bar_at(bfull_in, tb % kRingBlk), use_parity(tb, kRingBlk), p.ctl,
                                p.timeout_ns, 1))
                return;
            if (!__all_sync(kFull, ro) &&
                !mbar_wait_slow(bar_at(bempty_out, tl % kRingBlk), use_parity(tl, kRingBlk) ^ 1u,
                                p.ctl, p.timeout_ns, 2))
                return;
            if (!__all_sync(kFull, rc) &&
                !mbar_wait_slow(bar_at(cfull, tc % kCostSlots), use_parity(tc, kCostSlots), p.ctl,
                                p.timeout_ns, 7))
                return;
            if (kTwoCost && !__all_sync(kFull, rc0) &&
                !mbar_wait_slow(bar_at(cfull, t % kCostSlots), use_parity(t, kCostSlots), p.ctl,
                                p.timeout_ns, 7))
                return;
            float gA0[kSub], gA1[kSub], gB0[kSub], gB1[kSub];
            load_border(in0 ? smem_u32(&myring[ti % kRingBlk][0][0]) : inf_blk, gA0, gA1);
            load_border(in1 ? smem_u32(&myring[(ti + 1u) % kRingBlk][0][0]) : inf_blk, gB0, gB1);
            float cA[R][kSub], cB[R][kSub];
            load_costs<R, kRM>(cring, t, lane, cA);
            load_costs<R, kRM>(cring, t + 1u, lane, cB);
            if (in0) mbar_arrive(bar_at(bempty_in, ti % kRingBlk));
            if (in1) mbar_arrive(bar_at(bempty_in, (ti + 1u) % kRingBlk));
            mbar_arrive(bar_at(cempty, t % kCostSlots));
            mbar_arrive(bar_at(cempty, (t + 1u) % kCostSlots));

            float o0[kSub], o1[kSub];  // the strip's two bottom rows (lane 30)
            float ol[kSub];            // subsequence DP: row La-1 (lane of has_last)
            (void)ol;
            float fw[R];  // backpointer fields of a sub-chunk, bits 2u, 2u+1
            uint32_t word[R];
#pragma unroll
            for (int k = 0; k < R; ++k) fw[k] = 0.0f;
            sweep_full<R, kSubseq, kT>(cA, gA0, gA1, j0 == 0, is_origin, srcA, w12, ghost, mu, cur,
                                       prv, ylp, fw, o0, o1, ol, kl);
            if constexpr (kSubseq)
                if (has_last) store_lastrow(p.lastrow + j0, kSub, ol);
#pragma unroll
            for (int k = 0; k < R; ++k) word[k] = field_bits(fw[k], 0);
            if (to_ring && lane == kOutLane) {
                store_border(smem_u32(&nextring[to % kRingBlk][0][0]), o0, o1);
                mbar_arrive(bar_at(bfull_out, to % kRingBlk));
            }
#pragma unroll
            for (int k = 0; k < R; ++k) fw[k] = 0.0f;
            sweep_full<R, kSubseq, kT>(cB, gB0, gB1, false, is_origin, srcA, w12, ghost, mu, cur,
                                       prv, ylp, fw, o0, o1, ol, kl);
            if constexpr (kSubseq)
                if (has_last) store_lastrow(p.lastrow + j0 + kSub, kSub, ol);
#pragma unroll
            for (int k = 0; k < R; ++k) word[k] |= field_bits(fw[k], 1);
            if (to_ring && lane == kOutLane) {
                store_border(smem_u32(&nextring[(to + 1u) % kRingBlk][0][0]), o0, o1);
                mbar_arrive(bar_at(bfull_out, (to + 1u) % kRingBlk));
            }
            if constexpr (kT) {
#pragma unroll
                for (int k = 0; k < R; ++k) word[k] = transpose_fields(word[k]);
            }
            store_words<R>(p.bp + ((size_t)strip * p.nchunk + (size_t)(j0 >> 4)) * (32 * R) +
                               (size_t)lane * R,
                           word);
        }
        // the last, ragged word: its one or two sub-chunks one at a time
        for (int js = jfull; js < jend; js += kSub) {
            const int n = js / kSub;
            const int nsteps = min(kSub, Lb - js);
            const unsigned ti = rin + (unsigned)(n - rp.x), to = rout + (unsigned)(n - rg.x);
            const unsigned t = csub + (unsigned)(n - rg.x);
            const bool have_in = from_ring && n < rp.y;
            const bool need_out = to_ring && ((n - rg.x) & 3) == 0;
            const unsigned tl = to + 3u;
            if (have_in && !mbar_wait(bar_at(bfull_in, ti % kRingBlk), use_parity(ti, kRingBlk), p.ctl,
                                      p.timeout_ns, 1))
                return;
            if (need_out && !mbar_wait(bar_at(bempty_out, tl % kRingBlk),
                                       use_parity(tl, kRingBlk) ^ 1u, p.ctl, p.timeout_ns, 2))
                return;
            if (!mbar_wait(bar_at(cfull, t % kCostSlots), use_parity(t, kCostSlots), p.ctl,
                           p.timeout_ns, 7))
                return;
            float g0[kSub], g1[kSub], c[R][kSub];
            load_border(have_in ? smem_u32(&myring[ti % kRingBlk][0][0]) : inf_blk, g0, g1);
            load_costs<R, kRM>(cring, t, lane, c);
            if (have_in) mbar_arrive(bar_at(bempty_in, ti % kRingBlk));
            mbar_arrive(bar_at(cempty, t % kCostSlots));
            float o0[kSub], o1[kSub], ol[kSub], fw[R];
            (void)ol;
#pragma unroll
            for (int k = 0; k < R; ++k) fw[k] = 0.0f;
            sweep_sub<R, kSubseq, kT>(c, g0, g1, nsteps, js == 0, is_origin, srcA, w12, ghost, mu, cur,
                                      prv, ylp, fw, o0, o1, ol, kl);
            if constexpr (kSubseq)
                if (has_last) store_lastrow(p.lastrow + js, nsteps, ol);
            if (to_ring && lane == kOutLane) {
                store_border(smem_u32(&nextring[to % kRingBlk][0][0]), o0, o1);
                mbar_arrive(bar_at(bfull_out, to % kRingBlk));
            }
            // the word's fields: the first sub-chunk's are the low half
            const int h = (js / kSub) & 1;
            uint32_t word[R];
#pragma unroll
            for (int k = 0; k < R; ++k) word[k] = field_bits(fw[k], h);
            if (h == 0) {
                // keep the low half for the second sub-chunk, if there is one
                if (js + kSub < jend) {
#pragma unroll
                    for (int k = 0; k < R; ++k) tailw[k] = word[k];
                    continue;
                }
            } else {
#pragma unroll
                for (int k = 0; k < R; ++k) word[k] |= tailw[k];
            }
            if constexpr (kT) {
#pragma unroll
                for (int k = 0; k < R; ++k) word[k] = transpose_fields(word[k]);
            }
            store_words<R>(p.bp + ((size_t)strip * p.nchunk + (size_t)(js >> 4)) * (32 * R) +
                               (size_t)lane * R,
                           word);
        }
    } else {
        // costs of the first sub-chunk
        float c[R][kSub];
        if (!mbar_wait(bar_at(cfull, csub % kCostSlots), use_parity(csub, kCostSlots), p.ctl,
                       p.timeout_ns, 7))
            return;
        load_costs<R, kRM>(cring, csub, lane, c);
        mbar_arrive(bar_at(cempty, csub % kCostSlots));

        const int jend = min(rg.y * kSub, Lb);
        for (int j0 = rg.x * kSub; j0 < jend; j0 += kColsPerWord) {
            uint32_t word[R];
#pragma unroll
            for (int k = 0; k < R; ++k) word[k] = 0;
            // the two sub-chunks of a backpointer word: not unrolled (half the
            // code of the sweep loop; measured 4-5% faster on a long pair)
#pragma unroll 1
            for (int h = 0; h < kColsPerWord / kSub; ++h) {
                const int js = j0 + h * kSub;
                if (js >= jend) break;
                const int n = js / kSub;
                const int nsteps = min(kSub, Lb - js);
                const unsigned ti = rin + (unsigned)(n - rp.x), to = rout + (unsigned)(n - rg.x);
                const unsigned t = csub + (unsigned)(n - rg.x);

                // The three waits of a sub-chunk -- the border rows top-2, top-1
                // of columns js .. js+7 from the ring above (the group's top
                // border is +inf in group 0, and so are the columns the strip
                // above did not sweep: the +inf block inf_blk), every 4 blocks the
                // output ring (the consumer empties it in order, so once the
                // previous use of block to+3 is consumed so are those of to ..
                // to+2), and the costs (the cost warp runs up to kCostSlots
                // sub-chunks ahead, so they are normally there) -- are first
                // tested together without blocking, so that their latencies
                // overlap; only a barrier not yet complete is waited for.
                const bool have_in = from_ring && n < rp.y;
                const bool need_out = to_ring && ((n - rg.x) & 3) == 0;
                const bool need_cost = n > rg.x;
                const unsigned tl = to + 3u;
                const int rb = have_in ? mbar_test_wait(bar_at(bfull_in, ti % kRingBlk),
                                                        use_parity(ti, kRingBlk))
                                       : 1;
                const int ro = need_out ? mbar_test_wait(bar_at(bempty_out, tl % kRingBlk),
                                                         use_parity(tl, kRingBlk) ^ 1u)
                                        : 1;
                const int rc = need_cost ? mbar_test_wait(bar_at(cfull, t % kCostSlots),
                                                          use_parity(t, kCostSlots))
                                         : 1;
                if (!__all_sync(kFull, rb) &&
                    !mbar_wait_slow(bar_at(bfull_in, ti % kRingBlk), use_parity(ti, kRingBlk), p.ctl,
                                    p.timeout_ns, 1))
                    return;
                if (!__all_sync(kFull, ro) &&
                    !mbar_wait_slow(bar_at(bempty_out, tl % kRingBlk), use_parity(tl, kRingBlk) ^ 1u,
                                    p.ctl, p.timeout_ns, 2))
                    return;
                if (!__all_sync(kFull, rc) &&
                    !mbar_wait_slow(bar_at(cfull, t % kCostSlots), use_parity(t, kCostSlots), p.ctl,
                                    p.timeout_ns, 7))
                    return;
                float gv0[kSub], gv1[kSub];
                {
                    const unsigned s0 = have_in ? smem_u32(&myring[ti % kRingBlk][0][0]) : inf_blk;
                    const float4 a0 = lds128(s0), a1 = lds128(s0 + 16);
                    const float4 b0 = lds128(s0 + 32), b1 = lds128(s0 + 48);
                    gv0[0] = a0.x; gv0[1] = a0.y; gv0[2] = a0.z; gv0[3] = a0.w;
                    gv0[4] = a1.x; gv0[5] = a1.y; gv0[6] = a1.z; gv0[7] = a1.w;
                    gv1[0] = b0.x; gv1[1] = b0.y; gv1[2] = b0.z; gv1[3] = b0.w;
                    gv1[4] = b1.x; gv1[5] = b1.y; gv1[6] = b1.z; gv1[7] = b1.w;
                }
                // this sub-chunk's costs (loaded here rather than half-way through
                // the previous sub-chunk keeps the 8 steps below one straight-line
                // block: measured 8% faster)
                if (need_cost) load_costs<R, kRM>(cring, t, lane, c);
                if (have_in) mbar_arrive(bar_at(bempty_in, ti % kRingBlk));
                if (need_cost) mbar_arrive(bar_at(cempty, t % kCostSlots));
                float o0[kSub], o1[kSub];  // the strip's two bottom rows (lane 30)
                float ol[kSub];            // subsequence DP: row La-1 (lane of has_last)
                (void)ol;
                float fw[R];  // backpointer fields of the sub-chunk, bits 2u, 2u+1
#pragma unroll
                for (int k = 0; k < R; ++k) fw[k] = 0.0f;
                if (nsteps == kSub) {
#pragma unroll
                    for (int u = 0; u < kSub; ++u) {
                        float cu[R];
#pragma unroll
                        for (int k = 0; k < R; ++k) cu[k] = c[k][u];
                        dp_step<R, kSubseq, kT>(cu, u, srcA, w12, ghost, gv0[u], gv1[u],
                                            (kSubseq || ((h == 0) && (u == 0) && (j0 == 0))) &&
                                                is_origin,
                                            mu, cur, prv, ylp, fw, o0[u], o1[u]);
                        if constexpr (kSubseq) ol[u] = pick_row<R>(cur, kl);
                    }
                } else {
                    // the last, partial sub-chunk
#pragma unroll
                    for (int u = 0; u < kSub; ++u) {
                        if (u >= nsteps) break;
                        float cu[R];
#pragma unroll
                        for (int k = 0; k < R; ++k) cu[k] = c[k][u];
                        dp_step<R, kSubseq, kT>(cu, u, srcA, w12, ghost, gv0[u], gv1[u],
                                            (kSubseq || ((h == 0) && (u == 0) && (j0 == 0))) &&
                                                is_origin,
                                            mu, cur, prv, ylp, fw, o0[u], o1[u]);
                        if constexpr (kSubseq) ol[u] = pick_row<R>(cur, kl);
                    }
                }
                if constexpr (kSubseq) {
                    if (has_last) {  // row La-1 of these columns
                        float* dst = p.lastrow + js;
                        if (nsteps == kSub) {
                            reinterpret_cast<float4*>(dst)[0] = make_float4(ol[0], ol[1], ol[2], ol[3]);
                            reinterpret_cast<float4*>(dst)[1] = make_float4(ol[4], ol[5], ol[6], ol[7]);
                        } else {
#pragma unroll
                            for (int u = 0; u < kSub; ++u)
                                if (u < nsteps) dst[u] = ol[u];
                        }
                    }
                }
#pragma unroll
                for (int k = 0; k < R; ++k) word[k] |= field_bits(fw[k], h);
                if (to_ring && lane == kOutLane) {
                    const unsigned d0 = smem_u32(&nextring[to % kRingBlk][0][0]);
                    sts128(d0, make_float4(o0[0], o0[1], o0[2], o0[3]));
                    sts128(d0 + 16, make_float4(o0[4], o0[5], o0[6], o0[7]));
                    sts128(d0 + 32, make_float4(o1[0], o1[1], o1[2], o1[3]));
                    sts128(d0 + 48, make_float4(o1[4], o1[5], o1[6], o1[7]));
                    mbar_arrive(bar_at(bfull_out, to % kRingBlk));
                }

            }
            if constexpr (kT) {
#pragma unroll
                for (int k = 0; k < R; ++k) word[k] = transpose_fields(word[k]);
            }
            store_words<R>(p.bp + ((size_t)strip * p.nchunk + (size_t)(j0 >> 4)) * (32 * R) +
                               (size_t)lane * R,
                           word);
        }
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (!ghost && i0 + k == p.La - 1) *p.e_final = cur[k];
    if (kFlag) {
        // the strip's words are all stored: raise its flag for the band map
        __threadfence();
        __syncwarp();
        if (lane == 0) st_release_g(done + strip, p.epoch);
    }
}

// Reader warp (groups g > 0): the bottom rows of group g-1 from the global
// border into ring 0.  Lane v < 16 carries value v of every sub-chunk
// (column v % 8, row v / 8); loads run kAheadSub sub-chunks ahead, and a
// value whose tag is not yet this call's is re-polled (bounded).
constexpr int kAheadSub = 4;
__device__ __forceinline__ void run_reader(const DpArgs& p, int g, int lane, float (*ring0)[2][kSub],
                                           unsigned bfull0, unsigned bempty0, unsigned rbase,
                                           int nfirst, int nsub, int clo, int chi) {
    // blocks nfirst .. nsub-1 (this group's first strip's range); only columns
    // clo .. chi-1 were published above (the others read as +inf)
    const int Lb = p.Lb;
    clo = max(clo, 0);
    chi = min(chi, Lb);
    const unsigned long long* gin = p.gborder + (size_t)(g - 1) * Lb * 2;
    const unsigned epoch = p.epoch;
    const bool act_lane = lane < 2 * kSub;
    const int cofs = lane & (kSub - 1), row = (lane >> 3) & 1;
    unsigned long long pend[kAheadSub];
#pragma unroll
    for (int q = 0; q < kAheadSub; ++q) {
        const int col = (nfirst + q) * kSub + cofs;
        pend[q] = (act_lane && col >= clo && col < chi) ? ldg1(gin + (size_t)col * 2 + row) : 0ull;
    }
    for (int n0 = nfirst; n0 < nsub; n0 += kAheadSub) {
#pragma unroll
        for (int q = 0; q < kAheadSub; ++q) {
            const int n = n0 + q;
            if (n >= nsub) break;
            const int col = n * kSub + cofs;
            const bool act = act_lane && col >= clo && col < chi;
            int ok = !act || tag_of(pend[q]) == epoch;
            if (!__all_sync(kFull, ok)) {
                // each poll is a round trip to L2; status and deadline every 16 polls
                const long long t0 = __shfl_sync(kFull, global_ns(), 0);
                for (int poll = 1;; ++poll) {
                    if (!ok) {
                        pend[q] = ldg1(gin + (size_t)col * 2 + row);
                        ok = tag_of(pend[q]) == epoch;
                    }
                    if (__all_sync(kFull, ok)) break;
                    if ((poll & 15) == 0) {
                        if (__shfl_sync(kFull, read_status(p.ctl), 0) != 0) return;
                        const long long now = __shfl_sync(kFull, global_ns(), 0);
                        if (now - t0 > p.timeout_ns) {
                            if (lane == 0) raise_status(p.ctl, DTW_ERR_TIMEOUT, 3);
                            return;
                        }
                    }
                }
            }
            const unsigned t = rbase + (unsigned)(n - nfirst);
            if (!mbar_wait(bar_at(bempty0, t % kRingBlk), use_parity(t, kRingBlk) ^ 1u, p.ctl,
                           p.timeout_ns, 8))
                return;
            if (act_lane) ring0[t % kRingBlk][row][cofs] = act ? val_of(pend[q]) : INFINITY;
            mbar_arrive(bar_at(bfull0, t % kRingBlk));
            const int ncol = col + kAheadSub * kSub;
            if (act_lane && ncol >= clo && ncol < chi) pend[q] = ldg1(gin + (size_t)ncol * 2 + row);
        }
    }
}

// Writer warp: the last DP slot's bottom rows from ring NS to the global
// border of group g, as (value, epoch) words; lanes 0..15 store one
// coalesced 128-byte line per sub-chunk.
__device__ __forceinline__ void run_writer(const DpArgs& p, int g, int lane,
                                           float (*ringo)[2][kSub], unsigned bfullo,
                                           unsigned bemptyo, unsigned rbase, int nfirst,
                                           int nsub) {
    const int Lb = p.Lb;
    unsigned long long* gout = p.gborder + (size_t)g * Lb * 2;
    const unsigned epoch = p.epoch;
    const int cofs = lane & (kSub - 1), row = (lane >> 3) & 1;
    for (int n = nfirst; n < nsub; ++n) {
        const unsigned t = rbase + (unsigned)(n - nfirst);
        if (!mbar_wait(bar_at(bfullo, t % kRingBlk), use_parity(t, kRingBlk), p.ctl, p.timeout_ns,
                       9))
            return;
        const float v = ringo[t % kRingBlk][row][cofs];
        mbar_arrive(bar_at(bemptyo, t % kRingBlk));
        const int col = n * kSub + cofs;
        if (lane < 2 * kSub && col < Lb) stg1(gout + (size_t)col * 2 + row, pack(v, epoch));
    }
}

// Cluster links.  Between two CTAs of one cluster the border goes through
// a staging ring of kRingBlk blocks in the shared memory of the CTA below
// (`link`, full barriers `lfull` there, empty barriers `lempty` in the CTA
// above); the DP warps' own rings are untouched, so their sweep is the same
// code with or without clusters.  Producer and consumer count the link's
// uses as the blocks of the strip above's range, in order.

// Writer warp of a CTA with another CTA of its cluster below: every block of
// the last strip's range [nfirst, nsub) from ring NS into the staging ring of
// CTA crank + 1 (lanes 0..15: value v = column v % 8 of row v / 8), each
// value an asynchronous store completing 4 of the 64 bytes its full barrier
// expects.
__device__ __forceinline__ void run_link_writer(const DpArgs& p, int lane, float (*ringo)[2][kSub],
                                                unsigned bfullo, unsigned bemptyo, unsigned rbase,
                                                int nfirst, int nsub, unsigned link_s,
                                                unsigned lfull_s, unsigned lempty_s,
                                                unsigned lbase, unsigned crank) {
    const int cofs = lane & (kSub - 1), row = (lane >> 3) & 1;
    for (int n = nfirst; n < nsub; ++n) {
        const unsigned t = rbase + (unsigned)(n - nfirst);  // use of ring NS
        const unsigned u = lbase + (unsigned)(n - nfirst);  // use of the link
        if (!mbar_wait(bar_at(bfullo, t % kRingBlk), use_parity(t, kRingBlk), p.ctl, p.timeout_ns,
                       9))
            return;
        // the link block's previous use has been read below
        if (!mbar_wait(bar_at(lempty_s, u % kRingBlk), use_parity(u, kRingBlk) ^ 1u, p.ctl,
                       p.timeout_ns, 10))
            return;
        const float v = ringo[t % kRingBlk][row][cofs];
        mbar_arrive(bar_at(bemptyo, t % kRingBlk));
        if (lane < 2 * kSub)
            st_async_f32(map_rank(link_s + (u % kRingBlk) * (2 * kSub * 4) +
                                      (unsigned)(row * kSub + cofs) * 4u,
                                  crank + 1),
                         v, map_rank(bar_at(lfull_s, u % kRingBlk), crank + 1));
    }
}

// Reader warp of a CTA with another CTA of its cluster above: ring 0 for the
// first strip's range [nfirst, nsub) from the staging ring, which carries
// the strip above's range [pa, pb): blocks of it before nfirst (or after
// nsub) are consumed unread, blocks of the strip's range past pb read +inf.
// Lane 0 re-arms a consumed block's full barrier for its next use and then
// arrives on the sender's empty barrier, with a count that depends on the
// value it loaded (the warp's loads of the block are one instruction).
__device__ __forceinline__ void run_link_reader(const DpArgs& p, int lane, float (*ring0)[2][kSub],
                                                unsigned bfull0, unsigned bempty0, unsigned rbase,
                                                int nfirst, int nsub, int pa, int pb,
                                                float (*link)[2][kSub], unsigned lfull_s,
                                                unsigned lempty_s, unsigned lbase,
                                                unsigned crank) {
    const int cofs = lane & (kSub - 1), row = (lane >> 3) & 1;
    auto release = [&](unsigned u, unsigned dep) {
        if (lane == 0) {
            mbar_arrive_expect_tx(bar_at(lfull_s, u % kRingBlk), 2 * kSub * 4);
            mbar_arrive_remote_relaxed(map_rank(bar_at(lempty_s, u % kRingBlk), crank - 1),
                                       1u + zero_after(dep));
        }
        __syncwarp();
    };
    auto skip = [&](int n) -> int {
        const unsigned u = lbase + (unsigned)(n - pa);
        if (!mbar_wait(bar_at(lfull_s, u % kRingBlk), use_parity(u, kRingBlk), p.ctl,
                       p.timeout_ns, 11))
            return 0;
        release(u, 0u);
        return 1;
    };
    for (int n = pa; n < min(nfirst, pb); ++n)
        if (!skip(n)) return;
    for (int n = nfirst; n < nsub; ++n) {
        const unsigned t = rbase + (unsigned)(n - nfirst);  // use of ring 0
        float v = INFINITY;
        if (n >= pa && n < pb) {
            const unsigned u = lbase + (unsigned)(n - pa);
            if (!mbar_wait(bar_at(lfull_s, u % kRingBlk), use_parity(u, kRingBlk), p.ctl,
                           p.timeout_ns, 11))
                return;
            v = link[u % kRingBlk][row][cofs];
            release(u, __float_as_uint(v));
        }
        if (!mbar_wait(bar_at(bempty0, t % kRingBlk), use_parity(t, kRingBlk) ^ 1u, p.ctl,
                       p.timeout_ns, 8))
            return;
        if (lane < 2 * kSub) ring0[t % kRingBlk][row][cofs] = v;
        mbar_arrive(bar_at(bfull0, t % kRingBlk));
    }
    for (int n = max(pa, max(nsub, nfirst)); n < pb; ++n)
        if (!skip(n)) return;
}

// Band-map item `item` of the pair (band-major: band item / nseg, column
// segment item % nseg) by all NT threads of the CTA, once the strips covering
// the band have raised their flags.  The wait (thread 0) gives up when the
// call has failed elsewhere, or when no flag it waits for has come up for
// 8 x the handoff limit (DTW_ERR_TIMEOUT, detail 6): a strip's whole sweep
// lies between the item's start and its flag, not just one handoff.
template <int NT>
__device__ __noinline__ void run_bandmap_item(const DpArgs& p, const MapArgs& m, int item,
                                              int (*s_x)[NT][3]) {
    __shared__ int s_ok;
    const BtArgs& bt = m.bt;
    constexpr int kWidth = NT * kColsPerWord - 2 * kBand;
    const int nseg = (bt.Lb + kWidth - 1) / kWidth;
    const int b = item / nseg, segx = item - b * nseg;
    const int s0 = (b * kBand) / p.rps;
    const int s1 = (min((b + 1) * kBand, p.La) - 1) / p.rps;
    auto ready = [&]() -> int {
        if (threadIdx.x == 0) {
            int ok = 1;
            long long t0 = global_ns();
            for (int s = s0; s <= s1 && ok; ++s)
                for (int poll = 0;; ++poll) {
                    if (ld_acquire_g(m.done + s) == p.epoch) {
                        t0 = global_ns();
                        break;
                    }
                    if (read_status(p.ctl) != 0) {
                        ok = 0;
                        break;
                    }
                    if (global_ns() - t0 > 8 * p.timeout_ns) {
                        raise_status(p.ctl, DTW_ERR_TIMEOUT, 6);
                        ok = 0;
                        break;
                    }
                    if (poll >= 4) __nanosleep(256);
                }
            s_ok = ok;
        }
        __syncthreads();
        return s_ok;
    };
    if (bt.ranges)
        bandmap_segment<NT, true, true>(bt, b, segx, s_x, ready);
    else
        bandmap_segment<NT, false, true>(bt, b, segx, s_x, ready);
}

// NS strips per CTA.  Warps 0..NS-1: the strips' cost warps; NS..2NS-1:
// their DP warps; 2NS: the reader; 2NS+1: the writer.  Warp w runs on SM
// sub-partition w % 4, so for NS = 2 each DP warp has a sub-partition of its
// own and the helpers share those of the cost warps.  Persistent: a CTA
// takes strip groups from the ticket counter until none are left, so a
// group only ever waits on groups that started earlier.
// kMany: the groups come from a work queue over many pairs (`many`, `item0`,
// `ticket`; see launch_dp_split_many) instead of the pair `one`.
// kMap (one pair): tickets past the strip groups are the map.nbm band-map
// items of the pair's backtrace (map.bt, run_bandmap_item); every group has
// been taken by a running CTA before the first item is, so an item only
// waits on strips in progress.  For pairs whose groups outnumber the
// resident CTAs: the CTAs of the last round that find no group then map the
// bands above while the last strips sweep.  The launch bounds keep as many
// CTAs per SM as the DP alone fits (split_ctas_per_sm).
// kCl (one pair, no band map): the kernel runs in clusters of cn CTAs that
// take tickets together: ticket T gives CTA rank r the strip group
// T cn + r, so the border between two of a ticket's groups goes through
// distributed shared memory (run_link_writer, run_link_reader); only rank 0
// reads a global border and only rank cn - 1 writes one.  A CTA leaves only
// when its whole cluster does (no CTA's shared memory may disappear while a
// peer can still reach it).
template <int DP, int R, int NS, bool kMany, bool kBF, bool kSubseq = false, bool kT = false,
          bool kMap = false, bool kCl = false>
__global__ void __launch_bounds__(split_threads<DP, NS, kBF>(),
                                  (kMap ? split_ctas_per_sm(R, NS, DP, kBF) : 1))
    k_dp_split(const DpArgs one, const MapArgs map, const DpArgs* __restrict__ many,
               const int* __restrict__ item0, int nmany, int* ticket) {
    static_assert(!kCl || (!kMany && !kMap && !kSubseq), "clusters sweep one plain pair");
    constexpr int kThreads = split_threads<DP, NS, kBF>();
    constexpr int kNC = CostWide<DP, kBF>::kNC;  // cost warps per strip
    constexpr bool kWide = CostWide<DP, kBF>::kOn;
    using S = BStage<DP>;
    using M = SplitSmem<DP, R, kBF>;
    __shared__ __align__(16) float ring[NS + 1][kRingBlk][2][kSub];
    __shared__ __align__(8) unsigned long long bbar[NS * kNC][S::kSlots];
    __shared__ __align__(8) unsigned long long cfull[NS][kCostSlots];
    __shared__ __align__(8) unsigned long long cempty[NS][kCostSlots];
    __shared__ __align__(8) unsigned long long bfull[NS + 1][kRingBlk];
    __shared__ __align__(8) unsigned long long bempty[NS + 1][kRingBlk];
    __shared__ __align__(16) float s_inf[2][kSub];  // +inf border block, never written after
    __shared__ int s_group, s_pair;
    // cluster link into this CTA (staging ring, its full barriers) and out of
    // it (the empty barriers of the staging ring of the CTA below)
    __shared__ __align__(16) float link[kCl ? kRingBlk : 1][2][kSub];
    __shared__ __align__(8) unsigned long long lfull[kCl ? kRingBlk : 1];
    __shared__ __align__(8) unsigned long long lempty[kCl ? kRingBlk : 1];
    extern __shared__ __align__(128) unsigned char dyn[];  // NS * M::kStripBytes
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned crank = kCl ? cluster_rank() : 0u;
    const unsigned cn = kCl ? cluster_size() : 1u;
    // warps 0 .. kNC NS - 1: cost warps (strip slot wid % NS, half wid / NS);
    // then one DP warp per strip, the reader and the writer
    const int role = wid < kNC * NS ? 0
                                    : (wid < (kNC + 1) * NS ? 1 : (wid == (kNC + 1) * NS ? 2 : 3));
    const int w = role == 0 ? wid % NS : (role == 1 ? wid - kNC * NS : 0);  // strip slot
    const int half = role == 0 ? wid / NS : 0;
    unsigned char* mine = dyn + (size_t)w * M::kStripBytes;
    const unsigned cring_s = smem_u32(mine + M::kOperandBytes);
    const unsigned a_s = smem_u32(mine);                                  // kBF: A tile
    const unsigned b_s = smem_u32(mine + 32 * R * kBfStride * 2);         // kBF: B ring
    unsigned bbase = 0;  // kBF: lifetime count of this cost warp's B blocks
    const unsigned cfull_s = smem_u32(&cfull[w][0]);
    const unsigned cempty_s = smem_u32(&cempty[w][0]);

    BRing<DP> br;
    br.stage = reinterpret_cast<const float*>(mine);
    br.stage_s = smem_u32(mine);
    br.bar_s = smem_u32(&bbar[w][0]);
    br.base = 0;
    br.first = 0;
    br.nblk = 0;
    br.issued = br.waited = 0;
    // the wide FP32 cost warps: A tile, then a B ring per half (two chunks)
    using WS = BStage<DP, CostWide<DP, kBF>::kBSlots>;
    BRing<DP, CostWide<DP, kBF>::kBSlots> bw;
    bw.stage_s = smem_u32(mine + 32 * R * CostWide<DP, kBF>::kStride * 4 + half * WS::kWarpBytes);
    bw.stage = reinterpret_cast<const float*>(mine);  // (unused by the wide cost warp)
    bw.bar_s = smem_u32(&bbar[half * NS + w][0]);
    bw.base = 0;
    bw.first = 0;
    bw.nblk = 0;
    bw.issued = bw.waited = 0;
    if (threadIdx.x < 2 * kSub) (&s_inf[0][0])[threadIdx.x] = INFINITY;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS * kNC; ++s)
            for (int k = 0; k < S::kSlots; ++k) mbar_init(smem_u32(&bbar[s][k]), 1);
        for (int s = 0; s < NS; ++s) {
            for (int k = 0; k < kCostSlots; ++k) {
                mbar_init(smem_u32(&cfull[s][k]), kWarp);  // the lanes of the slot's cost warp
                mbar_init(smem_u32(&cempty[s][k]), kWarp);  // the DP warp's lanes
            }
        }
        for (int s = 0; s <= NS; ++s)
            for (int k = 0; k < kRingBlk; ++k) {
                // ring 0 is filled by the reader's lanes, the others by lane 30
                // of the DP warp above; every ring is emptied by a whole warp
                mbar_init(smem_u32(&bfull[s][k]), s == 0 ? kWarp : 1);
                mbar_init(smem_u32(&bempty[s][k]), kWarp);
            }
        if (kCl) {
            // the staging ring: a full barrier completes on the reader's
            // arrival and 64 bytes of asynchronous stores from the CTA above
            // (armed here for the first uses); an empty barrier (of the link
            // to the CTA below) on one arrival of that CTA's reader
            for (int k = 0; k < kRingBlk; ++k) {
                mbar_init(smem_u32(&lfull[k]), 1);
                mbar_init(smem_u32(&lempty[k]), 1);
            }
            if (crank > 0)
                for (int k = 0; k < kRingBlk; ++k)
                    mbar_arrive_expect_tx(smem_u32(&lfull[k]), 2 * kSub * 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if constexpr (kCl) cluster_sync_all();  // every CTA's barriers before any remote access
    // Lifetime sub-chunk counts of the cost rings and the border rings.
    unsigned csub[NS], rsub[NS + 1];
#pragma unroll
    for (int s = 0; s < NS; ++s) csub[s] = 0;
#pragma unroll
    for (int s = 0; s <= NS; ++s) rsub[s] = 0;
    unsigned lin = 0, lout = 0;  // uses of the cluster links into and out of this CTA

    for (;;) {
        if constexpr (kCl) {
            // every warp of the cluster finished the previous ticket; rank 0
            // takes the next one and hands it to every CTA of the cluster
            cluster_sync_all();
            if (crank == 0 && threadIdx.x == 0) {
                const int T = read_status(one.ctl) != 0 ? one.ngroups
                                                        : atomicAdd(&one.ctl->ticket, 1);
                for (unsigned r = 0; r < cn; ++r)
                    st_cluster_u32(map_rank(smem_u32(&s_pair), r), (unsigned)T);
            }
            cluster_sync_all();
            const int T = s_pair;
            if ((long long)T * cn >= one.ngroups) break;  // the whole cluster leaves
            if (threadIdx.x == 0) s_group = T * (int)cn + (int)crank;
        } else {
        __syncthreads();  // every warp finished the previous group
        }
        if (!kCl && threadIdx.x == 0) {
            if (kMany) {
                // item t -> (pair, group): the last pair whose first item is <= t
                const int t = atomicAdd(ticket, 1);
                int pi = -1, gi = 0;
                if (t < item0[nmany]) {
                    int lo = 0, hi = nmany - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (item0[mid] <= t)
                            lo = mid;
                        else
                            hi = mid - 1;
                    }
                    pi = lo;
                    gi = t - item0[lo];
                    if (read_status(many[pi].ctl) != 0) gi = -1;  // the pair has failed
                }
                s_pair = pi;
                s_group = gi;
            } else {
                s_pair = 0;
                s_group = read_status(one.ctl) != 0 ? one.ngroups + (kMap ? map.nbm : 0)
                                                    : atomicAdd(&one.ctl->ticket, 1);
            }
        }
        // +inf border: the top rows of group 0
        float* rf = &ring[0][0][0][0];
        for (int k = threadIdx.x; k < kRing * 2; k += blockDim.x) rf[k] = INFINITY;
        __syncthreads();
        if (kMany && s_pair < 0) return;
        if (kMany && s_group < 0) continue;  // nothing of a failed pair runs
        const DpArgs p = kMany ? many[s_pair] : one;
        const int g = s_group;
        if (kCl && g >= p.ngroups) continue;  // this CTA's group of the ticket does not exist
        if (g >= p.ngroups) {
            if constexpr (kMap) {
                if (g - p.ngroups < map.nbm) {
                    // left-neighbour exchange of the band map
                    __shared__ int s_bm[2][kThreads][3];
                    run_bandmap_item<kThreads>(p, map, g - p.ngroups, s_bm);
                    continue;
                }
            }
            return;
        }
        const GroupRoles gr = group_roles<NS>(p, g);
        const int strip = g * NS + w;
        // the sub-chunk ranges of the group's strips (all columns without a band)
        int2 rgs[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q)
            rgs[q] = q < gr.nstrips_here ? strip_range(p, g * NS + q) : make_int2(0, 0);
        if (role == 0) {
            if (w < gr.nstrips_here)
            {
                if constexpr (kBF)
                    run_cost_bf16<DP, R>(p, strip, lane, a_s, b_s, smem_u32(&bbar[w][0]), bbase,
                                         cring_s, cfull_s, cempty_s, csub[w]);
                else if constexpr (kWide)
                    run_cost_wide<DP, R>(p, strip, w, half, lane, reinterpret_cast<float*>(mine),
                                         cring_s, cfull_s, cempty_s, csub[w], bw);
                else
                    run_cost<DP, R>(p, strip, lane, cring_s, cfull_s, cempty_s, csub[w], br);
            }
        } else if (role == 1) {
            if (w < gr.nstrips_here)
                run_dp<R, NS, kBF, kSubseq, kT, kMap, (kBF || kWide), kWide>(p, gr, w, strip, lane, ring, smem_u32(&bfull[0][0]),
                                   smem_u32(&bempty[0][0]), rsub[w], rsub[w + 1], cring_s,
                                   cfull_s, cempty_s, csub[w], smem_u32(&s_inf[0][0]),
                                   kMap ? map.done : nullptr);
        } else if (role == 2) {
            if (gr.reader) {
                // the first strip's blocks; the strip above (last of the group
                // above) published its own range's columns
                const int2 above = strip_range(p, g * NS - 1);
                if (kCl && crank > 0)
                    run_link_reader(p, lane, ring[0], smem_u32(&bfull[0][0]),
                                    smem_u32(&bempty[0][0]), rsub[0], rgs[0].x, rgs[0].y, above.x,
                                    above.y, link, smem_u32(&lfull[0]), smem_u32(&lempty[0]), lin,
                                    crank);
                else
                    run_reader(p, g, lane, ring[0], smem_u32(&bfull[0][0]),
                               smem_u32(&bempty[0][0]), rsub[0], rgs[0].x, rgs[0].y,
                               above.x * kSub, above.y * kSub);
            }
        } else {
            if (gr.writer) {
                if (kCl && crank + 1 < cn)
                    run_link_writer(p, lane, ring[NS], smem_u32(&bfull[NS][0]),
                                    smem_u32(&bempty[NS][0]), rsub[NS], rgs[NS - 1].x,
                                    rgs[NS - 1].y, smem_u32(&link[0][0][0]), smem_u32(&lfull[0]),
                                    smem_u32(&lempty[0]), lout, crank);
                else
                    run_writer(p, g, lane, ring[NS], smem_u32(&bfull[NS][0]),
                               smem_u32(&bempty[NS][0]), rsub[NS], rgs[NS - 1].x, rgs[NS - 1].y);
            }
        }
        // ring uses of this group, in blocks of 8 columns: a cost ring the
        // strip's range; ring 0 the first strip's range; ring w (1 <= w < NS)
        // and ring NS the range of the strip that fills them
#pragma unroll
        for (int q = 0; q < NS; ++q)
            if (q < gr.nstrips_here) csub[q] += (unsigned)(rgs[q].y - rgs[q].x);
        if (ring_used<NS>(gr, 0)) rsub[0] += (unsigned)(rgs[0].y - rgs[0].x);
        if (kCl && crank > 0 && gr.reader) {  // the link carries the strip above's range
            const int2 above = strip_range(p, g * NS - 1);
            lin += (unsigned)(above.y - above.x);
        }
        if (kCl && crank + 1 < cn && gr.writer) lout += (unsigned)(rgs[NS - 1].y - rgs[NS - 1].x);
#pragma unroll
        for (int q = 1; q <= NS; ++q)
            if (ring_used<NS>(gr, q)) rsub[q] += (unsigned)(rgs[q - 1].y - rgs[q - 1].x);
    }
    if constexpr (kCl) cluster_sync_all();  // no peer reaches this CTA's shared memory any more
}

template <int DP, int R, int NS, bool kMany, bool kBF = false, bool kSubseq = false,
          bool kT = false, bool kMap = false>
cudaError_t launch_t(const DpArgs& a, const DpArgs* many, const int* item0, int n, int items,
                     int* ticket, int num_sms, cudaStream_t s, const MapArgs* map = nullptr) {
    static_assert(!kMap || (!kMany && !kSubseq), "the band map runs with one pair");
    constexpr int kThreads = split_threads<DP, NS, kBF>();
    const int smem = NS * SplitSmem<DP, R, kBF>::kStripBytes;
    auto* kern = k_dp_split<DP, R, NS, kMany, kBF, kSubseq, kT, kMap>;
    static DeviceSlots occupancy;
    int blocks_per_sm = 0;
    const cudaError_t e = blocks_per_sm_once(kern, kThreads, smem, occupancy, &blocks_per_sm);
    if (e != cudaSuccess) return e;
    int grid = blocks_per_sm * num_sms;
    if (kMap) {
        if (!map || !map->done || map->nbm <= 0) return cudaErrorInvalidValue;
        items += map->nbm;
    }
    if (grid > items) grid = items;
    kern<<<grid, kThreads, smem, s>>>(a, map ? *map : MapArgs{}, many, item0, n, ticket);
    return cudaGetLastError();
}

}  // namespace
}  // namespace pardtw
