// Exact DTW dynamic programming on the GPU (ParDTW's DP stage, Sec. II-D,
// Sec. III-B) with 2-bit backpointers (Sec. VI-D).
//
// Recurrence (Sec. V steps and weights), on the shifted cost C' = C - mu:
//   E[0][0] = C[0][0]
//   E[i][j] = min(E[i-1][j-1] + 2C', E[i-1][j-2] + 3C', E[i-2][j-1] + 3C')
// and D = E + mu*(i+j), so the arg-min decisions equal those of D in exact
// arithmetic (every step's weight equals its advance in i+j).
//
// Schedule.  With steps (1,1), (1,2), (2,1) a cell of column j reads only
// columns j-1 and j-2, so all cells of a column are independent.  ParDTW
// sweeps anti-diagonals for the same reason (cells of a diagonal only read
// the three previous diagonals, Sec. II-D); sweeping columns instead keeps
// every sweep step at full width (no fill and drain of diagonals) and makes
// the column of B a warp-uniform broadcast.
//
//   - A warp owns a strip of 30 consecutive rows of A, one row per lane
//     0..29, and sweeps all Lb columns; each lane keeps its row's two live
//     cumulative values and the normalised frame a_i in registers.
//   - Lanes 30 and 31 are "ghost" rows: they reproduce the two bottom rows of
//     the strip above.  A ghost lane runs the same step as a real one, but
//     its cost is 1e30 and the weight of its (1,2) candidate is 0, so that
//     candidate -- fed with the border value -- is always the minimum.  Rows
//     i-1 and i-2 of column j-1 then arrive for every lane by two rotating
//     shuffles (lane 0 reads lanes 31 and 30), with no per-lane fix-up.
//     Values >= 1e30 stand for unreachable cells and never reach a
//     reachable end cell, whose cost is far below.
//   - The border values come from a ring in shared memory.  Within a CTA the
//     warp above fills it and publishes its progress every kSub columns with
//     a release store that the reader acquires.  Across CTAs the bottom rows travel through
//     a border buffer in global memory whose 64-bit entries carry the call's
//     tag next to the value, so a matching tag proves the value is current;
//     warp 0 loads them kWin columns ahead and checks them kSub at a time.
//   - Per chunk of 16 columns the 16 cosine costs are formed first, as 16
//     independent FMA chains, then the 16 DP steps run without branches; the
//     only dependency chain left per step is shuffle -> FMA -> 3-input min.
//   - A CTA owns kWarpsPerGroup consecutive strips (a "strip group");
//     persistent CTAs take groups in order from an atomic ticket, so every
//     group a CTA waits on was taken earlier by a running CTA.
//   - Each lane packs 16 columns of 2-bit codes into a uint32; the warp
//     stores 32 consecutive words (128 bytes) per 16 columns.
//   - Every wait is bounded in time; on expiry the kernel records
//     DTW_ERR_TIMEOUT and all CTAs leave.
#include "dp_device.cuh"

namespace pardtw {
namespace {

constexpr int kGhost0 = kRowsPerStrip;  // first ghost lane (30)

// Part uu (0..15) of the next chunk's cost accumulation: flat indices
// DP*uu .. DP*uu+DP-1 of its feature-major 16 x DP block, i.e. feature
// d = idx / 16 of column idx % 16, read four at a time.
template <int DP>
__device__ __forceinline__ void next_cost_part(const float* nb, int uu, const float* na,
                                               float* cn) {
#pragma unroll
    for (int e = 0; e < DP; e += 4) {
        const int idx = DP * uu + e;
        const float4 b4 = *reinterpret_cast<const float4*>(nb + idx);
        const int d = idx / kColsPerWord, f = idx % kColsPerWord;
        cn[f] = fmaf(na[d], b4.x, cn[f]);
        cn[f + 1] = fmaf(na[d], b4.y, cn[f + 1]);
        cn[f + 2] = fmaf(na[d], b4.z, cn[f + 2]);
        cn[f + 3] = fmaf(na[d], b4.w, cn[f + 3]);
    }
}

// One DP step of column j for the warp's 32 lanes: no memory access and no
// branch.  Lane sources srcA = lane-1, srcB = lane-2 (mod 32) give rows i-1
// and i-2 of column j-1; x1p holds row i-1 of column j-2 (for a ghost lane:
// its own border value of column j).
__device__ __forceinline__ void dp_step(float cost, int u, int srcA, int srcB, float w12,
                                        bool origin_here, float mu, float& cur, float& x1p,
                                        float& x1, float& fw, float& out) {
    x1 = __shfl_sync(kFull, cur, srcA);        // E[i-1][j-1]
    const float x2 = __shfl_sync(kFull, cur, srcB);  // E[i-2][j-1]
    const float c0 = fmaf(2.0f, cost, x1);  // from (i-1, j-1)
    const float c1 = fmaf(w12, cost, x1p);  // from (i-1, j-2)
    const float c2 = fmaf(3.0f, cost, x2);  // from (i-2, j-1)
    float m = min3f(c0, c1, c2);
    // backpointer field (step_of_field) at bits 2u, 2u+1 of the sub-chunk's
    // accumulator
    fw = fmaf(eq_as_float(c0, m), (float)(1u << (2 * u)), fw);
    fw = fmaf(eq_as_float(c1, m), (float)(2u << (2 * u)), fw);
    m = origin_here ? cost + mu : m;  // E[0][0] = C[0][0]
    out = m;
    cur = m;
}

// One warp sweeps its strip (30 rows + 2 ghost lanes) over all columns.
template <int DP, int NW>
__device__ __forceinline__ void run_strip(const DpArgs& p, int g, int w, int lane,
                                          float (*ring)[kRingBlk][2][kSub], int* prod, int* cons,
                                          BRing<DP>& br) {
    using S = BStage<DP>;
    const int strip = g * NW + w;
    if (strip >= p.nstrips) return;
    const bool ghost = lane >= kGhost0;
    const int i = strip * kRowsPerStrip + lane;  // row of a real lane
    const int Lb = p.Lb;

    float na[DP];  // -a^_i (0 in ghost lanes)
    {
        const float4* s = reinterpret_cast<const float4*>(p.Ahat + (size_t)i * DP);
#pragma unroll
        for (int q = 0; q < DP / 4; ++q) {
            const float4 v = ghost ? make_float4(0.f, 0.f, 0.f, 0.f) : __ldg(s + q);
            na[4 * q] = -v.x;
            na[4 * q + 1] = -v.y;
            na[4 * q + 2] = -v.z;
            na[4 * q + 3] = -v.w;
        }
    }
    const bool to_ring = (w + 1 < NW) && (strip + 1 < p.nstrips);
    const bool to_global = (w == NW - 1) && (g + 1 < p.ngroups) && (g != p.skip_publish);
    const bool out_lane = (lane == kGhost0 - 2) || (lane == kGhost0 - 1);  // rows 28, 29
    const int out_comp = lane - (kGhost0 - 2);                             // 0 or 1
    float (*myring)[2][kSub] = ring[w];
    float (*nextring)[2][kSub] = ring[(w + 1) % NW];
    const int in_comp = (lane == 31) ? 1 : 0;  // lane 30: row top-2, lane 31: row top-1
    const unsigned prod_in = smem_u32(&prod[w]);
    const unsigned prod_out = smem_u32(&prod[(w + 1) % NW]);
    const unsigned cons_mine = smem_u32(&cons[w]);
    const unsigned cons_next = smem_u32(&cons[(w + 1) % NW]);
    unsigned long long* gout = p.gborder + (size_t)g * Lb * 2;
    const unsigned long long* gin = p.gborder + (size_t)(g > 0 ? g - 1 : 0) * Lb * 2;
    const float kcost = ghost ? kGhostCost : p.kcost;
    const float mu = p.mu;
    const float w12 = ghost ? 0.0f : 3.0f;
    const int srcA = (lane + 31) & 31, srcB = (lane + 30) & 31;
    const unsigned epoch = p.epoch;
    const bool is_origin = (i == 0);
    const bool from_global = (w == 0) && (g > 0);

    // B pipeline and, for warp 0 below another group, the border window
    br.begin(0, (p.nchunk * kColsPerWord + S::kBlk - 1) / S::kBlk);
    const int Lb_pad = p.nchunk * kColsPerWord;
    br.top_up(0, p.Bhat, Lb_pad, lane);
    unsigned long long g0 = 0, g1 = 0;
    if (from_global && lane < Lb) ldg2(gin + (size_t)lane * 2, g0, g1);

    // C' = (1 - mu) - a^_i . b^_j for the 16 columns of a chunk, each summed
    // one FMA per feature in feature order (bit-identical to dtw_cost).  The
    // costs of chunk k+1 are accumulated feature-major during the DP steps of
    // chunk k: step u issues the DP FMAs with flat index DP*u .. DP*u+DP-1 of
    // the chunk's 16 x DP block (index d*16 + column), 16 columns apart, so
    // they never wait on one another nor on the DP chain.
    float c[kColsPerWord];
    if (!br.wait(0, p.ctl, p.timeout_ns)) {
        br.drain();
        return;
    }
    {
        const float* cb = br.chunk(0);
#pragma unroll
        for (int u = 0; u < kColsPerWord; ++u) c[u] = kcost;
#pragma unroll
        for (int d = 0; d < DP; ++d) {
            const float4* v = reinterpret_cast<const float4*>(cb + d * kColsPerWord);
#pragma unroll
            for (int q = 0; q < kColsPerWord / 4; ++q) {
                const float4 b4 = v[q];
                c[4 * q] = fmaf(na[d], b4.x, c[4 * q]);
                c[4 * q + 1] = fmaf(na[d], b4.y, c[4 * q + 1]);
                c[4 * q + 2] = fmaf(na[d], b4.z, c[4 * q + 2]);
                c[4 * q + 3] = fmaf(na[d], b4.w, c[4 * q + 3]);
            }
        }
    }

    float cur = INFINITY;  // E[i][j-1]
    float x1p = INFINITY;  // E[i-1][j-2]; a ghost lane: its border value of column j
    float x1 = INFINITY;
    // The failure flag is loaded one chunk ahead of its test, so the load's
    // latency never stalls the sweep.
    int status_seen = 0;
    for (int j0 = 0; j0 < Lb; j0 += kColsPerWord) {
        if (__shfl_sync(kFull, status_seen, 0) != 0) {
            br.drain();
            return;
        }
        status_seen = read_status(p.ctl);
        // the next chunk's block of B frames (when it starts a new block)
        const int jn = j0 + kColsPerWord;
        const bool has_next = jn < Lb;
        if (has_next && (jn % S::kBlk) == 0) {
            const int q = jn / S::kBlk;
            if (!br.wait(q, p.ctl, p.timeout_ns)) {
                br.drain();
                return;
            }
            br.top_up(q, p.Bhat, Lb_pad, lane);
        }
        // the last chunk recomputes its own block into unused accumulators
        const float* nb = br.chunk(has_next ? jn / kColsPerWord : j0 / kColsPerWord);
        float cn[kColsPerWord];
#pragma unroll
        for (int u = 0; u < kColsPerWord; ++u) cn[u] = kcost;
        uint32_t word = 0;
#pragma unroll
        for (int h = 0; h < kColsPerWord / kSub; ++h) {
            const int js = j0 + h * kSub;
            if (js >= Lb) break;
            const int nsteps = min(kSub, Lb - js);
            const int b = (js / kSub) % kRingBlk;
            // border values of columns js .. js+nsteps-1
            if (from_global) {
                if (!refill_top(myring[b], js, lane, Lb, gin, epoch, g0, g1, p.ctl,
                                p.timeout_ns)) {
                    br.drain();
                    return;
                }
            } else if (w > 0) {
                if (!wait_counter_fast(prod_in, js + nsteps, p.ctl, p.timeout_ns, 1)) {
                    br.drain();
                    return;
                }
            }
            if (w > 0 && lane == 0) st_release_s(cons_mine, js);  // windows < js are read
            if (to_ring) {
                // the ring block about to be written must have been read below
                const int need = js + 2 * kSub - kRing;
                if (need > 0 && !wait_counter_fast(cons_next, need, p.ctl, p.timeout_ns, 2)) {
                    br.drain();
                    return;
                }
            }
            float gv[kSub];  // ghost lanes: border value of columns js .. js+kSub-1
            {
                const float4* src = reinterpret_cast<const float4*>(&myring[b][in_comp][0]);
                const float4 v0 = src[0], v1 = src[1];
                gv[0] = v0.x; gv[1] = v0.y; gv[2] = v0.z; gv[3] = v0.w;
                gv[4] = v1.x; gv[5] = v1.y; gv[6] = v1.z; gv[7] = v1.w;
            }
            x1p = ghost ? gv[0] : x1p;
            float o[kSub];  // rows 28, 29: own values of columns js .. js+kSub-1
            float fw = 0.0f;  // backpointer fields of the sub-chunk, bits 2u, 2u+1
            if (nsteps == kSub) {
#pragma unroll
                for (int u = 0; u < kSub; ++u) {
                    const int uu = h * kSub + u;
                    next_cost_part<DP>(nb, uu, na, cn);
                    dp_step(c[uu], u, srcA, srcB, w12, (uu == 0) && (j0 == 0) && is_origin,
                            mu, cur, x1p, x1, fw, o[u]);
                    x1p = (u + 1 < kSub && ghost) ? gv[u + 1 < kSub ? u + 1 : 0] : x1;
                }
            } else {
#pragma unroll
                for (int u = 0; u < kSub; ++u) {
                    const int uu = h * kSub + u;
                    if (u >= nsteps) break;
                    dp_step(c[uu], u, srcA, srcB, w12, (uu == 0) && (j0 == 0) && is_origin,
                            mu, cur, x1p, x1, fw, o[u]);
                    x1p = (u + 1 < kSub && ghost) ? gv[u + 1 < kSub ? u + 1 : 0] : x1;
                }
            }
            word |= field_bits(fw, h);
            if (to_ring) {
                if (out_lane) {
                    float4* dst = reinterpret_cast<float4*>(&nextring[b][out_comp][0]);
                    dst[0] = make_float4(o[0], o[1], o[2], o[3]);
                    dst[1] = make_float4(o[4], o[5], o[6], o[7]);
                }
                __syncwarp();
                // columns < js+nsteps of the bottom rows are in the ring below
                if (lane == kGhost0 - 1) st_release_s(prod_out, js + nsteps);
            } else if (to_global && out_lane) {
#pragma unroll
                for (int u = 0; u < kSub; ++u)
                    if (u < nsteps)
                        stg1(gout + (size_t)(js + u) * 2 + out_comp, pack(o[u], epoch));
            }
        }
        p.bp[((size_t)strip * p.nchunk + (size_t)(j0 >> 4)) * 32 + lane] = word;  // wpb = 32
#pragma unroll
        for (int u = 0; u < kColsPerWord; ++u) c[u] = cn[u];
    }
    if (!ghost && i == p.La - 1) *p.e_final = cur;
}

template <int DP, int NW>
__global__ void __launch_bounds__(NW * 32, DP <= 32 ? 2 : 1) k_dp(const DpArgs p) {
    using S = BStage<DP>;
    __shared__ __align__(16) float ring[NW][kRingBlk][2][kSub];
    __shared__ __align__(8) unsigned long long bars[NW][S::kSlots];
    __shared__ int prod[NW];
    __shared__ int cons[NW];
    __shared__ int s_group;
    extern __shared__ __align__(128) unsigned char bstage[];  // NW * S::kWarpBytes
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;

    BRing<DP> br;
    br.stage = reinterpret_cast<const float*>(bstage + (size_t)w * S::kWarpBytes);
    br.stage_s = smem_u32(bstage + (size_t)w * S::kWarpBytes);
    br.bar_s = smem_u32(&bars[w][0]);
    br.base = 0;
    br.first = 0;
    br.nblk = 0;
    br.issued = br.waited = 0;
    if (lane == 0) {
        for (int k = 0; k < S::kSlots; ++k) mbar_init(br.bar_s + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();

    for (;;) {
        __syncthreads();  // every warp finished the previous group
        if (threadIdx.x == 0) {
            s_group = read_status(p.ctl) != 0 ? p.ngroups : atomicAdd(&p.ctl->ticket, 1);
        }
        // +inf border: group 0's top rows, and nothing is read before it is written
        float* rf = &ring[0][0][0][0];
        for (int k = threadIdx.x; k < NW * kRing * 2; k += blockDim.x) rf[k] = INFINITY;
        if (threadIdx.x < NW) {
            prod[threadIdx.x] = 0;
            cons[threadIdx.x] = 0;
        }
        __syncthreads();
        const int g = s_group;
        if (g >= p.ngroups) return;
        run_strip<DP, NW>(p, g, w, lane, ring, prod, cons, br);
    }
}

template <int DP>
cudaError_t launch_dp_t(const DpArgs& a, int num_sms, cudaStream_t s) {
    constexpr int NW = kWarpsPerGroup;
    const int smem = NW * BStage<DP>::kWarpBytes;
    static DeviceSlots occupancy;
    int blocks_per_sm = 0;
    const cudaError_t e = blocks_per_sm_once(k_dp<DP, NW>, NW * 32, smem, occupancy,
                                             &blocks_per_sm);
    if (e != cudaSuccess) return e;
    int grid = blocks_per_sm * num_sms;
    if (grid > a.ngroups) grid = a.ngroups;
    k_dp<DP, NW><<<grid, NW * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_dp(const DpArgs& a, int dp, int num_sms, cudaStream_t s) {
    switch (dp) {
        case 4: return launch_dp_t<4>(a, num_sms, s);
        case 8: return launch_dp_t<8>(a, num_sms, s);
        case 12: return launch_dp_t<12>(a, num_sms, s);
        case 16: return launch_dp_t<16>(a, num_sms, s);
        case 32: return launch_dp_t<32>(a, num_sms, s);
        case 64: return launch_dp_t<64>(a, num_sms, s);
        case 128: return launch_dp_t<128>(a, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pardtw
