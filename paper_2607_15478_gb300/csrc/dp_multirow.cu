// Exact DTW dynamic programming with R rows of A per lane (R = 2 or 4), the
// fused-cost DP for feature dimensions up to 32.  Same recurrence, step set,
// weights and tie order as the one-row kernel (dp_kernel.cu, Sec. V,
// Sec. II-D); only the work decomposition differs.
//
//   - A warp owns a strip of 31 R rows: lane t (0..30) holds rows
//     31 R s + R t .. + R - 1.  Lane 31 is the ghost lane: its last two rows
//     reproduce the two bottom rows of the strip above (cost 1e30, weight 0
//     on the (1,2) candidate, which is fed with the border value, so the
//     minimum is the border value).
//   - Per column step a lane needs the last two rows of the lane above at
//     column j-1: two rotating shuffles serve all R rows; the other inputs
//     of rows 1..R-1 are the lane's own registers.  One set of shared-memory
//     loads of b_j and one pair of shuffles thus serve R cells, which is the
//     point: both go through the same memory-I/O queue, and the shuffles sit
//     on the step's dependency chain.
//   - The costs of the next 8 columns are accumulated feature-major during
//     the 8 DP steps of the current ones (12 R independent FMAs per step for
//     D = 12), each cost summed one FMA per feature in feature order.
//   - Synchronisation with the strip above and below, the global border
//     between strip groups, the TMA ring of B frames and the bounded waits
//     are those of dp_device.cuh.
#include "dp_device.cuh"

namespace pardtw {
namespace {

constexpr int kGhostLane = 31;
constexpr int kOutLane = 30;  // holds the strip's two bottom rows

// Part u (0..kSub-1) of the next sub-chunk's cost accumulation.  nb points at
// the 8 columns of the sub-chunk inside its chunk's feature-major block
// (column f' of feature d at nb[d * 16 + f']); flat index idx = d * 8 + f'.
template <int DP, int R>
__device__ __forceinline__ void next_cost_part(const float* nb, int u, const float (*na)[DP],
                                               float (*cn)[kSub]) {
#pragma unroll
    for (int e = 0; e < DP; e += 4) {
        const int idx = DP * u + e;
        const int d = idx / kSub, f = idx % kSub;
        const float4 b4 = *reinterpret_cast<const float4*>(nb + d * kColsPerWord + f);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            cn[k][f] = fmaf(na[k][d], b4.x, cn[k][f]);
            cn[k][f + 1] = fmaf(na[k][d], b4.y, cn[k][f + 1]);
            cn[k][f + 2] = fmaf(na[k][d], b4.z, cn[k][f + 2]);
            cn[k][f + 3] = fmaf(na[k][d], b4.w, cn[k][f + 3]);
        }
    }
}

template <int DP, int R, int NW>
__device__ __forceinline__ void run_strip(const DpArgs& p, int g, int w, int lane,
                                          float (*ring)[kRingBlk][2][kSub], int* prod, int* cons,
                                          BRing<DP>& br) {
    using S = BStage<DP>;
    constexpr int kRows = 31 * R;
    const int strip = g * NW + w;
    if (strip >= p.nstrips) return;
    const bool ghost = lane == kGhostLane;
    const int i0 = strip * kRows + lane * R;  // first row of a real lane
    const int Lb = p.Lb;

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
    const bool to_ring = (w + 1 < NW) && (strip + 1 < p.nstrips);
    const bool to_global = (w == NW - 1) && (g + 1 < p.ngroups) && (g != p.skip_publish);
    float (*myring)[2][kSub] = ring[w];
    float (*nextring)[2][kSub] = ring[(w + 1) % NW];
    const unsigned prod_in = smem_u32(&prod[w]);
    const unsigned prod_out = smem_u32(&prod[(w + 1) % NW]);
    const unsigned cons_mine = smem_u32(&cons[w]);
    const unsigned cons_next = smem_u32(&cons[(w + 1) % NW]);
    unsigned long long* gout = p.gborder + (size_t)g * Lb * 2;
    const unsigned long long* gin = p.gborder + (size_t)(g > 0 ? g - 1 : 0) * Lb * 2;
    const float kc = ghost ? kGhostCost : p.kcost;
    const float mu = p.mu;
    float w12[R];
#pragma unroll
    for (int k = 0; k < R; ++k) w12[k] = (ghost && k >= R - 2) ? 0.0f : 3.0f;
    const int srcA = (lane + 31) & 31;
    const unsigned epoch = p.epoch;
    const bool is_origin = (i0 == 0) && !ghost;
    const bool from_global = (w == 0) && (g > 0);

    // B pipeline and, for warp 0 below another group, the border window
    const int Lb_pad = p.nchunk * kColsPerWord;
    br.begin(0, (Lb_pad + S::kBlk - 1) / S::kBlk);
    br.top_up(0, p.Bhat, Lb_pad, lane);
    unsigned long long g0 = 0, g1 = 0;
    if (from_global && lane < Lb) ldg2(gin + (size_t)lane * 2, g0, g1);

    // costs C' = (1 - mu) - a^_i . b^_j of sub-chunk 0
    if (!br.wait(0, p.ctl, p.timeout_ns)) {
        br.drain();
        return;
    }
    float c[R][kSub];
    {
        const float* cb = br.chunk(0);
#pragma unroll
        for (int k = 0; k < R; ++k)
#pragma unroll
            for (int f = 0; f < kSub; ++f) c[k][f] = kc;
#pragma unroll
        for (int d = 0; d < DP; ++d)
#pragma unroll
            for (int f = 0; f < kSub; f += 4) {
                const float4 b4 = *reinterpret_cast<const float4*>(cb + d * kColsPerWord + f);
#pragma unroll
                for (int k = 0; k < R; ++k) {
                    c[k][f] = fmaf(na[k][d], b4.x, c[k][f]);
                    c[k][f + 1] = fmaf(na[k][d], b4.y, c[k][f + 1]);
                    c[k][f + 2] = fmaf(na[k][d], b4.z, c[k][f + 2]);
                    c[k][f + 3] = fmaf(na[k][d], b4.w, c[k][f + 3]);
                }
            }
    }

    float cur[R], prv[R];
#pragma unroll
    for (int k = 0; k < R; ++k) cur[k] = prv[k] = INFINITY;
    float ylp = INFINITY;
    // The failure flag is loaded one chunk ahead of its test, so the load's
    // latency never stalls the sweep.
    int status_seen = 0;
    for (int j0 = 0; j0 < Lb; j0 += kColsPerWord) {
        if (__shfl_sync(kFull, status_seen, 0) != 0) {
            br.drain();
            return;
        }
        status_seen = read_status(p.ctl);
        uint32_t word[R];
#pragma unroll
        for (int k = 0; k < R; ++k) word[k] = 0;
#pragma unroll
        for (int h = 0; h < kColsPerWord / kSub; ++h) {
            const int js = j0 + h * kSub;
            if (js >= Lb) break;
            const int nsteps = min(kSub, Lb - js);
            const int b = (js / kSub) % kRingBlk;
            // the next sub-chunk's frames: the other half of this chunk, or
            // the first half of the next chunk (waiting for its block when it
            // starts one); the last sub-chunk re-reads its own frames
            const bool has_next = js + kSub < Lb;
            const int k0 = j0 / kColsPerWord;
            if (h == 1 && has_next && ((j0 + kColsPerWord) % S::kBlk) == 0) {
                const int q = (j0 + kColsPerWord) / S::kBlk;
                if (!br.wait(q, p.ctl, p.timeout_ns)) {
                    br.drain();
                    return;
                }
                br.top_up(q, p.Bhat, Lb_pad, lane);
            }
            const float* nb = has_next ? (h == 0 ? br.chunk(k0) + kSub : br.chunk(k0 + 1))
                                       : br.chunk(k0) + h * kSub;
            float cn[R][kSub];
#pragma unroll
            for (int k = 0; k < R; ++k)
#pragma unroll
                for (int f = 0; f < kSub; ++f) cn[k][f] = kc;

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
            float gv0[kSub], gv1[kSub];  // border rows top-2, top-1 of columns js ..
            {
                const float4* s0 = reinterpret_cast<const float4*>(&myring[b][0][0]);
                const float4* s1 = reinterpret_cast<const float4*>(&myring[b][1][0]);
                const float4 a0 = s0[0], a1 = s0[1], b0 = s1[0], b1 = s1[1];
                gv0[0] = a0.x; gv0[1] = a0.y; gv0[2] = a0.z; gv0[3] = a0.w;
                gv0[4] = a1.x; gv0[5] = a1.y; gv0[6] = a1.z; gv0[7] = a1.w;
                gv1[0] = b0.x; gv1[1] = b0.y; gv1[2] = b0.z; gv1[3] = b0.w;
                gv1[4] = b1.x; gv1[5] = b1.y; gv1[6] = b1.z; gv1[7] = b1.w;
            }
            float o0[kSub], o1[kSub];  // the strip's two bottom rows (lane 30)
            float fw[R];  // backpointer fields of the sub-chunk, bits 2u, 2u+1
#pragma unroll
            for (int k = 0; k < R; ++k) fw[k] = 0.0f;
            if (nsteps == kSub) {
#pragma unroll
                for (int u = 0; u < kSub; ++u) {
                    next_cost_part<DP, R>(nb, u, na, cn);
                    float cu[R];
#pragma unroll
                    for (int k = 0; k < R; ++k) cu[k] = c[k][u];
                    dp_step<R>(cu, u, srcA, w12, ghost, gv0[u], gv1[u],
                               (h == 0) && (u == 0) && (j0 == 0) && is_origin, mu, cur, prv,
                               ylp, fw, o0[u], o1[u]);
                }
            } else {
#pragma unroll
                for (int u = 0; u < kSub; ++u) {
                    if (u >= nsteps) break;
                    float cu[R];
#pragma unroll
                    for (int k = 0; k < R; ++k) cu[k] = c[k][u];
                    dp_step<R>(cu, u, srcA, w12, ghost, gv0[u], gv1[u],
                               (h == 0) && (u == 0) && (j0 == 0) && is_origin, mu, cur, prv,
                               ylp, fw, o0[u], o1[u]);
                }
            }
#pragma unroll
            for (int k = 0; k < R; ++k) word[k] |= field_bits(fw[k], h);
            if (lane == kOutLane) {
                if (to_ring) {
                    float4* d0 = reinterpret_cast<float4*>(&nextring[b][0][0]);
                    float4* d1 = reinterpret_cast<float4*>(&nextring[b][1][0]);
                    d0[0] = make_float4(o0[0], o0[1], o0[2], o0[3]);
                    d0[1] = make_float4(o0[4], o0[5], o0[6], o0[7]);
                    d1[0] = make_float4(o1[0], o1[1], o1[2], o1[3]);
                    d1[1] = make_float4(o1[4], o1[5], o1[6], o1[7]);
                    // columns < js+nsteps of the bottom rows are in the ring below
                    st_release_s(prod_out, js + nsteps);
                } else if (to_global) {
#pragma unroll
                    for (int u = 0; u < kSub; ++u)
                        if (u < nsteps) {
                            stg1(gout + (size_t)(js + u) * 2, pack(o0[u], epoch));
                            stg1(gout + (size_t)(js + u) * 2 + 1, pack(o1[u], epoch));
                        }
                }
            }
#pragma unroll
            for (int k = 0; k < R; ++k)
#pragma unroll
                for (int f = 0; f < kSub; ++f) c[k][f] = cn[k][f];
        }
        store_words<R>(p.bp + ((size_t)strip * p.nchunk + (size_t)(j0 >> 4)) * (32 * R) +
                           (size_t)lane * R,
                       word);
    }
#pragma unroll
    for (int k = 0; k < R; ++k)
        if (!ghost && i0 + k == p.La - 1) *p.e_final = cur[k];
}

template <int DP, int R, int NW>
__global__ void __launch_bounds__(NW * 32, 1) k_dp_multirow(const DpArgs p) {
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
        run_strip<DP, R, NW>(p, g, w, lane, ring, prod, cons, br);
    }
}

template <int DP, int R>
cudaError_t launch_t(const DpArgs& a, int num_sms, cudaStream_t s) {
    constexpr int NW = kWarpsPerGroup;
    const int smem = NW * BStage<DP>::kWarpBytes;
    static DeviceSlots occupancy;
    int blocks_per_sm = 0;
    const cudaError_t e = blocks_per_sm_once(k_dp_multirow<DP, R, NW>, NW * 32, smem, occupancy,
                                             &blocks_per_sm);
    if (e != cudaSuccess) return e;
    int grid = blocks_per_sm * num_sms;
    if (grid > a.ngroups) grid = a.ngroups;
    k_dp_multirow<DP, R, NW><<<grid, NW * 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool multirow_supported(int dp, int R) {
    if (R == 2) return dp <= 32;
    if (R == 4) return dp <= 16;
    return false;
}

cudaError_t launch_dp_multirow(const DpArgs& a, int dp, int R, int num_sms, cudaStream_t s) {
    if (R == 2) {
        switch (dp) {
            case 4: return launch_t<4, 2>(a, num_sms, s);
            case 8: return launch_t<8, 2>(a, num_sms, s);
            case 12: return launch_t<12, 2>(a, num_sms, s);
            case 16: return launch_t<16, 2>(a, num_sms, s);
            case 32: return launch_t<32, 2>(a, num_sms, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (R == 4) {
        switch (dp) {
            case 4: return launch_t<4, 4>(a, num_sms, s);
            case 8: return launch_t<8, 4>(a, num_sms, s);
            case 12: return launch_t<12, 4>(a, num_sms, s);
            case 16: return launch_t<16, 4>(a, num_sms, s);
            default: return cudaErrorInvalidValue;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace pardtw
