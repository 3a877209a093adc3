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
//   - A warp owns a strip of 32 consecutive rows of A, one row per lane, and
//     sweeps all Lb columns; each lane keeps its row's two live cumulative
//     values in registers and the normalised frame a_i in registers.
//   - Rows i-1 and i-2 of column j-1 come from the lanes above through warp
//     shuffles; lanes 0 and 1 take the two bottom rows of the strip above
//     from a tagged ring in shared memory (strip above in the same CTA) or
//     from a tagged border buffer in global memory (strip above in another
//     CTA).  Ring and border entries carry a tag in the same 64-bit word as
//     the value, so a reader never needs a fence: a matching tag proves the
//     value is the one it waits for.
//   - A CTA owns kWarpsPerGroup consecutive strips (a "strip group");
//     persistent CTAs take groups in order from an atomic ticket, so every
//     group a CTA waits on was taken earlier by a running CTA.
//   - Each lane packs 16 columns of 2-bit codes into a uint32; the warp
//     stores 32 consecutive words (128 bytes) per 16 columns.
//   - Every wait is bounded in time; on expiry the kernel records
//     DTW_ERR_TIMEOUT and all CTAs leave.
#include <math.h>

#include "pardtw_common.cuh"

namespace pardtw {
namespace {

constexpr int kRing = 64;  // ring slots (columns) per warp
constexpr int kRingMask = kRing - 1;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long pack(float v, unsigned tag) {
    return ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(v);
}
__device__ __forceinline__ float val_of(unsigned long long e) { return __uint_as_float((unsigned)e); }
__device__ __forceinline__ unsigned tag_of(unsigned long long e) { return (unsigned)(e >> 32); }

__device__ __forceinline__ void lds2(const unsigned long long* p, unsigned long long& a,
                                     unsigned long long& b) {
    asm volatile("ld.volatile.shared.v2.u64 {%0, %1}, [%2];"
                 : "=l"(a), "=l"(b)
                 : "r"((unsigned)__cvta_generic_to_shared(p)));
}
__device__ __forceinline__ void sts2(unsigned long long* p, unsigned long long a,
                                     unsigned long long b) {
    asm volatile("st.volatile.shared.v2.u64 [%0], {%1, %2};" ::"r"(
                     (unsigned)__cvta_generic_to_shared(p)),
                 "l"(a), "l"(b));
}
// Border entries in global memory are two 64-bit words, each (value, tag);
// every word is read and written as one relaxed gpu-scope 64-bit access,
// which is single-copy atomic, so a reader can trust a word whose tag matches.
__device__ __forceinline__ void ldg2(const unsigned long long* p, unsigned long long& a,
                                     unsigned long long& b) {
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(a) : "l"(p));
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(b) : "l"(p + 1));
}
__device__ __forceinline__ void stg2(unsigned long long* p, unsigned long long a,
                                     unsigned long long b) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(a));
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p + 1), "l"(b));
}
__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int read_status(const DevCtl* c) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(&c->status));
    return v;
}
__device__ __forceinline__ void raise_status(DevCtl* c, int code, int detail) {
    if (atomicCAS(&c->status, 0, code) == 0) atomicExch(&c->detail, detail);
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float m;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(m) : "f"(a), "f"(b), "f"(c));
    return m;
}

struct Entry {
    unsigned long long e0, e1;
    int ok;
};

// Slow path of a ring read: poll the slot until its tags match in every
// lane, the call fails elsewhere, or the deadline passes.  Every decision is
// a warp vote or comes from lane 0: lanes of a warp are not guaranteed to
// execute a load together, so two lanes may see different tags, and a
// per-lane branch in front of the warp-wide shuffles would be unsafe.
__device__ __noinline__ Entry wait_ring_slot(const unsigned long long* slot, unsigned tag,
                                             DevCtl* ctl, long long timeout_ns, int where) {
    Entry r;
    const long long t0 = __shfl_sync(kFull, global_ns(), 0);
    for (;;) {
        __nanosleep(40);
        lds2(slot, r.e0, r.e1);
        if (__all_sync(kFull, tag_of(r.e0) == tag && tag_of(r.e1) == tag)) {
            r.ok = 1;
            return r;
        }
        const int st = __shfl_sync(kFull, read_status(ctl), 0);
        if (st != 0) break;
        const long long now = __shfl_sync(kFull, global_ns(), 0);
        if (now - t0 > timeout_ns) {
            if ((threadIdx.x & 31) == 0) raise_status(ctl, DTW_ERR_TIMEOUT, where);
            break;
        }
    }
    r.ok = 0;
    return r;
}

// Producer side of a ring: wait until the consumer warp has read far enough
// that the slots about to be overwritten are free.
__device__ __noinline__ int wait_consumer(const volatile int* cons, int need, DevCtl* ctl,
                                          long long timeout_ns) {
    const long long t0 = __shfl_sync(kFull, global_ns(), 0);
    for (;;) {
        __nanosleep(40);
        if (__shfl_sync(kFull, *cons, 0) >= need) return 1;
        if (__shfl_sync(kFull, read_status(ctl), 0) != 0) return 0;
        const long long now = __shfl_sync(kFull, global_ns(), 0);
        if (now - t0 > timeout_ns) {
            if ((threadIdx.x & 31) == 0) raise_status(ctl, DTW_ERR_TIMEOUT, 2);
            return 0;
        }
    }
}

// Warp 0 of a group: move the next 32 columns of the top border into its
// ring.  For group 0 the border is +inf (no rows above row 0).  Otherwise
// (g0, g1) hold the entries of columns [j0, j0+32) loaded one block earlier
// from the group above; they are validated by tag (re-polled if stale), then
// the loads of the following block are issued.
__device__ __forceinline__ int refill_top(unsigned long long* myring, int j0, int lane, int Lb,
                                          int g, const unsigned long long* gin, unsigned epoch,
                                          unsigned long long& g0, unsigned long long& g1,
                                          DevCtl* ctl, long long timeout_ns) {
    const int col = j0 + lane;
    if (g == 0) {
        if (col < Lb)
            sts2(myring + (col & kRingMask) * 2, pack(INFINITY, col + 1), pack(INFINITY, col + 1));
        __syncwarp();
        return 1;
    }
    if (j0 == 0 && col < Lb) ldg2(gin + (size_t)col * 2, g0, g1);
    int ok = col >= Lb || (tag_of(g0) == epoch && tag_of(g1) == epoch);
    if (!__all_sync(kFull, ok)) {
        const long long t0 = __shfl_sync(kFull, global_ns(), 0);
        for (;;) {
            __nanosleep(200);
            if (!ok) {
                ldg2(gin + (size_t)col * 2, g0, g1);
                ok = tag_of(g0) == epoch && tag_of(g1) == epoch;
            }
            if (__all_sync(kFull, ok)) break;
            if (__shfl_sync(kFull, read_status(ctl), 0) != 0) return 0;
            const long long now = __shfl_sync(kFull, global_ns(), 0);
            if (now - t0 > timeout_ns) {
                if (lane == 0) raise_status(ctl, DTW_ERR_TIMEOUT, 3);
                return 0;
            }
        }
    }
    if (col < Lb)
        sts2(myring + (col & kRingMask) * 2, pack(val_of(g0), col + 1), pack(val_of(g1), col + 1));
    if (col + 32 < Lb) ldg2(gin + (size_t)(col + 32) * 2, g0, g1);
    __syncwarp();
    return 1;
}

// The B frame of one column.  Small frames (DP <= 16) are loaded one step
// ahead into registers; larger ones are streamed from L1 inside the dot
// product to keep the register count bounded.
template <int DP, bool kHold = (DP <= 16)>
struct BFrame {
    float4 v[DP / 4];
    __device__ __forceinline__ void load(const float* Bhat, int j) {
        const float4* s = reinterpret_cast<const float4*>(Bhat + (size_t)j * DP);
#pragma unroll
        for (int q = 0; q < DP / 4; ++q) v[q] = __ldg(s + q);
    }
    __device__ __forceinline__ float dot_from(const float* na, float acc, const float*, int) const {
#pragma unroll
        for (int q = 0; q < DP / 4; ++q) {
            acc = fmaf(na[4 * q], v[q].x, acc);
            acc = fmaf(na[4 * q + 1], v[q].y, acc);
            acc = fmaf(na[4 * q + 2], v[q].z, acc);
            acc = fmaf(na[4 * q + 3], v[q].w, acc);
        }
        return acc;
    }
};
template <int DP>
struct BFrame<DP, false> {
    __device__ __forceinline__ void load(const float*, int) {}
    __device__ __forceinline__ float dot_from(const float* na, float acc, const float* Bhat,
                                              int j) const {
        const float4* s = reinterpret_cast<const float4*>(Bhat + (size_t)j * DP);
#pragma unroll
        for (int q = 0; q < DP / 4; ++q) {
            const float4 b = __ldg(s + q);
            acc = fmaf(na[4 * q], b.x, acc);
            acc = fmaf(na[4 * q + 1], b.y, acc);
            acc = fmaf(na[4 * q + 2], b.z, acc);
            acc = fmaf(na[4 * q + 3], b.w, acc);
        }
        return acc;
    }
};

// One warp sweeps its 32-row strip over all columns.
template <int DP, int NW>
__device__ __forceinline__ void run_strip(const DpArgs& p, int g, int w, int lane,
                                          unsigned long long (*ring)[kRing][2],
                                          volatile int* cons) {
    const int strip = g * NW + w;
    if (strip >= p.nstrips) return;
    const int i = strip * kRowsPerStrip + lane;
    const int Lb = p.Lb;

    float na[DP];  // -a^_i
    {
        const float4* s = reinterpret_cast<const float4*>(p.Ahat + (size_t)i * DP);
#pragma unroll
        for (int q = 0; q < DP / 4; ++q) {
            const float4 v = __ldg(s + q);
            na[4 * q] = -v.x;
            na[4 * q + 1] = -v.y;
            na[4 * q + 2] = -v.z;
            na[4 * q + 3] = -v.w;
        }
    }
    const bool to_ring = (w + 1 < NW) && (strip + 1 < p.nstrips);
    const bool to_global = (w == NW - 1) && (g + 1 < p.ngroups) && (g != p.skip_publish);
    unsigned long long* myring = &ring[w][0][0];
    unsigned long long* nextring = &ring[(w + 1) % NW][0][0];
    unsigned long long* gout = p.gborder + (size_t)g * Lb * 2;
    const unsigned long long* gin = p.gborder + (size_t)(g > 0 ? g - 1 : 0) * Lb * 2;
    const float kcost = p.kcost;
    const bool is_origin = (i == 0);

    float cur = INFINITY;  // E[i][j-1]
    float x1p = INFINITY;  // E[i-1][j-2]
    unsigned long long g0 = 0, g1 = 0;
    BFrame<DP> bcur;
    bcur.load(p.Bhat, 0);

    // The failure flag is loaded one chunk ahead of its test, so the load's
    // latency never stalls the sweep.
    int status_seen = 0;
    for (int j0 = 0; j0 < Lb; j0 += kColsPerWord) {
        if (__shfl_sync(kFull, status_seen, 0) != 0) return;
        status_seen = read_status(p.ctl);
        if (w > 0 && lane == 0) {
            __threadfence_block();
            cons[w] = j0;
        }
        if (to_ring) {
            const int need = j0 + kColsPerWord + 2 - kRing;
            if (need > 0 && __shfl_sync(kFull, cons[w + 1], 0) < need)
                if (!wait_consumer(&cons[w + 1], need, p.ctl, p.timeout_ns)) return;
        }
        if (w == 0 && (j0 & 31) == 0)
            if (!refill_top(myring, j0, lane, Lb, g, gin, p.epoch, g0, g1, p.ctl, p.timeout_ns))
                return;

        uint32_t word = 0;
#pragma unroll
        for (int u = 0; u < kColsPerWord; ++u) {
            const int j = j0 + u;
            if (j >= Lb) break;
            BFrame<DP> bnext;
            if (j + 1 < Lb) bnext.load(p.Bhat, j + 1);

            // C' = (1 - mu) - a^_i . b^_j, one FMA per feature in order
            const float acc = bcur.dot_from(na, kcost, p.Bhat, j);

            // the strip above: E[top-2][j-1], E[top-1][j-1]
            float t30 = INFINITY, t31 = INFINITY;
            if (j > 0) {
                const unsigned long long* slot = myring + ((j - 1) & kRingMask) * 2;
                Entry e;
                lds2(slot, e.e0, e.e1);
                if (!__all_sync(kFull, tag_of(e.e0) == (unsigned)j &&
                                           tag_of(e.e1) == (unsigned)j)) {
                    e = wait_ring_slot(slot, (unsigned)j, p.ctl, p.timeout_ns, 1);
                    if (!e.ok) return;
                }
                t30 = val_of(e.e0);
                t31 = val_of(e.e1);
            }
            float x1 = __shfl_up_sync(kFull, cur, 1);  // E[i-1][j-1]
            float x2 = __shfl_up_sync(kFull, cur, 2);  // E[i-2][j-1]
            if (lane == 0) {
                x1 = t31;
                x2 = t30;
            }
            if (lane == 1) x2 = t31;

            const float c0 = fmaf(2.0f, acc, x1);   // from (i-1, j-1)
            const float c1 = fmaf(3.0f, acc, x1p);  // from (i-1, j-2)
            const float c2 = fmaf(3.0f, acc, x2);   // from (i-2, j-1)
            float m = min3f(c0, c1, c2);
            const uint32_t code = (c0 == m) ? 0u : ((c1 == m) ? 1u : 2u);
            if (j == 0 && is_origin) m = acc + p.mu;  // E[0][0] = C[0][0]
            word |= code << (2 * u);

            // bottom two rows of this strip, column j-1, to the strip below
            if (lane == 31 && j > 0) {
                if (to_ring)
                    sts2(nextring + ((j - 1) & kRingMask) * 2, pack(x1, j), pack(cur, j));
                else if (to_global)
                    stg2(gout + (size_t)(j - 1) * 2, pack(x1, p.epoch), pack(cur, p.epoch));
            }
            x1p = x1;
            cur = m;
            bcur = bnext;
        }
        p.bp[((size_t)strip * p.nchunk + (size_t)(j0 >> 4)) * 32 + lane] = word;
    }
    // column Lb-1 of the bottom rows
    const float xl = __shfl_up_sync(kFull, cur, 1);
    if (lane == 31) {
        if (to_ring)
            sts2(nextring + ((Lb - 1) & kRingMask) * 2, pack(xl, Lb), pack(cur, Lb));
        else if (to_global)
            stg2(gout + (size_t)(Lb - 1) * 2, pack(xl, p.epoch), pack(cur, p.epoch));
    }
    if (i == p.La - 1) *p.e_final = cur;
}

template <int DP, int NW>
__global__ void __launch_bounds__(NW * 32, DP <= 32 ? 4 : 1) k_dp(const DpArgs p) {
    __shared__ __align__(16) unsigned long long ring[NW][kRing][2];
    __shared__ volatile int cons[NW];
    __shared__ int s_group;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        __syncthreads();  // every warp finished the previous group
        if (threadIdx.x == 0) {
            s_group = read_status(p.ctl) != 0 ? p.ngroups : atomicAdd(&p.ctl->ticket, 1);
        }
        for (int k = threadIdx.x; k < NW * kRing; k += blockDim.x) {
            ring[k / kRing][k % kRing][0] = 0ull;
            ring[k / kRing][k % kRing][1] = 0ull;
        }
        if (threadIdx.x < NW) cons[threadIdx.x] = 0;
        __syncthreads();
        const int g = s_group;
        if (g >= p.ngroups) return;
        run_strip<DP, NW>(p, g, w, lane, ring, cons);
    }
}

template <int DP>
cudaError_t launch_dp_t(const DpArgs& a, int num_sms, cudaStream_t s) {
    constexpr int NW = kWarpsPerGroup;
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        cudaError_t e =
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_dp<DP, NW>, NW * 32, 0);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    int grid = blocks_per_sm * num_sms;
    if (grid > a.ngroups) grid = a.ngroups;
    k_dp<DP, NW><<<grid, NW * 32, 0, s>>>(a);
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
