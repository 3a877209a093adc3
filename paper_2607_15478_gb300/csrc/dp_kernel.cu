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
#include <math.h>

#include "pardtw_common.cuh"

namespace pardtw {
namespace {

constexpr int kRing = 64;  // ring capacity (columns) per warp
constexpr int kSub = 8;    // columns between two progress synchronisations
constexpr int kRingBlk = kRing / kSub;  // ring blocks of kSub columns
constexpr int kGhost0 = kRowsPerStrip;  // first ghost lane (30)
constexpr float kGhostCost = 1e30f;
constexpr int kWin = 32;   // global border columns warp 0 keeps in flight
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned long long pack(float v, unsigned tag) {
    return ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(v);
}
__device__ __forceinline__ float val_of(unsigned long long e) { return __uint_as_float((unsigned)e); }
__device__ __forceinline__ unsigned tag_of(unsigned long long e) { return (unsigned)(e >> 32); }

// Shared-memory accessors.  The progress counters are accessed with
// acquire/release semantics; their asm carries a memory clobber, so the
// compiler keeps the plain ring loads and stores of a synchronisation step
// after the acquire and before the release.
__device__ __forceinline__ int ld_acquire_s(unsigned addr) {
    int v;
    asm volatile("ld.acquire.cta.shared.b32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_s(unsigned addr, int v) {
    asm volatile("st.release.cta.shared.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// Border entries in global memory are two 64-bit words, each (value, tag);
// every word is read and written as one relaxed gpu-scope 64-bit access,
// which is single-copy atomic, so a reader can trust a word whose tag matches.
__device__ __forceinline__ void ldg2(const unsigned long long* p, unsigned long long& a,
                                     unsigned long long& b) {
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(a) : "l"(p));
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(b) : "l"(p + 1));
}
__device__ __forceinline__ void stg1(unsigned long long* p, unsigned long long a) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(a) : "memory");
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

// Polls between two checks of the call's failure flag and of the deadline.
constexpr int kFastPolls = 128;

// Wait until the shared counter at `addr` reaches `need` (acquire loads in
// every lane; the decision is a warp vote, so the warp never splits in front
// of its shuffles).  Bounded: gives up when the call fails elsewhere or the
// deadline passes.
__device__ __noinline__ int wait_counter(unsigned addr, int need, DevCtl* ctl,
                                         long long timeout_ns, int where) {
    long long t0 = 0;
    for (int round = 0;; ++round) {
        for (int k = 0; k < kFastPolls; ++k)
            if (__all_sync(kFull, ld_acquire_s(addr) >= need)) return 1;
        const long long now = __shfl_sync(kFull, global_ns(), 0);
        if (round == 0) t0 = now;
        if (__shfl_sync(kFull, read_status(ctl), 0) != 0) return 0;
        if (now - t0 > timeout_ns) {
            if ((threadIdx.x & 31) == 0) raise_status(ctl, DTW_ERR_TIMEOUT, where);
            return 0;
        }
        if (round >= 8) __nanosleep(256);
    }
}
__device__ __forceinline__ int wait_counter_fast(unsigned addr, int need, DevCtl* ctl,
                                                 long long timeout_ns, int where) {
    if (__all_sync(kFull, ld_acquire_s(addr) >= need)) return 1;
    return wait_counter(addr, need, ctl, timeout_ns, where);
}

// Warp 0 of a group g > 0: columns [js, js+kSub) of the border above, held
// in the lanes l with (l - js) mod 32 < kSub (lane l holds the column
// congruent to l mod 32 of the current kWin window), are validated by tag
// (re-polled from L2 while stale), copied into the warp's own ring block,
// and replaced by the loads of the columns kWin further on.
__device__ __forceinline__ int refill_top(float (*blk)[kSub], int js, int lane, int Lb,
                                          const unsigned long long* gin, unsigned epoch,
                                          unsigned long long& g0, unsigned long long& g1,
                                          DevCtl* ctl, long long timeout_ns) {
    const int off = (lane - js) & (kWin - 1);
    const int col = js + off;
    const bool act = off < kSub && col < Lb;
    int ok = !act || (tag_of(g0) == epoch && tag_of(g1) == epoch);
    if (!__all_sync(kFull, ok)) {
        // each poll is a round trip to L2; status and deadline every 16 polls
        const long long t0 = __shfl_sync(kFull, global_ns(), 0);
        for (int poll = 1;; ++poll) {
            if (!ok) {
                ldg2(gin + (size_t)col * 2, g0, g1);
                ok = tag_of(g0) == epoch && tag_of(g1) == epoch;
            }
            if (__all_sync(kFull, ok)) break;
            if ((poll & 15) == 0) {
                if (__shfl_sync(kFull, read_status(ctl), 0) != 0) return 0;
                const long long now = __shfl_sync(kFull, global_ns(), 0);
                if (now - t0 > timeout_ns) {
                    if (lane == 0) raise_status(ctl, DTW_ERR_TIMEOUT, 3);
                    return 0;
                }
                if (poll >= 256) __nanosleep(256);
            }
        }
    }
    if (act) {
        blk[0][off] = val_of(g0);
        blk[1][off] = val_of(g1);
        if (col + kWin < Lb) ldg2(gin + (size_t)(col + kWin) * 2, g0, g1);
    }
    __syncwarp();
    return 1;
}

// B frames reach the cost computation through a per-warp ring of kSlots
// blocks in shared memory, filled by TMA bulk copies (cp.async.bulk) with
// one mbarrier per slot.  Block t of a warp's lifetime sits in slot
// t % kSlots; its mbarrier phase parity is (t / kSlots) & 1.  A copy is
// issued three blocks ahead of use, so the L2 latency never meets the
// sweep.  Only lane 0 issues; all lanes wait on the barrier.
template <int DP>
struct BStage {
    static constexpr int kBlk = DP <= 16 ? 64 : (DP <= 32 ? 32 : 16);  // frames per copy
    static constexpr int kSlots = 4;
    static constexpr int kAhead = kSlots - 1;
    static constexpr int kWarpBytes = kSlots * kBlk * DP * 4;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ int mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return (int)done;
}
// Lane 0: copy `bytes` from global `src` into shared `dst`, completing on `bar`.
__device__ __forceinline__ void tma_load(unsigned dst, const void* src, unsigned bytes,
                                         unsigned bar) {
    // earlier generic-proxy reads of this slot are ordered before the
    // async-proxy write
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

template <int DP>
struct BRing {
    using S = BStage<DP>;
    const float* stage;   // this warp's kSlots * kBlk frames
    unsigned stage_s;     // its shared address
    unsigned bar_s;       // shared address of this warp's kSlots mbarriers
    unsigned base;        // lifetime block number of block 0 of the current strip
    int nblk;             // blocks in the current strip (ceil(Lb / kBlk))
    int issued;           // blocks of this strip issued so far
    int waited;           // blocks of this strip known complete

    __device__ __forceinline__ void issue(int q, const float* Bhat, int Lb, int lane) {
        if (lane == 0) {
            const unsigned t = base + (unsigned)q;
            const int f0 = q * S::kBlk;
            const int nf = min(S::kBlk, Lb - f0);
            tma_load(stage_s + (t % S::kSlots) * (S::kBlk * DP * 4), Bhat + (size_t)f0 * DP,
                     (unsigned)(nf * DP * 4), bar_s + (t % S::kSlots) * 8);
        }
    }
    // Issue the blocks that fit ahead of block `q` (the one about to be read).
    __device__ __forceinline__ void top_up(int q, const float* Bhat, int Lb, int lane) {
        while (issued < nblk && issued <= q + S::kAhead) {
            issue(issued, Bhat, Lb, lane);
            ++issued;
        }
    }
    // Wait until block q is in shared memory (bounded); warp-uniform.
    __device__ __forceinline__ int wait(int q, DevCtl* ctl, long long timeout_ns) {
        const unsigned t = base + (unsigned)q;
        const unsigned bar = bar_s + (t % S::kSlots) * 8;
        const unsigned par = (t / S::kSlots) & 1u;
        if (__all_sync(kFull, mbar_try_wait(bar, par))) {
            waited = q + 1;
            return 1;
        }
        const long long t0 = __shfl_sync(kFull, global_ns(), 0);
        for (int poll = 1;; ++poll) {
            if (__all_sync(kFull, mbar_try_wait(bar, par))) {
                waited = q + 1;
                return 1;
            }
            if ((poll & 63) == 0) {
                if (__shfl_sync(kFull, read_status(ctl), 0) != 0) return 0;
                const long long now = __shfl_sync(kFull, global_ns(), 0);
                if (now - t0 > timeout_ns) {
                    if ((threadIdx.x & 31) == 0) raise_status(ctl, DTW_ERR_TIMEOUT, 4);
                    return 0;
                }
            }
        }
    }
    // Before leaving a strip early: let every issued copy land (bounded), so
    // no bulk copy is still writing this CTA's shared memory.
    __device__ __forceinline__ void drain() {
        for (int q = waited; q < issued; ++q) {
            const unsigned t = base + (unsigned)q;
            const unsigned bar = bar_s + (t % S::kSlots) * 8;
            const unsigned par = (t / S::kSlots) & 1u;
            const long long t0 = __shfl_sync(kFull, global_ns(), 0);
            while (!__all_sync(kFull, mbar_try_wait(bar, par))) {
                const long long now = __shfl_sync(kFull, global_ns(), 0);
                if (now - t0 > 1000000000LL) break;  // 1 s: give up on this copy
            }
        }
        waited = issued;
    }
    // Frame f of the strip (its block must be complete).
    __device__ __forceinline__ const float4* frame(int f) const {
        const unsigned t = base + (unsigned)(f / S::kBlk);
        return reinterpret_cast<const float4*>(stage + ((size_t)(t % S::kSlots) * S::kBlk +
                                                        (size_t)(f % S::kBlk)) * DP);
    }
};

// C' = (1 - mu) - a^_i . b^_j: one FMA per feature, in feature order, from
// the negated row a^_i held in registers and the frame b^_j in shared memory
// (broadcast reads: every lane reads the same address).
template <int DP>
__device__ __forceinline__ float cost_of(const float* na, float kcost, const float4* b) {
    float acc = kcost;
#pragma unroll
    for (int q = 0; q < DP / 4; ++q) {
        const float4 v = b[q];
        acc = fmaf(na[4 * q], v.x, acc);
        acc = fmaf(na[4 * q + 1], v.y, acc);
        acc = fmaf(na[4 * q + 2], v.z, acc);
        acc = fmaf(na[4 * q + 3], v.w, acc);
    }
    return acc;
}

// One DP step of column j for the warp's 32 lanes: no memory access and no
// branch.  Lane sources srcA = lane-1, srcB = lane-2 (mod 32) give rows i-1
// and i-2 of column j-1; x1p holds row i-1 of column j-2 (for a ghost lane:
// its own border value of column j).
__device__ __forceinline__ void dp_step(float cost, unsigned bit, int srcA, int srcB, float w12,
                                        bool origin_here, float mu, float& cur, float& x1p,
                                        float& x1, uint32_t& word, float& out) {
    x1 = __shfl_sync(kFull, cur, srcA);        // E[i-1][j-1]
    const float x2 = __shfl_sync(kFull, cur, srcB);  // E[i-2][j-1]
    const float c0 = fmaf(2.0f, cost, x1);  // from (i-1, j-1)
    const float c1 = fmaf(w12, cost, x1p);  // from (i-1, j-2)
    const float c2 = fmaf(3.0f, cost, x2);  // from (i-2, j-1)
    float m = min3f(c0, c1, c2);
    const uint32_t code = (c0 == m) ? 0u : ((c1 == m) ? 1u : 2u);
    m = origin_here ? cost + mu : m;  // E[0][0] = C[0][0]
    word |= code << bit;
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
    br.base += (unsigned)br.nblk;  // continue the lifetime block numbering
    br.nblk = (Lb + S::kBlk - 1) / S::kBlk;
    br.issued = 0;
    br.waited = 0;
    br.top_up(0, p.Bhat, Lb, lane);
    unsigned long long g0 = 0, g1 = 0;
    if (from_global && lane < Lb) ldg2(gin + (size_t)lane * 2, g0, g1);

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
        if ((j0 % S::kBlk) == 0) {
            const int q = j0 / S::kBlk;
            if (!br.wait(q, p.ctl, p.timeout_ns)) {
                br.drain();
                return;
            }
            br.top_up(q, p.Bhat, Lb, lane);
        }
        // the chunk's costs C' = (1 - mu) - a^_i . b^_j (1e30 in ghost lanes)
        float c[kColsPerWord];
        {
            const float4* fb = br.frame(j0);
            if (j0 + kColsPerWord <= Lb) {
#pragma unroll
                for (int u = 0; u < kColsPerWord; ++u)
                    c[u] = cost_of<DP>(na, kcost, fb + u * (DP / 4));
            } else {
#pragma unroll
                for (int u = 0; u < kColsPerWord; ++u)
                    c[u] = (j0 + u < Lb) ? cost_of<DP>(na, kcost, fb + u * (DP / 4)) : 0.f;
            }
        }
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
            if (nsteps == kSub) {
#pragma unroll
                for (int u = 0; u < kSub; ++u) {
                    const int uu = h * kSub + u;
                    dp_step(c[uu], 2u * uu, srcA, srcB, w12, (uu == 0) && (j0 == 0) && is_origin,
                            mu, cur, x1p, x1, word, o[u]);
                    x1p = (u + 1 < kSub && ghost) ? gv[u + 1 < kSub ? u + 1 : 0] : x1;
                }
            } else {
#pragma unroll
                for (int u = 0; u < kSub; ++u) {
                    const int uu = h * kSub + u;
                    if (u >= nsteps) break;
                    dp_step(c[uu], 2u * uu, srcA, srcB, w12, (uu == 0) && (j0 == 0) && is_origin,
                            mu, cur, x1p, x1, word, o[u]);
                    x1p = (u + 1 < kSub && ghost) ? gv[u + 1 < kSub ? u + 1 : 0] : x1;
                }
            }
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
        p.bp[((size_t)strip * p.nchunk + (size_t)(j0 >> 4)) * 32 + lane] = word;
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
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_dp<DP, NW>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_dp<DP, NW>, NW * 32,
                                                          smem);
        if (e != cudaSuccess) return e;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
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
