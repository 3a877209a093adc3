// Device-side building blocks shared by the DP kernels: tagged border
// entries, acquire/release progress counters, bounded waits, the top-border
// refill from global memory, and the TMA-fed ring of B frames.
// Internal to libpardtw; every translation unit gets its own copy.
#pragma once

#include <math.h>

#include "pardtw_common.cuh"

namespace pardtw {
namespace {


constexpr int kRing = 64;  // ring capacity (columns) per warp
constexpr int kSub = 8;    // columns between two progress synchronisations
constexpr int kRingBlk = kRing / kSub;  // ring blocks of kSub columns
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
__device__ __forceinline__ unsigned long long ldg1(const unsigned long long* p) {
    unsigned long long a;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(a) : "l"(p));
    return a;
}
__device__ __forceinline__ void stg1(unsigned long long* p, unsigned long long a) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(a) : "memory");
}
// Per-strip completion flags in global memory: released by the DP warp that
// finished the strip, acquired by the band-map items that read its words.
__device__ __forceinline__ void st_release_g(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_g(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
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

// B frames (chunk-transposed, see bt_index) reach the cost computation
// through a per-warp ring of kSlots blocks in shared memory, filled by TMA
// bulk copies (cp.async.bulk) with one mbarrier per slot.  Block t of a warp's lifetime sits in slot
// t % kSlots; its mbarrier phase parity is (t / kSlots) & 1.  A copy is
// issued three blocks ahead of use, so the L2 latency never meets the
// sweep.  Only lane 0 issues; all lanes wait on the barrier.  (The wide
// FP32 cost warps of dp_split.cuh use rings of two slots: a copy one block
// ahead, each block a whole 16-frame chunk.)
template <int DP, int kSlotsT = 4>
struct BStage {
    static constexpr int kBlk = DP <= 16 ? 64 : (DP <= 32 ? 32 : 16);  // frames per copy
    static constexpr int kSlots = kSlotsT;
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


// Explicit shared-memory vector accesses (32-bit shared addresses).  Both
// are compiler memory barriers, so they stay in program order with the
// barrier waits and arrivals and with plain shared-memory accesses.
__device__ __forceinline__ float4 lds128(unsigned addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}
__device__ __forceinline__ void sts128(unsigned addr, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w)
                 : "memory");
}

// Non-blocking test of the same condition as mbar_try_wait (never suspends
// the thread), for look-ahead checks placed between independent work.
__device__ __forceinline__ int mbar_test_wait(unsigned bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return (int)done;
}

// mbarrier arrive (release at CTA scope) by the calling thread.
__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// Wait (warp-uniform) until the phase of parity `par` of `bar` has completed.
// Bounded like every other wait: gives up when the call failed elsewhere or
// the deadline passed (raising DTW_ERR_TIMEOUT with detail `where`).
__device__ __noinline__ int mbar_wait_slow(unsigned bar, unsigned par, DevCtl* ctl,
                                           long long timeout_ns, int where) {
    const long long t0 = __shfl_sync(kFull, global_ns(), 0);
    for (int poll = 1;; ++poll) {
        if (__all_sync(kFull, mbar_try_wait(bar, par))) return 1;
        if ((poll & 63) == 0) {
            if (__shfl_sync(kFull, read_status(ctl), 0) != 0) return 0;
            const long long now = __shfl_sync(kFull, global_ns(), 0);
            if (now - t0 > timeout_ns) {
                if ((threadIdx.x & 31) == 0) raise_status(ctl, DTW_ERR_TIMEOUT, where);
                return 0;
            }
        }
    }
}
__device__ __forceinline__ int mbar_wait(unsigned bar, unsigned par, DevCtl* ctl,
                                         long long timeout_ns, int where) {
    if (__all_sync(kFull, mbar_try_wait(bar, par))) return 1;
    return mbar_wait_slow(bar, par, ctl, timeout_ns, where);
}

// ---- thread-block clusters: between the strip groups of two CTAs of one
// cluster the border travels through distributed shared memory.  The
// writer warp of the CTA above copies each block of its last strip's bottom
// rows into the staging ring of the CTA below with asynchronous stores that
// complete a transaction count on that CTA's full barrier (armed for 64
// bytes per use by the receiving reader warp), so no fence orders them; the
// reader warp below, once it holds a block's values in registers, re-arms
// the full barrier and arrives on the sender's empty barrier with a count
// that depends on a loaded value, so the arrival cannot be performed before
// the loads.
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_size() {
    unsigned n;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
    return n;
}
// Barrier of every thread of the cluster (shared-memory accesses before it
// are visible to the cluster after it).
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}
// The shared::cluster address of local shared address `addr` in CTA `rank`.
__device__ __forceinline__ unsigned map_rank(unsigned addr, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_u32(unsigned addr, unsigned v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// Asynchronous 4-byte store into the shared memory of another CTA of the
// cluster; completes 4 bytes of the transaction count of `remote_bar`, an
// mbarrier of that CTA (both shared::cluster addresses).
__device__ __forceinline__ void st_async_f32(unsigned addr, float v, unsigned remote_bar) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
        "r"(__float_as_uint(v)), "r"(remote_bar)
        : "memory");
}
// Arrive on a local mbarrier and expect `bytes` more transaction bytes for
// the phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
// 0, computed from x (a register dependency on x that the compiler keeps).
__device__ __forceinline__ unsigned zero_after(unsigned x) {
    unsigned z;
    asm volatile("and.b32 %0, %1, 0;" : "=r"(z) : "r"(x));
    return z;
}
// Relaxed arrival with `count` on an mbarrier of another CTA of the cluster.
__device__ __forceinline__ void mbar_arrive_remote_relaxed(unsigned remote_bar, unsigned count) {
    asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(remote_bar),
                 "r"(count)
                 : "memory");
}

template <int DP, int kSlotsT = 4>
struct BRing {
    using S = BStage<DP, kSlotsT>;
    const float* stage;   // this warp's kSlots * kBlk frames
    unsigned stage_s;     // its shared address
    unsigned bar_s;       // shared address of this warp's kSlots mbarriers
    unsigned base;        // lifetime block number of block `first` of the current strip
    int first;            // first block of B the current strip reads
    int nblk;             // blocks of B up to the end of the strip's columns
    int issued;           // blocks of this strip issued so far (first <= issued)
    int waited;           // blocks of this strip known complete

    // Copy block q (frames q*kBlk .., whole 16-frame chunks) of the
    // chunk-transposed B (Lb_pad frames) into its slot.
    // A new strip reading blocks q0 .. nb-1: the lifetime numbering continues
    // after the blocks the previous strip issued.
    __device__ __forceinline__ void begin(int q0, int nb) {
        base += (unsigned)(issued - first);
        first = issued = waited = q0;
        nblk = nb;
    }
    __device__ __forceinline__ void issue(int q, const float* Bt, int Lb_pad, int lane) {
        if (lane == 0) {
            const unsigned t = base + (unsigned)(q - first);
            const int f0 = q * S::kBlk;
            const int nf = min(S::kBlk, Lb_pad - f0);
            tma_load(stage_s + (t % S::kSlots) * (S::kBlk * DP * 4), Bt + (size_t)f0 * DP,
                     (unsigned)(nf * DP * 4), bar_s + (t % S::kSlots) * 8);
        }
    }
    // Issue the blocks that fit ahead of block `q` (the one about to be read).
    __device__ __forceinline__ void top_up(int q, const float* Bt, int Lb_pad, int lane) {
        while (issued < nblk && issued <= q + S::kAhead) {
            issue(issued, Bt, Lb_pad, lane);
            ++issued;
        }
    }
    // Wait until block q is in shared memory (bounded); warp-uniform.
    __device__ __forceinline__ int wait(int q, DevCtl* ctl, long long timeout_ns) {
        const unsigned t = base + (unsigned)(q - first);
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
            const unsigned t = base + (unsigned)(q - first);
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
    // Shared address of the 16 x DP feature-major values of chunk k.
    __device__ __forceinline__ unsigned chunk_s(int k) const {
        const int f = k * kColsPerWord;
        const unsigned t = base + (unsigned)(f / S::kBlk - first);
        return stage_s +
               (unsigned)(((t % S::kSlots) * S::kBlk + (unsigned)(f % S::kBlk)) * DP * 4);
    }
    // The 16 x DP feature-major values of chunk k (its block must be complete).
    __device__ __forceinline__ const float* chunk(int k) const {
        const int f = k * kColsPerWord;
        const unsigned t = base + (unsigned)(f / S::kBlk - first);
        return stage + ((size_t)(t % S::kSlots) * S::kBlk + (size_t)(f % S::kBlk)) * DP;
    }
};

// 1.0f if a == b, else 0.0f (one compare that yields a float).
__device__ __forceinline__ float eq_as_float(float a, float b) {
    float r;
    asm("set.eq.f32.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// One DP step of one column for the lane's R rows (no memory access, no
// branch).  cur[k] = E[row k][j-1], prv[k] = E[row k][j-2], ylp = E[row
// above][j-2]; g0, g1 = the ghost lane's border values of column j.  u is
// the column's place in its 8-column sub-chunk: the cell's backpointer
// field (see step_of_field) is added to fw[k] at bits 2u, 2u+1 by two FMAs
// of exact powers of two, so the code costs two compares and no integer or
// select instruction.
// kSubseq: the subsequence DTW of WSDTW (Sec. II-C), weights 1, 1, 2 for
// (1,1), (1,2), (2,1) instead of 2, 3, 3.  (w12 is no longer read: the
// ghost rows' zero weight became a select of the border value.)
// kT: the pair is swept transposed (rows of the kernel = frames of B), so
// the kernel's (1,2) candidate is the problem's (2,1) and vice versa; the
// problem's tie order (1,1), (1,2), (2,1) is then the kernel's c0, c2, c1.
// Bit 1 then records that c2 attains the minimum (one compare, as in the
// direct sweep), and transpose_fields turns the finished word into the
// kernel's decoding before it is stored.  Same cells, same values, same path.
template <int R, bool kSubseq = false, bool kT = false>
__device__ __forceinline__ void dp_step(const float* cost, int u, int srcA, const float* w12,
                                        bool ghost, float g0, float g1, bool origin_here,
                                        float mu, float* cur, float* prv, float& ylp, float* fw,
                                        float& o0, float& o1) {
    (void)w12;  // the (1,2) weight: 3 (1 in the subsequence DP) on every real row
    const float y1 = __shfl_sync(kFull, cur[R - 1], srcA);  // E[i0-1][j-1]
    const float y2 = __shfl_sync(kFull, cur[R - 2], srcA);  // E[i0-2][j-1]
    const float bit0 = (float)(1u << (2 * u)), bit1 = (float)(2u << (2 * u));
    float m[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const float x1 = (k == 0) ? y1 : cur[k - 1];                       // E[i-1][j-1]
        const float x2 = (k == 0) ? y2 : ((k == 1) ? y1 : cur[k - 2]);     // E[i-2][j-1]
        const float x1p = (k == 0) ? ylp : prv[k - 1];                     // E[i-1][j-2]
        constexpr float w11 = kSubseq ? 1.0f : 2.0f, w21 = kSubseq ? 2.0f : 3.0f;
        constexpr float w12c = kSubseq ? 1.0f : 3.0f;
        const float c0 = fmaf(w11, cost[k], x1);     // from (i-1, j-1)
        // from (i-1, j-2); the ghost lane's two rows take the border value
        // here (their other candidates carry the cost 1e30), the value that
        // a weight of 0 on this candidate gave, without an FMA reading three
        // registers (those issue at 0.64-0.83 per cycle on GB300, against
        // 0.91 with a constant operand)
        float c1 = fmaf(w12c, cost[k], x1p);
        if (k == R - 2) c1 = ghost ? g0 : c1;
        if (k == R - 1) c1 = ghost ? g1 : c1;
        const float c2 = fmaf(w21, cost[k], x2);     // from (i-2, j-1)
        float mk = min3f(c0, c1, c2);
        fw[k] = fmaf(eq_as_float(c0, mk), bit0, fw[k]);
        fw[k] = fmaf(eq_as_float(kT ? c2 : c1, mk), bit1, fw[k]);
        if (k == 0) mk = origin_here ? cost[0] + mu : mk;  // E[0][0] = C[0][0]
        m[k] = mk;
    }
    o0 = m[R - 2];
    o1 = m[R - 1];
    ylp = y1;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        prv[k] = cur[k];
        cur[k] = m[k];
    }
}

// A word of the transposed sweep, whose bit 1 of each field says that the
// kernel's c2 attains the minimum, in the decoding of step_of_field: where
// bit 0 is clear (the diagonal does not attain it), the step is c2's when c2
// attains the minimum, else c1's, so bit 1 is inverted there; where bit 0 is
// set the step is the diagonal whatever bit 1 holds.
__device__ __forceinline__ uint32_t transpose_fields(uint32_t w) {
    return w ^ (~(w << 1) & 0xAAAAAAAAu);
}

// The 16 field bits a sub-chunk accumulated, as the low or high half of a
// backpointer word (h = 0 or 1).  fw is an integer below 2^16 held exactly in
// a float, so fw + 2^23 is exact and its low 16 mantissa bits are fw: an add
// and a mask in the DP warp's per-sub-chunk tail instead of a float-to-integer
// conversion (2% of the sweep, measured on GB300).
__device__ __forceinline__ uint32_t field_bits(float fw, int h) {
    return (__float_as_uint(fw + 8388608.0f) & 0xFFFFu) << (16 * h);
}

// A lane's R backpointer words of one chunk, at word offset lane * R of the
// strip's block (vector stores where the offset is aligned for them).
template <int R>
__device__ __forceinline__ void store_words(uint32_t* dst, const uint32_t* word) {
    if constexpr (R == 2) {
        *reinterpret_cast<uint2*>(dst) = make_uint2(word[0], word[1]);
    } else if constexpr (R == 4) {
        *reinterpret_cast<uint4*>(dst) = make_uint4(word[0], word[1], word[2], word[3]);
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) dst[k] = word[k];
    }
}

}  // namespace
}  // namespace pardtw
