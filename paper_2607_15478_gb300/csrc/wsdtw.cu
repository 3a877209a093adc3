// Weakly-ordered Segmental DTW (WSDTW, Sec. II-C), steps 3 to 5 on the GPU.
// Steps 1 and 2 (the fragments of A and their subsequence DTW against all of
// B) run in the batched warp-pair DP (dp_split.cu, subsequence mode), which
// leaves every fragment's last row of cumulative costs (C_seg, step 3) and its
// 2-bit backtrace matrix.  Here:
//
//   k_seg_tile,  step 4, fragment k = 0 .. N-1 in turn (two launches each):
//   k_seg_fix      match[j]   = D_seg[k-1][j - delta_k] + C_seg[k][j]
//                               (= C_seg[0][j] for k = 0; +inf for j < delta_k)
//                  D_seg[k][j] = running minimum of match over j' <= j,
//                  arg[k][j]   = the first j' attaining it,
//                as a tiled prefix scan; then the end frames
//                e_{N-1} = arg[N-1][Lb-1], e_{k-1} = arg[k-1][e_k - delta_k].
//   k_bt_subseq  step 5, one warp per fragment: the walk from (last row,
//                e_k) back to row 0 through the fragment's backtrace matrix,
//                written backwards into the fragment's slots of a scratch path.
//   k_compact    the fragment paths one after another into the caller's path.
#include <atomic>

#include "dp_device.cuh"
#include "block_walk.cuh"

namespace pardtw {

namespace {

constexpr int kSegThreads = 1024;

// (value, index) minimum where the earlier index wins ties.
struct MinArg {
    float v;
    int j;
};
__device__ __forceinline__ MinArg better(MinArg a, MinArg b) {  // a is earlier
    return (b.v < a.v) ? b : a;
}

// Step 4 runs fragment by fragment; within fragment k the running minimum
// over j is a prefix scan of (value, column) pairs (the earlier column wins
// ties), done in tiles of kTile columns by two launches:
//   k_seg_tile   every tile: its match values (coalesced), their minimum into
//                agg[tile]; the last tile to finish (a counter, no waiting)
//                turns agg into exclusive carries for all tiles;
//   k_seg_fix    every tile: the block-wide inclusive scan of its match values
//                from its carry, written as D_seg[k][*] and arg[k][*].
constexpr int kTile = 1024;

__device__ __forceinline__ float seg_match(const float* cs, const float* prev, int k, int dk,
                                           int j) {
    if (k == 0) return cs[j];
    return j - dk >= 0 ? prev[j - dk] + cs[j] : INFINITY;
}

// Block-wide inclusive scan of one (value, column) per thread, earlier wins.
__device__ __forceinline__ MinArg block_scan_min(MinArg v, MinArg* s_warp) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        MinArg o;
        o.v = __shfl_up_sync(0xffffffffu, v.v, off);
        o.j = __shfl_up_sync(0xffffffffu, v.j, off);
        if (lane >= off) v = better(o, v);
    }
    if (lane == 31) s_warp[w] = v;
    __syncthreads();
    if (w == 0) {
        MinArg x = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : MinArg{INFINITY, -1};
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            MinArg o;
            o.v = __shfl_up_sync(0xffffffffu, x.v, off);
            o.j = __shfl_up_sync(0xffffffffu, x.j, off);
            if (lane >= off) x = better(o, x);
        }
        s_warp[lane] = x;  // inclusive prefix over warps
    }
    __syncthreads();
    if (w > 0) v = better(s_warp[w - 1], v);
    return v;
}

__global__ void __launch_bounds__(kTile)
    k_seg_tile(const WsFrag* __restrict__ fr, const float* __restrict__ lastrow, size_t stride,
               int N, int Lb, int k, const int* __restrict__ delta,
               const float* __restrict__ Dseg, MinArg* __restrict__ agg,
               unsigned* __restrict__ done, DevCtl* ctl) {
    __shared__ MinArg s_warp[32];
    __shared__ bool s_last;
    const int ntile = gridDim.x;
    const int j = blockIdx.x * kTile + threadIdx.x;
    const float* cs = lastrow + (size_t)k * stride;
    const float* prev = k > 0 ? Dseg + (size_t)(k - 1) * Lb : nullptr;
    const int dk = k > 0 ? delta[k] : 0;
    MinArg v{INFINITY, -1};
    if (j < Lb) v = MinArg{seg_match(cs, prev, k, dk, j), j};
    v = block_scan_min(v, s_warp);
    if (threadIdx.x == blockDim.x - 1) {
        agg[blockIdx.x] = v;
        __threadfence();
        s_last = atomicAdd(done, 1u) == (unsigned)ntile - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // the last tile: exclusive carries of all tiles, in tile order (a few
    // hundred tiles at most), then the counter is reset for the next launch
    __threadfence();
    if (threadIdx.x == 0) {
        // a fragment whose DP failed (a bounded wait expired) fails the call
        if (k == 0)
            for (int q = 0; q < N; ++q) {
                const int st = fr[q].pctl->status;
                if (st != 0) {
                    raise_status(ctl, st, 20);
                    break;
                }
            }
        MinArg run{INFINITY, -1};
        volatile MinArg* va = agg;  // written by the other tiles of this launch
        for (int t = 0; t < ntile; ++t) {
            const MinArg a{va[t].v, va[t].j};
            va[t].v = run.v;  // carry into tile t
            va[t].j = run.j;
            run = better(run, a);
        }
        *done = 0u;
    }
}

__global__ void __launch_bounds__(kTile)
    k_seg_fix(const float* __restrict__ lastrow, size_t stride, int N, int Lb, int k,
              const int* __restrict__ delta, float* __restrict__ Dseg, int* __restrict__ arg,
              const MinArg* __restrict__ agg, int* __restrict__ ends, float* __restrict__ total,
              DevCtl* ctl) {
    __shared__ MinArg s_warp[32];
    const int j = blockIdx.x * kTile + threadIdx.x;
    const float* cs = lastrow + (size_t)k * stride;
    const float* prev = k > 0 ? Dseg + (size_t)(k - 1) * Lb : nullptr;
    const int dk = k > 0 ? delta[k] : 0;
    MinArg v{INFINITY, -1};
    if (j < Lb) v = MinArg{seg_match(cs, prev, k, dk, j), j};
    v = better(agg[blockIdx.x], block_scan_min(v, s_warp));
    if (j < Lb) {
        Dseg[(size_t)k * Lb + j] = v.v;
        arg[(size_t)k * Lb + j] = v.j;
    }
    // the last fragment's last column: the total and the end frames
    if (k == N - 1 && j == Lb - 1) {
        if (ctl->status != 0) return;
        if (!(v.v < INFINITY)) {
            raise_status(ctl, DTW_ERR_UNREACHABLE, 21);
            return;
        }
        *total = v.v;
        int e = v.j;
        ends[N - 1] = e;
        for (int q = N - 1; q > 0; --q) {
            e = arg[(size_t)(q - 1) * Lb + (e - delta[q])];
            ends[q - 1] = e;
        }
    }
}

// One warp per fragment: the subsequence path from (len-1, e_k) to row 0
// (BlockWalker), stored backwards (ascending once read from slot
// row0 + len - n) as global (row of A, frame of B) pairs.  A step that
// leaves the fragment's cells raises DTW_ERR_CUDA (it cannot happen for a
// finite end cell).
__global__ void k_bt_subseq(const WsFrag* __restrict__ fr, int N, const int* __restrict__ ends,
                            int32_t* __restrict__ scratch, int* __restrict__ count,
                            DevCtl* ctl) {
    const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (k >= N) return;
    if (ctl->status != 0) {
        if (lane == 0) count[k] = 0;
        return;
    }
    const WsFrag f = fr[k];
    int i = f.len - 1, j = ends[k];
    int n = 0;
    int32_t* out = scratch + 2 * (size_t)(f.row0 + f.len - 1);
    BlockWalker w{f.bp, f.nchunk, f.rps, f.wpb, lane};
    w.start(i, max(j, 0));
    for (;;) {
        if (lane == 0) {
            out[-2 * n] = f.row0 + i;
            out[-2 * n + 1] = j;
        }
        ++n;
        if (i == 0) break;
        const uint32_t fl = w.field(j);
        const int di = field_di(fl);
        i -= di;
        j -= field_dj(fl);
        if (i < 0 || j < 0 || n >= f.len) {
            if (lane == 0) {
                raise_status(ctl, DTW_ERR_CUDA, 22);
                count[k] = 0;
            }
            return;
        }
        w.step(di, j, i > 0);
    }
    if (lane == 0) count[k] = n;
}

// The fragment paths one after another: fragment k's n_k pairs sit at the
// end of its slots [row0, row0 + len); *path_len = sum n_k (or -status).
__global__ void __launch_bounds__(kSegThreads)
    k_compact(const WsFrag* __restrict__ fr, int N, const int* __restrict__ count,
              const int32_t* __restrict__ scratch, int32_t* __restrict__ path,
              int* __restrict__ path_len, const DevCtl* ctl) {
    const int st = ctl->status;
    if (st != 0) {
        if (threadIdx.x == 0) *path_len = -st;
        return;
    }
    int base = 0;
    for (int k = 0; k < N; ++k) {
        const int n = count[k];
        const WsFrag f = fr[k];
        const int32_t* src = scratch + 2 * (size_t)(f.row0 + f.len - n);
        for (int q = threadIdx.x; q < 2 * n; q += blockDim.x) path[2 * (size_t)base + q] = src[q];
        base += n;
    }
    if (threadIdx.x == 0) *path_len = base;
}

}  // namespace

// Lexicographic (value, column) minimum: the same choice as better() when the
// columns of the two arguments are in order, for any order of arguments.
__device__ __forceinline__ MinArg lex_min(MinArg a, MinArg b) {
    return (b.v < a.v || (b.v == a.v && b.j < a.j)) ? b : a;
}

// Barrier over the CTAs of a cooperative launch (all resident at once):
// bar[0] counts arrivals, bar[1] is the generation the last arrival bumps.
// Bounded: a CTA gives up when the call has failed (any status) or after
// waiting timeout_ns (raising DTW_ERR_TIMEOUT, detail 23), and then returns
// false, as every CTA does once the call has failed.
__device__ __forceinline__ bool grid_barrier(unsigned* bar, DevCtl* ctl, long long timeout_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = ld_acquire_g(bar + 1);
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            st_release_g(bar + 1, g + 1);
        } else {
            const long long t0 = global_ns();
            while (ld_acquire_g(bar + 1) == g) {
                if (read_status(ctl) != 0) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > timeout_ns) {
                    raise_status(ctl, DTW_ERR_TIMEOUT, 23);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        s_ok = ok && read_status(ctl) == 0;
    }
    __syncthreads();
    return s_ok;
}

// The whole segment DP in one cooperative launch: one CTA per tile of kTile
// columns, fragments one after another, two bounded grid barriers per
// fragment (the tiles' minima complete; D_seg[k] complete before fragment
// k+1 reads it).  Same values and columns as k_seg_tile + k_seg_fix.
__global__ void __launch_bounds__(kTile)
    k_seg_all(const WsFrag* __restrict__ fr, const float* __restrict__ lastrow, size_t stride,
              int N, int Lb, const int* __restrict__ delta, float* __restrict__ Dseg,
              int* __restrict__ arg, MinArg* __restrict__ agg, unsigned* __restrict__ bar,
              int* __restrict__ ends, float* __restrict__ total, DevCtl* ctl,
              long long timeout_ns) {
    __shared__ MinArg s_warp[32];
    __shared__ MinArg s_carry;
    const int t = blockIdx.x;
    const int j = t * kTile + threadIdx.x;
    // a fragment whose DP failed (a bounded wait expired) fails the call
    if (t == 0 && threadIdx.x == 0)
        for (int q = 0; q < N; ++q) {
            const int st = fr[q].pctl->status;
            if (st != 0) {
                raise_status(ctl, st, 20);
                break;
            }
        }
    MinArg v{INFINITY, -1};
    for (int k = 0; k < N; ++k) {
        const float* cs = lastrow + (size_t)k * stride;
        const float* prev = k > 0 ? Dseg + (size_t)(k - 1) * Lb : nullptr;
        const int dk = k > 0 ? delta[k] : 0;
        v = MinArg{INFINITY, -1};
        if (j < Lb) {
            // D_seg[k-1] was written by other CTAs of this launch: read through L2
            const float m = k == 0 ? cs[j] : (j - dk >= 0 ? __ldcg(prev + j - dk) + cs[j] : INFINITY);
            v = MinArg{m, j};
        }
        v = block_scan_min(v, s_warp);
        if (threadIdx.x == blockDim.x - 1) {
            volatile MinArg* va = agg;
            va[t].v = v.v;
            va[t].j = v.j;
        }
        if (!grid_barrier(bar, ctl, timeout_ns)) return;
        // the carry into this tile: the minimum over the tiles before it
        if (threadIdx.x < 32) {
            MinArg c{INFINITY, -1};
            const volatile MinArg* va = agg;
            for (int q = threadIdx.x; q < t; q += 32) c = lex_min(c, MinArg{va[q].v, va[q].j});
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                MinArg o;
                o.v = __shfl_xor_sync(0xffffffffu, c.v, off);
                o.j = __shfl_xor_sync(0xffffffffu, c.j, off);
                c = lex_min(c, o);
            }
            if (threadIdx.x == 0) s_carry = c;
        }
        __syncthreads();
        v = better(s_carry, v);
        if (j < Lb) {
            Dseg[(size_t)k * Lb + j] = v.v;
            arg[(size_t)k * Lb + j] = v.j;
        }
        if (!grid_barrier(bar, ctl, timeout_ns)) return;
    }
    // the last fragment's last column: the total and the end frames
    if (j == Lb - 1) {
        if (ctl->status != 0) return;
        if (!(v.v < INFINITY)) {
            raise_status(ctl, DTW_ERR_UNREACHABLE, 21);
            return;
        }
        *total = v.v;
        int e = v.j;
        ends[N - 1] = e;
        for (int q = N - 1; q > 0; --q) {
            e = __ldcg(arg + (size_t)(q - 1) * Lb + (e - delta[q]));
            ends[q - 1] = e;
        }
    }
}

cudaError_t launch_seg_dp(const WsFrag* fr, const float* lastrow, size_t stride, int N, int Lb,
                          const int* delta, float* Dseg, int* arg, void* agg, unsigned* done,
                          int* ends, float* total, DevCtl* ctl, long long timeout_ns,
                          cudaStream_t s) {
    const int ntile = (Lb + kTile - 1) / kTile;
    cudaError_t e = cudaMemsetAsync(done, 0, 2 * sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    // one cooperative launch when every tile's CTA can be resident at once
    // (CTAs resident on the current device, looked up once per device)
    constexpr int kMaxDev = 64;
    static std::atomic<int> resident_of[kMaxDev];  // 0 = not looked up yet, else 1 + count
    int dev = 0, resident = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        dev = -1;
    }
    if (dev >= 0 && dev < kMaxDev && resident_of[dev].load() > 0) {
        resident = resident_of[dev].load() - 1;
    } else if (dev >= 0) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_seg_all, kTile, 0) !=
                cudaSuccess) {
            (void)cudaGetLastError();
        } else {
            resident = sms * per_sm;
            if (dev < kMaxDev) resident_of[dev].store(resident + 1);
        }
    }
    if (ntile <= resident) {
        MinArg* aggp = static_cast<MinArg*>(agg);
        void* args[] = {(void*)&fr,   (void*)&lastrow, (void*)&stride, (void*)&N,
                        (void*)&Lb,   (void*)&delta,   (void*)&Dseg,   (void*)&arg,
                        (void*)&aggp, (void*)&done,    (void*)&ends,   (void*)&total,
                        (void*)&ctl,  (void*)&timeout_ns};
        return cudaLaunchCooperativeKernel((const void*)k_seg_all, dim3(ntile), dim3(kTile), args,
                                           0, s);
    }
    for (int k = 0; k < N && e == cudaSuccess; ++k) {
        k_seg_tile<<<ntile, kTile, 0, s>>>(fr, lastrow, stride, N, Lb, k, delta, Dseg,
                                           static_cast<MinArg*>(agg), done, ctl);
        k_seg_fix<<<ntile, kTile, 0, s>>>(lastrow, stride, N, Lb, k, delta, Dseg, arg,
                                          static_cast<const MinArg*>(agg), ends, total, ctl);
        e = cudaGetLastError();
    }
    return e;
}

size_t seg_dp_scratch_bytes(int Lb) { return sizeof(MinArg) * (size_t)((Lb + kTile - 1) / kTile); }

cudaError_t launch_bt_subseq(const WsFrag* fr, int N, const int* ends, int32_t* scratch,
                             int* count, int32_t* path, int* path_len, DevCtl* ctl,
                             cudaStream_t s) {
    k_bt_subseq<<<(N + 3) / 4, 128, 0, s>>>(fr, N, ends, scratch, count, ctl);
    k_compact<<<1, kSegThreads, 0, s>>>(fr, N, count, scratch, path, path_len, ctl);
    return cudaGetLastError();
}

}  // namespace pardtw
