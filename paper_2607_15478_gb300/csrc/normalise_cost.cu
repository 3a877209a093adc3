// Per-frame L2 normalisation and the explicit cosine cost matrix.
//
// The cosine cost of Sec. IV is C[i][j] = 1 - (a_i . b_j) / (|a_i| |b_j|).
// The kernels normalise every frame once (a zero frame stays zero, so its
// cost against anything is 1) and then form 1 - a^_i . b^_j with one FP32
// fused multiply-add per feature, in feature order.  The DP kernel computes
// the cost of each cell the same way on the fly (Sec. II-D: the cost
// matrix is never stored); dtw_cost materialises it for inspection.
#include <cuda_bf16.h>

#include "pardtw_common.cuh"

namespace pardtw {

int padded_dim(int D) {
    static const int sizes[] = {4, 8, 12, 16, 32, 64, 128};
    for (int s : sizes)
        if (D <= s) return s;
    return 0;
}

// One thread per frame.  A is written row-major (La_pad x dp), B
// chunk-transposed (bt_index, Lb_pad frames).  Frames of A beyond La, frames
// of B beyond Lb and feature slots beyond D are zero.  Thread 0 also clears
// the control words of the call.
__device__ __forceinline__ void normalise_frame(int t, const float* __restrict__ A, int La,
                                                int La_pad, const float* __restrict__ B, int Lb,
                                                int Lb_pad, int D, int dp,
                                                float* __restrict__ Ahat, float* __restrict__ Bt,
                                                DevCtl* ctl) {
    if (t == 0) {
        ctl->status = 0;
        ctl->detail = 0;
        ctl->ticket = 0;
    }
    const float* src;
    bool valid, is_a;
    int k;
    if (t < La_pad) {
        k = t;
        src = A + (size_t)t * D;
        valid = t < La;
        is_a = true;
    } else if (t < La_pad + Lb_pad) {
        k = t - La_pad;
        src = B + (size_t)k * D;
        valid = k < Lb;
        is_a = false;
    } else {
        return;
    }
    float ss = 0.f;
    if (valid)
        for (int d = 0; d < D; ++d) {
            const float v = src[d];
            ss = fmaf(v, v, ss);
        }
    const float r = ss > 0.f ? 1.0f / sqrtf(ss) : 0.f;
    for (int d = 0; d < dp; ++d) {
        const float v = (valid && d < D) ? src[d] * r : 0.f;
        if (is_a)
            Ahat[(size_t)k * dp + d] = v;
        else
            Bt[bt_index(k, d, dp)] = v;
    }
}

__global__ void k_normalise(const float* __restrict__ A, int La, int La_pad,
                            const float* __restrict__ B, int Lb, int Lb_pad, int D, int dp,
                            float* __restrict__ Ahat, float* __restrict__ Bt, DevCtl* ctl) {
    normalise_frame(blockIdx.x * blockDim.x + threadIdx.x, A, La, La_pad, B, Lb, Lb_pad, D, dp,
                    Ahat, Bt, ctl);
}

// One pair per blockIdx.y (the grid covers the largest pair); also clears the
// batch's work-queue ticket.
__global__ void k_normalise_many(const NormArgs* __restrict__ many, int D, int dp, int* ticket) {
    const NormArgs& a = many[blockIdx.y];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0 && blockIdx.y == 0) *ticket = 0;
    normalise_frame(t, a.A, a.La, a.La_pad, a.B, a.Lb, a.Lb_pad, D, dp, a.Ahat, a.Bt, a.ctl);
}

// A replayed batch graph starts with this: a new tag for the border entries
// of every pair (entries left by the previous replay carry the old one).
__global__ void k_bump_epoch(DpArgs* many, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    unsigned e = many[k].epoch + 1u;
    many[k].epoch = e == 0u ? 1u : e;
}

cudaError_t launch_bump_epoch(DpArgs* many, int n, cudaStream_t s) {
    k_bump_epoch<<<(n + 127) / 128, 128, 0, s>>>(many, n);
    return cudaGetLastError();
}

cudaError_t launch_normalise(const float* A, int La, int La_pad, const float* B, int Lb,
                             int Lb_pad, int D, int dp, float* Ahat, float* Bt, DevCtl* ctl,
                             cudaStream_t s) {
    const int n = La_pad + Lb_pad;
    const int threads = 256;
    k_normalise<<<(n + threads - 1) / threads, threads, 0, s>>>(A, La, La_pad, B, Lb, Lb_pad, D,
                                                                dp, Ahat, Bt, ctl);
    return cudaGetLastError();
}

// One warp per frame of B: normalise in FP32 (the same sum of squares and
// reciprocal square root as k_normalise), round each feature to bf16.
__global__ void k_pack_b_bf16(const float* __restrict__ B, int Lb, int Lb_pad, int D,
                              __nv_bfloat16* __restrict__ Bbf) {
    const int f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (f >= Lb_pad) return;
    float r = 0.f;
    if (f < Lb && lane == 0) {
        float ss = 0.f;
        for (int d = 0; d < D; ++d) {
            const float v = B[(size_t)f * D + d];
            ss = fmaf(v, v, ss);
        }
        r = ss > 0.f ? 1.0f / sqrtf(ss) : 0.f;
    }
    r = __shfl_sync(0xffffffffu, r, 0);
    for (int d = lane; d < kBfStride; d += 32) {
        const float v = (f < Lb && d < D) ? B[(size_t)f * D + d] * r : 0.f;
        Bbf[(size_t)f * kBfStride + d] = __float2bfloat16_rn(v);
    }
}

cudaError_t launch_pack_b_bf16(const float* B, int Lb, int Lb_pad, int D, void* Bbf,
                               cudaStream_t s) {
    const int warps = 8;
    k_pack_b_bf16<<<(Lb_pad + warps - 1) / warps, warps * 32, 0, s>>>(
        B, Lb, Lb_pad, D, static_cast<__nv_bfloat16*>(Bbf));
    return cudaGetLastError();
}

cudaError_t launch_normalise_many(const NormArgs* many, int n, int max_frames, int D, int dp,
                                  int* ticket, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    dim3 grid((unsigned)((max_frames + threads - 1) / threads), (unsigned)n);
    k_normalise_many<<<grid, threads, 0, s>>>(many, D, dp, ticket);
    return cudaGetLastError();
}

// C[i][j] = 1 - sum_d a^_i[d] b^_j[d], accumulated as fma(-a, b, acc) from 1
// in feature order -- bit-identical to the cost the DP kernel uses.
// Writing the matrix is the whole cost of this kernel (4 bytes a cell against
// (La + Lb) * D * 4 bytes read), so it is laid out for the HBM write: a block
// of 256 threads covers kCostCols columns and takes tiles of kCostRows rows
// (about 8192 blocks, each over several tiles); thread (tx, ty) makes the 4 x 4
// cells of columns 4 tx .. 4 tx + 3 and rows 4 ty .. 4 ty + 3 of each tile.
// b^ comes as one 16-byte word per feature (bt_index puts 16 consecutive frames
// of a feature side by side), a^ as 16-byte broadcast loads (a warp holds one
// ty), and each row of 4 results is one 16-byte store when the rows are
// 16-byte aligned (Lb % 4 == 0), else four 4-byte stores.  Loading b^ per tile
// from the chunk layout costs ~8 L1 wavefronts per warp load (a warp's 128
// columns span 8 chunks): that, not HBM, bounded the first form of this kernel
// (3.3 TB/s against 7.6 for a plain write), hence the registers below.
constexpr int kCostRows = 16, kCostCols = 256, kCostMaxDp = 128;

// The rows i0 .. i0+3 of a thread's tile against its 4 columns, features
// d0 .. d0+3 (b[u]: the 4 columns' values of feature d0 + u).
__device__ __forceinline__ void cost_fma4(float (&acc)[4][4], const float4 (&a)[4],
                                          const float4 (&b)[4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float av[4] = {a[r].x, a[r].y, a[r].z, a[r].w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            acc[r][0] = fmaf(-av[u], b[u].x, acc[r][0]);
            acc[r][1] = fmaf(-av[u], b[u].y, acc[r][1]);
            acc[r][2] = fmaf(-av[u], b[u].z, acc[r][2]);
            acc[r][3] = fmaf(-av[u], b[u].w, acc[r][3]);
        }
    }
}

__device__ __forceinline__ void cost_store4(const float (&acc)[4][4], int i0, int La, int j,
                                            int Lb, float* __restrict__ C, int vec) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + r;
        if (i >= La) continue;
        float* out = C + (size_t)i * Lb + j;
        if (vec && j + 3 < Lb) {
            __stcs(reinterpret_cast<float4*>(out),
                   make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]));
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (j + c < Lb) __stcs(out + c, acc[r][c]);
        }
    }
}

// DP <= 16: the thread's 4 columns of b^ stay in registers over all its row
// tiles (DP float4 words), so a tile costs only the 4 rows' values of a^ (one
// broadcast load per 4 features and row) and the stores.  Other widths load
// b^ per tile (L1 hits).
template <int DP>
__global__ void __launch_bounds__(256) k_cost(const float* __restrict__ Ahat, int La,
                                              const float* __restrict__ Bt, int Lb, int dp,
                                              float* __restrict__ C, int vec) {
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    const int j = blockIdx.x * kCostCols + 4 * tx;
    if (j >= Lb) return;  // Bt holds whole chunks of 16 frames: j .. j+3 exist
    if (DP > 0) dp = DP;
    const float* bcol = Bt + bt_index(j, 0, dp);  // feature d at bcol + 16 d
    constexpr int kRegD = DP > 0 ? DP : 4;
    float4 breg[kRegD];
    if constexpr (DP > 0) {
#pragma unroll
        for (int d = 0; d < DP; ++d)
            breg[d] = __ldg(reinterpret_cast<const float4*>(bcol + (size_t)d * 16));
    }
    for (int i0 = blockIdx.y * kCostRows + 4 * ty; i0 < La; i0 += gridDim.y * kCostRows) {
        float acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 1.0f;
        const float* arow[4];  // rows beyond La read row La - 1 (never stored)
#pragma unroll
        for (int r = 0; r < 4; ++r) arow[r] = Ahat + (size_t)min(i0 + r, La - 1) * dp;
        if constexpr (DP > 0) {
#pragma unroll
            for (int d0 = 0; d0 < DP; d0 += 4) {
                float4 a[4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    a[r] = __ldg(reinterpret_cast<const float4*>(arow[r] + d0));
                const float4 b[4] = {breg[d0], breg[d0 + 1], breg[d0 + 2], breg[d0 + 3]};
                cost_fma4(acc, a, b);
            }
        } else {
            for (int d0 = 0; d0 < dp; d0 += 4) {
                float4 a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    b[u] = __ldg(reinterpret_cast<const float4*>(bcol + (size_t)(d0 + u) * 16));
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    a[r] = __ldg(reinterpret_cast<const float4*>(arow[r] + d0));
                cost_fma4(acc, a, b);
            }
        }
        cost_store4(acc, i0, La, j, Lb, C, vec);
    }
}

cudaError_t launch_cost(const float* Ahat, int La, const float* Bt, int Lb, int dp, float* C,
                        cudaStream_t s) {
    if (dp > kCostMaxDp || dp % 4 != 0) return cudaErrorInvalidValue;
    const int gx = (Lb + kCostCols - 1) / kCostCols;
    const int ty = (La + kCostRows - 1) / kCostRows;
    // about 8192 blocks: each takes several row tiles, reusing its columns
    int gy = (8192 + gx - 1) / gx;
    if (gy > ty) gy = ty;
    if (gy > 65535) gy = 65535;
    const dim3 grid((unsigned)gx, (unsigned)gy);
    const int vec = (Lb % 4 == 0 && reinterpret_cast<uintptr_t>(C) % 16 == 0) ? 1 : 0;
    switch (dp) {
        case 4: k_cost<4><<<grid, 256, 0, s>>>(Ahat, La, Bt, Lb, dp, C, vec); break;
        case 8: k_cost<8><<<grid, 256, 0, s>>>(Ahat, La, Bt, Lb, dp, C, vec); break;
        case 12: k_cost<12><<<grid, 256, 0, s>>>(Ahat, La, Bt, Lb, dp, C, vec); break;
        case 16: k_cost<16><<<grid, 256, 0, s>>>(Ahat, La, Bt, Lb, dp, C, vec); break;
        default: k_cost<0><<<grid, 256, 0, s>>>(Ahat, La, Bt, Lb, dp, C, vec); break;
    }
    return cudaGetLastError();
}

}  // namespace pardtw
