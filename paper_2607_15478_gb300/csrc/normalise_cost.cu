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
// Block: 256 threads = 8 rows x 32 column lanes; each lane writes 4 columns
// of its row per pass.
__global__ void k_cost(const float* __restrict__ Ahat, int La, const float* __restrict__ Bt,
                       int Lb, int dp, float* __restrict__ C) {
    const int lane = threadIdx.x & 31;
    for (int i = blockIdx.y * 8 + (threadIdx.x >> 5); i < La; i += gridDim.y * 8) {
        const float* a = Ahat + (size_t)i * dp;
        for (int j0 = blockIdx.x * 128 + lane; j0 < Lb; j0 += gridDim.x * 128) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = j0 + 32 * q;
                if (j >= Lb) break;
                float acc = 1.0f;
                for (int d = 0; d < dp; ++d) acc = fmaf(-a[d], Bt[bt_index(j, d, dp)], acc);
                C[(size_t)i * Lb + j] = acc;
            }
        }
    }
}

cudaError_t launch_cost(const float* Ahat, int La, const float* Bt, int Lb, int dp, float* C,
                        cudaStream_t s) {
    const int gx = (Lb + 127) / 128 < 64 ? (Lb + 127) / 128 : 64;
    const int gy = (La + 7) / 8 < 32768 ? (La + 7) / 8 : 32768;
    dim3 grid((unsigned)gx, (unsigned)gy);
    k_cost<<<grid, 256, 0, s>>>(Ahat, La, Bt, Lb, dp, C);
    return cudaGetLastError();
}

}  // namespace pardtw
