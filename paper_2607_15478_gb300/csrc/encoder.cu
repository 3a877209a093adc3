// Band encoder of the learned band (dtw_align_learned): a small 1-D
// convolutional network over the sequences averaged over `ds` frames.  The
// paper only names bands and multiscale DTW as ways to cut the quadratic cost
// (Sec. II); the network, its loss and its use are this library's.
//
//   x      = pooled frames (mean of ds frames), L2-normalised   [Lc][D]
//   h1     = relu(conv5(x,  W1) + b1)                            [Lc][64]
//   h2     = relu(conv5(h1, W2) + b2)                            [Lc][64]
//   h3     = relu(conv5(h2, W3) + b3)                            [Lc][64]
//   z      = W4 h3 + b4,  e = z / |z|  (the embedding)           [Lc][16]
//   s      = W5 . h3 + b5 (half-width logit; rows of A only)     [Lc]
//   halfwidth = wmin * (wmax / wmin)^sigmoid(s)   in fine frames
//
// conv5 is a 1-D convolution of width 5 with zero padding 2:
//   y[l][co] = sum_{ci, t} W[co][ci][t] x[l + t - 2][ci].
// The coarse alignment is the exact DTW of eA against eB (cosine cost), and
// the band around its upsampled path has the predicted half-width.
//
// Training (dtw_encoder_grad): mode 0 is a contrastive loss on the
// embeddings, for each coarse row i of A a softmax over the coarse columns
// within kWin of the column c_i that the exact path matches to the row,
// loss_i = -log softmax_j(eA_i . eB_j / tau)[c_i]; mode 1 fits the width head
// (trunk frozen) with a pinball loss at quantile kQ to the half-width the
// band of the coarse path needs to hold the exact path.  Gradients are the
// hand-derived backward passes of the layers above (no autodiff), summed into
// the caller's gradient array with atomics.
//
// Kernels: k_pool_norm, k_conv (forward, and backward-data with transposed
// flipped weights), k_conv_wgrad, k_embed, k_embed_bwd, k_outer (reductions
// sum_l u[l][a] v[l][b] for the head weights), k_targets*, k_loss_emb,
// k_width_target, k_loss_width, k_adam.
#include "pardtw_common.cuh"

#include <cuda_bf16.h>

namespace pardtw {

namespace {

constexpr int kC = kEncChannels;   // 64
constexpr int kE = kEncEmbed;      // 16
constexpr int kK = kEncKernel;     // 5
constexpr int kPad = kK / 2;
constexpr int kWin = 16;           // contrastive window half-width (coarse columns)
constexpr float kTau = 0.1f;       // softmax temperature
constexpr float kQ = 0.9f;         // pinball quantile of the width loss
constexpr float kMargin = 64.0f;   // fine frames added to the needed half-width

__device__ __forceinline__ float round_bf16(float x) {
    return __bfloat162float(__float2bfloat16_rn(x));
}

// Mean of each window of ds frames (the last may be shorter), L2-normalised
// (a zero mean stays zero).  One thread per pooled frame.
__global__ void k_pool_norm(const float* __restrict__ X, int L, int D, int ds,
                            float* __restrict__ Y) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int Lc = (L + ds - 1) / ds;
    if (c >= Lc) return;
    const int f0 = c * ds, f1 = min(f0 + ds, L);
    float ss = 0.f;
    for (int d = 0; d < D; ++d) {
        float acc = 0.f;
        for (int f = f0; f < f1; ++f) acc += X[(size_t)f * D + d];
        acc /= (float)(f1 - f0);
        Y[(size_t)c * D + d] = acc;
        ss = fmaf(acc, acc, ss);
    }
    const float r = ss > 0.f ? rsqrtf(ss) : 0.f;
    for (int d = 0; d < D; ++d) Y[(size_t)c * D + d] *= r;
}

// Generic conv5 over kTL rows per block, all kC output channels:
//   Y[l][co] = bias[co] + sum_{ci < Cin, t} Wt(ci, t, co) * Xm[l + t - 2][ci]
// Xm = X masked by (mask > 0) where mask is given (the relu derivative of
// the layer whose gradient X is).  Wt(ci, t, co) = W[co][ci][t] (forward,
// W: [kC][Cin][kK]) or, with kBwd, W[ci][co][kK-1-t] (backward data: W is the
// forward weight [Cin_b = kC][Cout_b][kK] read transposed and flipped).
// kBF16: inputs and weights rounded to bf16 (products exact in FP32, FP32
// accumulation).
// Thread t computes rows 4 (t / 16) .. + 3 and channels 4 (t % 16) .. + 3 of
// the tile, each output by the same FMAs in the same order (input channel
// outer, tap inner) as one thread per output would: per input channel 8 rows
// of X and 5 x 4 weights from shared memory feed 80 FMAs (one thread per
// channel and 16 rows read 17 values for 16; measured 52 us a layer of 15779
// rows at Cin = 64).
constexpr int kTL = 64;
constexpr int kConvThreads = 256;
constexpr int kXS = kTL + 2 * kPad;  // rows of X per input channel in shared memory
static_assert(kTL == 64 && kC == 64 && kConvThreads == 256, "4 x 4 outputs a thread");

template <bool kBwd, bool kBF16>
__global__ void __launch_bounds__(kConvThreads)
    k_conv(const float* __restrict__ X, const float* __restrict__ mask, int L, int Cin,
           const float* __restrict__ W, const float* __restrict__ bias, int relu,
           float* __restrict__ Y) {
    extern __shared__ __align__(16) float sm[];
    float* Ws = sm;                       // [Cin * kK][kC]
    float* Xs = sm + Cin * kK * kC;       // [Cin][kXS]
    const int l0 = blockIdx.x * kTL;
    const int tid = threadIdx.x;
    for (int k = tid; k < Cin * kK * kC; k += kConvThreads) {
        const int co = k % kC, ct = k / kC, ci = ct / kK, t = ct % kK;
        float w = kBwd ? W[((size_t)ci * kC + co) * kK + (kK - 1 - t)]
                       : W[((size_t)co * Cin + ci) * kK + t];
        Ws[k] = kBF16 ? round_bf16(w) : w;
    }
    for (int k = tid; k < kXS * Cin; k += kConvThreads) {
        const int r = k / Cin, ci = k % Cin;
        const int l = l0 + r - kPad;
        float v = 0.f;
        if (l >= 0 && l < L) {
            v = X[(size_t)l * Cin + ci];
            if (mask && !(mask[(size_t)l * Cin + ci] > 0.f)) v = 0.f;
        }
        Xs[ci * kXS + r] = kBF16 ? round_bf16(v) : v;
    }
    __syncthreads();
    const int cg = tid % 16, rg = tid / 16;  // channels 4 cg .., rows 4 rg ..
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int ci = 0; ci < Cin; ++ci) {
        // rows 4 rg .. 4 rg + 7 of the tile (with the halo): the taps' inputs
        const float4 xa = *reinterpret_cast<const float4*>(Xs + ci * kXS + 4 * rg);
        const float4 xb = *reinterpret_cast<const float4*>(Xs + ci * kXS + 4 * rg + 4);
        const float x[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
        for (int t = 0; t < kK; ++t) {
            const float4 w4 = *reinterpret_cast<const float4*>(Ws + (ci * kK + t) * kC + 4 * cg);
            const float w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(w[j], x[i + t], acc[i][j]);
        }
    }
    float b[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) b[j] = bias ? bias[4 * cg + j] : 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int l = l0 + 4 * rg + i;
        if (l < L) {
            float y[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                y[j] = acc[i][j] + b[j];
                if (relu) y[j] = fmaxf(y[j], 0.f);
            }
            *reinterpret_cast<float4*>(Y + (size_t)l * kC + 4 * cg) =
                make_float4(y[0], y[1], y[2], y[3]);
        }
    }
}

// Weight gradient of a conv5 layer over a tile of kTW rows:
//   dW[co][ci][t] += sum_l dYm[l][co] X[l + t - 2][ci],  db[co] += sum_l dYm[l][co]
// dYm = dY masked by (Yout > 0) (the layer's relu).  Thread (co, cg) owns the
// input channels ci = cg, cg + 4, ... (up to kCPT of them) for all t.
constexpr int kTW = 128;
template <int kCPT>
__global__ void __launch_bounds__(kConvThreads)
    k_conv_wgrad(const float* __restrict__ X, int L, int Cin, const float* __restrict__ dY,
                 const float* __restrict__ Yout, float* __restrict__ dW, float* __restrict__ db) {
    extern __shared__ float sm[];
    float* Gs = sm;                       // [kTW][kC]
    float* Xs = sm + kTW * kC;            // [kTW + 2 kPad][Cin]
    const int l0 = blockIdx.x * kTW;
    const int tid = threadIdx.x;
    for (int k = tid; k < kTW * kC; k += kConvThreads) {
        const int r = k / kC, co = k % kC;
        const int l = l0 + r;
        float g = 0.f;
        if (l < L) {
            const size_t o = (size_t)l * kC + co;
            g = Yout[o] > 0.f ? dY[o] : 0.f;
        }
        Gs[k] = g;
    }
    for (int k = tid; k < (kTW + 2 * kPad) * Cin; k += kConvThreads) {
        const int r = k / Cin, ci = k % Cin;
        const int l = l0 + r - kPad;
        Xs[k] = (l >= 0 && l < L) ? X[(size_t)l * Cin + ci] : 0.f;
    }
    __syncthreads();
    const int co = tid % kC, cg = tid / kC;
    float acc[kCPT][kK];
    float bacc = 0.f;
#pragma unroll
    for (int q = 0; q < kCPT; ++q)
#pragma unroll
        for (int t = 0; t < kK; ++t) acc[q][t] = 0.f;
    for (int r = 0; r < kTW; ++r) {
        const float g = Gs[r * kC + co];
        bacc += g;
#pragma unroll
        for (int q = 0; q < kCPT; ++q) {
            const int ci = cg + 4 * q;
            if (ci < Cin) {
#pragma unroll
                for (int t = 0; t < kK; ++t) acc[q][t] = fmaf(g, Xs[(r + t) * Cin + ci], acc[q][t]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kCPT; ++q) {
        const int ci = cg + 4 * q;
        if (ci < Cin)
#pragma unroll
            for (int t = 0; t < kK; ++t) atomicAdd(&dW[((size_t)co * Cin + ci) * kK + t], acc[q][t]);
    }
    if (cg == 0) atomicAdd(&db[co], bacc);
}

// Heads, one thread per row: z = W4 h3 + b4, e = z / |z| (invn = 1/|z|, 0
// for z = 0), s = W5 . h3 + b5 and the half-width in fine frames.
__global__ void k_embed(const float* __restrict__ H, int L, const float* __restrict__ W4,
                        const float* __restrict__ b4, const float* __restrict__ W5,
                        const float* __restrict__ b5, int bf16, float wmin, float wmax,
                        float* __restrict__ Emb, float* __restrict__ invn, float* __restrict__ S,
                        float* __restrict__ HW) {
    __shared__ float w4[kE * kC], w5[kC], bb[kE + 1];
    for (int k = threadIdx.x; k < kE * kC; k += blockDim.x)
        w4[k] = bf16 ? round_bf16(W4[k]) : W4[k];
    for (int k = threadIdx.x; k < kC; k += blockDim.x) w5[k] = W5[k];
    if (threadIdx.x < kE) bb[threadIdx.x] = b4[threadIdx.x];
    if (threadIdx.x == 0) bb[kE] = b5[0];
    __syncthreads();
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    float z[kE];
#pragma unroll
    for (int e = 0; e < kE; ++e) z[e] = 0.f;
    float s = 0.f;
    const float4* h4 = reinterpret_cast<const float4*>(H + (size_t)l * kC);
    for (int c4 = 0; c4 < kC / 4; ++c4) {
        const float4 v = h4[c4];
        const float hv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = 4 * c4 + u;
            const float hc = bf16 ? round_bf16(hv[u]) : hv[u];
#pragma unroll
            for (int e = 0; e < kE; ++e) z[e] = fmaf(w4[e * kC + c], hc, z[e]);
            s = fmaf(w5[c], hv[u], s);
        }
    }
    float ss = 0.f;
#pragma unroll
    for (int e = 0; e < kE; ++e) {
        z[e] += bb[e];
        ss = fmaf(z[e], z[e], ss);
    }
    const float r = ss > 0.f ? rsqrtf(ss) : 0.f;
#pragma unroll
    for (int e = 0; e < kE; ++e) Emb[(size_t)l * kE + e] = z[e] * r;
    if (invn) invn[l] = r;
    s += bb[kE];
    if (S) S[l] = s;
    if (HW) {
        const float sg = 1.f / (1.f + expf(-s));
        HW[l] = wmin * exp2f(sg * log2f(wmax / wmin));
    }
}

// Backward of the embedding head for one row: ge = dL/de -> dz = (ge - e (e.ge))
// * invn, stored in place of ge; dH[l][c] = sum_e W4[e][c] dz[e].
__global__ void k_embed_bwd(const float* __restrict__ Emb, const float* __restrict__ invn, int L,
                            const float* __restrict__ W4, float* __restrict__ G,
                            float* __restrict__ dH) {
    __shared__ float w4[kE * kC];
    for (int k = threadIdx.x; k < kE * kC; k += blockDim.x) w4[k] = W4[k];
    __syncthreads();
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    float e[kE], g[kE], dot = 0.f;
#pragma unroll
    for (int k = 0; k < kE; ++k) {
        e[k] = Emb[(size_t)l * kE + k];
        g[k] = G[(size_t)l * kE + k];
        dot = fmaf(e[k], g[k], dot);
    }
    const float r = invn[l];
#pragma unroll
    for (int k = 0; k < kE; ++k) {
        g[k] = (g[k] - e[k] * dot) * r;
        G[(size_t)l * kE + k] = g[k];
    }
    for (int c = 0; c < kC; ++c) {
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < kE; ++k) acc = fmaf(w4[k * kC + c], g[k], acc);
        dH[(size_t)l * kC + c] = acc;
    }
}

// out[a][b] += sum_l U[l][a] V[l][b] for a < na, b < nb (V = null: all ones,
// i.e. column sums of U), over a tile of 256 rows per block.  na * nb <= 1024.
__global__ void k_outer(const float* __restrict__ U, int na, const float* __restrict__ V, int nb,
                        int L, float* __restrict__ out) {
    __shared__ float us[64][kE], vs[64][kC];
    const int l0 = blockIdx.x * 256;
    const int n = na * nb;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int r0 = l0; r0 < min(l0 + 256, L); r0 += 64) {
        __syncthreads();
        for (int k = threadIdx.x; k < 64 * na; k += blockDim.x) {
            const int r = k / na, a = k % na;
            us[r][a] = (r0 + r < L) ? U[(size_t)(r0 + r) * na + a] : 0.f;
        }
        for (int k = threadIdx.x; k < 64 * nb; k += blockDim.x) {
            const int r = k / nb, b = k % nb;
            vs[r][b] = (r0 + r < L) ? (V ? V[(size_t)(r0 + r) * nb + b] : 1.f) : 0.f;
        }
        __syncthreads();
        for (int q = 0; q < 4; ++q) {
            const int o = threadIdx.x + q * blockDim.x;
            if (o < n) {
                const int a = o / nb, b = o % nb;
                for (int r = 0; r < 64; ++r) acc[q] = fmaf(us[r][a], vs[r][b], acc[q]);
            }
        }
    }
    for (int q = 0; q < 4; ++q) {
        const int o = threadIdx.x + q * blockDim.x;
        if (o < n) atomicAdd(&out[o], acc[q]);
    }
}

// Coarse column matched to every coarse row of A by the exact fine path:
// the mean column of the path entries in the row's ds fine rows, divided by
// ds.  Pass 1 sums (one thread per path entry), pass 2 divides.
__global__ void k_targets_sum(const int32_t* __restrict__ path, const int* __restrict__ plen,
                              int ds, unsigned long long* __restrict__ jsum,
                              int* __restrict__ cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= *plen) return;
    const int i = path[2 * k] / ds;
    atomicAdd(&jsum[i], (unsigned long long)path[2 * k + 1]);
    atomicAdd(&cnt[i], 1);
}
__global__ void k_targets_fin(const unsigned long long* __restrict__ jsum,
                              const int* __restrict__ cnt, int Lac, int Lbc, int ds,
                              int* __restrict__ tgt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Lac) return;
    const int n = cnt[i];
    // every fine row lies on a path except rows a (2,1) step skips; a coarse
    // row of ds >= 2 fine rows always holds one
    const double m = n > 0 ? (double)jsum[i] / n : 0.0;
    tgt[i] = min((int)(m / ds), Lbc - 1);
}

// Contrastive loss, one thread per coarse row i of A (see the file comment).
// gA[i] = dL/deA_i is written; dL/deB_j is added to gB with atomics.  The
// loss is the mean over rows.
__global__ void k_loss_emb(const float* __restrict__ eA, int Lac, const float* __restrict__ eB,
                           int Lbc, const int* __restrict__ tgt, float* __restrict__ gA,
                           float* __restrict__ gB, float* __restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Lac) return;
    float a[kE];
#pragma unroll
    for (int e = 0; e < kE; ++e) a[e] = eA[(size_t)i * kE + e];
    const int c = tgt[i];
    const int j0 = max(c - kWin, 0), j1 = min(c + kWin, Lbc - 1);
    float lg[2 * kWin + 1];
    float mx = -INFINITY;
    for (int j = j0; j <= j1; ++j) {
        float d = 0.f;
#pragma unroll
        for (int e = 0; e < kE; ++e) d = fmaf(a[e], eB[(size_t)j * kE + e], d);
        lg[j - j0] = d / kTau;
        mx = fmaxf(mx, lg[j - j0]);
    }
    float se = 0.f;
    for (int j = j0; j <= j1; ++j) se += expf(lg[j - j0] - mx);
    const float lse = mx + logf(se);
    const float inv_n = 1.f / (float)Lac;
    atomicAdd(loss, (lse - lg[c - j0]) * inv_n);
    float ga[kE];
#pragma unroll
    for (int e = 0; e < kE; ++e) ga[e] = 0.f;
    for (int j = j0; j <= j1; ++j) {
        const float pj = expf(lg[j - j0] - lse) - (j == c ? 1.f : 0.f);
        const float w = pj * inv_n / kTau;
#pragma unroll
        for (int e = 0; e < kE; ++e) {
            ga[e] = fmaf(w, eB[(size_t)j * kE + e], ga[e]);
            atomicAdd(&gB[(size_t)j * kE + e], w * a[e]);
        }
    }
#pragma unroll
    for (int e = 0; e < kE; ++e) gA[(size_t)i * kE + e] = ga[e];
}

// Width target of every coarse row i of A, in [0, 1] on the log scale of the
// half-width: the band of the coarse path at w = 0 over coarse rows
// i-1 .. i+1 spans fine columns [jmin ds, (jmax + 1) ds - 1]; the row needs
// the distance from that span of the exact path's columns in its fine rows,
// plus kMargin, as half-width.
__global__ void k_width_target(const int32_t* __restrict__ cpath, const int* __restrict__ clen,
                               const int32_t* __restrict__ path, const int* __restrict__ plen,
                               int ds, int Lac, float wmin, float wmax, float* __restrict__ wt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Lac) return;
    const int nc = *clen, nf = *plen;
    float need = 0.f;
    if (nc > 0) {
        int lo = 0, hi = nc;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cpath[2 * mid] < i - 1) lo = mid + 1; else hi = mid;
        }
        int jmin = 0x7fffffff, jmax = -1;
        for (int k = lo; k < nc && cpath[2 * k] <= i + 1; ++k) {
            jmin = min(jmin, cpath[2 * k + 1]);
            jmax = max(jmax, cpath[2 * k + 1]);
        }
        const int f0 = jmin * ds, f1 = (jmax + 1) * ds - 1;
        lo = 0;
        hi = nf;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (path[2 * mid] < i * ds) lo = mid + 1; else hi = mid;
        }
        for (int k = lo; k < nf && path[2 * k] < (i + 1) * ds; ++k) {
            const int j = path[2 * k + 1];
            need = fmaxf(need, (float)max(max(f0 - j, j - f1), 0));
        }
    } else {
        need = wmax;
    }
    const float t = log2f((need + kMargin) / wmin) / log2f(wmax / wmin);
    wt[i] = fminf(fmaxf(t, 0.f), 1.f);
}

// Pinball loss of sigmoid(s_i) against wt_i at quantile kQ (mean over rows);
// ds[i] = dL/ds_i.
__global__ void k_loss_width(const float* __restrict__ S, const float* __restrict__ wt, int Lac,
                             float* __restrict__ dS, float* __restrict__ loss) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Lac) return;
    const float p = 1.f / (1.f + expf(-S[i]));
    const float d = wt[i] - p;
    const float inv_n = 1.f / (float)Lac;
    atomicAdd(loss, (d > 0.f ? kQ * d : (kQ - 1.f) * d) * inv_n);
    const float dp = d > 0.f ? -kQ : (1.f - kQ);
    dS[i] = dp * p * (1.f - p) * inv_n;
}

// Adam (bias-corrected), then the gradient is zeroed for the next step.
__global__ void k_adam(int n, float* __restrict__ P, float* __restrict__ G, float* __restrict__ M,
                       float* __restrict__ V, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float g = G[k];
    const float m = b1 * M[k] + (1.f - b1) * g;
    const float v = b2 * V[k] + (1.f - b2) * g * g;
    M[k] = m;
    V[k] = v;
    P[k] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    G[k] = 0.f;
}

template <bool kBwd, bool kBF16>
cudaError_t conv_t(const float* X, const float* mask, int L, int Cin, const float* W,
                   const float* b, int relu, float* Y, cudaStream_t s) {
    const int smem = (Cin * kK * kC + (kTL + 2 * kPad) * Cin) * (int)sizeof(float);
    static DeviceSlots raised;
    const cudaError_t e = raise_smem_once(k_conv<kBwd, kBF16>,
                                          (kC * kK * kC + (kTL + 2 * kPad) * kC) * 4, raised);
    if (e != cudaSuccess) return e;
    k_conv<kBwd, kBF16><<<(L + kTL - 1) / kTL, kConvThreads, smem, s>>>(X, mask, L, Cin, W, b,
                                                                       relu, Y);
    return cudaGetLastError();
}

template <int kCPT>
cudaError_t wgrad_t(const float* X, int L, int Cin, const float* dY, const float* Yout, float* dW,
                    float* db, cudaStream_t s) {
    const int smem = (kTW * kC + (kTW + 2 * kPad) * Cin) * (int)sizeof(float);
    static DeviceSlots raised;
    const cudaError_t e = raise_smem_once(k_conv_wgrad<kCPT>,
                                          (kTW * kC + (kTW + 2 * kPad) * kC) * 4, raised);
    if (e != cudaSuccess) return e;
    k_conv_wgrad<kCPT><<<(L + kTW - 1) / kTW, kConvThreads, smem, s>>>(X, L, Cin, dY, Yout, dW,
                                                                      db);
    return cudaGetLastError();
}

}  // namespace

EncLayout enc_layout(int D) {
    EncLayout p;
    size_t o = 0;
    p.W1 = o; o += (size_t)kC * D * kK;
    p.b1 = o; o += kC;
    p.W2 = o; o += (size_t)kC * kC * kK;
    p.b2 = o; o += kC;
    p.W3 = o; o += (size_t)kC * kC * kK;
    p.b3 = o; o += kC;
    p.W4 = o; o += (size_t)kE * kC;
    p.b4 = o; o += kE;
    p.W5 = o; o += kC;
    p.b5 = o; o += 1;
    p.count = o;
    return p;
}

cudaError_t launch_pool_norm(const float* X, int L, int D, int ds, float* Y, cudaStream_t s) {
    const int Lc = (L + ds - 1) / ds;
    k_pool_norm<<<(Lc + 127) / 128, 128, 0, s>>>(X, L, D, ds, Y);
    return cudaGetLastError();
}

cudaError_t launch_conv(const float* X, const float* mask, int L, int Cin, const float* W,
                        const float* b, int relu, int bwd, int bf16, float* Y, cudaStream_t s) {
    if (Cin < 1 || Cin > kC) return cudaErrorInvalidValue;
    if (bwd) return bf16 ? cudaErrorInvalidValue : conv_t<true, false>(X, mask, L, Cin, W, b, relu, Y, s);
    return bf16 ? conv_t<false, true>(X, mask, L, Cin, W, b, relu, Y, s)
                : conv_t<false, false>(X, mask, L, Cin, W, b, relu, Y, s);
}

cudaError_t launch_conv_wgrad(const float* X, int L, int Cin, const float* dY, const float* Yout,
                              float* dW, float* db, cudaStream_t s) {
    const int cpt = (Cin + 3) / 4;
    if (cpt <= 4) return wgrad_t<4>(X, L, Cin, dY, Yout, dW, db, s);
    if (cpt <= 8) return wgrad_t<8>(X, L, Cin, dY, Yout, dW, db, s);
    if (cpt <= 16) return wgrad_t<16>(X, L, Cin, dY, Yout, dW, db, s);
    return cudaErrorInvalidValue;
}

cudaError_t launch_embed(const float* H, int L, const float* params, const EncLayout& p, int bf16,
                         float wmin, float wmax, float* Emb, float* invn, float* S, float* HW,
                         cudaStream_t s) {
    k_embed<<<(L + 127) / 128, 128, 0, s>>>(H, L, params + p.W4, params + p.b4, params + p.W5,
                                           params + p.b5, bf16, wmin, wmax, Emb, invn, S, HW);
    return cudaGetLastError();
}

cudaError_t launch_embed_bwd(const float* Emb, const float* invn, int L, const float* W4,
                             float* G, float* dH, cudaStream_t s) {
    k_embed_bwd<<<(L + 127) / 128, 128, 0, s>>>(Emb, invn, L, W4, G, dH);
    return cudaGetLastError();
}

cudaError_t launch_outer(const float* U, int na, const float* V, int nb, int L, float* out,
                         cudaStream_t s) {
    if (na < 1 || na > kE || nb < 1 || nb > kC || na * nb > 1024) return cudaErrorInvalidValue;
    k_outer<<<(L + 255) / 256, 256, 0, s>>>(U, na, V, nb, L, out);
    return cudaGetLastError();
}

cudaError_t launch_targets(const int32_t* path, const int* plen, int cap, int ds, int Lac, int Lbc,
                           unsigned long long* jsum, int* cnt, int* tgt, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(jsum, 0, sizeof(unsigned long long) * Lac, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int) * Lac, s);
    if (e != cudaSuccess) return e;
    k_targets_sum<<<(cap + 255) / 256, 256, 0, s>>>(path, plen, ds, jsum, cnt);
    k_targets_fin<<<(Lac + 255) / 256, 256, 0, s>>>(jsum, cnt, Lac, Lbc, ds, tgt);
    return cudaGetLastError();
}

cudaError_t launch_loss_emb(const float* eA, int Lac, const float* eB, int Lbc, const int* tgt,
                            float* gA, float* gB, float* loss, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(gB, 0, sizeof(float) * (size_t)Lbc * kE, s);
    if (e != cudaSuccess) return e;
    k_loss_emb<<<(Lac + 127) / 128, 128, 0, s>>>(eA, Lac, eB, Lbc, tgt, gA, gB, loss);
    return cudaGetLastError();
}

cudaError_t launch_width_target(const int32_t* cpath, const int* clen, const int32_t* path,
                                const int* plen, int ds, int Lac, float wmin, float wmax,
                                float* wt, cudaStream_t s) {
    k_width_target<<<(Lac + 127) / 128, 128, 0, s>>>(cpath, clen, path, plen, ds, Lac, wmin, wmax,
                                                     wt);
    return cudaGetLastError();
}

cudaError_t launch_loss_width(const float* S, const float* wt, int Lac, float* dS, float* loss,
                              cudaStream_t s) {
    k_loss_width<<<(Lac + 255) / 256, 256, 0, s>>>(S, wt, Lac, dS, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(int n, float* P, float* G, float* M, float* V, int step, float lr,
                        float b1, float b2, float eps, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(n, P, G, M, V, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace pardtw
