// Learned window proposal: training kernels (forward with stored
// activations, BCE-with-logits loss, backward, Adam), all on CUDA cores with
// fp32 accumulation. Activations a1, a2 are stored in bf16 exactly as the
// inference kernel stores them; a3 and h stay fp32. Every reduction runs in
// a fixed order (no floating-point atomics), so a training step is
// deterministic and resuming from a checkpoint reproduces the same run.
//
// Layout: for each pyramid level of the batch, planar activation maps
// a1[16][H1][W1], a2[32][H2][W2] (bf16), a3[32][H3][W3] (fp32) at offsets of
// a TrainLevel table; h, dh on the cell atlas (row cell_row + cy, pitch P);
// logits, labels and dz at the score-map offsets of the level.
#include "pd_internal.h"

#include <cuda_bf16.h>

namespace pd {
namespace {

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// ---- forward: 3x3 stride-2 pad-1 conv + bias + relu, one thread per output
// position, all output channels. IN: planar input (bf16, or the u8 level with
// the input table when CIN == 1).
template <int CIN, int COUT, bool FROM_IMAGE, bool OUT_BF16>
__global__ void __launch_bounds__(256) t_conv_fwd(const TrainLevel *__restrict__ tl, const LevelDesc *__restrict__ levels,
                                                  const uint8_t *__restrict__ pyr, const float *__restrict__ in_tab,
                                                  const __nv_bfloat16 *__restrict__ in_act, int layer,
                                                  const float *__restrict__ w, const float *__restrict__ b,
                                                  void *out_act) {
    const TrainLevel T = tl[blockIdx.y];
    const LevelDesc L = levels[T.level];
    int Hi, Wi, Ho, Wo;
    int64_t in_off, out_off;
    if (layer == 1) { Hi = L.Hk; Wi = L.Wk; Ho = T.H1; Wo = T.W1; in_off = 0; out_off = T.a1; }
    else if (layer == 2) { Hi = T.H1; Wi = T.W1; Ho = T.H2; Wo = T.W2; in_off = T.a1; out_off = T.a2; }
    else { Hi = T.H2; Wi = T.W2; Ho = T.H3; Wo = T.W3; in_off = T.a2; out_off = T.a3; }
    __shared__ float ws[COUT * CIN * 9];
    __shared__ float bs[COUT];
    for (int i = threadIdx.x; i < COUT * CIN * 9; i += blockDim.x) ws[i] = w[i];
    for (int i = threadIdx.x; i < COUT; i += blockDim.x) bs[i] = b[i];
    __syncthreads();
    const int n = Ho * Wo;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int i = p / Wo, j = p - i * Wo;
        float acc[COUT];
#pragma unroll
        for (int o = 0; o < COUT; ++o) acc[o] = bs[o];
        for (int c = 0; c < CIN; ++c) {
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const int y = 2 * i + dy - 1;
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int x = 2 * j + dx - 1;
                    float v = 0.f;
                    if (y >= 0 && y < Hi && x >= 0 && x < Wi) {
                        if (FROM_IMAGE) v = in_tab[pyr[L.img_off + (int64_t)y * L.img_pitch + x]];
                        else v = bf(in_act[in_off + ((int64_t)c * Hi + y) * Wi + x]);
                    }
#pragma unroll
                    for (int o = 0; o < COUT; ++o) acc[o] = fmaf(ws[(o * CIN + c) * 9 + dy * 3 + dx], v, acc[o]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < COUT; ++o) {
            const float a = fmaxf(acc[o], 0.f);
            if (OUT_BF16)
                reinterpret_cast<__nv_bfloat16 *>(out_act)[out_off + ((int64_t)o * Ho + i) * Wo + j] = __float2bfloat16_rn(a);
            else
                reinterpret_cast<float *>(out_act)[out_off + ((int64_t)o * Ho + i) * Wo + j] = a;
        }
    }
}

// ---- head: h = bh + wh . a3 on the cells of the level
__global__ void t_head_fwd(const TrainLevel *__restrict__ tl, const LevelDesc *__restrict__ levels,
                           const float *__restrict__ a3, const float *__restrict__ wh,
                           const float *__restrict__ bh, float *__restrict__ hmap, int32_t hp) {
    const TrainLevel T = tl[blockIdx.y];
    const LevelDesc L = levels[T.level];
    const int n = L.Hc * L.Wc;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int cy = p / L.Wc, cx = p - cy * L.Wc;
        float h = bh[0];
        for (int c = 0; c < 32; ++c) h = fmaf(wh[c], a3[T.a3 + ((int64_t)c * T.H3 + cy) * T.W3 + cx], h);
        hmap[(int64_t)(L.cell_row + cy) * hp + cx] = h;
    }
}

// ---- BCE with logits: per window dz = (p y (s - 1) + (1 - y) s) / N, loss
// terms; labels y = score > thr. One block per level, fixed-order sums.
__global__ void t_loss(const TrainLevel *__restrict__ tl, const LevelDesc *__restrict__ levels,
                       const float *__restrict__ logits, const float *__restrict__ scores, float thr,
                       float pos_weight, float inv_n, float *__restrict__ dz, float *__restrict__ level_loss) {
    const TrainLevel T = tl[blockIdx.x];
    const LevelDesc L = levels[T.level];
    const int n = L.rows * L.cols;
    float part = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float z = logits[L.score_off + i];
        const float y = scores[L.score_off + i] > thr ? 1.f : 0.f;
        // log sigmoid(z) = -softplus(-z), log(1 - sigmoid(z)) = -softplus(z)
        const float sp_neg = fmaxf(-z, 0.f) + log1pf(expf(-fabsf(z)));
        const float sp_pos = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));
        part += pos_weight * y * sp_neg + (1.f - y) * sp_pos;
        const float s = 1.f / (1.f + expf(-z));
        dz[L.score_off + i] = (pos_weight * y * (s - 1.f) + (1.f - y) * s) * inv_n;
    }
    __shared__ float red[256];
    red[threadIdx.x] = part;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) level_loss[blockIdx.x] = red[0] * inv_n;
}

// ---- pooling backward into h: dh[c] = sum over the windows that see cell c
// of V[r][s] dz[window] (a gather: no atomics)
__global__ void t_pool_bwd_h(const TrainLevel *__restrict__ tl, const LevelDesc *__restrict__ levels,
                             const float *__restrict__ dz, const float *__restrict__ v,
                             float *__restrict__ dh, int32_t hp) {
    const TrainLevel T = tl[blockIdx.y];
    const LevelDesc L = levels[T.level];
    const int n = L.Hc * L.Wc;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int cy = p / L.Wc, cx = p - cy * L.Wc;
        float g = 0.f;
        for (int r = 0; r < 16; ++r) {
            const int wy = cy - r;
            if (wy < 0 || wy >= L.rows) continue;
            for (int s = 0; s < 8; ++s) {
                const int wx = cx - s;
                if (wx < 0 || wx >= L.cols) continue;
                g = fmaf(v[r * 8 + s], dz[L.score_off + (int64_t)wy * L.cols + wx], g);
            }
        }
        dh[(int64_t)(L.cell_row + cy) * hp + cx] = g;
    }
}

// Block-wide sum of `v` in a fixed order (256 threads).
__device__ __forceinline__ float block_sum(float v, float *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const float r = red[0];
    __syncthreads();
    return r;
}

// ---- gradients of V, bv, wh, bh: one block per parameter, looping over the
// levels in order. Block q: 0..127 V, 128 bv, 129..160 wh, 161 bh; results go
// to their places in the flat parameter order.
__global__ void __launch_bounds__(256) t_small_grads(const TrainLevel *__restrict__ tl, int n_tl,
                                                     const LevelDesc *__restrict__ levels,
                                                     const float *__restrict__ dz, const float *__restrict__ hmap,
                                                     const float *__restrict__ dh, int32_t hp,
                                                     const float *__restrict__ a3, float *__restrict__ grad_out) {
    __shared__ float red[256];
    const int q = blockIdx.x;
    float acc = 0.f;
    for (int k = 0; k < n_tl; ++k) {
        const TrainLevel T = tl[k];
        const LevelDesc L = levels[T.level];
        float part = 0.f;
        if (q < 129) {
            const int n = L.rows * L.cols;
            const int r = q / 8, s = q % 8;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int wy = i / L.cols, wx = i - wy * L.cols;
                const float d = dz[L.score_off + i];
                part += q == 128 ? d : d * hmap[(int64_t)(L.cell_row + wy + r) * hp + wx + s];
            }
        } else {
            const int n = L.Hc * L.Wc;
            const int c = q - 129;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int cy = i / L.Wc, cx = i - cy * L.Wc;
                const float d = dh[(int64_t)(L.cell_row + cy) * hp + cx];
                part += q == 161 ? d : d * a3[T.a3 + ((int64_t)c * T.H3 + cy) * T.W3 + cx];
            }
        }
        acc += block_sum(part, red);
    }
    if (threadIdx.x == 0) {
        const int at = q < 128 ? kOffV + q : q == 128 ? kOffBv : q < 161 ? kOffWh + (q - 129) : kOffBh;
        grad_out[at] = acc;
    }
}

// ---- dz3[c][cell] = wh[c] dh[cell] (a3 > 0), zero outside the cells used
__global__ void t_head_bwd(const TrainLevel *__restrict__ tl, const LevelDesc *__restrict__ levels,
                           const float *__restrict__ dh, int32_t hp, const float *__restrict__ wh,
                           const float *__restrict__ a3, float *__restrict__ dz3) {
    const TrainLevel T = tl[blockIdx.y];
    const LevelDesc L = levels[T.level];
    const int n = 32 * T.H3 * T.W3;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int c = p / (T.H3 * T.W3), r = p - c * T.H3 * T.W3;
        const int cy = r / T.W3, cx = r - cy * T.W3;
        float g = 0.f;
        if (cy < L.Hc && cx < L.Wc && a3[T.a3 + p] > 0.f) g = wh[c] * dh[(int64_t)(L.cell_row + cy) * hp + cx];
        dz3[T.a3 + p] = g;
    }
}

// ---- data gradient of a 3x3 stride-2 conv, times the relu mask of its input:
// dz_in[c][y][x] = (a_in > 0) * sum_{o,dy,dx} w[o][c][dy][dx] dz_out[o][(y+1-dy)/2][(x+1-dx)/2]
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) t_conv_bwd_data(const TrainLevel *__restrict__ tl, int layer,
                                                       const float *__restrict__ w,
                                                       const float *__restrict__ dz_out,
                                                       const __nv_bfloat16 *__restrict__ a_in,
                                                       float *__restrict__ dz_in) {
    const TrainLevel T = tl[blockIdx.y];
    int Hi, Wi, Ho, Wo;
    int64_t in_off, out_off;
    if (layer == 3) { Hi = T.H2; Wi = T.W2; Ho = T.H3; Wo = T.W3; in_off = T.a2; out_off = T.a3; }
    else { Hi = T.H1; Wi = T.W1; Ho = T.H2; Wo = T.W2; in_off = T.a1; out_off = T.a2; }
    __shared__ float ws[COUT * CIN * 9];
    for (int i = threadIdx.x; i < COUT * CIN * 9; i += blockDim.x) ws[i] = w[i];
    __syncthreads();
    const int n = CIN * Hi * Wi;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int c = p / (Hi * Wi), r = p - c * Hi * Wi;
        const int y = r / Wi, x = r - y * Wi;
        float g = 0.f;
        if (bf(a_in[in_off + p]) > 0.f) {
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const int ty = y + 1 - dy;
                if (ty < 0 || (ty & 1) || (ty >> 1) >= Ho) continue;
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int tx = x + 1 - dx;
                    if (tx < 0 || (tx & 1) || (tx >> 1) >= Wo) continue;
                    const int64_t base = out_off + (int64_t)(ty >> 1) * Wo + (tx >> 1);
                    for (int o = 0; o < COUT; ++o)
                        g = fmaf(ws[(o * CIN + c) * 9 + dy * 3 + dx], dz_out[base + (int64_t)o * Ho * Wo], g);
                }
            }
        }
        dz_in[in_off + p] = g;
    }
}

// ---- weight gradient of a 3x3 stride-2 conv: one block per (o, c) pair,
// 9 taps (+ the bias when c == 0), fixed-order sums over levels and positions.
template <int CIN, int COUT, bool FROM_IMAGE>
__global__ void __launch_bounds__(256) t_conv_bwd_weight(const TrainLevel *__restrict__ tl, int n_tl,
                                                         const LevelDesc *__restrict__ levels, int layer,
                                                         const uint8_t *__restrict__ pyr,
                                                         const float *__restrict__ in_tab,
                                                         const __nv_bfloat16 *__restrict__ a_in,
                                                         const float *__restrict__ dz_out,
                                                         float *__restrict__ gw, float *__restrict__ gb) {
    __shared__ float red[256];
    const int o = blockIdx.x / CIN, c = blockIdx.x % CIN;
    float acc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) acc[k] = 0.f;
    for (int lv = 0; lv < n_tl; ++lv) {
        const TrainLevel T = tl[lv];
        const LevelDesc L = levels[T.level];
        int Hi, Wi, Ho, Wo;
        int64_t in_off, out_off;
        if (layer == 1) { Hi = L.Hk; Wi = L.Wk; Ho = T.H1; Wo = T.W1; in_off = 0; out_off = T.a1; }
        else if (layer == 2) { Hi = T.H1; Wi = T.W1; Ho = T.H2; Wo = T.W2; in_off = T.a1; out_off = T.a2; }
        else { Hi = T.H2; Wi = T.W2; Ho = T.H3; Wo = T.W3; in_off = T.a2; out_off = T.a3; }
        float part[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) part[k] = 0.f;
        const int n = Ho * Wo;
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int i = p / Wo, j = p - i * Wo;
            const float d = dz_out[out_off + (int64_t)o * n + p];
            if (d == 0.f) continue;
#pragma unroll
            for (int dy = 0; dy < 3; ++dy) {
                const int y = 2 * i + dy - 1;
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int x = 2 * j + dx - 1;
                    float v = 0.f;
                    if (y >= 0 && y < Hi && x >= 0 && x < Wi) {
                        if (FROM_IMAGE) v = in_tab[pyr[L.img_off + (int64_t)y * L.img_pitch + x]];
                        else v = bf(a_in[in_off + ((int64_t)c * Hi + y) * Wi + x]);
                    }
                    part[dy * 3 + dx] = fmaf(d, v, part[dy * 3 + dx]);
                }
            }
            part[9] += d;
        }
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[k] += block_sum(part[k], red);
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < 9; ++k) gw[(o * CIN + c) * 9 + k] = acc[k];
        if (c == 0) gb[o] = acc[9];
    }
}

// dz of a stored relu layer output: dz = (a > 0) * g, where g came from the
// data gradient of the next layer (already masked there), so layer-2 and
// layer-1 dz are the outputs of t_conv_bwd_data.

// ---- the working copy the forward pass uses: conv weights rounded to bf16
__global__ void t_round(const float *__restrict__ master, float *__restrict__ wr, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool conv_w = i < kOffB1 || (i >= kOffW2 && i < kOffB2) || (i >= kOffW3 && i < kOffB3);
        wr[i] = conv_w ? __bfloat162float(__float2bfloat16_rn(master[i])) : master[i];
    }
}

// ---- Adam on the fp32 master parameters
__global__ void t_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

}  // namespace

cudaError_t launch_train_step(cudaStream_t s, const TrainArgs &a) {
    const dim3 blk(256);
    const int gx = 48;
    const int nl = a.n_levels;
    if (nl <= 0) return cudaSuccess;
    const dim3 g2(gx, nl);
    // forward
    t_conv_fwd<1, 16, true, true><<<g2, blk, 0, s>>>(a.tl, a.levels, a.pyr, a.w.in_tab, nullptr, 1, a.wr + kOffW1,
                                                     a.wr + kOffB1, a.act16);
    t_conv_fwd<16, 32, false, true><<<g2, blk, 0, s>>>(a.tl, a.levels, a.pyr, a.w.in_tab, a.act16, 2, a.wr + kOffW2,
                                                       a.wr + kOffB2, a.act16);
    t_conv_fwd<32, 32, false, false><<<g2, blk, 0, s>>>(a.tl, a.levels, a.pyr, a.w.in_tab, a.act16, 3, a.wr + kOffW3,
                                                        a.wr + kOffB3, a.act32);
    t_head_fwd<<<g2, blk, 0, s>>>(a.tl, a.levels, a.act32, a.wr + kOffWh, a.wr + kOffBh, a.hmap, a.hp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // pooling forward: the inference pooling kernel (identical sums) over the
    // batch's levels (the training levels are all levels of the batch, in order)
    CnnWeights pw = a.w;
    pw.v = a.wr + kOffV;
    pw.bv = a.wr + kOffBv;
    e = launch_cnn(s, a.levels, nl, nullptr, nullptr, 0, pw, a.hmap, a.hp, a.logits, a.pool_tiles, nullptr);  // pooling only
    if (e != cudaSuccess) return e;
    // loss and backward
    t_loss<<<nl, 256, 0, s>>>(a.tl, a.levels, a.logits, a.scores, a.label_thr, a.pos_weight, a.inv_n, a.dz,
                              a.level_loss);
    t_pool_bwd_h<<<g2, blk, 0, s>>>(a.tl, a.levels, a.dz, a.wr + kOffV, a.dh, a.hp);
    t_small_grads<<<162, 256, 0, s>>>(a.tl, nl, a.levels, a.dz, a.hmap, a.dh, a.hp, a.act32, a.grad);
    t_head_bwd<<<g2, blk, 0, s>>>(a.tl, a.levels, a.dh, a.hp, a.wr + kOffWh, a.act32, a.dz32);
    t_conv_bwd_weight<32, 32, false><<<32 * 32, 256, 0, s>>>(a.tl, nl, a.levels, 3, a.pyr, a.w.in_tab, a.act16,
                                                             a.dz32, a.grad + kOffW3, a.grad + kOffB3);
    t_conv_bwd_data<32, 32><<<g2, blk, 0, s>>>(a.tl, 3, a.wr + kOffW3, a.dz32, a.act16, a.dz16);
    t_conv_bwd_weight<16, 32, false><<<32 * 16, 256, 0, s>>>(a.tl, nl, a.levels, 2, a.pyr, a.w.in_tab, a.act16,
                                                             a.dz16, a.grad + kOffW2, a.grad + kOffB2);
    t_conv_bwd_data<16, 32><<<g2, blk, 0, s>>>(a.tl, 2, a.wr + kOffW2, a.dz16, a.act16, a.dz16);
    t_conv_bwd_weight<1, 16, true><<<16, 256, 0, s>>>(a.tl, nl, a.levels, 1, a.pyr, a.w.in_tab, nullptr, a.dz16,
                                                      a.grad + kOffW1, a.grad + kOffB1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.lr > 0.f) {
        t_adam<<<64, 256, 0, s>>>(a.master, a.m, a.v, a.grad, kCnnParams, a.lr, a.beta1, a.beta2, a.eps, a.c1, a.c2);
        t_round<<<64, 256, 0, s>>>(a.master, a.wr, kCnnParams);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_round_params(cudaStream_t s, const float *master, float *wr) {
    t_round<<<64, 256, 0, s>>>(master, wr, kCnnParams);
    return cudaGetLastError();
}

}  // namespace pd
