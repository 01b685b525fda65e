// The paper's kernel schemes for LBP, HOG and the window SVM (Sections
// 4.2-4.4: LBP Naive / Scalable, HOG Global / Local / Shared, Naive and
// Warp-level SVM), written for this GPU over the same readings as the fused
// kernels (clamped borders, uniform-LBP bins, one global cell grid with
// bilinear votes, L2-Hys and L1-sqrt blocks), so that their results can be
// checked against the same oracle and their speed compared with the fused
// kernels. With per-block HOG the HOG schemes are Algorithm 5 as the paper
// lays it out: one thread per 16x16 block walks its 256 pixels into a 36-bin
// histogram (global, local or shared memory), written to the 36-plane
// per-block layout that the fused cells kernel also produces. They are separate stages with materialised intermediates, as in
// the paper: an LBP bin image, gradient magnitude / orientation images and a
// block-feature array.
#include "pd_internal.h"

#include <math.h>

#include <algorithm>

namespace pd {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Stencil: uniform-LBP bin of every pixel of the 8Wc x 8Hc cell grid (the 8
// clockwise neighbours from the top-left, neighbour >= centre gives 1,
// borders clamped to the level).
__global__ void k_lbp_codes(const uint8_t *__restrict__ img, int Wk, int Hk, int pitch, int gw, int gh,
                            const uint8_t *__restrict__ bin_of, uint8_t *__restrict__ codes) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= gw || y >= gh) return;
    auto px = [&](int yy, int xx) {
        return (int)img[(size_t)clampi(yy, 0, Hk - 1) * pitch + clampi(xx, 0, Wk - 1)];
    };
    const int c = px(y, x);
    const int code = (px(y - 1, x - 1) >= c) | ((px(y - 1, x) >= c) << 1) | ((px(y - 1, x + 1) >= c) << 2) |
                     ((px(y, x + 1) >= c) << 3) | ((px(y + 1, x + 1) >= c) << 4) | ((px(y + 1, x) >= c) << 5) |
                     ((px(y + 1, x - 1) >= c) << 6) | ((px(y, x - 1) >= c) << 7);
    codes[(size_t)y * gw + x] = bin_of[code];
}

// Naive LBP histograms: one thread per cell counts its 64 bins (Map).
__global__ void k_lbp_cells_naive(const uint8_t *__restrict__ codes, int gw, int Wc, int Hc,
                                  uint8_t *__restrict__ lbp, int64_t lbp_plane, int cell_pitch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Wc * Hc) return;
    const int cy = i / Wc, cx = i - cy * Wc;
    uint8_t cnt[kLbpBins];
    for (int t = 0; t < kLbpBins; ++t) cnt[t] = 0;
    for (int dy = 0; dy < 8; ++dy)
        for (int dx = 0; dx < 8; ++dx) ++cnt[codes[(size_t)(8 * cy + dy) * gw + 8 * cx + dx]];
    for (int t = 0; t < kLbpBins; ++t) lbp[(int64_t)t * lbp_plane + (int64_t)cy * cell_pitch + cx] = cnt[t];
}

// Scalable LBP histograms: one thread per pixel adds to its cell (Scatter,
// atomics), then one thread per (bin, cell) writes the count out.
__global__ void k_lbp_scatter(const uint8_t *__restrict__ codes, int gw, int gh, int Wc,
                              uint32_t *__restrict__ hist) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= gw || y >= gh) return;
    atomicAdd(&hist[((size_t)(y >> 3) * Wc + (x >> 3)) * kLbpBins + codes[(size_t)y * gw + x]], 1u);
}
__global__ void k_lbp_pack(const uint32_t *__restrict__ hist, int Wc, int Hc, uint8_t *__restrict__ lbp,
                           int64_t lbp_plane, int cell_pitch) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Wc * Hc * kLbpBins) return;
    const int t = i / (Wc * Hc), c = i - t * (Wc * Hc), cy = c / Wc, cx = c - cy * Wc;
    lbp[(int64_t)t * lbp_plane + (int64_t)cy * cell_pitch + cx] = (uint8_t)hist[(size_t)c * kLbpBins + t];
}

// Stencil: gradient magnitude and orientation (in bin units minus one half:
// theta / 20 - 0.5, theta in [0, 180)) of every grid pixel, central
// differences with clamped borders.
__global__ void k_gradient(const uint8_t *__restrict__ img, int Wk, int Hk, int pitch, int gw, int gh,
                           float *__restrict__ mag, float *__restrict__ pos) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= gw || y >= gh) return;
    auto px = [&](int yy, int xx) {
        return (int)img[(size_t)clampi(yy, 0, Hk - 1) * pitch + clampi(xx, 0, Wk - 1)];
    };
    const int gx = px(y, x + 1) - px(y, x - 1), gy = px(y + 1, x) - px(y - 1, x);
    float theta = atan2f((float)gy, (float)gx) * (180.0f / 3.14159265358979f);
    if (theta < 0.f) theta += 180.f;
    if (theta >= 180.f) theta -= 180.f;
    mag[(size_t)y * gw + x] = sqrtf((float)(gx * gx + gy * gy));
    pos[(size_t)y * gw + x] = theta / 20.f - 0.5f;
}

// Weight of pixel coordinate p (grid) in cell c along one axis: bilinear
// between the two nearest cell centres 8c + 3.5, clamped into [0, n).
__device__ __forceinline__ float axis_weight(int p, int c, int n) {
    const float u = ((float)p - 3.5f) * 0.125f;
    const float f = floorf(u);
    const float w1 = u - f;
    const int c0 = clampi((int)f, 0, n - 1), c1 = clampi((int)f + 1, 0, n - 1);
    return (c0 == c ? 1.f - w1 : 0.f) + (c1 == c ? w1 : 0.f);
}

// HOG cell histograms, one thread per cell (large-grain): the votes of the
// grid pixels within 4 pixels of the cell's 8 x 8 block, accumulated in
// global memory (MODE 0), a local array (1) or shared memory (2).
template <int MODE>
__global__ void k_hog_cells(const float *__restrict__ mag, const float *__restrict__ pos, int gw, int gh, int Wc,
                            int Hc, float *__restrict__ hog, int64_t hog_plane, int cell_pitch) {
    __shared__ float sh[kHogBins][kT];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Wc * Hc) return;
    const int cy = i / Wc, cx = i - cy * Wc;
    float *out = hog + (int64_t)cy * cell_pitch + cx;
    float loc[kHogBins];
    for (int b = 0; b < kHogBins; ++b) {
        if (MODE == 0) out[(int64_t)b * hog_plane] = 0.f;
        if (MODE == 1) loc[b] = 0.f;
        if (MODE == 2) sh[b][threadIdx.x] = 0.f;
    }
    const int y0 = max(8 * cy - 4, 0), y1 = min(8 * cy + 12, gh);
    const int x0 = max(8 * cx - 4, 0), x1 = min(8 * cx + 12, gw);
    for (int y = y0; y < y1; ++y) {
        const float wy = axis_weight(y, cy, Hc);
        if (wy == 0.f) continue;
        for (int x = x0; x < x1; ++x) {
            const float w = wy * axis_weight(x, cx, Wc);
            if (w == 0.f) continue;
            const float bp = pos[(size_t)y * gw + x], m = mag[(size_t)y * gw + x] * w;
            const float bf = floorf(bp);
            const float o1 = bp - bf;
            const int bi = (int)bf;
            const int b0 = bi < 0 ? kHogBins - 1 : bi, b1 = bi + 1 >= kHogBins ? 0 : bi + 1;
            if (MODE == 0) {
                out[(int64_t)b0 * hog_plane] += m * (1.f - o1);
                out[(int64_t)b1 * hog_plane] += m * o1;
            } else if (MODE == 1) {
                loc[b0] += m * (1.f - o1);
                loc[b1] += m * o1;
            } else {
                sh[b0][threadIdx.x] += m * (1.f - o1);
                sh[b1][threadIdx.x] += m * o1;
            }
        }
    }
    if (MODE == 1)
        for (int b = 0; b < kHogBins; ++b) out[(int64_t)b * hog_plane] = loc[b];
    if (MODE == 2)
        for (int b = 0; b < kHogBins; ++b) out[(int64_t)b * hog_plane] = sh[b][threadIdx.x];
}

// Per-block HOG histograms (Algorithm 5), one thread per block: its 16 x 16
// pixels vote bilinearly towards the block's cell centres (local 3.5 and
// 11.5), votes leaving the block dropped; the histogram lives in global
// memory (MODE 0: the block's own 36 output values), a local array (1) or
// shared memory (2). Output: place q of the block is plane 9 q + bin of cell
// (by + q / 2, bx + q % 2).
template <int MODE>
__global__ void k_hog_blocks(const float *__restrict__ mag, const float *__restrict__ pos, int gw, int Wb, int Hb,
                             float *__restrict__ hog, int64_t hog_plane, int cell_pitch) {
    __shared__ float sh[MODE == 2 ? kHogDim : 1][kT];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Wb * Hb) return;
    const int by = i / Wb, bx = i - by * Wb;
    auto at = [&](int t) {  // output value t = 9 q + bin of this block
        const int q = t / kHogBins;
        return hog + (int64_t)t * hog_plane + (int64_t)(by + (q >> 1)) * cell_pitch + bx + (q & 1);
    };
    float loc[MODE == 1 ? kHogDim : 1];
    for (int t = 0; t < kHogDim; ++t) {
        if (MODE == 0) *at(t) = 0.f;
        if (MODE == 1) loc[t] = 0.f;
        if (MODE == 2) sh[t][threadIdx.x] = 0.f;
    }
    auto add = [&](int t, float v) {
        if (MODE == 0) *at(t) += v;
        if (MODE == 1) loc[t] += v;
        if (MODE == 2) sh[t][threadIdx.x] += v;
    };
    for (int iy = 0; iy < 16; ++iy) {
        const float uy = ((float)iy - 3.5f) * 0.125f;
        const float fy = floorf(uy);
        const float vy = uy - fy;
        const int a0 = (int)fy;  // -1, 0 or 1; a0 + 1 in 0..2
        for (int ix = 0; ix < 16; ++ix) {
            const float ux = ((float)ix - 3.5f) * 0.125f;
            const float fx = floorf(ux);
            const float vx = ux - fx;
            const int c0 = (int)fx;
            const size_t p = (size_t)(8 * by + iy) * gw + 8 * bx + ix;
            const float bp = pos[p], m = mag[p];
            const float bf = floorf(bp);
            const float o1 = bp - bf;
            const int bi = (int)bf;
            const int b0 = bi < 0 ? kHogBins - 1 : bi, b1 = bi + 1 >= kHogBins ? 0 : bi + 1;
            for (int da = 0; da < 2; ++da) {
                const int a = a0 + da;
                if (a < 0 || a > 1) continue;
                const float wa = da ? vy : 1.f - vy;
                for (int db = 0; db < 2; ++db) {
                    const int b = c0 + db;
                    if (b < 0 || b > 1) continue;
                    const float w = m * wa * (db ? vx : 1.f - vx);
                    add((2 * a + b) * kHogBins + b0, w * (1.f - o1));
                    add((2 * a + b) * kHogBins + b1, w * o1);
                }
            }
        }
    }
    if (MODE == 1)
        for (int t = 0; t < kHogDim; ++t) *at(t) = loc[t];
    if (MODE == 2)
        for (int t = 0; t < kHogDim; ++t) *at(t) = sh[t][threadIdx.x];
}

// Block features, one thread per block: the 2 x 2 cells' 36 HOG values with
// L2-Hys, then the summed LBP counts with L1-sqrt (a block holds 256 pixels).
// qs = 9 reads the per-block layout (cell of place q from planes 9 q ..).
__global__ void k_blocks(const float *__restrict__ hog, int64_t hog_plane, const uint8_t *__restrict__ lbp,
                         int64_t lbp_plane, int cell_pitch, int Wb, int Hb, float clip, int qs,
                         float *__restrict__ feat) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Wb * Hb) return;
    const int by = i / Wb, bx = i - by * Wb;
    float *f = feat + (size_t)i * kFeat;
    float s = 0.f;
    for (int q = 0; q < 4; ++q)
        for (int b = 0; b < kHogBins; ++b) {
            const float v =
                hog[(int64_t)(qs * q + b) * hog_plane + (int64_t)(by + (q >> 1)) * cell_pitch + bx + (q & 1)];
            f[9 * q + b] = v;
            s += v * v;
        }
    const float i1 = 1.0f / sqrtf(s + 1.0f);
    float s2 = 0.f;
    for (int t = 0; t < kHogDim; ++t) {
        f[t] = fminf(f[t] * i1, clip);
        s2 += f[t] * f[t];
    }
    const float i2 = 1.0f / sqrtf(s2 + 1e-6f);
    for (int t = 0; t < kHogDim; ++t) f[t] *= i2;
    for (int t = 0; t < kLbpBins; ++t) {
        int c = 0;
        for (int q = 0; q < 4; ++q)
            c += lbp[(int64_t)t * lbp_plane + (int64_t)(by + (q >> 1)) * cell_pitch + bx + (q & 1)];
        f[kHogDim + t] = sqrtf((float)c * (1.0f / 256.0f));
    }
}

// Naive SVM: one thread per window dot product. Template layout [t][i][8].
__global__ void k_svm_naive(const float *__restrict__ feat, int Wb, const float *__restrict__ wt, float bias,
                            int rows, int cols, float *__restrict__ scores) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int wy = i / cols, wx = i - wy * cols;
    float s = 0.f;
    for (int bi = 0; bi < kWinBH; ++bi)
        for (int bj = 0; bj < kWinBW; ++bj) {
            const float *f = feat + ((size_t)(wy + bi) * Wb + wx + bj) * kFeat;
            for (int t = 0; t < kFeat; ++t) s = fmaf(f[t], wt[((size_t)t * kWinBH + bi) * kWPad + bj], s);
        }
    scores[i] = s + bias;
}

// Warp-level SVM: one warp per window; lane l takes products l, l + 32, ...
// of the 9,975 (block row, block column, feature) terms, then a shuffle
// reduction.
__global__ void k_svm_warp(const float *__restrict__ feat, int Wb, const float *__restrict__ wt, float bias,
                           int rows, int cols, float *__restrict__ scores) {
    const int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wi >= rows * cols) return;
    const int wy = wi / cols, wx = wi - wy * cols;
    float s = 0.f;
    for (int e = lane; e < kWinBH * kWinBW * kFeat; e += 32) {
        const int bi = e / (kWinBW * kFeat), r = e - bi * (kWinBW * kFeat), bj = r / kFeat, t = r - bj * kFeat;
        s = fmaf(feat[((size_t)(wy + bi) * Wb + wx + bj) * kFeat + t], wt[((size_t)t * kWinBH + bi) * kWPad + bj], s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) scores[wi] = s + bias;
}

}  // namespace

size_t scheme_cells_scratch(int Wk, int Hk) {
    const size_t gw = 8 * (size_t)(Wk / 8), gh = 8 * (size_t)(Hk / 8);
    const size_t cells = (size_t)(Wk / 8) * (Hk / 8);
    return ((gw * gh + 255) & ~(size_t)255) + 2 * gw * gh * 4 + cells * kLbpBins * 4 + 1024;
}

cudaError_t launch_scheme_cells(cudaStream_t s, int scheme, const uint8_t *img, int Wk, int Hk, int pitch, float *hog,
                                int64_t hog_plane, uint8_t *lbp, int64_t lbp_plane, int cell_pitch,
                                const uint8_t *bin_of, unsigned char *scratch, bool per_block) {
    const int Wc = Wk / 8, Hc = Hk / 8, gw = 8 * Wc, gh = 8 * Hc;
    if (Wc == 0 || Hc == 0) return cudaSuccess;
    uint8_t *codes = scratch;
    float *mag = reinterpret_cast<float *>(scratch + (((size_t)gw * gh + 255) & ~(size_t)255));
    float *pos = mag + (size_t)gw * gh;
    uint32_t *hist = reinterpret_cast<uint32_t *>(pos + (size_t)gw * gh);
    const dim3 pix((gw + kT - 1) / kT, gh);
    const int cells_blocks = (Wc * Hc + kT - 1) / kT;
    if (scheme == PD_SCHEME_LBP_NAIVE || scheme == PD_SCHEME_LBP_SCALABLE) {
        k_lbp_codes<<<pix, kT, 0, s>>>(img, Wk, Hk, pitch, gw, gh, bin_of, codes);
        if (scheme == PD_SCHEME_LBP_NAIVE) {
            k_lbp_cells_naive<<<cells_blocks, kT, 0, s>>>(codes, gw, Wc, Hc, lbp, lbp_plane, cell_pitch);
        } else {
            cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)Wc * Hc * kLbpBins * 4, s);
            if (e != cudaSuccess) return e;
            k_lbp_scatter<<<pix, kT, 0, s>>>(codes, gw, gh, Wc, hist);
            k_lbp_pack<<<(Wc * Hc * kLbpBins + kT - 1) / kT, kT, 0, s>>>(hist, Wc, Hc, lbp, lbp_plane, cell_pitch);
        }
    } else {
        k_gradient<<<pix, kT, 0, s>>>(img, Wk, Hk, pitch, gw, gh, mag, pos);
        const int Wb = Wc - 1, Hb = Hc - 1, blk = (Wb * Hb + kT - 1) / kT;
        if (per_block) {
            if (Wb <= 0 || Hb <= 0) return cudaGetLastError();
            if (scheme == PD_SCHEME_HOG_GLOBAL)
                k_hog_blocks<0><<<blk, kT, 0, s>>>(mag, pos, gw, Wb, Hb, hog, hog_plane, cell_pitch);
            else if (scheme == PD_SCHEME_HOG_LOCAL)
                k_hog_blocks<1><<<blk, kT, 0, s>>>(mag, pos, gw, Wb, Hb, hog, hog_plane, cell_pitch);
            else
                k_hog_blocks<2><<<blk, kT, 0, s>>>(mag, pos, gw, Wb, Hb, hog, hog_plane, cell_pitch);
        } else if (scheme == PD_SCHEME_HOG_GLOBAL)
            k_hog_cells<0><<<cells_blocks, kT, 0, s>>>(mag, pos, gw, gh, Wc, Hc, hog, hog_plane, cell_pitch);
        else if (scheme == PD_SCHEME_HOG_LOCAL)
            k_hog_cells<1><<<cells_blocks, kT, 0, s>>>(mag, pos, gw, gh, Wc, Hc, hog, hog_plane, cell_pitch);
        else
            k_hog_cells<2><<<cells_blocks, kT, 0, s>>>(mag, pos, gw, gh, Wc, Hc, hog, hog_plane, cell_pitch);
    }
    return cudaGetLastError();
}

size_t scheme_scores_scratch(int cells_x, int cells_y) {
    return (size_t)std::max(cells_x - 1, 0) * std::max(cells_y - 1, 0) * kFeat * 4 + 256;
}

cudaError_t launch_scheme_scores(cudaStream_t s, int scheme, const float *hog, int64_t hog_plane,
                                 const uint8_t *lbp, int64_t lbp_plane, int cell_pitch, int cells_x, int cells_y,
                                 const float *wt, float bias, float clip, float *scores, unsigned char *scratch,
                                 bool per_block) {
    const int Wb = cells_x - 1, Hb = cells_y - 1, rows = cells_y - kWinBH, cols = cells_x - kWinBW;
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    float *feat = reinterpret_cast<float *>(scratch);
    k_blocks<<<(Wb * Hb + kT - 1) / kT, kT, 0, s>>>(hog, hog_plane, lbp, lbp_plane, cell_pitch, Wb, Hb, clip,
                                                    per_block ? kHogBins : 0, feat);
    if (scheme == PD_SCHEME_SVM_NAIVE)
        k_svm_naive<<<(rows * cols + kT - 1) / kT, kT, 0, s>>>(feat, Wb, wt, bias, rows, cols, scores);
    else
        k_svm_warp<<<(rows * cols * 32 + kT - 1) / kT, kT, 0, s>>>(feat, Wb, wt, bias, rows, cols, scores);
    return cudaGetLastError();
}

}  // namespace pd
