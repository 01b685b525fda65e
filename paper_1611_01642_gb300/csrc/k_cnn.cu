// Learned window proposal: inference kernels.
//
// The paper has no learned stage; this network predicts which windows of a
// pyramid level can score above the SVM threshold, so that the sparse path
// computes HOG/LBP cells and window scores only where they matter:
//   x  = bf16(L/255 - 0.5)
//   a1 = relu(conv3x3 s2 (1 -> 16)),  a2 = relu(conv3x3 s2 (16 -> 32)),
//   a3 = relu(conv3x3 s2 (32 -> 32)) (one per 8x8 cell),
//   h  = wh . a3 + bh (1x1 head),   z[wy][wx] = bv + sum V[r][s] h[wy+r][wx+s].
// bf16 inputs, weights and stored activations; fp32 accumulation.
//
// k_cnn_fwd: one CTA (8 warps) per 8x8 tile of cells. It stages the 71x71
// input pixels, computes the 35x35x16 layer-1 activations on CUDA cores, the
// 17x17x32 layer-2 activations and the 8x8x32 layer-3 activations as implicit
// GEMMs on the tensor cores (mma.sync m16n8k16 bf16 -> fp32; the A operand is
// gathered from shared memory laid out position-major with padded strides so
// that the stride-2 gathers are bank-conflict free), and writes h.
// Zero padding of every convolution is the zero activation outside each
// layer's grid.
// k_cnn_pool: one thread per window, z from 128 taps of h.
#include "pd_internal.h"

#include <cuda_bf16.h>

namespace pd {
namespace {

constexpr int kThreads = 256;
constexpr int T3 = 8;            // layer-3 tile (cells)
constexpr int R2 = 2 * T3 + 1;   // 17 layer-2 positions per side
constexpr int R1 = 2 * R2 + 1;   // 35 layer-1 positions per side
constexpr int R0 = 2 * R1 + 1;   // 71 pixels per side
constexpr int S1W = 10;          // layer-1 position stride in 32-bit words (16 ch + 4 pad bf16)
constexpr int S2W = 18;          // layer-2 position stride in words (32 ch + 4 pad bf16)
constexpr int M2 = R2 * R2;      // 289 layer-2 positions
constexpr int M2T = (M2 + 15) / 16;  // 19 m-tiles

struct CnnSmem {
    float x[R0][R0 + 1];
    uint32_t a1[R1 * R1 * S1W];
    uint32_t a2[M2 * S2W];
    float w1[16][9];
    float b1[16];
    float b2[32];
    float b3[32];
    float wh[32];
    float hpart[2][64];
    float tab[256];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(kThreads) k_cnn_fwd(const LevelDesc *__restrict__ levels,
                                                      const uint8_t *__restrict__ pyr,
                                                      const CnnItem *__restrict__ items,
                                                      const CnnWeights wts, float *__restrict__ hmap,
                                                      int32_t hmap_pitch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CnnSmem &S = *reinterpret_cast<CnnSmem *>(smem_raw);
    const CnnItem it = items[blockIdx.x];
    const LevelDesc L = levels[it.level];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    const int Hk = L.Hk, Wk = L.Wk;
    const int H1 = (Hk + 1) / 2, W1 = (Wk + 1) / 2;
    const int H2 = (H1 + 1) / 2, W2 = (W1 + 1) / 2;
    const int y3 = it.cy0, x3 = it.cx0;                  // tile origin (cells)
    const int y2 = 2 * y3 - 1, x2 = 2 * x3 - 1;          // layer-2 region origin
    const int y1 = 2 * y2 - 1, x1 = 2 * x2 - 1;          // layer-1 region origin
    const int y0 = 2 * y1 - 1, x0 = 2 * x1 - 1;          // pixel region origin
    const uint8_t *img = pyr + L.img_off;

    for (int i = tid; i < 256; i += kThreads) S.tab[i] = wts.in_tab[i];
    for (int i = tid; i < 16 * 9; i += kThreads) (&S.w1[0][0])[i] = wts.w1[i];
    if (tid < 16) S.b1[tid] = wts.b1[tid];
    if (tid < 32) {
        S.b2[tid] = wts.b2[tid];
        S.b3[tid] = wts.b3[tid];
        S.wh[tid] = wts.wh[tid];
    }
    __syncthreads();
    // ---- input pixels (zero outside the level: the padding of layer 1)
    for (int i = tid; i < R0 * R0; i += kThreads) {
        const int r = i / R0, c = i - r * R0;
        const int y = y0 + r, x = x0 + c;
        float v = 0.f;
        if (y >= 0 && y < Hk && x >= 0 && x < Wk) v = S.tab[img[(size_t)y * L.img_pitch + x]];
        S.x[r][c] = v;
    }
    __syncthreads();
    // ---- layer 1 on CUDA cores: 35x35 positions x 16 channels
    for (int p = tid; p < R1 * R1; p += kThreads) {
        const int r = p / R1, c = p - r * R1;
        const int yy = y1 + r, xx = x1 + c;
        uint32_t *dst = &S.a1[p * S1W];
        if (yy < 0 || yy >= H1 || xx < 0 || xx >= W1) {
#pragma unroll
            for (int k = 0; k < 8; ++k) dst[k] = 0u;
            continue;
        }
        float in[9];
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) in[dy * 3 + dx] = S.x[2 * r + dy][2 * c + dx];
#pragma unroll
        for (int o = 0; o < 16; o += 2) {
            float s0 = S.b1[o], s1 = S.b1[o + 1];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                s0 = fmaf(S.w1[o][k], in[k], s0);
                s1 = fmaf(S.w1[o + 1][k], in[k], s1);
            }
            dst[o >> 1] = pack_bf16(fmaxf(s0, 0.f), fmaxf(s1, 0.f));
        }
    }
    // layer-2 weights as mma B fragments (9 taps x 4 n-tiles x 2 regs)
    uint32_t bw2[9][4][2];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const uint2 v = reinterpret_cast<const uint2 *>(wts.w2frag)[(tap * 4 + nt) * 32 + lane];
            bw2[tap][nt][0] = v.x;
            bw2[tap][nt][1] = v.y;
        }
    __syncthreads();
    // ---- layer 2 on tensor cores: 289 positions x 32 channels, K = 9 x 16
    for (int mt = warp; mt < M2T; mt += kThreads / 32) {
        const int p0 = mt * 16 + g, p1 = p0 + 8;
        const int q0 = min(p0, M2 - 1), q1 = min(p1, M2 - 1);  // padding rows reuse a valid row
        const int r0 = q0 / R2, c0 = q0 - r0 * R2, r1 = q1 / R2, c1 = q1 - r1 * R2;
        float acc[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[nt][e] = 0.f;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const uint32_t *s0 = &S.a1[((2 * r0 + dy) * R1 + 2 * c0 + dx) * S1W];
                const uint32_t *s1 = &S.a1[((2 * r1 + dy) * R1 + 2 * c1 + dx) * S1W];
                const uint32_t a0 = s0[t], a1 = s1[t], a2 = s0[4 + t], a3 = s1[4 + t];
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
                    mma_bf16(acc[nt], a0, a1, a2, a3, bw2[dy * 3 + dx][nt][0], bw2[dy * 3 + dx][nt][1]);
            }
        // epilogue: bias, relu, bf16, zero outside the layer-2 grid
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int p = half ? p1 : p0;
            if (p >= M2) continue;
            const int r = p / R2, c = p - r * R2;
            const bool inside = (y2 + r) >= 0 && (y2 + r) < H2 && (x2 + c) >= 0 && (x2 + c) < W2;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int co = nt * 8 + 2 * t;
                float v0 = acc[nt][2 * half] + S.b2[co], v1 = acc[nt][2 * half + 1] + S.b2[co + 1];
                v0 = inside ? fmaxf(v0, 0.f) : 0.f;
                v1 = inside ? fmaxf(v1, 0.f) : 0.f;
                S.a2[p * S2W + (co >> 1)] = pack_bf16(v0, v1);
            }
        }
    }
    __syncthreads();
    // ---- layer 3 on tensor cores: 64 positions x 32 channels, K = 9 x 32;
    // warp w: m-tile w & 3, n-tiles 2*(w >> 2) .. +1
    {
        const int mt = warp & 3, nh = warp >> 2;
        const int p0 = mt * 16 + g, p1 = p0 + 8;
        const int r0 = p0 >> 3, c0 = p0 & 7, r1 = p1 >> 3, c1 = p1 & 7;
        float acc[2][4];
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[j][e] = 0.f;
        const uint2 *w3 = reinterpret_cast<const uint2 *>(wts.w3frag);
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const uint32_t *s0 = &S.a2[((2 * r0 + dy) * R2 + 2 * c0 + dx) * S2W];
                const uint32_t *s1 = &S.a2[((2 * r1 + dy) * R2 + 2 * c1 + dx) * S2W];
#pragma unroll
                for (int kh = 0; kh < 2; ++kh) {
                    const uint32_t a0 = s0[kh * 8 + t], a1 = s1[kh * 8 + t];
                    const uint32_t a2 = s0[kh * 8 + 4 + t], a3 = s1[kh * 8 + 4 + t];
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const uint2 b = __ldg(&w3[(((dy * 3 + dx) * 2 + kh) * 4 + 2 * nh + j) * 32 + lane]);
                        mma_bf16(acc[j], a0, a1, a2, a3, b.x, b.y);
                    }
                }
            }
        // bias, relu, head partial over this lane's 4 channels, reduce over t
        float h0 = 0.f, h1 = 0.f;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int co = (2 * nh + j) * 8 + 2 * t;
            h0 = fmaf(fmaxf(acc[j][0] + S.b3[co], 0.f), S.wh[co], h0);
            h0 = fmaf(fmaxf(acc[j][1] + S.b3[co + 1], 0.f), S.wh[co + 1], h0);
            h1 = fmaf(fmaxf(acc[j][2] + S.b3[co], 0.f), S.wh[co], h1);
            h1 = fmaf(fmaxf(acc[j][3] + S.b3[co + 1], 0.f), S.wh[co + 1], h1);
        }
        h0 += __shfl_xor_sync(0xffffffffu, h0, 1);
        h0 += __shfl_xor_sync(0xffffffffu, h0, 2);
        h1 += __shfl_xor_sync(0xffffffffu, h1, 1);
        h1 += __shfl_xor_sync(0xffffffffu, h1, 2);
        if (t == 0) {
            S.hpart[nh][p0] = h0;
            S.hpart[nh][p1] = h1;
        }
    }
    __syncthreads();
    if (tid < 64) {
        const int cy = y3 + (tid >> 3), cx = x3 + (tid & 7);
        if (cy < L.Hc && cx < L.Wc)
            hmap[(int64_t)(L.cell_row + cy) * hmap_pitch + cx] = wts.bh[0] + S.hpart[0][tid] + S.hpart[1][tid];
    }
}

// One thread per window: z = bv + sum_{r<16, s<8} V[r][s] h[wy+r][wx+s].
__global__ void __launch_bounds__(256) k_cnn_pool(const LevelDesc *__restrict__ levels, int n_levels,
                                                  const float *__restrict__ hmap, int32_t hmap_pitch,
                                                  const float *__restrict__ v, const float *__restrict__ bvp,
                                                  float *__restrict__ logits) {
    __shared__ float V[16 * 8];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) V[i] = v[i];
    __syncthreads();
    const LevelDesc L = levels[blockIdx.y];
    const int n = L.rows * L.cols;
    const float bv = bvp[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int wy = i / L.cols, wx = i - wy * L.cols;
        const float *hp = hmap + (int64_t)(L.cell_row + wy) * hmap_pitch + wx;
        float z = bv;
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int s = 0; s < 8; ++s) z = fmaf(V[r * 8 + s], hp[(int64_t)r * hmap_pitch + s], z);
        logits[L.score_off + i] = z;
    }
    (void)n_levels;
}

}  // namespace

cudaError_t init_cnn() {
    return cudaFuncSetAttribute(k_cnn_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CnnSmem));
}

cudaError_t launch_cnn(cudaStream_t s, const LevelDesc *d_levels, int n_levels, const uint8_t *pyr,
                       const CnnItem *d_items, int n_items, const CnnWeights &w, float *hmap,
                       int32_t hmap_pitch, float *logits) {
    if (n_items > 0) {
        k_cnn_fwd<<<n_items, kThreads, sizeof(CnnSmem), s>>>(d_levels, pyr, d_items, w, hmap, hmap_pitch);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_levels > 0) {
        dim3 grid(32, n_levels);
        k_cnn_pool<<<grid, 256, 0, s>>>(d_levels, n_levels, hmap, hmap_pitch, w.v, w.bv, logits);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace pd
