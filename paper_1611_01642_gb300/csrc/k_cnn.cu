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
// k_cnn_fwd: persistent CTAs (8 warps, two per SM), each walking 8x8-cell
// tiles. The 72x80 input bytes of the next tile are fetched with cp.async
// while the current tile is computed. Per tile: the pixels become bf16 x
// (zero outside the level: the padding of layer 1); layer 1 runs on the
// tensor cores as a GEMM over 4x4 pixel patches (a stride-2 3x3 window at
// (2r-1, 2c-1) is the top-left 3x3 of the 4x4 patch there; the 7 extra taps
// carry zero weights), giving 35x35x16 activations; layer 2 (17x17x32,
// K = 9 taps x 16) and layer 3 (8x8x32, K = 9 x 32) are implicit GEMMs on
// the tensor cores (mma.sync m16n8k16 bf16 -> fp32) whose A operand is
// gathered from shared memory laid out position-major with padded strides
// so that the stride-2 gathers are bank-conflict free; the 1x1 head gives h.
// Zero padding of every convolution is the zero activation outside each
// layer's grid.
#include "pd_internal.h"

#include <cuda_bf16.h>

#include <algorithm>

namespace pd {
namespace {

constexpr int kThreads = 256;
constexpr int T3 = 8;            // layer-3 tile (cells)
constexpr int R2 = 2 * T3 + 1;   // 17 layer-2 positions per side
constexpr int R1 = 2 * R2 + 1;   // 35 layer-1 positions per side
constexpr int XR = 2 * R1 + 2;   // 72 pixel rows/columns under the 4x4 patches
constexpr int kRawW = 80;        // staged bytes per row: pixels x0-1 .. x0+78, ten 8-byte chunks
constexpr int kChunks = kRawW / 8;
constexpr int XBW = 44;          // bf16 pixel row stride in words (72 used, padded for banks)
// Activations are stored as 16-byte rows of 8 bf16 channels, split by
// channel group and by column parity: plane (group, parity) holds the
// positions of that parity, row-major with (columns + 1) / 2 columns. A
// stride-2 tap then reads 8 consecutive 16-byte rows (one ldmatrix 8x8
// matrix, conflict free), and the epilogue writes them with stmatrix. Plane
// strides are padded to 4 (mod 8) 16-byte units so that the two parities of
// 8 consecutive positions fall on disjoint banks.
constexpr int C1P = (R1 + 1) / 2;  // 18 plane columns of layer 1
constexpr int PS1 = 636;           // layer-1 plane stride (35 x 18 = 630, padded), 16-byte units
constexpr int C2P = (R2 + 1) / 2;  // 9 plane columns of layer 2
constexpr int PS2 = 156;           // layer-2 plane stride (17 x 9 = 153, padded)
static_assert(PS1 >= R1 * C1P && PS1 % 8 == 4 && PS2 >= R2 * C2P && PS2 % 8 == 4, "plane strides");
constexpr int M1 = R1 * R1;      // 1225 layer-1 positions
constexpr int M1T = (M1 + 15) / 16;  // 77 m-tiles
constexpr int M2 = R2 * R2;      // 289 layer-2 positions
constexpr int M2T = (M2 + 15) / 16;  // 19 m-tiles
constexpr int kW3Frag = 9 * 2 * 4 * 32;  // uint2 layer-3 B fragments
constexpr float kInv255 = 1.0f / 255.0f;   // float32 nearest to 1/255

struct CnnSmem {
    uint8_t raw[2][XR][kRawW];   // input bytes, double buffered
    uint4 a1[2 * 2 * PS1];       // [channel group 0..1][parity] planes of layer 1
    union {
        uint32_t xb[XR * XBW];   // bf16 pixel pairs (dead once layer 1 is done)
        uint4 a2[4 * 2 * PS2];   // [channel group 0..3][parity] planes of layer 2
    } u;
    uint2 w3[kW3Frag];
    float b1[16];
    float b2[32];
    float b3[32];
    float wh[32];
    float hpart[2][64];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// relu of both values, rounded to bf16 and packed (lo in the low half)
__device__ __forceinline__ uint32_t relu_pack_bf16(float lo, float hi) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Four 8x8 bf16 matrices from / to shared memory; lane l gives the address
// of row l % 8 of matrix l / 8; register i holds matrix i in the mma
// fragment layout (row lane / 4, columns 2 (lane % 4), +1).
template <int OFF>
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4+%5];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr), "n"(OFF)
                 : "memory");
}
__device__ __forceinline__ void stsm_x4(uint32_t addr, uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
    asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(r0), "r"(r1),
                 "r"(r2), "r"(r3)
                 : "memory");
}

// 8-byte asynchronous copy global -> shared; bytes past n are zero-filled.
__device__ __forceinline__ void cp_async8(void *dst, const void *src, int n) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Stages the bytes of pixel rows y0 .. y0+71 and columns x0-1 .. x0+78 of an
// item (x0 = 8 cx0 - 7, so every chunk starts on an 8-byte boundary of the
// level row; level rows are 16-byte aligned). Chunks outside the level read
// nothing (zero fill); the conversion below zeroes those pixels anyway.
__device__ __forceinline__ void stage_input(uint8_t (*raw)[kRawW], const CnnItem *__restrict__ items,
                                            const LevelDesc *__restrict__ levels, const uint8_t *__restrict__ pyr,
                                            int item, int tid) {
    const CnnItem it = items[item];
    const LevelDesc L = levels[it.level];
    const int y0 = 8 * it.cy0 - 7, xs = 8 * it.cx0 - 8;
    const uint8_t *img = pyr + L.img_off;
    for (int k = tid; k < XR * kChunks; k += kThreads) {
        const int r = k / kChunks, q = k - r * kChunks;
        const int y = y0 + r, x = xs + 8 * q;
        int n = 0;
        const uint8_t *src = img;
        if (y >= 0 && y < L.Hk && x >= 0) {
            n = min(max(L.Wk - x, 0), 8);
            if (n > 0) src = img + (size_t)y * L.img_pitch + x;
        }
        cp_async8(&raw[r][8 * q], src, n);
    }
}

__global__ void __launch_bounds__(kThreads, 2) k_cnn_fwd(const LevelDesc *__restrict__ levels,
                                                         const uint8_t *__restrict__ pyr,
                                                         const CnnItem *__restrict__ items, int n_items,
                                                         const CnnWeights wts, float *__restrict__ hmap,
                                                         int32_t hmap_pitch) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CnnSmem &S = *reinterpret_cast<CnnSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    int item = blockIdx.x;
    if (item >= n_items) return;
    stage_input(S.raw[0], items, levels, pyr, item, tid);
    cp_async_commit();

    for (int i = tid; i < kW3Frag; i += kThreads) S.w3[i] = reinterpret_cast<const uint2 *>(wts.w3frag)[i];
    if (tid < 16) S.b1[tid] = wts.b1[tid];
    if (tid < 32) {
        S.b2[tid] = wts.b2[tid];
        S.b3[tid] = wts.b3[tid];
        S.wh[tid] = wts.wh[tid];
    }
    // layer-1 B fragments: B[k][n] = w1[n][ky][kx], k = 4 ky + kx, zero for ky = 3 or kx = 3
    uint32_t bw1[2][2];
#pragma unroll
    for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int hk = 0; hk < 2; ++hk) {
            const int o = nt * 8 + g, ky = (t >> 1) + 2 * hk, kx = 2 * (t & 1);
            const float lo = (ky < 3 && kx < 3) ? wts.w1[o * 9 + ky * 3 + kx] : 0.f;
            const float hi = (ky < 3 && kx + 1 < 3) ? wts.w1[o * 9 + ky * 3 + kx + 1] : 0.f;
            bw1[nt][hk] = pack_bf16(lo, hi);
        }
    // layer-2 B fragments (9 taps x 4 n-tiles x 2 regs), kept in registers
    uint32_t bw2[9][4][2];
#pragma unroll
    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const uint2 v = reinterpret_cast<const uint2 *>(wts.w2frag)[(tap * 4 + nt) * 32 + lane];
            bw2[tap][nt][0] = v.x;
            bw2[tap][nt][1] = v.y;
        }
    const float bh = wts.bh[0];
    const uint32_t a1_base = static_cast<uint32_t>(__cvta_generic_to_shared(&S.a1[0]));
    const uint32_t a2_base = static_cast<uint32_t>(__cvta_generic_to_shared(&S.u.a2[0]));

    for (int iter = 0; item < n_items; ++iter, item += gridDim.x) {
        const int cur = iter & 1;
        const int next = item + gridDim.x;
        if (next < n_items) stage_input(S.raw[cur ^ 1], items, levels, pyr, next, tid);
        cp_async_commit();
        cp_async_wait_prev();  // this thread's copies of the current tile have landed
        __syncthreads();       // everyone's have; the previous tile is finished

        const CnnItem it = items[item];
        const LevelDesc L = levels[it.level];
        const int Hk = L.Hk, Wk = L.Wk;
        const int H1 = (Hk + 1) / 2, W1 = (Wk + 1) / 2;
        const int H2 = (H1 + 1) / 2, W2 = (W1 + 1) / 2;
        const int y3 = it.cy0, x3 = it.cx0;                  // tile origin (cells)
        const int y2 = 2 * y3 - 1, x2 = 2 * x3 - 1;          // layer-2 region origin
        const int y1 = 2 * y2 - 1, x1 = 2 * x2 - 1;          // layer-1 region origin
        const int y0 = 2 * y1 - 1, x0 = 2 * x1 - 1;          // pixel region origin
        const bool interior1 = y1 >= 0 && x1 >= 0 && y1 + R1 <= H1 && x1 + R1 <= W1;
        const bool interior2 = y2 >= 0 && x2 >= 0 && y2 + R2 <= H2 && x2 + R2 <= W2;

        // ---- pixels -> bf16 x; xb[r][c] = x(y0 + r, x0 + c) = raw[r][c + 1].
        // x = bf16(L/255 - 0.5): one fma in float32 rounded once to bf16 equals
        // the correctly rounded value for all 256 inputs (checked exhaustively
        // against exact rational arithmetic when this path was written).
        for (int k = tid; k < XR * (XR / 4); k += kThreads) {
            const int r = k / (XR / 4), j = k - r * (XR / 4);
            const uint32_t *rw = reinterpret_cast<const uint32_t *>(S.raw[cur][r]);
            const uint32_t v = __byte_perm(rw[j], rw[j + 1], 0x4321);
            const int y = y0 + r, xc = x0 + 4 * j;
            const bool rin = y >= 0 && y < Hk;
            float e[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int x = xc + b;
                e[b] = (rin && x >= 0 && x < Wk) ? fmaf((float)((v >> (8 * b)) & 255u), kInv255, -0.5f) : 0.f;
            }
            *reinterpret_cast<uint2 *>(&S.u.xb[r * XBW + 2 * j]) = make_uint2(pack_bf16(e[0], e[1]), pack_bf16(e[2], e[3]));
        }
        __syncthreads();
        // ---- layer 1 on tensor cores: 1225 positions x 16 channels, K = 16 (4x4 patch)
        for (int mt = warp; mt < M1T; mt += kThreads / 32) {
            const int p0 = mt * 16 + g, p1 = p0 + 8;
            const int q0 = min(p0, M1 - 1), q1 = min(p1, M1 - 1);  // padding rows repeat the last row
            const int r0 = q0 / R1, c0 = q0 - r0 * R1, r1 = q1 / R1, c1 = q1 - r1 * R1;
            const uint32_t *x0w = &S.u.xb[(2 * r0 + (t >> 1)) * XBW + c0 + (t & 1)];
            const uint32_t *x1w = &S.u.xb[(2 * r1 + (t >> 1)) * XBW + c1 + (t & 1)];
            const uint32_t a0 = x0w[0], a1 = x1w[0], a2 = x0w[2 * XBW], a3 = x1w[2 * XBW];
            float acc[2][4];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                acc[nt][0] = acc[nt][2] = S.b1[nt * 8 + 2 * t];
                acc[nt][1] = acc[nt][3] = S.b1[nt * 8 + 2 * t + 1];
                mma_bf16(acc[nt], a0, a1, a2, a3, bw1[nt][0], bw1[nt][1]);
            }
            const bool in0 = interior1 || ((y1 + r0) >= 0 && (y1 + r0) < H1 && (x1 + c0) >= 0 && (x1 + c0) < W1);
            const bool in1 = interior1 || ((y1 + r1) >= 0 && (y1 + r1) < H1 && (x1 + c1) >= 0 && (x1 + c1) < W1);
            // this lane's row address: row (l % 8) + 8 ((l / 8) & 1) of the tile, channel group l / 16
            const int ps = min(mt * 16 + (lane & 15), M1 - 1);
            const int pr = ps / R1, pc = ps - pr * R1;
            const uint32_t dst = a1_base + ((((lane >> 4) * 2 + (pc & 1)) * PS1 + pr * C1P + (pc >> 1)) << 4);
            stsm_x4(dst, in0 ? relu_pack_bf16(acc[0][0], acc[0][1]) : 0u,
                    in1 ? relu_pack_bf16(acc[0][2], acc[0][3]) : 0u, in0 ? relu_pack_bf16(acc[1][0], acc[1][1]) : 0u,
                    in1 ? relu_pack_bf16(acc[1][2], acc[1][3]) : 0u);
        }
        __syncthreads();
        // ---- layer 2 on tensor cores: 289 positions x 32 channels, K = 9 taps x 16
        for (int mt = warp; mt < M2T; mt += kThreads / 32) {
            const int p0 = mt * 16 + g, p1 = p0 + 8;
            const int q0 = min(p0, M2 - 1), q1 = min(p1, M2 - 1);
            const int r0 = q0 / R2, c0 = q0 - r0 * R2, r1 = q1 / R2, c1 = q1 - r1 * R2;
            // A rows: lane l reads output row (l % 8) + 8 ((l / 8) & 1), channel group l / 16;
            // tap (dy, dx) is layer-1 position (2r + dy, 2c + dx): parity dx & 1, plane column c + dx / 2
            const int ls = min(mt * 16 + (lane & 15), M2 - 1);
            const int lr = ls / R2, lc = ls - lr * R2;
            const uint32_t src = a1_base + ((((lane >> 4) * 2) * PS1 + 2 * lr * C1P + lc) << 4);
            float acc[4][4];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                acc[nt][0] = acc[nt][2] = S.b2[nt * 8 + 2 * t];
                acc[nt][1] = acc[nt][3] = S.b2[nt * 8 + 2 * t + 1];
            }
#define PD_L2_TAP(DY, DX)                                                                                   \
    {                                                                                                     \
        uint32_t a0, a1, a2, a3;                                                                          \
        ldsm_x4<((((DX) & 1) * PS1 + (DY) * C1P + ((DX) >> 1)) << 4)>(src, a0, a1, a2, a3);                \
        _Pragma("unroll") for (int nt = 0; nt < 4; ++nt)                                                  \
            mma_bf16(acc[nt], a0, a1, a2, a3, bw2[(DY) * 3 + (DX)][nt][0], bw2[(DY) * 3 + (DX)][nt][1]);   \
    }
            PD_L2_TAP(0, 0) PD_L2_TAP(0, 1) PD_L2_TAP(0, 2)
            PD_L2_TAP(1, 0) PD_L2_TAP(1, 1) PD_L2_TAP(1, 2)
            PD_L2_TAP(2, 0) PD_L2_TAP(2, 1) PD_L2_TAP(2, 2)
#undef PD_L2_TAP
            const bool in0 = interior2 || ((y2 + r0) >= 0 && (y2 + r0) < H2 && (x2 + c0) >= 0 && (x2 + c0) < W2);
            const bool in1 = interior2 || ((y2 + r1) >= 0 && (y2 + r1) < H2 && (x2 + c1) >= 0 && (x2 + c1) < W2);
            // channel groups 2h + (l / 16) of output row (l % 8) + 8 ((l / 8) & 1)
            const uint32_t dst = a2_base + ((((lane >> 4) * 2 + (lc & 1)) * PS2 + lr * C2P + (lc >> 1)) << 4);
#pragma unroll
            for (int h = 0; h < 2; ++h)
                stsm_x4(dst + ((4 * h * PS2) << 4),
                        in0 ? relu_pack_bf16(acc[2 * h][0], acc[2 * h][1]) : 0u,
                        in1 ? relu_pack_bf16(acc[2 * h][2], acc[2 * h][3]) : 0u,
                        in0 ? relu_pack_bf16(acc[2 * h + 1][0], acc[2 * h + 1][1]) : 0u,
                        in1 ? relu_pack_bf16(acc[2 * h + 1][2], acc[2 * h + 1][3]) : 0u);
        }
        __syncthreads();
        // ---- layer 3 on tensor cores: 64 positions x 32 channels, K = 9 x 32;
        // warp w: m-tile w & 3, n-tiles 2*(w >> 2) .. +1
        {
            const int mt = warp & 3, nh = warp >> 2;
            const int p0 = mt * 16 + g, p1 = p0 + 8;
            float acc2[2][2][4];  // [k-half][n-tile]: four independent mma chains
#pragma unroll
            for (int kh = 0; kh < 2; ++kh)
#pragma unroll
                for (int j = 0; j < 2; ++j)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc2[kh][j][e] = 0.f;
            // A rows: lane l reads output position (l % 8) + 8 ((l / 8) & 1) of the m-tile,
            // channel group 2 kh + l / 16
            const int lp = mt * 16 + (lane & 15);
            const int lr = lp >> 3, lc = lp & 7;
            const uint32_t src = a2_base + ((((lane >> 4) * 2) * PS2 + 2 * lr * C2P + lc) << 4);
#define PD_L3_TAP(DY, DX, KH)                                                                                  \
    {                                                                                                        \
        uint32_t a0, a1, a2, a3;                                                                             \
        ldsm_x4<(((2 * (KH) * 2 + ((DX) & 1)) * PS2 + (DY) * C2P + ((DX) >> 1)) << 4)>(src, a0, a1, a2, a3);  \
        _Pragma("unroll") for (int j = 0; j < 2; ++j) {                                                     \
            const uint2 b = S.w3[((((DY) * 3 + (DX)) * 2 + (KH)) * 4 + 2 * nh + j) * 32 + lane];             \
            mma_bf16(acc2[KH][j], a0, a1, a2, a3, b.x, b.y);                                                 \
        }                                                                                                    \
    }
            PD_L3_TAP(0, 0, 0) PD_L3_TAP(0, 0, 1) PD_L3_TAP(0, 1, 0) PD_L3_TAP(0, 1, 1) PD_L3_TAP(0, 2, 0)
            PD_L3_TAP(0, 2, 1) PD_L3_TAP(1, 0, 0) PD_L3_TAP(1, 0, 1) PD_L3_TAP(1, 1, 0) PD_L3_TAP(1, 1, 1)
            PD_L3_TAP(1, 2, 0) PD_L3_TAP(1, 2, 1) PD_L3_TAP(2, 0, 0) PD_L3_TAP(2, 0, 1) PD_L3_TAP(2, 1, 0)
            PD_L3_TAP(2, 1, 1) PD_L3_TAP(2, 2, 0) PD_L3_TAP(2, 2, 1)
#undef PD_L3_TAP
            float acc[2][4];
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[j][e] = acc2[0][j][e] + acc2[1][j][e];
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
                hmap[(int64_t)(L.cell_row + cy) * hmap_pitch + cx] = bh + S.hpart[0][tid] + S.hpart[1][tid];
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Window pooling z[wy][wx] = bv + sum_{r<16, s<8} V[r][s] h[wy+r][wx+s]: one
// CTA per (level, 64 x 16 window tile); the tile's 31 x 71 cells of h are
// staged in shared memory; each thread computes 4 consecutive windows of one
// row (8 taps x 4 windows per h row from 11 staged values), in a fixed order.
constexpr int kPoolHW = kPoolTW + 8;                    // 72 staged columns (71 used)
constexpr int kPoolHH = kPoolTH + kWinBH;               // 31 staged rows

__global__ void __launch_bounds__(256) k_cnn_pool(const LevelDesc *__restrict__ levels,
                                                  const float *__restrict__ hmap, int32_t hmap_pitch,
                                                  const float *__restrict__ v, const float *__restrict__ bvp,
                                                  float *__restrict__ logits) {
    __shared__ __align__(16) float V[16 * 8];
    __shared__ __align__(16) float Hs[kPoolHH][kPoolHW];
    const LevelDesc L = levels[blockIdx.y];
    const int tiles_x = (L.cols + kPoolTW - 1) / kPoolTW;
    const int ty = blockIdx.x / max(tiles_x, 1), tx = blockIdx.x - ty * max(tiles_x, 1);
    const int wy0 = ty * kPoolTH, wx0 = tx * kPoolTW;
    if (L.rows == 0 || wy0 >= L.rows) return;  // CTA-uniform
    for (int i = threadIdx.x; i < 128; i += blockDim.x) V[i] = v[i];
    for (int i = threadIdx.x; i < kPoolHH * kPoolHW; i += blockDim.x) {
        const int r = i / kPoolHW, c = i - r * kPoolHW;
        const int cy = wy0 + r, cx = wx0 + c;
        Hs[r][c] = (cy < L.Hc && cx < L.Wc) ? hmap[(int64_t)(L.cell_row + cy) * hmap_pitch + cx] : 0.f;
    }
    __syncthreads();
    const int ry = threadIdx.x >> 4, qx = 4 * (threadIdx.x & 15);
    const float bv = bvp[0];
    float z[4] = {bv, bv, bv, bv};
#pragma unroll 4
    for (int r = 0; r < 16; ++r) {
        const float4 h0 = *reinterpret_cast<const float4 *>(&Hs[ry + r][qx]);
        const float4 h1 = *reinterpret_cast<const float4 *>(&Hs[ry + r][qx + 4]);
        const float4 h2 = *reinterpret_cast<const float4 *>(&Hs[ry + r][qx + 8]);
        const float hv[12] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w, h2.x, h2.y, h2.z, h2.w};
        const float4 v0 = *reinterpret_cast<const float4 *>(&V[r * 8]);
        const float4 v1 = *reinterpret_cast<const float4 *>(&V[r * 8 + 4]);
        const float vv[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int x = 0; x < 4; ++x) z[x] = fmaf(vv[s], hv[x + s], z[x]);
    }
    const int wy = wy0 + ry;
    if (wy < L.rows) {
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int wx = wx0 + qx + x;
            if (wx < L.cols) logits[L.score_off + (int64_t)wy * L.cols + wx] = z[x];
        }
    }
}

int g_cnn_grid = 0;  // persistent CTAs: two per SM

}  // namespace

cudaError_t init_cnn() {
    if (g_cnn_grid == 0) {
        int dev = 0, sms = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_cnn_grid = 2 * sms;
    }
    return cudaFuncSetAttribute(k_cnn_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(CnnSmem));
}

cudaError_t launch_cnn(cudaStream_t s, const LevelDesc *d_levels, int n_levels, const uint8_t *pyr,
                       const CnnItem *d_items, int n_items, const CnnWeights &w, float *hmap,
                       int32_t hmap_pitch, float *logits, int pool_tiles) {
    if (n_items > 0) {
        const int grid = std::min(n_items, g_cnn_grid > 0 ? g_cnn_grid : n_items);
        k_cnn_fwd<<<grid, kThreads, sizeof(CnnSmem), s>>>(d_levels, pyr, d_items, n_items, w, hmap, hmap_pitch);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (n_levels > 0 && pool_tiles > 0) {
        // enough x-blocks for the largest level's 64 x 16 tiles; the others leave early
        dim3 grid(pool_tiles, n_levels);
        k_cnn_pool<<<grid, 256, 0, s>>>(d_levels, hmap, hmap_pitch, w.v, w.bv, logits);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace pd
