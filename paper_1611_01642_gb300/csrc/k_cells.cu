// K2 + K3 -- HOG and uniform-LBP cell histograms of one pyramid level
// (Section 4.2, Algorithms 1-2; Section 4.3, Algorithms 4-5).
//
// One CTA of 128 threads owns a tile of 15 x 8 cells (120 x 64 pixels). It
// first stages the 130 x 74 pixel region it reads (the tile, the 4 pixels on
// each side whose HOG votes still reach it, and the 1-pixel gradient halo,
// with the level's clamp-to-edge border baked in) in shared memory with one
// burst of coalesced loads. Thread t then owns pixel column
// x = 8*cx0 - 4 + t and walks down the rows [8*cy0 - 4, 8*cy0 + 68) with its
// 3x3 neighbourhood in registers.
//
// Per pixel:
//  * LBP (Algorithm 1): 8 comparisons with the clockwise neighbours (a
//    neighbour >= centre gives 1), uniform-pattern bin via a 256-entry table,
//    and a shared-memory integer count of its own cell (Algorithm 2; integer
//    atomics on two 16-bit counters per word, so the counts are exact and
//    order independent).
//  * HOG (Algorithm 4): central differences with clamped borders, magnitude
//    sqrt(gx^2 + gy^2), unsigned orientation atan2 folded into [0, 180).
//    The vote is linear between the two nearest of 9 orientation bins and
//    bilinear between the two nearest cell centres (8c + 3.5) on each axis,
//    clamped into the cell grid (Algorithm 5's interpolation on one global
//    cell grid). The vertical part is accumulated per column in the thread's
//    own shared-memory slots (no atomics, fixed row order); the horizontal
//    part is a fixed-order weighted sum over the 16 columns that reach each
//    cell. The result is therefore deterministic.
//
// The walk proceeds in bands of 8 rows: band k covers pixel rows
// [8(cy0+k)-4, 8(cy0+k)+4), which vote only into cell rows cy0+k-1 and
// cy0+k, so after band k cell row cy0+k-1 is final: the CTA reduces it
// horizontally, stores it and recycles its slots. Per-column HOG partial sums
// and LBP counts therefore live in rings of 2 cell rows, which keeps the CTA
// at ~23 KB of shared memory (many CTAs per SM).
// Outputs go to plane-major cell atlases: hog[b][row][cx] (f32),
// lbp[bin][row][cx] (u8, counts <= 64).
#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kThreads = 128;
constexpr int kTW = kCellTW;          // 15 cells
constexpr int kTH = kCellTH;          // 8 cells
constexpr int kCols = 8 * kTW + 8;    // 128 columns (one per thread)
constexpr int kPixCols = kCols + 2;   // + gradient / LBP halo
constexpr int kPixRows = 8 * kTH + 10;
constexpr int kRing = 2;              // open cell rows
constexpr int kRPitch = kCols + kCols / 32;    // padded column index: c + c/32
constexpr int kLbpWords = (kLbpBins + 1) / 2;  // two 16-bit counters per word

struct CellSmem {
    float R[kRing][kHogBins][kRPitch];      // vertical HOG partial sums per column
    uint32_t cnt[kRing][kTW][kLbpWords];    // LBP counts of the open cell rows
    uint8_t map[256];                       // LBP code -> uniform bin
    uint8_t pix[kPixRows][kPixCols];        // [8cy0-5, 8cy0+69) x [8cx0-5, 8cx0+125), clamped
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }
__device__ __forceinline__ int rcol(int c) { return c + (c >> 5); }

__global__ void __launch_bounds__(kThreads) k_cells(const LevelDesc *__restrict__ levels,
                                                    const uint8_t *__restrict__ pyr,
                                                    CellAtlas atlas,
                                                    const CellItem *__restrict__ items,
                                                    const uint8_t *__restrict__ lbp_map) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CellSmem &S = *reinterpret_cast<CellSmem *>(smem_raw);
    const CellItem it = items[blockIdx.x];
    const LevelDesc L = levels[it.level];
    const int tid = threadIdx.x;
    const uint8_t *img = pyr + L.img_off;
    const int pitch = L.img_pitch;
    const int Wk = L.Wk, Hk = L.Hk, Wc = L.Wc, Hc = L.Hc;
    const int gridW = 8 * Wc, gridH = 8 * Hc;

    for (int i = tid; i < kRing * kHogBins * kRPitch; i += kThreads) (&S.R[0][0][0])[i] = 0.f;
    for (int i = tid; i < kRing * kTW * kLbpWords; i += kThreads) (&S.cnt[0][0][0])[i] = 0u;
    for (int i = tid; i < 256; i += kThreads) S.map[i] = lbp_map[i];
    const int px0 = 8 * it.cx0 - 5, py0 = 8 * it.cy0 - 5;
    {
        const int c0 = tid, c1 = tid + kThreads;
        const int x0c = clampi(px0 + c0, 0, Wk - 1);
        const int x1c = clampi(px0 + c1, 0, Wk - 1);
#pragma unroll 8
        for (int r = 0; r < kPixRows; ++r) {
            const uint8_t *p = img + (size_t)clampi(py0 + r, 0, Hk - 1) * pitch;
            S.pix[r][c0] = p[x0c];
            if (c1 < kPixCols) S.pix[r][c1] = p[x1c];
        }
    }
    __syncthreads();

    const int x = 8 * it.cx0 - 4 + tid;
    const bool active = x >= 0 && x < gridW;
    const int sc = x - px0;  // shared-memory column of x
    const bool core_x = (x >= 8 * it.cx0) && (x < 8 * it.cx0 + 8 * kTW);
    const int cxl = (x >> 3) - it.cx0;
    const int rc = rcol(tid);
    const int n_rows = min(kTH, Hc - it.cy0);  // cell rows of this tile inside the level

    for (int band = 0; band <= n_rows; ++band) {
        const int yb = 8 * (it.cy0 + band) - 4;
        const int y_begin = max(yb, 0);
        const int y_end = min(yb + 8, gridH);
        if (active && y_begin < y_end) {
            auto row = [&](int yy, int &l, int &m, int &r) {
                const uint8_t *p = &S.pix[yy - py0][sc];
                l = p[-1];
                m = p[0];
                r = p[1];
            };
            int al, am, ar, bl, bm, br, cl, cm, cr;
            row(y_begin - 1, al, am, ar);
            row(y_begin, bl, bm, br);
            for (int y = y_begin; y < y_end; ++y) {
                row(y + 1, cl, cm, cr);
                // ---- HOG vote
                const int gx = br - bl;
                const int gy = cm - am;
                const float mag = sqrtf((float)(gx * gx + gy * gy));
                float th = atan2f((float)gy, (float)gx) * 57.295779513082320876f;
                if (th < 0.f) th += 180.f;
                if (th >= 180.f) th -= 180.f;
                const float bpos = th * 0.05f - 0.5f;
                const float bf = floorf(bpos);
                const float o1 = bpos - bf, o0 = 1.f - o1;
                int b0 = (int)bf;
                int b1 = b0 + 1;
                b0 = b0 < 0 ? b0 + kHogBins : b0;
                b1 = b1 >= kHogBins ? b1 - kHogBins : b1;
                b0 = clampi(b0, 0, kHogBins - 1);  // theta is in [0, 180): a no-op kept as a guard
                b1 = clampi(b1, 0, kHogBins - 1);
                const float uy = ((float)y - 3.5f) * 0.125f;
                const float fy = floorf(uy);
                const float wy1 = uy - fy, wy0 = 1.f - wy1;
                const int cy0 = clampi((int)fy, 0, Hc - 1) - it.cy0;
                const int cy1 = clampi((int)fy + 1, 0, Hc - 1) - it.cy0;
                if (cy0 >= 0 && cy0 < kTH) {
                    float *R0 = &S.R[cy0 & 1][0][rc];
                    R0[b0 * kRPitch] += mag * o0 * wy0;
                    R0[b1 * kRPitch] += mag * o1 * wy0;
                }
                if (cy1 >= 0 && cy1 < kTH) {
                    float *R1 = &S.R[cy1 & 1][0][rc];
                    R1[b0 * kRPitch] += mag * o0 * wy1;
                    R1[b1 * kRPitch] += mag * o1 * wy1;
                }
                // ---- LBP code and count (core pixels only)
                const int cyl = (y >> 3) - it.cy0;
                if (core_x && cyl >= 0 && cyl < kTH) {
                    const int c = bm;
                    const int code = (al >= c) | ((am >= c) << 1) | ((ar >= c) << 2) |
                                     ((br >= c) << 3) | ((cr >= c) << 4) | ((cm >= c) << 5) |
                                     ((cl >= c) << 6) | ((bl >= c) << 7);
                    const int bin = S.map[code];
                    atomicAdd(&S.cnt[cyl & 1][cxl][bin >> 1], 1u << ((bin & 1) << 4));
                }
                al = bl; am = bm; ar = br;
                bl = cl; bm = cm; br = cr;
            }
        }
        __syncthreads();
        // ---- cell row cyl = band - 1 is final: horizontal HOG reduction, stores
        const int cyl = band - 1;
        if (cyl >= 0) {
            const int cy = it.cy0 + cyl;
            float(*R)[kRPitch] = S.R[cyl & 1];
            for (int i = tid; i < kTW * kHogBins; i += kThreads) {
                const int cxo = i % kTW, b = i / kTW;
                const int cx = it.cx0 + cxo;
                if (cx >= Wc) continue;
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int xx = 8 * cx - 4 + k;
                    if (xx < 0 || xx >= gridW) continue;
                    // the two cell votes of column xx, clamped into the grid
                    const float ux = ((float)xx - 3.5f) * 0.125f;
                    const float fx = floorf(ux);
                    const float wx1 = ux - fx;
                    float w = 0.f;
                    if (clampi((int)fx, 0, Wc - 1) == cx) w += 1.f - wx1;
                    if (clampi((int)fx + 1, 0, Wc - 1) == cx) w += wx1;
                    acc += w * R[b][rcol(8 * cxo + k)];
                }
                atlas.hog[(int64_t)b * atlas.hog_plane + (int64_t)(L.cell_row + cy) * atlas.pitch + cx] = acc;
            }
            for (int i = tid; i < kLbpBins * kTW; i += kThreads) {
                const int cxo = i % kTW, bin = i / kTW;
                const int cx = it.cx0 + cxo;
                if (cx >= Wc) continue;
                const uint32_t v = S.cnt[cyl & 1][cxo][bin >> 1];
                atlas.lbp[(int64_t)bin * atlas.lbp_plane + (int64_t)(L.cell_row + cy) * atlas.pitch + cx] =
                    (uint8_t)((v >> ((bin & 1) << 4)) & 0xffffu);
            }
            __syncthreads();
            // recycle the slots of cell row cyl for cell row cyl + 2
            for (int i = tid; i < kHogBins * kRPitch; i += kThreads) (&R[0][0])[i] = 0.f;
            for (int i = tid; i < kTW * kLbpWords; i += kThreads) (&S.cnt[cyl & 1][0][0])[i] = 0u;
            __syncthreads();
        }
    }
}

}  // namespace

cudaError_t init_cells() {
    return cudaFuncSetAttribute(k_cells, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(CellSmem));
}

cudaError_t launch_cells(cudaStream_t s, const LevelDesc *d_levels, const uint8_t *pyr,
                         CellAtlas atlas, const CellItem *d_items, int n_items,
                         const uint8_t *d_lbp_map) {
    if (n_items <= 0) return cudaSuccess;
    const int smem = (int)sizeof(CellSmem);
    k_cells<<<n_items, kThreads, smem, s>>>(d_levels, pyr, atlas, d_items, d_lbp_map);
    return cudaGetLastError();
}

}  // namespace pd
