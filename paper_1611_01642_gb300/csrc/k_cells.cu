// K2 + K3 -- HOG and uniform-LBP cell histograms of one pyramid level
// (Section 4.2, Algorithms 1-2; Section 4.3, Algorithms 4-5).
//
// One CTA of 128 threads owns a tile of 15 x 8 cells (120 x 64 pixels). It
// first stages the 130 x 74 pixel region it reads (the tile, the 4 pixels on
// each side whose HOG votes still reach it, and the 1-pixel gradient halo,
// with the level's clamp-to-edge border baked in) in shared memory with one
// burst of coalesced loads. Thread t then owns pixel column
// x = 8*cx0 - 4 + t and walks down the rows [8*cy0 - 4, 8*cy0 + 68) with its
// 3x3 neighbourhood kept in registers (one new row of 3 bytes per step).
//
// Per pixel:
//  * LBP (Algorithm 1): 8 comparisons with the clockwise neighbours (a
//    neighbour >= centre gives 1), uniform-pattern bin via a 256-entry table,
//    and a shared-memory integer count of its own cell (Algorithm 2; integer
//    atomics, so the counts are exact and order independent).
//  * HOG (Algorithm 4): central differences with clamped borders, magnitude
//    sqrt(gx^2 + gy^2), unsigned orientation atan2 folded into [0, 180).
//    The vote is linear between the two nearest of 9 orientation bins and
//    bilinear between the two nearest cell centres (8c + 3.5) on each axis,
//    clamped into the cell grid (Algorithm 5's interpolation on one global
//    cell grid). The vertical part is accumulated per column in the thread's
//    own shared-memory slots (no atomics, fixed row order); the horizontal
//    part is a fixed-order weighted sum over the 16 columns that reach each
//    cell. The result is therefore deterministic.
// Outputs go to plane-major cell atlases: hog[b][row][cx] (f32),
// lbp[bin][row][cx] (u8, counts <= 64).
#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kThreads = 128;
constexpr int kTW = kCellTW;   // 15 cells
constexpr int kTH = kCellTH;   // 8 cells
constexpr int kCols = 8 * kTW + 8;  // 128 columns (one per thread)
constexpr int kPixCols = kCols + 2;  // + gradient / LBP halo
constexpr int kPixRows = 8 * kTH + 10;

struct CellSmem {
    float R[kTH][kHogBins][kCols];       // vertical HOG partial sums per column
    uint32_t cnt[kTH][kTW][kLbpBins];    // LBP counts per cell
    uint8_t map[256];                    // LBP code -> uniform bin
    uint8_t pix[kPixRows][kPixCols];     // pixels [8cy0-5, 8cy0+69) x [8cx0-5, 8cx0+125), clamped
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

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

#pragma unroll
    for (int r = 0; r < kTH; ++r)
#pragma unroll
        for (int b = 0; b < kHogBins; ++b) S.R[r][b][tid] = 0.f;
    for (int i = tid; i < kTH * kTW * kLbpBins; i += kThreads) (&S.cnt[0][0][0])[i] = 0u;
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
    const int gridW = 8 * Wc, gridH = 8 * Hc;
    if (x >= 0 && x < gridW) {
        const int sc = x - px0;  // shared-memory column of x (x-1 and x+1 are its neighbours)
        const bool core_x = (x >= 8 * it.cx0) && (x < 8 * it.cx0 + 8 * kTW);
        const int cxl = (x >> 3) - it.cx0;
        const int y_begin = max(8 * it.cy0 - 4, 0);
        const int y_end = min(8 * it.cy0 + 8 * kTH + 4, gridH);
        // rolling 3x3 neighbourhood: rows y-1 (a), y (b), y+1 (c)
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
                S.R[cy0][b0][tid] += mag * o0 * wy0;
                S.R[cy0][b1][tid] += mag * o1 * wy0;
            }
            if (cy1 >= 0 && cy1 < kTH) {
                S.R[cy1][b0][tid] += mag * o0 * wy1;
                S.R[cy1][b1][tid] += mag * o1 * wy1;
            }
            // ---- LBP code and count (core pixels only)
            const int cyl = (y >> 3) - it.cy0;
            if (core_x && cyl >= 0 && cyl < kTH) {
                const int c = bm;
                const int code = (al >= c) | ((am >= c) << 1) | ((ar >= c) << 2) | ((br >= c) << 3) |
                                 ((cr >= c) << 4) | ((cm >= c) << 5) | ((cl >= c) << 6) |
                                 ((bl >= c) << 7);
                atomicAdd(&S.cnt[cyl][cxl][S.map[code]], 1u);
            }
            al = bl; am = bm; ar = br;
            bl = cl; bm = cm; br = cr;
        }
    }
    __syncthreads();

    // ---- horizontal HOG reduction and stores
    for (int i = tid; i < kTH * kTW * kHogBins; i += kThreads) {
        const int b = i % kHogBins;
        const int cxl = (i / kHogBins) % kTW;
        const int cyl = i / (kHogBins * kTW);
        const int cx = it.cx0 + cxl, cy = it.cy0 + cyl;
        if (cx >= Wc || cy >= Hc) continue;
        float acc = 0.f;
        for (int xx = 8 * cx - 4; xx < 8 * cx + 12; ++xx) {
            if (xx < 0 || xx >= gridW) continue;
            const float ux = ((float)xx - 3.5f) * 0.125f;
            const float fx = floorf(ux);
            const float wx1 = ux - fx, wx0 = 1.f - wx1;
            float w = 0.f;
            if (clampi((int)fx, 0, Wc - 1) == cx) w += wx0;
            if (clampi((int)fx + 1, 0, Wc - 1) == cx) w += wx1;
            acc += w * S.R[cyl][b][xx - (8 * it.cx0 - 4)];
        }
        atlas.hog[(int64_t)b * atlas.hog_plane + (int64_t)(L.cell_row + cy) * atlas.pitch + cx] = acc;
    }
    for (int i = tid; i < kLbpBins * kTH * kTW; i += kThreads) {
        const int cxl = i % kTW;
        const int cyl = (i / kTW) % kTH;
        const int bin = i / (kTW * kTH);
        const int cx = it.cx0 + cxl, cy = it.cy0 + cyl;
        if (cx >= Wc || cy >= Hc) continue;
        atlas.lbp[(int64_t)bin * atlas.lbp_plane + (int64_t)(L.cell_row + cy) * atlas.pitch + cx] =
            (uint8_t)S.cnt[cyl][cxl][bin];
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
