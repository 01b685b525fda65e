// K2 + K3 with per-block HOG -- HOG and uniform-LBP cell histograms of one
// pyramid level (Section 4.2, Algorithms 1-2; Section 4.3, Algorithms 4-5),
// the HOG histograms restricted to each 16x16 block (kFeatHogBlock below).
// The shared-cell features (the default) run on the warp-per-strip kernel of
// k_cells_warp.cu; this CTA-per-tile kernel keeps the general FEAT template
// it was written with.
//
// One CTA of 128 threads owns a tile of 15 x 8 cells (120 x 64 pixels). It
// first stages the 130 x 74 pixel region it reads (the tile, the 4 pixels on
// each side whose HOG votes still reach it, and the 1-pixel gradient halo,
// with the level's clamp-to-edge border baked in) in shared memory with one
// burst of coalesced 16-byte loads. Thread t then owns pixel column
// x = 8*cx0 - 4 + t and walks down the rows [8*cy0 - 4, 8*cy0 + 68) with its
// 3x3 neighbourhood in registers.
//
// Per pixel:
//  * LBP (Algorithm 1): 8 comparisons with the clockwise neighbours (a
//    neighbour >= centre gives 1), and a shared-memory integer count of its
//    own cell (Algorithm 2; integer atomics on two 16-bit counters per word,
//    so the counts are exact and order independent); a 256-entry table maps
//    the code straight to its uniform bin's counter word and increment.
//  * HOG (Algorithm 4): central differences with clamped borders, magnitude
//    sqrt(gx^2 + gy^2), unsigned orientation in [0, 180). The orientation is
//    evaluated directly in bin units: the gradient is folded into the upper
//    half plane, reduced to an octant so that z = min/max in [0, 1], and
//    atan(z) comes from an odd polynomial z*P(z^2) of degree 13 whose
//    coefficients were fitted for this kernel (weighted least squares on
//    Chebyshev nodes of [0, 1]) and then scaled to bin units; its float32
//    evaluation is within 1e-6 of a bin (2e-5 degrees) of the true
//    arctangent, and the vote is
//    continuous in the angle, so the histogram error stays far below the
//    1e-4 parity bar.
//    The vote is linear between the two nearest of 9 orientation bins and
//    bilinear between the two nearest cell centres (8c + 3.5) on each axis,
//    clamped into the cell grid (Algorithm 5's interpolation on one global
//    cell grid). The vertical part is accumulated per column in the thread's
//    own shared-memory slots (no atomics, fixed row order); the horizontal
//    part is a fixed-order weighted sum over the 16 columns that reach each
//    cell, one thread per (cell, bin). The result is therefore deterministic.
//
// The walk proceeds in bands of 8 rows: band k covers pixel rows
// [8(cy0+k)-4, 8(cy0+k)+4), which vote only into cell rows cy0+k-1 and
// cy0+k, so after band k cell row cy0+k-1 is final: the CTA reduces it
// horizontally, stores it and recycles its slots. Per-column HOG partial sums
// and LBP counts therefore live in rings of 2 cell rows, which keeps the CTA
// at ~23 KB of shared memory (many CTAs per SM).
// Outputs go to plane-major cell atlases: hog[b][row][cx] (f32),
// lbp[bin][row][cx] (u8, counts <= 64). `feat` selects the features computed
// (HOG, LBP or both: the HOG-SVM and LBP-SVM pipelines of Section 4.1 skip
// the other one).
//
// Per-block HOG (kFeatHogBlock, Algorithm 5 read per 16x16 block): a block's
// 4 cell histograms take only the block's own pixels, with the votes of the
// shared grid left unclamped (a vote towards a cell outside the block is
// dropped). Cell (cy, cx) sits at one of 4 places q = 2a + b of the blocks
// that contain it (a = 0: it is the block's top cell, so the block spans
// pixel rows [8cy, 8cy + 16); a = 1: rows [8cy - 8, 8cy + 8); b likewise on
// x), and the kernel writes its 4 restricted histograms Q_q to planes
// 9q + bin. Block (by, bx) is then [Q_0(by, bx), Q_1(by, bx+1),
// Q_2(by+1, bx), Q_3(by+1, bx+1)]. Of the pixel rows that vote into cell row
// t, those in [8t, 8t + 12) belong to a = 0 and those in [8t - 4, 8t + 8) to
// a = 1: a band row votes into both a's of one of its two cell rows and one
// a of the other (3 vertical slots per pixel instead of 2). On x, the 4
// column sums of a cell's two groups are split in halves: b = 0 drops the
// first half of its own group, b = 1 the second half of the next one.
#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kThreads = 128;
constexpr int kTW = kCellTW;          // 15 cells
constexpr int kTH = kCellTH;          // 8 cells
constexpr int kCols = 8 * kTW + 8;    // 128 columns (one per thread)
constexpr int kPixCols = kCols + 16;  // + gradient / LBP halo, from a 16-byte boundary
constexpr int kPixRows = 8 * kTH + 10;
constexpr int kRing = 2;              // open cell rows
constexpr int kRPitch = kCols;                 // bin stride: a multiple of 32 banks
static_assert(kCols == kThreads, "one pixel column (and its vote slots) per thread");
constexpr int kLbpWords = (kLbpBins + 1) / 2;  // two 16-bit counters per word

template <int NA>
struct CellSmem {
    int4 yv[kPixRows];                      // per pixel row: ring slot / weight of its two cell votes
    float R[kRing][NA][kHogBins][kRPitch];  // vertical HOG partial sums per column (NA = 2: per a)
    float WA[kCols];                        // per column: weight of its vote to the left cell of its group
    float WB[kCols];                        // per column: weight of its vote to its group's own cell
    uint32_t cnt[kRing][kTW][kLbpWords];    // LBP counts of the open cell rows
    uint2 map[256];                         // LBP code -> (counter word byte offset, increment)
    uint8_t pix[kPixRows][kPixCols];        // rows [8cy0-5, 8cy0+69) x columns from xs, clamped
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// atan(z) * 9/pi (radians -> 20-degree bins) for z in [0, 1]: the fitted
// polynomial's coefficients scaled by 9/pi and rounded to float.
__device__ __forceinline__ float atan_bins01(float z) {
    const float s = z * z;
    float p = 0.019514326006174088f;
    p = fmaf(p, s, -0.09626893699169159f);
    p = fmaf(p, s, 0.22810496389865875f);
    p = fmaf(p, s, -0.3791072964668274f);
    p = fmaf(p, s, 0.5674521327018738f);
    p = fmaf(p, s, -0.9544723033905029f);
    p = fmaf(p, s, 2.8647778034210205f);
    return p * z;
}

// Unsigned orientation of (gx, gy) in bin units: theta_degrees / 20, in
// [0, 9] (9 only for theta = 180 degrees, the same orientation as 0: both
// give the same two votes below).
__device__ __forceinline__ float orientation_bins(int gx, int gy) {
    const int ax = abs(gx), ay = abs(gy);
    const float mx = (float)max(ax, ay), mn = (float)min(ax, ay);
    // mx is 0 or >= 1, so adding 1e-30 changes nothing but the 0 / 0 case
    // (which becomes 0 without a branch)
    const float z = __fdividef(mn, mx + 1e-30f);
    float phi = atan_bins01(z);                // angle of (|gx|, |gy|) to the nearer axis
    if (ay > ax) phi = 4.5f - phi;             // 90 degrees - phi
    return (gx ^ gy) < 0 ? 9.0f - phi : phi;   // opposite signs: mirror into (90, 180)
}

template <int FEAT>
__global__ void __launch_bounds__(kThreads) k_cells(const LevelDesc *__restrict__ levels,
                                                    const uint8_t *__restrict__ pyr,
                                                    CellAtlas atlas,
                                                    const CellItem *__restrict__ items,
                                                    const uint8_t *__restrict__ lbp_map,
                                                    const uint32_t *__restrict__ c_flag) {
    constexpr int feat = FEAT;
    constexpr bool pb = (FEAT & kFeatHogBlock) != 0;  // per-block HOG
    constexpr int NA = pb ? 2 : 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CellSmem<NA> &S = *reinterpret_cast<CellSmem<NA> *>(smem_raw);
    if (c_flag && !c_flag[blockIdx.x]) return;  // sparse path: no kept window needs these cells
    const CellItem it = items[blockIdx.x];
    const LevelDesc L = levels[it.level];
    const int tid = threadIdx.x;
    const uint8_t *img = pyr + L.img_off;
    const int pitch = L.img_pitch;
    const int Wk = L.Wk, Hk = L.Hk, Wc = L.Wc, Hc = L.Hc;
    const int gridW = 8 * Wc, gridH = 8 * Hc;

    for (int i = tid; i < kRing * NA * kHogBins * kRPitch; i += kThreads) (&S.R[0][0][0][0])[i] = 0.f;
    for (int i = tid; i < kRing * kTW * kLbpWords; i += kThreads) (&S.cnt[0][0][0])[i] = 0u;
    for (int i = tid; i < 256; i += kThreads) {
        // uniform bin -> its 16-bit counter: word (byte offset) and increment
        const int bn = lbp_map[i];
        S.map[i] = make_uint2((uint32_t)(bn >> 1) * 4u, 1u << ((bn & 1) << 4));
    }
    const int px0 = 8 * it.cx0 - 5, py0 = 8 * it.cy0 - 5;
    for (int r = tid; r < kPixRows; r += kThreads) {
        // row y votes into cell rows floor(u), floor(u)+1 (u = (y-3.5)/8,
        // clamped into the grid; per-block: unclamped, rows outside the grid
        // dropped) with weights 1-frac, frac; slot -1 = not in this tile
        const int y = py0 + r;
        const float uy = ((float)y - 3.5f) * 0.125f;
        const float fy = floorf(uy);
        const float w1 = uy - fy;
        const int f0 = (int)fy;
        const int c0 = (pb ? (f0 >= 0 && f0 < Hc ? f0 : -(1 << 20)) : clampi(f0, 0, Hc - 1)) - it.cy0;
        const int c1 = (pb ? (f0 + 1 < Hc ? f0 + 1 : -(1 << 20)) : clampi(f0 + 1, 0, Hc - 1)) - it.cy0;
        int4 e;
        e.x = (c0 >= 0 && c0 < kTH) ? (c0 & 1) : -1;
        e.y = (c1 >= 0 && c1 < kTH) ? (c1 & 1) : -1;
        e.z = __float_as_int(1.f - w1);
        e.w = __float_as_int(w1);
        S.yv[r] = e;
    }
    static_assert(kPixCols % 16 == 0 && kPixCols >= kCols + 13, "16-byte chunks covering the halo");
    // Staging: rows [py0, py0 + kPixRows) and the 144 columns from
    // xs = 8 cx0 - 8 rounded down to a multiple of 16 (they hold the 130
    // columns [px0, px0 + 130) the tile reads), in 16-byte chunks: one
    // 16-byte load each where the chunk lies inside the level row (and the
    // level is 16-byte aligned), else byte loads clamped to the level.
    const int xs = (px0 - 3) & ~15;
    {
        constexpr int kChunks = kPixCols / 16;
        const bool al = ((reinterpret_cast<uintptr_t>(img) | (uintptr_t)pitch) & 15u) == 0;
        for (int i = tid; i < kPixRows * kChunks; i += kThreads) {
            const int r = i / kChunks, q = i - r * kChunks;
            const int x0 = xs + 16 * q;
            const uint8_t *row = img + (size_t)clampi(py0 + r, 0, Hk - 1) * pitch;
            uint4 v;
            if (al && x0 >= 0 && x0 + 16 <= Wk) {
                v = *reinterpret_cast<const uint4 *>(row + x0);
            } else {
                uint32_t wv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    uint32_t wd = 0;
#pragma unroll
                    for (int j = 0; j < 4; ++j) wd |= (uint32_t)row[clampi(x0 + 4 * k + j, 0, Wk - 1)] << (8 * j);
                    wv[k] = wd;
                }
                v = make_uint4(wv[0], wv[1], wv[2], wv[3]);
            }
            reinterpret_cast<uint4 *>(S.pix[r])[q] = v;
        }
    }
    __syncthreads();

    const int x = 8 * it.cx0 - 4 + tid;
    const bool active = x >= 0 && x < gridW;
    const int sc = x - xs;  // shared-memory column of x
    const bool core_x = (x >= 8 * it.cx0) && (x < 8 * it.cx0 + 8 * kTW);
    const int cxl = (x >> 3) - it.cx0;
    const int rc = tid;
    // Horizontal vote of this column: pixel column x reaches cells
    // cx0+g-1 and cx0+g (g = tid/8) with weights wA, wB (clamped into the grid,
    // unclamped for per-block HOG; zero outside it).
    float wA = 0.f, wB = 0.f;
    if (active) {
        const float ux = ((float)x - 3.5f) * 0.125f;
        const float fx = floorf(ux);
        const float w1 = ux - fx, w0 = 1.f - w1;
        const int c0 = pb ? (int)fx : clampi((int)fx, 0, Wc - 1);
        const int c1 = pb ? (int)fx + 1 : clampi((int)fx + 1, 0, Wc - 1);
        const int left = it.cx0 + (tid >> 3) - 1, own = left + 1;
        wA = (c0 == left ? w0 : 0.f) + (c1 == left ? w1 : 0.f);
        wB = (c0 == own ? w0 : 0.f) + (c1 == own ? w1 : 0.f);
    }
    S.WA[tid] = wA;
    S.WB[tid] = wB;
    const int n_rows = min(kTH, Hc - it.cy0);  // cell rows of this tile inside the level

    for (int band = 0; band <= n_rows; ++band) {
        // band rows yb .. yb+7 (the staged region holds yb-1 .. yb+8, clamped to
        // the level); rows outside the cell grid [0, gridH) are skipped
        const int yb = 8 * (it.cy0 + band) - 4;
        if (active) {
            auto row = [&](int yy, int &l, int &m, int &r) {
                const uint8_t *p = &S.pix[yy - py0][sc];
                l = p[-1];
                m = p[0];
                r = p[1];
            };
            int al, am, ar, bl, bm, br;
            row(yb - 1, al, am, ar);
            row(yb, bl, bm, br);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int y = yb + k;
                int cl, cm, cr;
                row(y + 1, cl, cm, cr);
                if (y >= 0 && y < gridH && (feat & kFeatHog)) {
                    // ---- HOG vote
                    const int gx = br - bl;
                    const int gy = cm - am;
                    const float m2 = (float)(gx * gx + gy * gy);
                    // m2 is 0 or >= 1: the 1e-30 only turns 0 * inf into 0
                    const float mag = m2 * rsqrtf(m2 + 1e-30f);
                    // bpos in [-0.5, 8.5]: floor in [-1, 8], so b0 = -1 wraps to 8
                    // and b1 = 9 to 0 (bpos -0.5 and 8.5 give the same votes)
                    const float bpos = orientation_bins(gx, gy) - 0.5f;
                    const float bf = floorf(bpos);
                    const float o1 = bpos - bf, o0 = 1.f - o1;
                    const int bi = (int)bf;
                    const int b0 = bi < 0 ? kHogBins - 1 : bi;
                    const int b1 = bi + 1 >= kHogBins ? 0 : bi + 1;
                    const int4 yv = S.yv[y - py0];
                    const float mo1 = mag * o1, mo0 = mag - mo1;
                    if constexpr (!pb) {
                        if (yv.x >= 0) {
                            const float w = __int_as_float(yv.z);
                            float *R0 = &S.R[yv.x][0][0][rc];
                            R0[b0 * kRPitch] += mo0 * w;
                            R0[b1 * kRPitch] += mo1 * w;
                        }
                        if (yv.y >= 0) {
                            const float w = __int_as_float(yv.w);
                            float *R1 = &S.R[yv.y][0][0][rc];
                            R1[b0 * kRPitch] += mo0 * w;
                            R1[b1 * kRPitch] += mo1 * w;
                        }
                    } else {
                        // a band row above the band's centre (k < 4) lies in both a's
                        // of the upper cell row and in a = 1 of the lower one; below
                        // it (k >= 4), in a = 0 of the upper and both of the lower
                        if (yv.x >= 0) {
                            const float w = __int_as_float(yv.z);
                            const float v0 = mo0 * w, v1 = mo1 * w;
                            float *R0 = &S.R[yv.x][0][0][rc];
                            R0[b0 * kRPitch] += v0;
                            R0[b1 * kRPitch] += v1;
                            if (k < 4) {
                                R0 += kHogBins * kRPitch;
                                R0[b0 * kRPitch] += v0;
                                R0[b1 * kRPitch] += v1;
                            }
                        }
                        if (yv.y >= 0) {
                            const float w = __int_as_float(yv.w);
                            const float v0 = mo0 * w, v1 = mo1 * w;
                            float *R1 = &S.R[yv.y][NA - 1][0][rc];
                            R1[b0 * kRPitch] += v0;
                            R1[b1 * kRPitch] += v1;
                            if (k >= 4) {
                                R1 -= kHogBins * kRPitch;
                                R1[b0 * kRPitch] += v0;
                                R1[b1 * kRPitch] += v1;
                            }
                        }
                    }
                }
                if (y >= 0 && y < gridH && (feat & kFeatLbp)) {
                    // ---- LBP code and count (core pixels only; the cell row is
                    // band - 1 for k < 4, band for k >= 4)
                    const int cyl = band - 1 + (k >= 4 ? 1 : 0);
                    if (core_x && cyl >= 0 && cyl < kTH) {
                        const int c = bm;
                        const int code = (al >= c) | ((am >= c) << 1) | ((ar >= c) << 2) |
                                         ((br >= c) << 3) | ((cr >= c) << 4) | ((cm >= c) << 5) |
                                         ((cl >= c) << 6) | ((bl >= c) << 7);
                        const uint2 e = S.map[code];
                        atomicAdd(reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(&S.cnt[cyl & 1][cxl][0]) + e.x), e.y);
                    }
                }
                al = bl; am = bm; ar = br;
                bl = cl; bm = cm; br = cr;
            }
        }
        __syncthreads();
        // ---- cell row cyl = band - 1 is final: horizontal HOG sums, stores
        const int cyl = band - 1;
        if (cyl >= 0) {
            const int cy = it.cy0 + cyl;
            const int64_t row = (int64_t)(L.cell_row + cy) * atlas.pitch;
            const float(*R)[kRPitch] = S.R[cyl & 1][0];
            // HOG: one thread per (bin, cell): own group with WB, next group with WA
            if (pb) {
                // per-block: halves of both groups for each a; b = 0 drops the
                // first half of the own group, b = 1 the second half of the next
                for (int o = tid; o < 2 * kHogBins * kTW; o += kThreads) {
                    const int a = o / (kHogBins * kTW), ob = o - a * (kHogBins * kTW);
                    const int bin = ob / kTW, cxo = ob - bin * kTW;
                    const int cx = it.cx0 + cxo;
                    if (cx >= Wc) continue;
                    const float *Ra = &S.R[cyl & 1][a][bin][8 * cxo];
                    float h[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float4 v = reinterpret_cast<const float4 *>(Ra)[k];
                        const float4 w = reinterpret_cast<const float4 *>(k < 2 ? &S.WB[8 * cxo] : &S.WA[8 * cxo + 8])[k & 1];
                        float acc = w.x * v.x;
                        acc = fmaf(w.y, v.y, acc);
                        acc = fmaf(w.z, v.z, acc);
                        acc = fmaf(w.w, v.w, acc);
                        h[k] = acc;
                    }
                    const int64_t at = row + cx;
                    atlas.hog[(int64_t)((2 * a) * kHogBins + bin) * atlas.hog_plane + at] = (h[1] + h[2]) + h[3];
                    atlas.hog[(int64_t)((2 * a + 1) * kHogBins + bin) * atlas.hog_plane + at] = (h[0] + h[1]) + h[2];
                }
            }
            for (int o = tid; o < ((feat & kFeatHog) && !pb ? kHogBins * kTW : 0); o += kThreads) {
                const int b = o / kTW, cxo = o - b * kTW;
                const int cx = it.cx0 + cxo;
                if (cx >= Wc) continue;
                const float4 *r4 = reinterpret_cast<const float4 *>(&R[b][8 * cxo]);
                const float4 *wb4 = reinterpret_cast<const float4 *>(&S.WB[8 * cxo]);
                const float4 *wa4 = reinterpret_cast<const float4 *>(&S.WA[8 * cxo + 8]);
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float4 v = r4[k], w = wb4[k];
                    acc = fmaf(w.x, v.x, acc);
                    acc = fmaf(w.y, v.y, acc);
                    acc = fmaf(w.z, v.z, acc);
                    acc = fmaf(w.w, v.w, acc);
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float4 v = r4[2 + k], w = wa4[k];
                    acc = fmaf(w.x, v.x, acc);
                    acc = fmaf(w.y, v.y, acc);
                    acc = fmaf(w.z, v.z, acc);
                    acc = fmaf(w.w, v.w, acc);
                }
                atlas.hog[(int64_t)b * atlas.hog_plane + row + cx] = acc;
            }
            // LBP: one thread per counter word (two bins) of a cell
            for (int o = tid; o < ((feat & kFeatLbp) ? kLbpWords * kTW : 0); o += kThreads) {
                const int wd = o / kTW, cxo = o - wd * kTW;
                const int cx = it.cx0 + cxo;
                const uint32_t v = S.cnt[cyl & 1][cxo][wd];
                S.cnt[cyl & 1][cxo][wd] = 0u;  // recycled for cell row cyl + 2
                if (cx >= Wc) continue;
                atlas.lbp[(int64_t)(2 * wd) * atlas.lbp_plane + row + cx] = (uint8_t)(v & 0xffffu);
                if (2 * wd + 1 < kLbpBins)
                    atlas.lbp[(int64_t)(2 * wd + 1) * atlas.lbp_plane + row + cx] = (uint8_t)(v >> 16);
            }
            __syncthreads();
            // recycle the HOG slots of cell row cyl for cell row cyl + 2: only
            // this thread votes into its column, so it clears it itself
#pragma unroll
            for (int a = 0; a < NA; ++a)
#pragma unroll
                for (int b = 0; b < kHogBins; ++b) S.R[cyl & 1][a][b][tid] = 0.f;
        }
    }
}

}  // namespace

namespace {
using CellFn = void (*)(const LevelDesc *, const uint8_t *, CellAtlas, const CellItem *, const uint8_t *,
                        const uint32_t *);
constexpr int kBlk = kFeatHogBlock;
// per-block HOG only (the shared-cell features run on the warp-per-strip kernel)
const CellFn kCellFns[2] = {k_cells<kFeatHog | kFeatLbp | kBlk>, k_cells<kFeatHog | kBlk>};
const int kCellSmem = (int)sizeof(CellSmem<2>);
}  // namespace

cudaError_t init_cells() {
    for (int i = 0; i < 2; ++i) {
        const cudaError_t e = cudaFuncSetAttribute(kCellFns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, kCellSmem);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_cells(cudaStream_t s, const LevelDesc *d_levels, const uint8_t *pyr,
                         CellAtlas atlas, const CellItem *d_items, int n_items,
                         const uint8_t *d_lbp_map, const uint32_t *c_flag, int feat) {
    if (!(feat & kFeatHogBlock)) return cudaErrorInvalidValue;
    if (n_items <= 0) return cudaSuccess;
    const int k = (feat & kFeatLbp) ? 0 : 1;
    kCellFns[k]<<<n_items, kThreads, kCellSmem, s>>>(d_levels, pyr, atlas, d_items, d_lbp_map, c_flag);
    return cudaGetLastError();
}

}  // namespace pd
