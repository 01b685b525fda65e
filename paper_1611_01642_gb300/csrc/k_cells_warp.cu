// K2 + K3 -- HOG and uniform-LBP cell histograms of the pyramid levels
// (Section 4.2, Algorithms 1-2; Section 4.3, Algorithms 4-5), one warp per
// strip of cells, four pixel columns per lane.
//
// Persistent warps (4 per CTA, independent of each other) take strips from a
// queue, tallest first. A strip is 15 cells wide and up to kStripTiles cell
// tiles (8 cell rows each) tall; the planner takes shorter strips, down to 2
// cell rows, when a batch is small. Its warp walks the 128 pixel columns
// [8 cx0 - 4, 8 cx0 + 124) (the strip and the 4 columns on each side whose
// HOG votes still reach it): lane t owns columns 8 cx0 - 4 + 4t .. + 3, which
// lie in one cell (strip cell (t - 1) / 2; lanes 0 and 31 lie in the
// neighbouring strips). The warp walks the pixel rows from the top in bands
// of 8: band k covers the rows [8 (cy0 + k) - 4, 8 (cy0 + k) + 4), which vote
// only into cell rows cy0 + k - 1 and cy0 + k, so after band k cell row
// cy0 + k - 1 is final and the warp writes it out. A tall strip walks the
// 4-row vertical halo of a band once per strip.
//
// Per row a lane loads three aligned 32-bit words of the level row (its own
// 4 bytes and its neighbours'; byte loads clamped to the level at its left
// and right edges), one row pair ahead, and keeps the rows above and below
// in registers. For its 4 pixels:
//  * LBP (Algorithm 1) on packed bytes. For bytes n, c: n >= c exactly when
//    the subtraction n - c does not borrow out of bit 7, which is the
//    majority of (n7, not c7, bit 7 of (n | 0x80) - (c & 0x7f)); one
//    subtraction and one 3-input logic operation compare 4 pixels with one
//    neighbour, and the 8 comparison words fold into 4 codes. A 256-entry
//    table gives each code's uniform bin as an 8-bit counter of a word of the
//    lane's own counters ([word][lane] layout: the shared-memory atomics never
//    collide; exact and order independent; Algorithm 2). A cell's counts are
//    the sum of its two lanes' counters (each <= 32), written out after the
//    band's first 4 rows, which complete cell row cy0 + k - 1.
//  * HOG (Algorithm 4). One byte permute and two dp2a (weights +1, -1) give
//    the central differences of two pixels; the accumulator 0x4B400000 makes
//    the 32-bit result the float 1.5 * 2^23 + g, so one multiply-add turns it
//    into g / 2 (exact). Magnitude sqrt(gx^2 + gy^2); unsigned orientation in
//    bin units (degrees / 20): the angle phi of (|gx|, |gy|) is 45 degrees +
//    atan(t) with t = (|gy| - |gx|) / (|gy| + |gx|) in [-1, 1], where an odd
//    polynomial t P(t^2) of degree 13 fitted to atan on [0, 1] (weighted
//    least squares on Chebyshev nodes, scaled to bin units; error < 1e-6
//    bin) holds; theta is phi or 180 degrees - phi as the signs of gx and gy
//    agree or not (one sign flip, no branch). The vote is linear between the
//    two nearest of the 9 bins and between the two cell rows of the band
//    (weights (7.5 - k) / 8 and (k + 0.5) / 8 for band row k), and bilinear
//    on x through the columns' weights in the epilogue.
//    floor(theta / 20deg - 0.5) comes from rounding 2 (theta - 1) to an even
//    integer by adding 3 * 2^23, where floats are spaced by 2 (a tie gives
//    the other neighbour with weight 1, the same votes); the residual e in
//    [-1, 1] gives the lower and upper bins' weights (1 - e) / 2 and
//    (1 + e) / 2 with one multiply-add each, and the float's bits are the
//    bin number plus a constant, so they index the column's vote slots
//    directly. There are 11 slots per column, slot s holding bin
//    (s - 1) mod 9 (bin -1 and bin 9 wrap), which the epilogue folds back:
//    the loop needs no wrap logic.
//    The slots of lane t's 4 columns sit at 4t + (j ^ ((t >> 3) & 3)), so
//    that a warp's data-dependent scatter hits 32 distinct banks and the
//    epilogue reads them with one 16-byte load. Rows outside the cell grid
//    vote with weight 0 and count nothing (no branch).
// HOG epilogue of cell row r: each lane forms, per bin, the weighted sums of
// its 4 columns for its own cell and for the neighbouring cell they reach;
// three shuffles add the 4 lanes that reach a cell (fixed order:
// deterministic). The LBP counts go out bin-plane by bin-plane, one byte per
// cell, lanes on consecutive cells (coalesced). At the top and bottom of a
// level the votes of the clamped cell row (Algorithm 5's interpolation
// clamped into the grid) are added into the first and last row before they
// are written. The result does not depend on the strip height: every cell
// row sums its votes in the same order.
//
// Sparse path: c_flag marks the 15 x 8-cell tiles to compute; a band is
// walked when one of its two cell rows lies in a marked tile, and a cell
// row is written when its tile is marked.
#include <algorithm>
#include <type_traits>
#include <utility>

#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kWarps = 4;                        // strips per CTA
constexpr int kSCols = 8 * kCellTW + 8;          // 128 pixel columns walked per strip
static_assert(kSCols == 4 * 32, "four pixel columns per lane");
constexpr int kSlots = kHogBins + 2;             // vote slots per column (bins -1 .. 9)
constexpr int kRingStride = kSlots * kSCols;     // floats per open cell row
constexpr int kCntWords = (kLbpBins + 3) / 4;    // words of four 8-bit counters per cell
constexpr uint32_t kHi = 0x80808080u;
constexpr float kMagic = 12582912.0f;            // 1.5 * 2^23: dp2a accumulator
constexpr uint32_t kMagicBits = 0x4B400000u;
constexpr float kMagic2 = 25165824.0f;           // 3 * 2^23 (spacing 2): rounds to even integers
constexpr uint32_t kMagic2Bits = 0x4BC00000u;

struct WarpSmem {
    float R[2 * kRingStride];       // HOG vote slots of the 2 open cell rows
    uint32_t cnt[kCntWords * 32];   // LBP counters of the open cell row: [word][lane], lane-private
};
struct StripSmem {
    uint2 map[256];                 // LBP code -> (counter word index, increment)
    WarpSmem w[kWarps];
};

struct Row {
    uint32_t l, c, r;  // bytes x - 1 .. x + 2, x .. x + 3, x + 1 .. x + 4 of a lane's columns
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// c + b.byte0 - b.byte1 (lo) / c + b.byte2 - b.byte3 (hi), bytes unsigned
__device__ __forceinline__ int dp2a_diff_lo(uint32_t b, int c) {
    int d;
    asm("dp2a.lo.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(0xFFFF0001u), "r"(b), "r"(c));
    return d;
}
__device__ __forceinline__ int dp2a_diff_hi(uint32_t b, int c) {
    int d;
    asm("dp2a.hi.s32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(0xFFFF0001u), "r"(b), "r"(c));
    return d;
}

// Operands here are 0 or >= 1e-30 (never subnormal), so the flush-to-zero
// forms are exact.
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 2 atan(z) * 9/pi / z as a polynomial in s = z^2 (|z| <= 1): the fitted
// coefficients scaled to 20-degree bins and doubled (exact: every step of
// the evaluation scales by 2).
__device__ __forceinline__ float atan_bins2_poly(float s) {
    float p = 2.0f * 0.019514326006174088f;
    p = fmaf(p, s, 2.0f * -0.09626893699169159f);
    p = fmaf(p, s, 2.0f * 0.22810496389865875f);
    p = fmaf(p, s, 2.0f * -0.3791072964668274f);
    p = fmaf(p, s, 2.0f * 0.5674521327018738f);
    p = fmaf(p, s, 2.0f * -0.9544723033905029f);
    return fmaf(p, s, 2.0f * 2.8647778034210205f);
}

template <class F, int... I>
__device__ __forceinline__ void static_for(F &&f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}

// 4 pixels' n >= c comparisons, as bit 7 of each byte (other bits 0).
__device__ __forceinline__ uint32_t ge4(uint32_t n, uint32_t c_lo, uint32_t c_not7) {
    const uint32_t t = (n | kHi) - c_lo;
    const uint32_t n7 = n & kHi;
    return (n7 & c_not7) | (t & (n7 | c_not7));
}

template <int FEAT>
__global__ void __launch_bounds__(kWarps * 32, 4)
    k_cells_warp(const LevelDesc *__restrict__ levels, const uint8_t *__restrict__ pyr, CellAtlas atlas,
                 const StripItem *__restrict__ items, int n_items, int *__restrict__ queue,
                 const uint8_t *__restrict__ lbp_map, const uint32_t *__restrict__ c_flag) {
    constexpr bool kHog = (FEAT & kFeatHog) != 0, kLbp = (FEAT & kFeatLbp) != 0;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StripSmem &S = *reinterpret_cast<StripSmem *>(smem_raw);
    if (kLbp) {
        for (int i = threadIdx.x; i < 256; i += kWarps * 32) {
            const int bn = lbp_map[i];
            S.map[i] = make_uint2((uint32_t)(bn >> 2) * 32u, 1u << ((bn & 3) * 8));
        }
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    WarpSmem &Wm = S.w[threadIdx.x >> 5];
    // persistent warps: each takes the next strip (tallest first) until none is left
    for (;;) {
        int item = lane == 0 ? atomicAdd(queue, 1) : 0;
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) return;
        const StripItem it = items[item];
        const LevelDesc L = levels[it.level];
        const uint8_t *img = pyr + L.img_off;
        const int pitch = L.img_pitch, Wk = L.Wk, Hk = L.Hk, Wc = L.Wc, Hc = L.Hc;
        const int gridH = 8 * Hc;
        const int cx0 = it.cx0, cy0 = it.cy0, nb = it.cy1 - it.cy0;
        const int tx = cx0 / kCellTW;
        const int x = 8 * cx0 - 4 + 4 * lane;  // first pixel column of this lane
        const bool fast = (((reinterpret_cast<uintptr_t>(img) | (uintptr_t)pitch) & 3u) == 0) && x >= 4 &&
                          x + 8 <= Wk;

        if (kHog)
            for (int i = lane; i < 2 * kRingStride / 4; i += 32)
                reinterpret_cast<float4 *>(Wm.R)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (kLbp)
            for (int i = lane; i < kCntWords * 32; i += 32) Wm.cnt[i] = 0u;

        // ---- lane constants
        const int sw = (lane >> 3) & 3;
        // float index of slot 0 of pixel j's column, less the bias of the rounded angle's bits
        uint32_t vb[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) vb[j] = (uint32_t)(4 * lane + (j ^ sw)) + 128u - kMagic2Bits * 128u;
        // epilogue x-weights by slot position p (column j = p ^ sw): own cell, neighbour cell
        float wo[4], wn[4];
        {
            const int own = cx0 + ((lane - 1) >> 1);
            const int nbr = own + ((lane & 1) ? -1 : 1);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int xc = x + (p ^ sw);
                float a = 0.f, b = 0.f;
                if (xc >= 0 && xc < 8 * Wc) {
                    const float ux = ((float)xc - 3.5f) * 0.125f;
                    const float fx = floorf(ux);
                    const float w1 = ux - fx, w0 = 1.f - w1;
                    const int c0 = clampi((int)fx, 0, Wc - 1), c1 = clampi((int)fx + 1, 0, Wc - 1);
                    a = (c0 == own ? w0 : 0.f) + (c1 == own ? w1 : 0.f);
                    b = (c0 == nbr ? w0 : 0.f) + (c1 == nbr ? w1 : 0.f);
                }
                wo[p] = a;
                wn[p] = b;
            }
        }
        const bool core = (unsigned)(lane - 1) < 30u;  // lanes 1..30 own strip pixels (LBP)
        __syncwarp();

        // ---- rows
        auto fetch = [&](int y, uint32_t (&w)[3]) {
            const uint8_t *row = img + (size_t)clampi(y, 0, Hk - 1) * pitch;
            if (fast) {
                const uint32_t *p = reinterpret_cast<const uint32_t *>(row + x);
                w[0] = __ldg(p - 1);
                w[1] = __ldg(p);
                w[2] = __ldg(p + 1);
            } else {
                uint32_t v[6];
#pragma unroll
                for (int i = 0; i < 6; ++i) v[i] = __ldg(row + clampi(x - 1 + i, 0, Wk - 1));
                w[0] = v[0] << 24;
                w[1] = v[1] | (v[2] << 8) | (v[3] << 16) | (v[4] << 24);
                w[2] = v[5];
            }
        };
        auto mkrow = [](const uint32_t (&w)[3]) {
            Row r;
            r.l = __funnelshift_r(w[0], w[1], 24);
            r.c = w[1];
            r.r = __funnelshift_r(w[1], w[2], 8);
            return r;
        };
        auto need = [&](int r) -> bool {  // strip cell row r is computed
            if (r < 0 || r >= nb) return false;
            return !c_flag || c_flag[L.citem0 + ((cy0 + r) / kCellTH) * L.ctx + tx] != 0u;
        };

        // ---- one pixel row (rows a / b / c = y - 1, y, y + 1): HOG votes with
        // weights wa, wb into the vote slots at float indices va[j] (cell row
        // band - 1) and va[j] + dB (cell row band); LBP counts into the lane's counters
        // (a row outside the cell grid votes with weight 0 and counts nothing)
        auto pixel_row = [&](const Row &ra, const Row &rb, const Row &rc, float wa, float wb, const uint32_t (&va)[4],
                             int dB, bool valid) {
            if (kHog) {
                const uint32_t P01 = __byte_perm(rb.r, rb.l, 0x5140), P23 = __byte_perm(rb.r, rb.l, 0x7362);
                const uint32_t Q01 = __byte_perm(rc.c, ra.c, 0x5140), Q23 = __byte_perm(rc.c, ra.c, 0x7362);
                const int gxb[4] = {dp2a_diff_lo(P01, (int)kMagicBits), dp2a_diff_hi(P01, (int)kMagicBits),
                                    dp2a_diff_lo(P23, (int)kMagicBits), dp2a_diff_hi(P23, (int)kMagicBits)};
                const int gyb[4] = {dp2a_diff_lo(Q01, (int)kMagicBits), dp2a_diff_hi(Q01, (int)kMagicBits),
                                    dp2a_diff_lo(Q23, (int)kMagicBits), dp2a_diff_hi(Q23, (int)kMagicBits)};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // half gradients, exact: (1.5 * 2^23 + g) / 2 - 0.75 * 2^23
                    const float hx = fmaf(__int_as_float(gxb[j]), 0.5f, -0.5f * kMagic);
                    const float hy = fmaf(__int_as_float(gyb[j]), 0.5f, -0.5f * kMagic);
                    const float hm = sqrt_approx(fmaf(hx, hx, hy * hy));  // magnitude / 2
                    const float ax = fabsf(hx), ay = fabsf(hy);
                    // phi = atan(ay / ax) = 45deg + atan(t), t = (ay - ax) / (ay + ax) in [-1, 1];
                    // ax + ay is 0 or >= 0.5: the 1e-30 only turns 0 / 0 into 0
                    const float t = (ay - ax) * rcp_approx(ax + ay + 1e-30f);
                    const float u = fmaf(-t, atan_bins2_poly(t * t), 4.5f);  // 2 (4.5 - phi) in bins, in [0, 9]
                    // theta = phi (same signs) or 9 - phi (opposite signs); the vote position is
                    // theta - 0.5, rounded below through theta - 1: p2 = 2 (theta - 1) = 7 -/+ u
                    const uint32_t flip = (__float_as_uint(hx) ^ __float_as_uint(hy)) & 0x80000000u;
                    const float p2 = 7.0f - __uint_as_float(__float_as_uint(u) ^ flip);
                    const float r2 = p2 + kMagic2;                // 2 round(theta - 1) + 3 * 2^23
                    const float e2 = p2 - (r2 - kMagic2);         // 2 (theta - 1 - round(...)), in [-1, 1]
                    const int oa = (int)((uint32_t)__float_as_int(r2) * 128u + va[j]);
                    float *v = Wm.R + oa;
                    float *w = Wm.R + (oa + dB);
                    // upper / lower bin: magnitude times (1 +/- e2) / 2
                    const float mo1 = fmaf(hm, e2, hm), mo0 = fmaf(-hm, e2, hm);
                    v[0] = fmaf(mo0, wa, v[0]);
                    v[kSCols] = fmaf(mo1, wa, v[kSCols]);
                    w[0] = fmaf(mo0, wb, w[0]);
                    w[kSCols] = fmaf(mo1, wb, w[kSCols]);
                }
            }
            if (kLbp) {
                const uint32_t clo = rb.c & ~kHi, cn7 = ~rb.c & kHi;
                const uint32_t code = (ge4(ra.l, clo, cn7) >> 7) | (ge4(ra.c, clo, cn7) >> 6) |
                                      (ge4(ra.r, clo, cn7) >> 5) | (ge4(rb.r, clo, cn7) >> 4) |
                                      (ge4(rc.r, clo, cn7) >> 3) | (ge4(rc.c, clo, cn7) >> 2) |
                                      (ge4(rc.l, clo, cn7) >> 1) | ge4(rb.l, clo, cn7);
                if (core && valid) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const uint2 e = S.map[(code >> (8 * j)) & 0xffu];
                        atomicAdd(&Wm.cnt[(int)e.x + lane], e.y);
                    }
                }
            }
        };

        // ---- LBP of cell row r = band - 1 is final after the band's first 4 rows:
        // a cell's counts are its two lanes' counters; write them, clear
        auto emit_lbp = [&](int band, bool walked) {
            __syncwarp();  // every lane's counts of row r are in
            const int r = band - 1;
            const int c = lane & 15, half = lane >> 4;
            if (walked && need(r) && c < kCellTW && cx0 + c < Wc) {
                const int64_t pl = atlas.lbp_plane;
                // bin planes 32 half .. 32 half + 31 of cell c
                uint8_t *dst = atlas.lbp + (int64_t)(L.cell_row + cy0 + r) * atlas.pitch + cx0 + c + 32 * half * pl;
                const uint32_t *cw = Wm.cnt + half * 8 * 32 + 2 * c + 1;
                const int nw = half ? kCntWords - 8 : 8;
#pragma unroll 1
                for (int i = 0; i < nw; ++i) {
                    const uint32_t val = cw[i * 32] + cw[i * 32 + 1];  // counts <= 32 each: no carry
                    dst[0] = (uint8_t)val;
                    dst[pl] = (uint8_t)(val >> 8);
                    dst[2 * pl] = (uint8_t)(val >> 16);
                    if (32 * half + 4 * i + 3 < kLbpBins) dst[3 * pl] = (uint8_t)(val >> 24);
                    dst += 4 * pl;
                }
            }
            __syncwarp();  // read before cleared
#pragma unroll
            for (int wd = 0; wd < kCntWords; ++wd) Wm.cnt[wd * 32 + lane] = 0u;
        };

        // ---- HOG of cell row r = band - 1 is final: write it, recycle its slots
        auto emit = [&](int band, bool walked) {
            const int ringA = (band + 1) & 1, ringB = band & 1;
            const int r = band - 1;
            const bool out = walked && need(r);
            const int64_t rowoff = (int64_t)(L.cell_row + cy0 + r) * atlas.pitch;
            if (kHog) {
                float *Ra = Wm.R + ringA * kRingStride + 4 * lane;
                if (walked && band == 0 && cy0 == 0) {
                    // top of the level: the rows above cell row 0 vote into row 0
                    float *Rb = Wm.R + ringB * kRingStride + 4 * lane;
#pragma unroll
                    for (int s = 0; s < kSlots; ++s) {
                        float4 a = *reinterpret_cast<float4 *>(Ra + s * kSCols);
                        float4 &b = *reinterpret_cast<float4 *>(Rb + s * kSCols);
                        b.x += a.x;
                        b.y += a.y;
                        b.z += a.z;
                        b.w += a.w;
                    }
                }
                if (out) {
                    if (band == nb && cy0 + nb == Hc) {
                        // bottom of the level: the rows below the last cell row vote into it
                        const float *Rb = Wm.R + ringB * kRingStride + 4 * lane;
#pragma unroll
                        for (int s = 0; s < kSlots; ++s) {
                            float4 &a = *reinterpret_cast<float4 *>(Ra + s * kSCols);
                            const float4 b = *reinterpret_cast<const float4 *>(Rb + s * kSCols);
                            a.x += b.x;
                            a.y += b.y;
                            a.z += b.z;
                            a.w += b.w;
                        }
                    }
                    const bool st = (lane & 1) && lane <= 2 * kCellTW - 1 && cx0 + ((lane - 1) >> 1) < Wc;
                    float *dst = atlas.hog + rowoff + cx0 + ((lane - 1) >> 1);
#pragma unroll
                    for (int h = 0; h < kHogBins; ++h) {
                        // bin h is slot h + 1; bin 0 also slot 10, bin 8 also slot 0
                        float4 v = *reinterpret_cast<const float4 *>(Ra + (h + 1) * kSCols);
                        if (h == 0 || h == kHogBins - 1) {
                            const float4 u = *reinterpret_cast<const float4 *>(Ra + (h == 0 ? kSlots - 1 : 0) * kSCols);
                            v.x += u.x;
                            v.y += u.y;
                            v.z += u.z;
                            v.w += u.w;
                        }
                        float own = wo[0] * v.x;
                        own = fmaf(wo[1], v.y, own);
                        own = fmaf(wo[2], v.z, own);
                        own = fmaf(wo[3], v.w, own);
                        float nbv = wn[0] * v.x;
                        nbv = fmaf(wn[1], v.y, nbv);
                        nbv = fmaf(wn[2], v.z, nbv);
                        nbv = fmaf(wn[3], v.w, nbv);
                        // cell (t - 1) / 2 at odd lane t: own(t) + own(t + 1) + nb(t - 1) + nb(t + 2)
                        const float o_next = __shfl_down_sync(0xffffffffu, own, 1);
                        const float n_prev = __shfl_up_sync(0xffffffffu, nbv, 1);
                        const float n_next2 = __shfl_down_sync(0xffffffffu, nbv, 2);
                        const float tot = ((own + o_next) + n_prev) + n_next2;
                        if (st) dst[(int64_t)h * atlas.hog_plane] = tot;
                    }
                }
                // clear the slots of row r for row r + 2 (only this lane wrote them)
#pragma unroll
                for (int s = 0; s < kSlots; ++s)
                    *reinterpret_cast<float4 *>(Ra + s * kSCols) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };

        // ---- the walk: bands 0..nb. Rows arrive in pairs, the next pair loaded
        // while the current one is processed (across band boundaries too).
        uint32_t p0[3], p1[3];
        Row ra, rb;
        bool have = false;   // p0, p1 and ra, rb hold this band's first rows
        bool walked_prev = false;
#pragma unroll 1
        for (int band = 0; band <= nb; ++band) {
            const int yb = 8 * (cy0 + band) - 4;
            if (!(need(band - 1) || need(band))) {
                if (walked_prev) {  // recycle row band - 1's slots and counters
                    emit(band, false);
                    if (kLbp) emit_lbp(band, false);
                }
                have = false;
                walked_prev = false;
                continue;
            }
            if (!have) {
                uint32_t w[3];
                fetch(yb - 1, w);
                ra = mkrow(w);
                fetch(yb, w);
                rb = mkrow(w);
                fetch(yb + 1, p0);
                fetch(yb + 2, p1);
            }
            const bool pf = band + 1 <= nb && (need(band) || need(band + 1));
            const int ringA = (band + 1) & 1;
            const int dB = (ringA ? -1 : 1) * kRingStride;  // floats from row band - 1's slots to row band's
            uint32_t va[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) va[j] = vb[j] + (uint32_t)(ringA * kRingStride);
#pragma unroll 1
            for (int i = 0; i < 4; ++i) {
                const Row c0 = mkrow(p0), c1 = mkrow(p1);
                if (i < 3 || pf) {
                    fetch(yb + 3 + 2 * i, p0);
                    fetch(yb + 4 + 2 * i, p1);
                }
                // band rows k = 2i, 2i + 1: weights (7.5 - k) / 8 and (k + 0.5) / 8;
                // LBP cell row band - 1 for k < 4, band for k >= 4
                const float wa0 = (7.5f - 2 * i) * 0.125f;
                const int y = yb + 2 * i;
                const bool v0 = y >= 0 && y < gridH, v1 = y + 1 >= 0 && y + 1 < gridH;
                pixel_row(ra, rb, c0, v0 ? wa0 : 0.f, v0 ? 1.f - wa0 : 0.f, va, dB, v0);
                pixel_row(rb, c0, c1, v1 ? wa0 - 0.125f : 0.f, v1 ? 1.125f - wa0 : 0.f, va, dB, v1);
                ra = c0;
                rb = c1;
                if (kLbp && i == 1) emit_lbp(band, true);
            }
            emit(band, true);
            have = pf;
            walked_prev = true;
        }
        __syncwarp();  // the next strip reuses the warp's shared memory
    }
}

using StripFn = void (*)(const LevelDesc *, const uint8_t *, CellAtlas, const StripItem *, int, int *,
                         const uint8_t *, const uint32_t *);
const StripFn kStripFns[3] = {k_cells_warp<kFeatHog | kFeatLbp>, k_cells_warp<kFeatHog>,
                              k_cells_warp<kFeatLbp>};

int strip_fn_index(int feat) {
    if (feat == kFeatHog) return 1;
    if (feat == kFeatLbp) return 2;
    return 0;
}

}  // namespace

cudaError_t init_cells_warp() {
    for (int i = 0; i < 3; ++i) {
        const cudaError_t e =
            cudaFuncSetAttribute(kStripFns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(StripSmem));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_cells_warp(cudaStream_t s, const LevelDesc *d_levels, const uint8_t *pyr, CellAtlas atlas,
                              const StripItem *d_items, int n_items, int *d_queue, int sm_count,
                              const uint8_t *d_lbp_map, const uint32_t *c_flag, int feat) {
    if (n_items <= 0) return cudaSuccess;
    // resident CTAs: 4 per SM (shared memory); the warps share the strip queue. A
    // small plan gets one CTA per strip, so that its warps spread over the SMs.
    static_assert(kWarps * 4 == kStripWarpsPerSm, "resident warps per SM");
    const int grid = std::min(n_items, 4 * sm_count);
    kStripFns[strip_fn_index(feat)]<<<grid, kWarps * 32, sizeof(StripSmem), s>>>(d_levels, pyr, atlas, d_items,
                                                                                 n_items, d_queue, d_lbp_map, c_flag);
    return cudaGetLastError();
}

}  // namespace pd
