// K1 -- image pyramid (Section 4.4, pyramidal sliding window; Section 4.1 step 2).
//
// Every pyramid level is a fixed-point bilinear resample (11-bit weights) of
// the frame itself, not of the previous level (downsampled levels, and the
// optional upsampled ones placed before them). One CTA owns a 128x32 source
// tile of one frame: it stages the tile (+1 pixel of right/bottom halo) in
// shared memory once and then writes, for every level of that frame, the
// output pixels whose top-left source sample falls inside the tile. The
// frame is therefore read from HBM exactly once for all levels, and each
// level pixel is written exactly once.
//
// Per output coordinate the host planner precomputes the Q11 source index
// and weight (packed as x0 << 11 | a), so the kernel does only integer
// multiply-adds:  out = ((2048-ay)*((2048-ax)*I00 + ax*I01)
//                        + ay*((2048-ax)*I10 + ax*I11) + 2^21) >> 22.
#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kThreads = 256;
constexpr int kTileW = kResizeTW;       // 128
constexpr int kTileH = kResizeTH;       // 32
constexpr int kSmemW = kTileW + 4;      // 129 used, padded
constexpr int kSmemH = kTileH + 1;      // 33

__global__ void __launch_bounds__(kThreads) k_resize(const FrameDesc *__restrict__ frames,
                                                     const LevelDesc *__restrict__ levels,
                                                     const int32_t *__restrict__ tabs,
                                                     uint8_t *__restrict__ pyr,
                                                     const ResizeItem *__restrict__ items) {
    __shared__ uint8_t tile[kSmemH][kSmemW];
    __shared__ int4 ranges[PD_MAX_LEVELS];  // xs, xe, ys, ye per level

    const ResizeItem it = items[blockIdx.x];
    const FrameDesc fd = frames[it.frame];
    const int tid = threadIdx.x;

    // Stage the source tile [x0, x0+129) x [y0, y0+33) clamped to the frame
    // (independent loads, unrolled so that many are in flight: the frame may
    // be read straight from pinned host memory).
#pragma unroll 6
    for (int i = tid; i < kSmemH * (kTileW + 1); i += kThreads) {
        int r = i / (kTileW + 1), c = i - r * (kTileW + 1);
        int y = min(it.y0 + r, fd.H - 1), x = min(it.x0 + c, fd.W - 1);
        tile[r][c] = fd.ptr[(size_t)y * fd.pitch + x];
    }
    // Output ranges of every level (one thread per level), from the
    // planner's per-tile boundary tables.
    for (int k = tid; k < fd.n_levels; k += kThreads) {
        const LevelDesc L = levels[fd.first_level + k];
        const int tx = it.x0 / kTileW, ty = it.y0 / kTileH;
        int4 r;
        r.x = __ldg(tabs + L.xbnd_off + tx);
        r.y = __ldg(tabs + L.xbnd_off + tx + 1);
        r.z = __ldg(tabs + L.ybnd_off + ty);
        r.w = __ldg(tabs + L.ybnd_off + ty + 1);
        ranges[k] = r;
    }
    __syncthreads();

    // two adjacent output columns per thread (they share the row lookups and
    // the address work): 64 column pairs x 4 rows per pass
    const int tx = tid & 63, ty = tid >> 6;
    for (int k = 0; k < fd.n_levels; ++k) {
        const int4 r = ranges[k];
        // (an upsampled level has more than 128 output columns per tile: passes of 128)
        for (int x = r.x + 2 * tx; x < r.y; x += 128) {
            const bool two = x + 1 < r.y;
            const LevelDesc L = levels[fd.first_level + k];
            const int32_t ex0 = __ldg(tabs + L.xtab_off + x);
            const int32_t ex1 = two ? __ldg(tabs + L.xtab_off + x + 1) : ex0;
            const int a0 = (ex0 >> 11) - it.x0, ax0 = ex0 & 2047;
            const int b0 = min((ex0 >> 11) + 1, fd.W - 1) - it.x0;
            const int a1 = (ex1 >> 11) - it.x0, ax1 = ex1 & 2047;
            const int b1 = min((ex1 >> 11) + 1, fd.W - 1) - it.x0;
            uint8_t *out = pyr + L.img_off + x;
            for (int y = r.z + ty; y < r.w; y += 4) {
                const int32_t ey = __ldg(tabs + L.ytab_off + y);
                const int sy0 = (ey >> 11) - it.y0, ay = ey & 2047;
                const int sy1 = min((ey >> 11) + 1, fd.H - 1) - it.y0;
                const uint8_t *t0 = tile[sy0], *t1 = tile[sy1];
                const int top0 = (2048 - ax0) * t0[a0] + ax0 * t0[b0];
                const int bot0 = (2048 - ax0) * t1[a0] + ax0 * t1[b0];
                const int top1 = (2048 - ax1) * t0[a1] + ax1 * t0[b1];
                const int bot1 = (2048 - ax1) * t1[a1] + ax1 * t1[b1];
                uint8_t *o = out + (size_t)y * L.img_pitch;
                o[0] = (uint8_t)(((2048 - ay) * top0 + ay * bot0 + (1 << 21)) >> 22);
                if (two) o[1] = (uint8_t)(((2048 - ay) * top1 + ay * bot1 + (1 << 21)) >> 22);
            }
        }
    }
}

}  // namespace

cudaError_t launch_resize(cudaStream_t s, const FrameDesc *d_frames, const LevelDesc *d_levels,
                          const int32_t *d_tabs, uint8_t *pyr, const ResizeItem *d_items,
                          int n_items) {
    if (n_items <= 0) return cudaSuccess;
    k_resize<<<n_items, kThreads, 0, s>>>(d_frames, d_levels, d_tabs, pyr, d_items);
    return cudaGetLastError();
}

}  // namespace pd
