// K1 -- image pyramid (Section 4.4, pyramidal sliding window; Section 4.1 step 2).
//
// Every pyramid level is a fixed-point bilinear resample (11-bit weights) of
// the frame itself, not of the previous level (downsampled levels, and the
// optional upsampled ones placed before them). One CTA owns a 128x32 source
// tile of one frame: it stages the tile (plus a right halo of up to 32
// columns and one bottom row) in shared memory once and then writes, for
// every level of that frame, the output pixels it owns. The frame is read
// from HBM once for all levels, and each level pixel is written once.
//
// Ownership: output row y belongs to the tile row holding its top source row;
// output columns go in groups of 4 (one 32-bit store), and a group belongs to
// the tile column holding the top-left source sample of its first column. A
// group's other columns may reach into the halo (32 columns); levels whose
// groups would reach past it (downsampling by more than 10) use groups of 1
// column.
//
// The staged tile is rewritten as "quads": quad (r, c) holds the four taps
// I(r,c), I(r,c+1), I(r+1,c), I(r+1,c+1) of a source position in one 32-bit
// word, so one shared-memory load gives all taps of an output pixel. With
// the column weights packed as two 16-bit halves W = (2048-ax) | ax << 16,
// two dp2a instructions give the horizontal sums of both rows,
//   top = (2048-ax) I00 + ax I01,   bot = (2048-ax) I10 + ax I11,
// and out = (4 (2048-ay) top + 4 ay bot + 2^23) >> 24 is the Q11 rounding
//   ((2048-ay) top + ay bot + 2^21) >> 22
// scaled by 4 (exact: 4 (2^30 + 2^21) < 2^32), so the output byte is byte 3
// of the 32-bit sum and byte permutes pack four outputs into one store.
// The planner precomputes every column's packed weights and the index of its
// quad, per level (small tables, read through L1), so the inner loop is
// shared-memory loads, dp2a and multiply-adds.
// The level at scale 1 (the identity) is a 16-byte copy of the staged tile.
#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kThreads = 256;
constexpr int kTW = kResizeTW;                 // 128 source columns per tile
constexpr int kTH = kResizeTH;                 // 32 source rows per tile
constexpr int kTP = 176;                       // staged byte row pitch (>= kResizeBW + 8, 16-byte multiple)
constexpr int kQP = kResizeQP;                 // quad row pitch in words
constexpr int kML = PD_MAX_LEVELS;
constexpr int kStageIters = ((kTH + 1) * ((kResizeBW + 3) / 4) + kThreads - 1) / kThreads;  // staged words per thread
static_assert(kTP >= kResizeBW + 8 && kTP % 16 == 0, "staged row pitch");
static_assert(kQP > (kResizeBW - 2) + ((kResizeBW - 2) >> 5) && kQP % 32 == 1 && kQP <= 256, "quad row pitch");

// Dynamic shared memory layout (bytes).
constexpr int kOffTile = 0;
constexpr int kOffQuad = kOffTile + (kTH + 1) * kTP;
constexpr int kOffRng = kOffQuad + ((kTH * kQP * 4 + 15) & ~15);  // int4 per level: first group, groups, first row, rows
constexpr int kOffCnt = kOffRng + kML * 16;             // int per level: warp tasks (-1: the copied level)
constexpr int kOffPre = kOffCnt + kML * 4;              // int per level + 1: first task
constexpr int kOffMisc = kOffPre + (kML + 1) * 4;       // copied level, task counter
constexpr int kOffLvl = (kOffMisc + 16 + 15) & ~15;     // per level: the fields the task loop reads
constexpr int kSmemBytes = kOffLvl + kML * 32;
static_assert(kOffQuad % 16 == 0 && kOffRng % 16 == 0, "alignment");

// One output pixel: its quad (taps) at shared-memory byte address qa, packed
// column weights and scaled row weights; the output byte is byte 3.
__device__ __forceinline__ uint32_t q11_pixel(uint32_t qa, uint32_t wx, uint32_t wt, uint32_t wb) {
    uint32_t q;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(q) : "r"(qa));
    const uint32_t top = __dp2a_lo(wx, q, 0u);
    const uint32_t bot = __dp2a_hi(wx, q, 0u);
    return wt * top + wb * bot + (1u << 23);
}

// Bytes 3 of four sums -> one word (output bytes in column order).
__device__ __forceinline__ uint32_t pack4(uint32_t o0, uint32_t o1, uint32_t o2, uint32_t o3) {
    return __byte_perm(__byte_perm(o0, o1, 0x0073), __byte_perm(o2, o3, 0x0073), 0x5410);
}

// kCG column groups per warp task; the warp's lanes are kCG groups x kRS row slices.
template <int kCG>
__global__ void __launch_bounds__(kThreads, 6) k_resize(const FrameDesc *__restrict__ frames,
                                                        const LevelDesc *__restrict__ levels,
                                                        const int32_t *__restrict__ tabs,
                                                        uint8_t *__restrict__ pyr,
                                                        const ResizeItem *__restrict__ items) {
    constexpr int kRS = 32 / kCG;
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t *tile = smem + kOffTile;
    uint32_t *quad = reinterpret_cast<uint32_t *>(smem + kOffQuad);
    int4 *s_rng = reinterpret_cast<int4 *>(smem + kOffRng);
    int *s_cnt = reinterpret_cast<int *>(smem + kOffCnt);
    int *s_pre = reinterpret_cast<int *>(smem + kOffPre);
    int *s_misc = reinterpret_cast<int *>(smem + kOffMisc);
    // per level: {img_off lo, img_off hi, pitch, Wk}, {rgroup, xtab_off, xq_off, ytab_off}
    int4 *s_lvl = reinterpret_cast<int4 *>(smem + kOffLvl);

    const ResizeItem it = items[blockIdx.x];
    const FrameDesc fd = frames[it.frame];
    const int tid = threadIdx.x, lane = tid & 31;
    const int n = fd.n_levels;
    const int tcx = it.x0 / kTW, tcy = it.y0 / kTH;


    // Stage source rows y0 .. y0+32 (clamped to the frame), bytes [x0, x0 + bw)
    // with columns at or past the right edge replaced by the last one. Aligned
    // 32-bit loads, each holding at least one byte of the row, realigned by a
    // funnel shift (the frame may be read straight from pinned host memory).
    // The level set-up below runs while the loads are in flight.
    {
        const int bw = fd.rbw;
        const int nw = (bw + 3) >> 2;
        const int nvalid = min(bw, fd.W - it.x0);
        uint32_t w0[kStageIters], w1[kStageIters];
#pragma unroll
        for (int u = 0; u < kStageIters; ++u) {
            const int i = tid + u * kThreads;
            w0[u] = w1[u] = 0u;
            if (i < (kTH + 1) * nw) {
                const int r = i / nw, j = i - r * nw;
                const int y = min(it.y0 + r, fd.H - 1);
                const uintptr_t a = reinterpret_cast<uintptr_t>(fd.ptr + (size_t)y * fd.pitch + it.x0);
                const int m = (int)(a & 3);
                const uintptr_t last = a + nvalid - 1;
                const uintptr_t w0a = a - m + 4 * (uintptr_t)j;
                if (w0a <= last) w0[u] = *reinterpret_cast<const uint32_t *>(w0a);
                if (m && w0a + 4 <= last) w1[u] = *reinterpret_cast<const uint32_t *>(w0a + 4);
            }
        }
        // Per level: the groups and rows this tile owns, and whether the level is
        // the identity with 16-byte aligned rows (copied, not resampled).
        for (int k = tid; k < n; k += kThreads) {
            const LevelDesc &L = levels[fd.first_level + k];
            const int gs = __ldg(tabs + L.xbnd_off + tcx), ge = __ldg(tabs + L.xbnd_off + tcx + 1);
            const int rs = __ldg(tabs + L.ybnd_off + tcy), re = __ldg(tabs + L.ybnd_off + tcy + 1);
            const bool copy = L.Wk == fd.W && L.Hk == fd.H && L.img_pitch % 16 == 0 &&
                              ((reinterpret_cast<uintptr_t>(pyr + L.img_off)) & 15) == 0;
            const int ng = ge - gs, nr = re - rs;
            const bool work = !copy && ng > 0 && nr > 0;
            s_rng[k] = make_int4(gs, ng, rs, nr);
            s_lvl[2 * k] = make_int4((int)(uint32_t)(uint64_t)L.img_off, (int)((uint64_t)L.img_off >> 32),
                                     L.img_pitch, L.Wk);
            s_lvl[2 * k + 1] = make_int4(L.rgroup, L.xtab_off, L.xq_off, L.ytab_off);
            // warp tasks (-1 marks the copied level: a frame has at most one level of scale 1)
            s_cnt[k] = copy ? -1 : work ? (ng + kCG - 1) / kCG : 0;
        }
        if (tid == 0) s_misc[1] = 0;
#pragma unroll
        for (int u = 0; u < kStageIters; ++u) {
            const int i = tid + u * kThreads;
            if (i < (kTH + 1) * nw) {
                const int r = i / nw, j = i - r * nw;
                const int y = min(it.y0 + r, fd.H - 1);
                const uint8_t *p = fd.ptr + (size_t)y * fd.pitch + it.x0;
                const int m = (int)(reinterpret_cast<uintptr_t>(p) & 3);
                uint32_t w = __funnelshift_r(w0[u], w1[u], 8 * m);
                if (4 * j + 4 > nvalid) {
                    const uint32_t e = p[nvalid - 1];
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (4 * j + b >= nvalid) w = (w & ~(0xffu << (8 * b))) | (e << (8 * b));
                }
                *reinterpret_cast<uint32_t *>(tile + r * kTP + 4 * j) = w;
            }
        }
    }
    __syncthreads();

    // Warp 0: prefix sum of the levels' warp tasks (n <= 96 = 3 per lane), and
    // the copied level.
    if (tid < 32) {
        int u[3], su = 0, cp = -1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int k = 3 * tid + i;
            const int c = k < n ? s_cnt[k] : 0;
            if (c < 0) cp = k;
            u[i] = max(c, 0);
            su += u[i];
        }
        cp = __reduce_max_sync(0xffffffffu, cp);
        int iu = su;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, iu, o);
            if (tid >= o) iu += a;
        }
        int ru = iu - su;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int k = 3 * tid + i;
            if (k < n) s_pre[k] = ru;
            ru += u[i];
        }
        if (tid == 31) s_pre[n] = iu;
        if (tid == 0) s_misc[0] = cp;
    }

    // Quads: quad (r, c) = [I(r,c), I(r,c+1), I(r+1,c), I(r+1,c+1)] for c < bw - 1,
    // at word resize_quad_index(c) of quad row r (the skew spreads strided reads over banks).
    {
        const int nq4 = (fd.rbw - 1 + 3) >> 2;
        for (int i = tid; i < kTH * nq4; i += kThreads) {
            const int r = i / nq4, j = i - r * nq4;
            const uint8_t *t0 = tile + r * kTP + 4 * j;
            const uint32_t a0 = *reinterpret_cast<const uint32_t *>(t0);
            const uint32_t a1 = *reinterpret_cast<const uint32_t *>(t0 + 4);
            const uint32_t b0 = *reinterpret_cast<const uint32_t *>(t0 + kTP);
            const uint32_t b1 = *reinterpret_cast<const uint32_t *>(t0 + kTP + 4);
            uint32_t *q = quad + r * kQP + resize_quad_index(4 * j);
            q[0] = __byte_perm(a0, b0, 0x5410);
            q[1] = __byte_perm(a0, b0, 0x6521);
            q[2] = __byte_perm(a0, b0, 0x7632);
            q[3] = __byte_perm(__byte_perm(a0, a1, 0x0043), __byte_perm(b0, b1, 0x0043), 0x5410);
        }
    }
    __syncthreads();

    // The identity level: 16-byte copies of the staged rows.
    const int kc = s_misc[0];
    if (kc >= 0) {
        const LevelDesc &L = levels[fd.first_level + kc];
        const int r = tid >> 3, c = (tid & 7) * 16;
        const int y = it.y0 + r, x = it.x0 + c;
        if (y < L.Hk && x < L.Wk) {
            const uint4 v = *reinterpret_cast<const uint4 *>(tile + r * kTP + c);
            uint8_t *o = pyr + L.img_off + (size_t)y * L.img_pitch + x;
            if (x + 16 <= L.Wk) {
                *reinterpret_cast<uint4 *>(o) = v;
            } else {
                const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int b = 0; b < 16; ++b)
                    if (x + b < L.Wk) o[b] = (uint8_t)(wv[b >> 2] >> (8 * (b & 3)));
            }
        }
    }
    __syncthreads();

    // Every other level: warp tasks of kCG column groups x all the tile's rows
    // of the level, taken from a shared counter. Lane = (row slice j, group c):
    // it keeps its group's weights and quad addresses in registers and walks
    // rows j, j + 4, ... (consecutive groups of a row store 32 contiguous bytes).
    const int total = s_pre[n];
    const uint32_t quad_base =
        (uint32_t)__cvta_generic_to_shared(quad) - (uint32_t)(it.y0 * kQP * 4);
    const int c = lane & (kCG - 1), j = lane / kCG;
    int k = -1;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(&s_misc[1], 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= total) break;
        while (t >= s_pre[k + 1]) ++k;
        const int4 rg = s_rng[k];
        const int g = (t - s_pre[k]) * kCG + c;
        if (g < rg.y) {
        const int4 la = s_lvl[2 * k], lb = s_lvl[2 * k + 1];
        const int64_t img_off = (int64_t)(((uint64_t)(uint32_t)la.y << 32) | (uint32_t)la.x);
        const int gg = rg.x + g;
        const int4 wx = __ldg(reinterpret_cast<const int4 *>(tabs + lb.y) + gg);
        const uint32_t qo = (uint32_t)__ldg(tabs + lb.z + gg);
        const int G = lb.x, Wk = la.w, pitch = la.z;
        const int x = G * gg;
        const int y0 = rg.z + j, re = rg.z + rg.w;
        const int nrow = y0 < re ? (re - y0 + kRS - 1) / kRS : 0;
        const int2 *yp = reinterpret_cast<const int2 *>(tabs + lb.w) + y0;
        uint8_t *op = pyr + img_off + x + (size_t)y0 * pitch;
        const size_t ostep = (size_t)kRS * pitch;
        if (G == 4) {
            const uint32_t a0 = quad_base + 4u * (qo & 255u), a1 = quad_base + 4u * ((qo >> 8) & 255u);
            const uint32_t a2 = quad_base + 4u * ((qo >> 16) & 255u), a3 = quad_base + 4u * (qo >> 24);
            // row entry: byte offset of the top source row's quad row, packed scaled row weights
            auto px4 = [&](int2 e, uint32_t &o0, uint32_t &o1, uint32_t &o2, uint32_t &o3) {
                const uint32_t ro = (uint32_t)e.x;
                const uint32_t wt = (uint32_t)e.y & 0xffffu, wb = (uint32_t)e.y >> 16;
                o0 = q11_pixel(a0 + ro, (uint32_t)wx.x, wt, wb);
                o1 = q11_pixel(a1 + ro, (uint32_t)wx.y, wt, wb);
                o2 = q11_pixel(a2 + ro, (uint32_t)wx.z, wt, wb);
                o3 = q11_pixel(a3 + ro, (uint32_t)wx.w, wt, wb);
            };
            if (x + 4 <= Wk && ((reinterpret_cast<uintptr_t>(pyr + img_off) | (uintptr_t)pitch) & 3) == 0) {
#pragma unroll 2
                for (int i = 0; i < nrow; ++i, yp += kRS, op += ostep) {
                    uint32_t o0, o1, o2, o3;
                    px4(__ldg(yp), o0, o1, o2, o3);
                    *reinterpret_cast<uint32_t *>(op) = pack4(o0, o1, o2, o3);
                }
            } else {
                for (int i = 0; i < nrow; ++i, yp += kRS, op += ostep) {
                    uint32_t ov[4];
                    px4(__ldg(yp), ov[0], ov[1], ov[2], ov[3]);
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (x + b < Wk) op[b] = (uint8_t)(ov[b] >> 24);
                }
            }
        } else {
            const uint32_t a0 = quad_base + 4u * (qo & 255u);
            for (int i = 0; i < nrow; ++i, yp += kRS, op += ostep) {
                const int2 e = __ldg(yp);
                *op = (uint8_t)(q11_pixel(a0 + (uint32_t)e.x, (uint32_t)wx.x, (uint32_t)e.y & 0xffffu,
                                          (uint32_t)e.y >> 16) >> 24);
            }
        }
        }
    }
}

}  // namespace

cudaError_t init_resize() {
    cudaError_t e = cudaFuncSetAttribute(k_resize<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resize<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_resize<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    return e;
}

cudaError_t launch_resize(cudaStream_t s, const FrameDesc *d_frames, const LevelDesc *d_levels,
                          const int32_t *d_tabs, uint8_t *pyr, const ResizeItem *d_items,
                          int n_items, int k1_groups) {
    if (n_items <= 0) return cudaSuccess;
    if (k1_groups == 4)
        k_resize<4><<<n_items, kThreads, kSmemBytes, s>>>(d_frames, d_levels, d_tabs, pyr, d_items);
    else if (k1_groups == 16)
        k_resize<16><<<n_items, kThreads, kSmemBytes, s>>>(d_frames, d_levels, d_tabs, pyr, d_items);
    else
        k_resize<8><<<n_items, kThreads, kSmemBytes, s>>>(d_frames, d_levels, d_tabs, pyr, d_items);
    return cudaGetLastError();
}

}  // namespace pd
