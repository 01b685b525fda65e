// K4 on the tensor cores -- block normalisation fused with the sliding-window
// linear SVM (Section 4.4, Algorithm 6; block features of Sections 4.2-4.3).
//
// score[wy][wx] = b + sum_{i<15} sum_{j<7} < f[wy+i][wx+j], w[i][j] >
// with f[by][bx] the 95-value block feature (36 L2-Hys HOG values of the 2x2
// cells, then the 59 L1-sqrt LBP values of their summed counts).
//
// Per block row r of a level this is one GEMM: P[bx][(i, j)] =
// < f[r][bx], w[i][j] > for all 105 template positions (M = blocks of the
// row, N = 105 padded to 112, K = 95 padded to 96). Window (wy, wx) then
// collects P_{wy+i}[wx+j][(i, j)] over its 15 x 7 positions: the j terms
// come from the 7 neighbouring blocks of one block row, the i terms from 15
// consecutive block rows. The GEMM runs on tcgen05 (bf16 operands, fp32
// accumulators in tensor memory); fp32 accuracy is kept by splitting both
// operands into bf16 high and low parts, x = xh + xl and w = wh + wl, and
// summing xh.wh + xl.wh + xh.wl (K = 3 x 96; the dropped xl.wl and the
// rounding of the low parts are below 2^-16 of |x w| per term).
//
// One persistent CTA per SM (8 warps) takes items from a queue: an item is a
// strip of up to 104 window columns and up to 64 window rows of one level.
// It walks the strip's block rows top to bottom:
//  * TMA (cp.async.bulk.tensor.3d) brings cell rows into a ring of four
//    slots: the 9 HOG planes (f32) and the 59 LBP count planes (u8) of the
//    strip's 112 + 16 cells; the LBP counts of a staged row are replaced in
//    place by the sums of horizontally adjacent cells.
//  * Producers: threads 0-127 build the HOG part of one A row each (36 cell
//    values, L2-Hys, bf16 split), threads 128-255 the LBP part (2 x 2 count
//    sum, L1-sqrt and its bf16 split from a 512-entry table). A row m holds
//    block wx0 + 26 (m / 32) + m % 32: every warp of 32 rows covers 26
//    windows and the 6 blocks to their right, so the j terms stay inside a
//    warp and move with shuffles.
//  * Thread 0 issues the 18 MMAs of the row (K-major, no-swizzle canonical
//    layouts in shared memory; D in one of two 128-column TMEM buffers) and
//    commits them to an mbarrier. The A operand is double buffered: the
//    producers build row r + 1 while row r's MMAs run.
//  * Epilogue of row r - 1 (all warps; warp w reads TMEM lanes 32 (w % 4)
//    and half w / 4 of the 105 columns): lane l sums P[l + j][(i, j)] over j
//    with shuffles and adds it to the running score of window row r - 1 - i.
//    Warps of half 0 carry i = 0..7, half 1 i = 8..14; a window row's partial
//    sum passes from half 0 to half 1 through shared memory, so every score
//    is b plus its terms in the fixed order (i, j) = (0,0), (0,1), ...: the
//    result does not depend on how the level is cut into items.
// Sparse path: a window is scored when every cell tile under it was
// computed; block rows that no such window needs are skipped, other windows
// get -inf. Waits are bounded (1 s): a wait that gives up sets the error
// word and the CTA drains its copies and MMAs, frees its tensor memory and
// leaves.
#include "pd_internal.h"

#include <cuda_bf16.h>

namespace pd {
namespace {

constexpr int kThreads = 256;
constexpr int kM = 128;               // A rows = TMEM lanes
constexpr int kN = 112;               // 105 template positions, padded
constexpr int kWinPerWarp = 26;
constexpr int kChunks = 24;           // 16-byte K chunks per operand row: 12 high + 12 low
constexpr int kSBO = kChunks * 128;   // bytes per 8-row group
constexpr int kHogX = 112;            // HOG cells per staged row (TMA box width)
constexpr int kLbpX = 128;            // LBP cells per staged row (box width, from a 16-cell boundary)
constexpr int kSlots = 4;
constexpr uint32_t kTmemCols = 256;   // two accumulator buffers of 128 columns
constexpr uint64_t kWaitNs = 1000000000ull;
static_assert(4 * kWinPerWarp == kTcStrip, "strip width");
static_assert(kWinPerWarp + kWinBW - 1 <= 32, "window blocks inside a warp");

struct Slot {
    float hog[kHogBins][kHogX];       // 4032 B
    uint8_t pad0[64];
    uint8_t lbp[kLbpBins][kLbpX];     // 7552 B
    uint8_t pad1[128];
};
static_assert(sizeof(Slot) % 128 == 0 && offsetof(Slot, lbp) % 128 == 0, "TMA destinations");

struct TcSmem {
    uint8_t a[2][16 * kSBO];          // A operands, double buffered
    uint8_t b[14 * kSBO];             // B operand: template high | low parts
    Slot slot[kSlots];                // staged cell rows
    uint32_t tab[512];                // sum of 4 cell counts -> bf16 high | low << 16 of sqrt(S / 256)
    float handoff[2][kM];             // window-row partial sums from half 0 to half 1
    uint32_t win_ok[kTcChunk][4];     // sparse: window of the strip is scored
    uint8_t row_ok[kTcChunk];         // sparse: window row holds a scored window
    uint8_t tflag[16][16];            // sparse: cell-tile flags of the item's region
    unsigned long long cbar[kSlots];  // cell row arrival
    unsigned long long mbar[2];       // MMA completion per accumulator buffer
    unsigned long long wbar;          // unused spare barrier slot
    uint32_t tmem;
    int item;
};
static_assert(offsetof(TcSmem, slot) % 128 == 0 && offsetof(TcSmem, b) % 1024 == 0, "alignment");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool bar_wait(unsigned long long *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    uint32_t ok = 0;
    const uint64_t t0 = global_ns();
    while (true) {
        asm volatile(
            "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok || global_ns() - t0 > kWaitNs) break;
    }
    return ok != 0;
}
__device__ __forceinline__ void tma_3d(void *dst, const CUtensorMap *map, unsigned long long *bar, int x, int y,
                                       int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// ---- tcgen05
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {  // K chunk stride 128 B, row group stride kSBO
    return (uint64_t)((saddr >> 4) & 0x3fff) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(kSBO >> 4) << 32) |
           (1ull << 46);
}
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);  // f32 D, bf16 A and B, K-major, N, M
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

#define PD_LD_X8(taddr, v, o)                                                                              \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"                 \
                 : "=f"(v[o + 0]), "=f"(v[o + 1]), "=f"(v[o + 2]), "=f"(v[o + 3]), "=f"(v[o + 4]),         \
                   "=f"(v[o + 5]), "=f"(v[o + 6]), "=f"(v[o + 7])                                           \
                 : "r"(taddr))
#define PD_LD_X16(taddr, v, o)                                                                             \
    asm volatile(                                                                                          \
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "  \
        "[%16];"                                                                                           \
        : "=f"(v[o + 0]), "=f"(v[o + 1]), "=f"(v[o + 2]), "=f"(v[o + 3]), "=f"(v[o + 4]), "=f"(v[o + 5]),   \
          "=f"(v[o + 6]), "=f"(v[o + 7]), "=f"(v[o + 8]), "=f"(v[o + 9]), "=f"(v[o + 10]), "=f"(v[o + 11]), \
          "=f"(v[o + 12]), "=f"(v[o + 13]), "=f"(v[o + 14]), "=f"(v[o + 15])                                \
        : "r"(taddr))

// bf16 high and low parts of two floats, packed (first float in the low half)
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    uint32_t h, l;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(b), "f"(a));
    const float ah = __uint_as_float(h << 16), bh = __uint_as_float(h & 0xffff0000u);
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(l) : "f"(b - bh), "f"(a - ah));
    hi = h;
    lo = l;
}
__device__ __forceinline__ void st_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1,%2,%3,%4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ void st_v2(uint32_t addr, uint32_t a, uint32_t b) {
    asm volatile("st.shared.v2.b32 [%0], {%1,%2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}

// HOG part of A row m (features 0..35): cells (r, c), (r, c+1), (r+1, c),
// (r+1, c+1) of slots s0 (row r) and s1 (row r + 1), L2-Hys.
__device__ __forceinline__ void build_hog(const Slot &s0, const Slot &s1, int c, bool valid, float clip,
                                          uint32_t row) {
    float v[36];
#pragma unroll
    for (int b = 0; b < kHogBins; ++b) {
        v[b] = s0.hog[b][c];
        v[9 + b] = s0.hog[b][c + 1];
        v[18 + b] = s1.hog[b][c];
        v[27 + b] = s1.hog[b][c + 1];
    }
    float ss = 0.f;
#pragma unroll
    for (int t = 0; t < 36; ++t) ss = fmaf(v[t], v[t], ss);
    const float i1 = 1.0f / sqrtf(ss + 1.0f);
    float s2 = 0.f;
#pragma unroll
    for (int t = 0; t < 36; ++t) {
        v[t] = fminf(v[t] * i1, clip);
        s2 = fmaf(v[t], v[t], s2);
    }
    const float i2 = 1.0f / sqrtf(s2 + 1e-6f);
    uint32_t hi[18], lo[18];
#pragma unroll
    for (int p = 0; p < 18; ++p) {
        const float a = valid ? v[2 * p] * i2 : 0.f, b = valid ? v[2 * p + 1] * i2 : 0.f;
        split2(a, b, hi[p], lo[p]);
    }
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) {
        st_v4(row + ch * 128, hi[4 * ch], hi[4 * ch + 1], hi[4 * ch + 2], hi[4 * ch + 3]);
        st_v4(row + (12 + ch) * 128, lo[4 * ch], lo[4 * ch + 1], lo[4 * ch + 2], lo[4 * ch + 3]);
    }
    st_v2(row + 4 * 128, hi[16], hi[17]);
    st_v2(row + 16 * 128, lo[16], lo[17]);
}

// LBP part of A row m (features 36..95): the staged rows hold sums of
// horizontally adjacent cells, so cells (r, c..c+1) + (r+1, c..c+1) are two
// loads; the table gives the bf16 split of sqrt(S / 256).
__device__ __forceinline__ void build_lbp(const Slot &s0, const Slot &s1, const uint32_t *tab, int c, bool valid,
                                          uint32_t row) {
    uint32_t e[60];
#pragma unroll
    for (int t = 0; t < kLbpBins; ++t) e[t] = valid ? tab[(uint32_t)s0.lbp[t][c] + (uint32_t)s1.lbp[t][c]] : 0u;
    e[59] = 0u;
    uint32_t hi[30], lo[30];
#pragma unroll
    for (int p = 0; p < 30; ++p) {
        hi[p] = __byte_perm(e[2 * p], e[2 * p + 1], 0x5410);
        lo[p] = __byte_perm(e[2 * p], e[2 * p + 1], 0x7632);
    }
    st_v2(row + 4 * 128 + 8, hi[0], hi[1]);
    st_v2(row + 16 * 128 + 8, lo[0], lo[1]);
#pragma unroll
    for (int ch = 5; ch < 12; ++ch) {
        const int p = 2 + 4 * (ch - 5);
        st_v4(row + ch * 128, hi[p], hi[p + 1], hi[p + 2], hi[p + 3]);
        st_v4(row + (12 + ch) * 128, lo[p], lo[p + 1], lo[p + 2], lo[p + 3]);
    }
}

// In place: LBP count c[t][x] -> c[t][x] + c[t][x + 1] (x < 127) of a
// staged row. One warp per plane row; counts are at most 64, and the 7-bit
// mask keeps bytes that hold no valid count from carrying into a neighbour.
__device__ __forceinline__ void pair_sums(Slot &s, int tid) {
    for (int w = tid; w < kLbpBins * 32; w += kThreads) {
        uint32_t *row = reinterpret_cast<uint32_t *>(s.lbp[w >> 5]);
        const int k = w & 31;
        const uint32_t x = row[k] & 0x7f7f7f7fu;
        const uint32_t y = k < 31 ? row[k + 1] & 0x7f7f7f7fu : 0u;
        __syncwarp();
        row[k] = x + __funnelshift_r(x, y, 8);
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    k_svm_tc(const __grid_constant__ CUtensorMap hog_map, const __grid_constant__ CUtensorMap lbp_map,
             const LevelDesc *__restrict__ levels, const TcItem *__restrict__ items, int n_items,
             int *__restrict__ queue, const float *__restrict__ wt, float bias, float clip,
             float *__restrict__ scores, const uint32_t *__restrict__ c_flag, unsigned *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (smem_u32(smem_raw) & 1023u) {  // operand and TMA alignment: never expected
        if (tid == 0) atomicOr(err, kErrTimeout);
        return;
    }
    if (tid == 0) {
        for (int s = 0; s < kSlots; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.cbar[s])));
        for (int s = 0; s < 2; ++s)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar[s])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // B operand: template position n = 7 i + j (rows), feature t (K); high
    // parts in chunks 0..11, low parts in chunks 12..23
    for (int e = tid; e < kN * 96; e += kThreads) {
        const int n = e / 96, t = e - 96 * (e / 96);
        const int i = n / kWinBW, j = n - kWinBW * (n / kWinBW);
        const float w = (n < kWinBH * kWinBW && t < kFeat) ? wt[((size_t)t * kWinBH + i) * kWPad + j] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(w);
        const __nv_bfloat16 l = __float2bfloat16_rn(w - __bfloat162float(h));
        const uint32_t off = (n >> 3) * kSBO + (t >> 3) * 128 + (n & 7) * 16 + (t & 7) * 2;
        *reinterpret_cast<__nv_bfloat16 *>(S.b + off) = h;
        *reinterpret_cast<__nv_bfloat16 *>(S.b + off + 12 * 128) = l;
    }
    for (int s = tid; s < 512; s += kThreads) {
        uint32_t e = 0u;
        if (s <= 256) {
            const float f = sqrtf((float)s * (1.0f / 256.0f));
            const __nv_bfloat16 h = __float2bfloat16_rn(f);
            const __nv_bfloat16 l = __float2bfloat16_rn(f - __bfloat162float(h));
            e = (uint32_t)__bfloat16_as_ushort(h) | ((uint32_t)__bfloat16_as_ushort(l) << 16);
        }
        S.tab[s] = e;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t a_base = smem_u32(S.a[0]), b_base = smem_u32(S.b);

    // CTA-uniform pipeline state
    uint32_t nrow = 0;      // block rows processed (A buffer, D buffer and MMA barrier phase)
    uint32_t ncell = 0;     // cell rows loaded (slot and its barrier phase)
    uint32_t issued = 0;    // thread 0: cell rows whose load was issued
    int fail = 0;           // warp-uniform: a wait of this warp gave up
    // bounded wait, decided for the whole warp (shuffles and tcgen05.ld below
    // need every lane)
    auto uwait = [&](unsigned long long *bar, uint32_t parity) -> bool {
        const bool ok = __all_sync(0xffffffffu, !fail && bar_wait(bar, parity));
        if (!ok) fail = 1;
        return ok;
    };

    const int q = warp & 3, half = warp >> 2;
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.f;

    for (;;) {
        if (tid == 0) S.item = atomicAdd(queue, 1);
        __syncthreads();
        const int item = S.item;
        if (item >= n_items) break;
        const TcItem it = items[item];
        const LevelDesc L = levels[it.level];
        const int wend = min(it.wx0 + kTcStrip, L.cols);
        const int nrows = it.wy1 - it.wy0;
        const bool sparse = c_flag != nullptr;
        const int xl = it.wx0 & ~15;   // LBP box origin (16-byte boundary)

        // ---- sparse: which windows of the item are scored
        if (sparse) {
            const int ty0 = it.wy0 / kCellTH, ty1 = (it.wy1 - 1 + kWinBH) / kCellTH;
            const int tx0 = it.wx0 / kCellTW, tx1 = (wend - 1 + kWinBW) / kCellTW;
            const int ntx = tx1 - tx0 + 1, nt = (ty1 - ty0 + 1) * ntx;
            for (int i = tid; i < nt; i += kThreads) {
                const int ty = ty0 + i / ntx, tx = tx0 + i % ntx;
                S.tflag[ty - ty0][tx - tx0] = c_flag[L.citem0 + ty * L.ctx + tx] != 0u;
            }
            __syncthreads();
            for (int row = warp; row < nrows; row += kThreads / 32) {
                const int wy = it.wy0 + row;
                const int a0 = wy / kCellTH - ty0, a1 = (wy + kWinBH) / kCellTH - ty0;
                uint32_t any = 0u;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int wx = it.wx0 + 32 * k + lane;
                    bool ok = wx < wend && 32 * k + lane < kTcStrip;
                    if (ok) {
                        const int c0 = wx / kCellTW - tx0, c1 = (wx + kWinBW) / kCellTW - tx0;
                        for (int a = a0; a <= a1; ++a)
                            for (int c = c0; c <= c1; ++c) ok = ok && S.tflag[a][c];
                    }
                    const uint32_t bits = __ballot_sync(0xffffffffu, ok);
                    if (lane == 0) S.win_ok[row][k] = bits;
                    any |= bits;
                }
                if (lane == 0) S.row_ok[row] = any != 0u;
                if (!any)  // no scored window in this row: it is never reached below
                    for (int wx = it.wx0 + lane; wx < wend; wx += 32)
                        scores[L.score_off + (int64_t)wy * L.cols + wx] = -INFINITY;
            }
            __syncthreads();
        }

        // ---- runs of block rows: [ra, rb]
        int r_next = it.wy0;
        const int r_last = it.wy1 - 1 + kWinBH - 1;
        while (r_next <= r_last) {
            int ra, rb;
            if (!sparse) {
                ra = it.wy0;
                rb = r_last;
            } else {
                int wy = max(r_next - (kWinBH - 1), it.wy0);
                while (wy < it.wy1 && !S.row_ok[wy - it.wy0]) ++wy;
                if (wy >= it.wy1) break;
                ra = wy;
                rb = wy + kWinBH - 1;
                for (int w2 = wy + 1; w2 < it.wy1 && w2 <= rb; ++w2)
                    if (S.row_ok[w2 - it.wy0]) rb = w2 + kWinBH - 1;
            }
            const int n_cell = rb - ra + 2;  // cell rows ra .. rb + 1
            auto slot_of = [&](int u) -> Slot & { return S.slot[(ncell + u) % kSlots]; };
            auto issue = [&](int u) {  // thread 0: load cell row ra + u
                const uint32_t idx = ncell + u;
                Slot &s = S.slot[idx % kSlots];
                unsigned long long *bar = &S.cbar[idx % kSlots];
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                             "r"((uint32_t)(sizeof(float) * kHogBins * kHogX + kLbpBins * kLbpX))
                             : "memory");
                tma_3d(&s.hog[0][0], &hog_map, bar, it.wx0, L.cell_row + ra + u, 0);
                tma_3d(&s.lbp[0][0], &lbp_map, bar, xl, L.cell_row + ra + u, 0);
                ++issued;
            };
            auto wait_cell = [&](int u) -> bool {
                const uint32_t idx = ncell + u;
                return uwait(&S.cbar[idx % kSlots], (idx / kSlots) & 1u);
            };
            if (tid == 0)
                for (int u = 0; u < min(kSlots, n_cell); ++u) issue(u);
            // the first two rows: arrival and pair sums
            for (int u = 0; u < 2; ++u)
                if (wait_cell(u)) pair_sums(slot_of(u), tid);
            if (__syncthreads_or(fail)) goto abort;

            for (int r = ra; r <= rb + 1; ++r) {
                const int u = r - ra;
                if (r <= rb) {
                    // pair sums of cell row r + 2 (first used by block row r + 1)
                    if (u + 2 < n_cell && wait_cell(u + 2)) pair_sums(slot_of(u + 2), tid);
                    // block features of row r -> A[nrow & 1]
                    if (!fail) {
                        const int m = tid & (kM - 1);
                        const int c = kWinPerWarp * (m >> 5) + (m & 31);
                        const bool valid = it.wx0 + c < L.Wc - 1;
                        const uint32_t row = a_base + (nrow & 1) * (16 * kSBO) + (m >> 3) * kSBO + (m & 7) * 16;
                        if (tid < kM)
                            build_hog(slot_of(u), slot_of(u + 1), c, valid, clip, row);
                        else
                            build_lbp(slot_of(u), slot_of(u + 1), S.tab, c + it.wx0 - xl, valid, row);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A -> tensor cores
                }
                if (__syncthreads_or(fail)) goto abort;
                if (r <= rb && tid == 0) {
                    tc_fence_after();
                    const uint32_t d = tmem + (nrow & 1) * 128;
                    const uint32_t a0 = a_base + (nrow & 1) * (16 * kSBO);
#pragma unroll
                    for (int s = 0; s < 6; ++s) umma(d, umma_desc(a0 + 256 * s), umma_desc(b_base + 256 * s), s > 0);
#pragma unroll
                    for (int s = 0; s < 6; ++s)
                        umma(d, umma_desc(a0 + 12 * 128 + 256 * s), umma_desc(b_base + 256 * s), 1);
#pragma unroll
                    for (int s = 0; s < 6; ++s)
                        umma(d, umma_desc(a0 + 256 * s), umma_desc(b_base + 12 * 128 + 256 * s), 1);
                    umma_commit(&S.mbar[nrow & 1]);
                    // cell row r is no longer read: its slot takes row r + 4
                    if (u + kSlots < n_cell) issue(u + kSlots);
                }
                // ---- epilogue of block row r - 1
                if (r > ra) {
                    const uint32_t k = nrow - 1;  // its index
                    const int rr = r - 1;
                    if (uwait(&S.mbar[k & 1], (k >> 1) & 1u)) {
                        tc_fence_after();
                        const uint32_t t0 = tmem + ((uint32_t)(32 * q) << 16) + (k & 1) * 128;
                        if (half == 0) {
                            float v[56];
                            PD_LD_X16(t0, v, 0);
                            PD_LD_X16(t0 + 16, v, 16);
                            PD_LD_X16(t0 + 32, v, 32);
                            PD_LD_X8(t0 + 48, v, 48);
                            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                            acc[0] = bias;
#pragma unroll
                            for (int i = 0; i < 8; ++i)
#pragma unroll
                                for (int j = 0; j < kWinBW; ++j) {
                                    const float x = v[kWinBW * i + j];
                                    acc[i] += j ? __shfl_down_sync(0xffffffffu, x, j) : x;
                                }
                            S.handoff[(rr - 7) & 1][32 * q + lane] = acc[7];
#pragma unroll
                            for (int i = 7; i > 0; --i) acc[i] = acc[i - 1];
                        } else {
                            float v[56];
                            PD_LD_X8(t0 + 56, v, 0);
                            PD_LD_X16(t0 + 64, v, 8);
                            PD_LD_X16(t0 + 80, v, 24);
                            PD_LD_X16(t0 + 96, v, 40);
                            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                            acc[0] = S.handoff[(rr - 8) & 1][32 * q + lane];
#pragma unroll
                            for (int i = 0; i < 7; ++i)
#pragma unroll
                                for (int j = 0; j < kWinBW; ++j) {
                                    const float x = v[kWinBW * i + j];
                                    acc[i] += j ? __shfl_down_sync(0xffffffffu, x, j) : x;
                                }
                            const int wy = rr - (kWinBH - 1);
                            const int wl = kWinPerWarp * q + lane;
                            const int wx = it.wx0 + wl;
                            if (wy >= it.wy0 && lane < kWinPerWarp && wx < wend) {
                                const bool ok = !sparse || ((S.win_ok[wy - it.wy0][wl >> 5] >> (wl & 31)) & 1u);
                                scores[L.score_off + (int64_t)wy * L.cols + wx] = ok ? acc[6] : -INFINITY;
                            }
#pragma unroll
                            for (int i = 6; i > 0; --i) acc[i] = acc[i - 1];
                        }
                        tc_fence_before();
                    }
                }
                if (r <= rb) ++nrow;
            }
            ncell += n_cell;
            if (__syncthreads_or(fail)) goto abort;
            r_next = rb + 1;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    return;

abort:
    // a wait gave up: drain this CTA's copies and MMAs (bounded), free the
    // tensor memory and leave
    if (tid == 0) {
        atomicOr(err, kErrTimeout);
        // the last load of each slot (earlier ones completed before their slot was reused)
        for (uint32_t idx = max(ncell, issued > kSlots ? issued - kSlots : 0u); idx < issued; ++idx)
            bar_wait(&S.cbar[idx % kSlots], (idx / kSlots) & 1u);
        if (nrow > 0) bar_wait(&S.mbar[(nrow - 1) & 1], ((nrow - 1) >> 1) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

#undef PD_LD_X8
#undef PD_LD_X16

}  // namespace

cudaError_t init_svm_tc() {
    return cudaFuncSetAttribute(k_svm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem));
}

int svm_tc_smem_bytes() { return (int)sizeof(TcSmem); }

cudaError_t launch_svm_tc(cudaStream_t s, const CUtensorMap &hog_map, const CUtensorMap &lbp_map,
                          const LevelDesc *d_levels, const TcItem *d_items, int n_items, int *d_queue, int grid,
                          const float *d_w, float bias, float clip, float *scores, const uint32_t *c_flag,
                          unsigned *d_err) {
    if (n_items <= 0) return cudaSuccess;
    grid = grid < n_items ? grid : n_items;
    k_svm_tc<<<grid, kThreads, sizeof(TcSmem), s>>>(hog_map, lbp_map, d_levels, d_items, n_items, d_queue, d_w,
                                                    bias, clip, scores, c_flag, d_err);
    return cudaGetLastError();
}

}  // namespace pd
