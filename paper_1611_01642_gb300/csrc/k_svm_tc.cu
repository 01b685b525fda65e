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
// One persistent CTA per SM takes items from a queue: an item is a strip of
// up to 104 window columns and up to 64 window rows of one level, walked one
// block row at a time by a warp-specialised pipeline (mbarriers between the
// roles, bounded waits):
//  * 8 producer warps: first all of them replace a staged row's LBP counts
//    by sums of horizontally adjacent cells (in place); then they write the
//    A operand straight into tensor memory (tcgen05.st: row m = lane m, two
//    bf16 per column), row m holding block wx0 + 26 (m / 32) + m % 32: warps
//    0-3 the 36 values of its 2x2 HOG cells (L2-Hys, bf16 split) and LBP
//    bins 0..9, warps 4-7 LBP bins 10..58 (the 2 x 2 count sums, L1-sqrt
//    and its bf16 split from a 512-entry table; the split balances the two
//    groups' work per row). Every group of 32 rows
//    covers 26 windows and the 6 blocks to their right, so the j terms of a
//    window stay inside one warp of the epilogue;
//  * one thread (lane 0 of the first epilogue warp, between its epilogue
//    rows) issues the TMA (cp.async.bulk.tensor.3d) of cell rows into a ring
//    of four slots (the 9 HOG planes, f32, and the 59 LBP count planes, u8,
//    of the strip's 112 + 16 cells) and the 18 MMAs of every block row (A in
//    tensor memory, the template's B operand K-major no-swizzle canonical in
//    shared memory, D in one of two 128-column TMEM buffers), committed to
//    the A-free and D-full barriers;
//  * 4 epilogue warps (warp e reads TMEM lanes 32 e .. 32 e + 31): lane l adds
//    P[l + j][(i, j)] (a shuffle by j) to the running score of window row
//    r - i, for all 105 positions, in the fixed order (i, j) = (0,0), (0,1),
//    ..., so every score is b plus its terms in one order whatever the item
//    cut; window row r - 14 is complete and stored.
// The A operand (two 96-column TMEM stages) and the accumulators are double
// buffered, so the producers build row r + 1 and the epilogue reads row
// r - 1 while row r's MMAs run.
// Per-block HOG (Algorithm 5 read per block): each staged cell row holds 36
// HOG planes, the cell's 4 block-restricted histograms (plane 9 q + bin, q =
// its place in the block); a block takes q = 0, 1 from row r and q = 2, 3
// from row r + 1, and nothing else changes.
// Sparse path: a window is scored when every cell tile under it was
// computed; block rows that no such window needs are skipped, other windows
// get -inf. A wait that gives up (1 s) sets the error word and a CTA flag
// that ends every role's waits; the CTA then drains its copies and MMAs,
// frees its tensor memory and leaves.
#include "pd_internal.h"

#include <cuda_bf16.h>

namespace pd {
namespace {

constexpr int kWarps = 12;            // 4 HOG, 4 LBP, 4 epilogue (one thread of which also issues)
constexpr int kProducers = 8;         // producer warps
constexpr int kThreads = 32 * kWarps;
constexpr int kM = 128;               // A rows = TMEM lanes
constexpr int kN = 112;               // 105 template positions, padded
constexpr int kWinPerWarp = 26;
constexpr int kChunks = 24;           // 16-byte K chunks per operand row: 12 high + 12 low
constexpr int kSBO = kChunks * 128;   // bytes per 8-row group
constexpr int kHogX = 112;            // HOG cells per staged row (TMA box width)
constexpr int kLbpX = 128;            // LBP cells per staged row (box width, from a 16-cell boundary)
constexpr int kSlots = 4;
constexpr uint32_t kTmemCols = 512;   // two accumulator buffers of 128 columns, two A stages of 96
constexpr uint32_t kTmemA = 256;      // first A stage column (bf16 pairs: high parts 0..47, low 48..95)
constexpr uint64_t kWaitNs = 1000000000ull;
constexpr int kProducerBarrier = 1;   // named barrier of the producer warps
constexpr int kHogLbpPairs = 5;       // LBP bin pairs built by the HOG warps (the LBP warps take the rest)
static_assert(4 * kWinPerWarp == kTcStrip, "strip width");
static_assert(kWinPerWarp + kWinBW - 1 <= 32, "window blocks inside a warp");

template <int HP>  // HOG planes per cell row: 9, or 36 for per-block HOG
struct SlotT {
    static constexpr int kPlanes = HP;
    float hog[HP][kHogX];                       // 4032 B (16128 B per-block)
    alignas(128) uint8_t lbp[kLbpBins][kLbpX];  // 7552 B
    uint8_t pad1[128];
};
static_assert(sizeof(SlotT<9>) == 11776 && offsetof(SlotT<9>, lbp) == 4096, "slot layout");
static_assert(sizeof(SlotT<36>) % 128 == 0 && offsetof(SlotT<36>, lbp) % 128 == 0, "TMA destinations");

template <int HP>
struct TcSmemT {
    uint8_t b[14 * kSBO];             // B operand: template high | low parts
    SlotT<HP> slot[kSlots];           // staged cell rows
    uint32_t tab[512];                // sum of 4 cell counts -> bf16 high | low << 16 of sqrt(S / 256)
    uint32_t win_ok[kTcChunk][4];     // sparse: window of the strip is scored
    uint8_t row_ok[kTcChunk];         // sparse: window row holds a scored window
    uint8_t tflag[16][16];            // sparse: cell-tile flags of the item's region
    unsigned long long cfull[kSlots];   // cell row arrived (TMA transaction count)
    unsigned long long cempty[kSlots];  // cell row no longer read (8 producer warps)
    unsigned long long afull[2];        // A operand written (8 producer warps)
    unsigned long long aempty[2];       // A operand read by the MMAs (commit)
    unsigned long long dfull[2];        // accumulators written (commit)
    unsigned long long dempty[2];       // accumulators read (4 epilogue warps)
    uint32_t tmem;
    int item;
    volatile int failed;
};
static_assert(offsetof(TcSmemT<9>, slot) % 128 == 0 && offsetof(TcSmemT<36>, slot) % 128 == 0, "alignment");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool try_wait(unsigned long long *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity`; gives up after 1 s (and marks the CTA
// failed) or as soon as another role has marked it failed.
template <class SM>
__device__ __forceinline__ bool bar_wait(SM &S, unsigned long long *bar, uint32_t parity, unsigned *err) {
    if (try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!S.failed) {
        if (try_wait(bar, parity)) return true;
        if (global_ns() - t0 > kWaitNs) {
            S.failed = 1;
            atomicOr(err, kErrTimeout);
            break;
        }
    }
    return false;
}
// Drain wait (after a failure): bounded, ignores the failed flag.
__device__ __forceinline__ void drain_wait(unsigned long long *bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    while (!try_wait(bar, parity) && global_ns() - t0 < kWaitNs) {
    }
}
__device__ __forceinline__ void arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
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
// A from tensor memory (lane m = row m, K packed two bf16 per column)
__device__ __forceinline__ void umma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d),
        "r"(a_tmem), "l"(b), "r"(kIdesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

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
// this thread's TMEM lane: 4, 8 or 16 consecutive 32-bit columns from taddr
__device__ __forceinline__ void tst1(uint32_t t, const uint32_t *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(t), "r"(v[0]) : "memory");
}
__device__ __forceinline__ void tst2(uint32_t t, const uint32_t *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1,%2};" ::"r"(t), "r"(v[0]), "r"(v[1]) : "memory");
}
__device__ __forceinline__ void tst4(uint32_t t, const uint32_t *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};" ::"r"(t), "r"(v[0]), "r"(v[1]),
                 "r"(v[2]), "r"(v[3])
                 : "memory");
}
__device__ __forceinline__ void tst8(uint32_t t, const uint32_t *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(t), "r"(v[0]),
                 "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
                 : "memory");
}
__device__ __forceinline__ void tst16(uint32_t t, const uint32_t *v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(t),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

// LBP features of A row m for bins [T0, T0 + 2 NP) (bin 59 is the zero pad):
// the staged rows hold sums of horizontally adjacent cells, so cells
// (r, c..c+1) + (r+1, c..c+1) are two loads; the table gives the bf16 split
// of sqrt(S / 256), packed two bins per word.
template <int T0, int NP, class Slot>
__device__ __forceinline__ void lbp_pairs(const Slot &s0, const Slot &s1, const uint32_t *tab, int c, uint32_t *hi,
                                          uint32_t *lo) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int t = T0 + 2 * p;
        const uint32_t e0 = tab[(uint32_t)s0.lbp[t][c] + (uint32_t)s1.lbp[t][c]];
        const uint32_t e1 = t + 1 < kLbpBins ? tab[(uint32_t)s0.lbp[t + 1][c] + (uint32_t)s1.lbp[t + 1][c]] : 0u;
        hi[p] = __byte_perm(e0, e1, 0x5410);
        lo[p] = __byte_perm(e0, e1, 0x7632);
    }
}

// Features 0..45 of A row m into its TMEM lane (columns a + f / 2 for the high
// parts, a + 48 + f / 2 for the low parts): the 36 HOG values of its cells
// (r, c), (r, c+1), (r+1, c), (r+1, c+1) (slots s0 = row r, s1 = row r + 1) in
// the template's order (cells TL, TR, BL, BR, 9 bins each), L2-Hys, bf16
// split; then LBP bins 0..9 (LBP column cl).
template <class Slot>
__device__ __forceinline__ void build_hog(const Slot &s0, const Slot &s1, const uint32_t *tab, int c, int cl,
                                          float clip, uint32_t a) {
    constexpr int pq = Slot::kPlanes == 36 ? kHogBins : 0;  // per-block: plane set of the cell's place
    float v[36];
#pragma unroll
    for (int b = 0; b < kHogBins; ++b) {
        v[b] = s0.hog[b][c];
        v[9 + b] = s0.hog[pq + b][c + 1];
        v[18 + b] = s1.hog[2 * pq + b][c];
        v[27 + b] = s1.hog[3 * pq + b][c + 1];
    }
    // sums of squares in four interleaved partial sums (independent chains)
    float q[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int t = 0; t < 36; ++t) q[t & 3] = fmaf(v[t], v[t], q[t & 3]);
    const float i1 = rsqrtf((q[0] + q[1]) + (q[2] + q[3]) + 1.0f);
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = 0.f;
#pragma unroll
    for (int t = 0; t < 36; ++t) {
        v[t] = fminf(v[t] * i1, clip);
        q[t & 3] = fmaf(v[t], v[t], q[t & 3]);
    }
    const float i2 = rsqrtf((q[0] + q[1]) + (q[2] + q[3]) + 1e-6f);
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int p = 0; p < 16; ++p) split2(v[2 * p] * i2, v[2 * p + 1] * i2, hi[p], lo[p]);
    tst16(a, hi);        // features 0..31
    tst16(a + 48, lo);
    // features 32..35 (HOG) and the first kHogLbpPairs LBP bin pairs
    split2(v[32] * i2, v[33] * i2, hi[0], lo[0]);
    split2(v[34] * i2, v[35] * i2, hi[1], lo[1]);
    static_assert(kHogLbpPairs == 5, "TMEM column split");
    lbp_pairs<0, kHogLbpPairs>(s0, s1, tab, cl, hi + 2, lo + 2);  // columns 16..22
    tst4(a + 16, hi);
    tst2(a + 20, hi + 4);
    tst1(a + 22, hi + 6);
    tst4(a + 64, lo);
    tst2(a + 68, lo + 4);
    tst1(a + 70, lo + 6);
}

// Features 46..95 of A row m (LBP bins 10..58 and the zero pad): columns
// a + 23 .. a + 47 and a + 71 .. a + 95.
template <class Slot>
__device__ __forceinline__ void build_lbp(const Slot &s0, const Slot &s1, const uint32_t *tab, int cl, uint32_t a) {
    uint32_t hi[25], lo[25];
    lbp_pairs<2 * kHogLbpPairs, 30 - kHogLbpPairs>(s0, s1, tab, cl, hi, lo);  // bins 10..59: columns 23..47
    tst1(a + 23, hi);
    tst8(a + 24, hi + 1);
    tst16(a + 32, hi + 9);
    tst1(a + 71, lo);
    tst8(a + 72, lo + 1);
    tst16(a + 80, lo + 9);
}

// In place, by the 256 producer threads: LBP count c[t][x] -> c[t][x] +
// c[t][x + 1] (x < 127) of a staged row. A warp takes whole plane rows (word
// k of the row per lane), all its loads first; counts are at most 64, and
// the 7-bit mask keeps bytes that hold no valid count from carrying into a
// neighbour.
constexpr int kPairIters = (kLbpBins * 32 + 255) / 256;  // 8
template <class Slot>
__device__ __forceinline__ void pair_sums(Slot &s, int pt) {
    uint32_t x[kPairIters], y[kPairIters];
    const int k = pt & 31;
#pragma unroll
    for (int n = 0; n < kPairIters; ++n) {
        const int w = pt + 256 * n;
        if (w < kLbpBins * 32) {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(s.lbp[w >> 5]);
            x[n] = row[k] & 0x7f7f7f7fu;
            y[n] = k < 31 ? row[k + 1] & 0x7f7f7f7fu : 0u;
        }
    }
    __syncwarp();
#pragma unroll
    for (int n = 0; n < kPairIters; ++n) {
        const int w = pt + 256 * n;
        if (w < kLbpBins * 32) reinterpret_cast<uint32_t *>(s.lbp[w >> 5])[k] = x[n] + __funnelshift_r(x[n], y[n], 8);
    }
}

// named barrier of the producer warps
__device__ __forceinline__ void producer_barrier() {
    asm volatile("bar.sync %0, %1;" ::"n"(kProducerBarrier), "n"(32 * kProducers) : "memory");
}

template <int HP>
__global__ void __launch_bounds__(kThreads, 1)
    k_svm_tc(const __grid_constant__ CUtensorMap hog_map, const __grid_constant__ CUtensorMap lbp_map,
             const LevelDesc *__restrict__ levels, const TcItem *__restrict__ items, int n_items,
             int *__restrict__ queue, const float *__restrict__ wt, float bias, float clip,
             float *__restrict__ scores, const uint32_t *__restrict__ c_flag, unsigned *__restrict__ err,
             const CUtensorMap *__restrict__ level_maps) {
    using Slot = SlotT<HP>;
    using TcSmem = TcSmemT<HP>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (smem_u32(smem_raw) & 1023u) {  // operand and TMA alignment: never expected
        if (tid == 0) atomicOr(err, kErrTimeout);
        return;
    }
    if (tid == 0) {
        auto init = [](unsigned long long *bar, uint32_t count) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
        };
        for (int s = 0; s < kSlots; ++s) {
            init(&S.cfull[s], 1);
            init(&S.cempty[s], kProducers);
        }
        for (int s = 0; s < 2; ++s) {
            init(&S.afull[s], kProducers);
            init(&S.aempty[s], 1);
            init(&S.dfull[s], 1);
            init(&S.dempty[s], 4);
        }
        S.failed = 0;
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
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B -> tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    const uint32_t b_base = smem_u32(S.b);

    // pipeline counters, advanced identically by every role
    uint32_t nrow = 0;      // block rows (A buffer, D buffer, their barrier phases)
    uint32_t ncell = 0;     // cell rows loaded (slot and its barrier phases)
    uint32_t issued = 0, committed = 0;  // control thread: loads issued, MMA rows committed

    for (;;) {
        if (tid == 0) S.item = atomicAdd(queue, 1);
        __syncthreads();
        const int item = S.item;
        if (item >= n_items || S.failed) break;
        const TcItem it = items[item];
        const LevelDesc L = levels[it.level];
        const int wend = min(it.wx0 + kTcStrip, L.cols);
        const int nrows = it.wy1 - it.wy0;
        const bool sparse = c_flag != nullptr;
        const int xl = it.wx0 & ~15;   // LBP box origin (16-byte boundary)

        // ---- sparse: which windows of the item are scored (all threads)
        if (sparse) {
            const int ty0 = it.wy0 / kCellTH, ty1 = (it.wy1 - 1 + kWinBH) / kCellTH;
            const int tx0 = it.wx0 / kCellTW, tx1 = (wend - 1 + kWinBW) / kCellTW;
            const int ntx = tx1 - tx0 + 1, nt = (ty1 - ty0 + 1) * ntx;
            for (int i = tid; i < nt; i += kThreads) {
                const int ty = ty0 + i / ntx, tx = tx0 + i % ntx;
                S.tflag[ty - ty0][tx - tx0] = c_flag[L.citem0 + ty * L.ctx + tx] != 0u;
            }
            __syncthreads();
            for (int row = warp; row < nrows; row += kWarps) {
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
                if (!any)  // no scored window in this row: it is never stored below
                    for (int wx = it.wx0 + lane; wx < wend; wx += 32)
                        scores[L.score_off + (int64_t)wy * L.cols + wx] = -INFINITY;
            }
            __syncthreads();
        }

        // ---- runs of block rows [ra, rb]; every role walks the same runs
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
            const int n_blk = rb - ra + 1;
            auto slot_of = [&](int u) -> Slot & { return S.slot[(ncell + u) % kSlots]; };
            // bounded wait by every lane of a warp, decided for the whole warp
            auto warp_wait = [&](unsigned long long *bar, uint32_t parity) {
                return __all_sync(0xffffffffu, bar_wait(S, bar, parity, err));
            };
            auto cell_wait = [&](int u) {  // cell row ra + u has arrived
                const uint32_t idx = ncell + u;
                return warp_wait(&S.cfull[idx % kSlots], (idx / kSlots) & 1u);
            };

            if (warp < kProducers) {
                // ---- producers: warps 0-3 HOG and LBP bins 0..9, warps 4-7
                // LBP bins 10..58, for rows 32 (w % 4) + lane
                const bool is_lbp = warp >= 4;
                const int m = 32 * (warp & 3) + lane;
                const int c = kWinPerWarp * (m >> 5) + (m & 31);
                const int cl = c + it.wx0 - xl;
                // (a row whose block lies past the level's last block holds whatever
                // the staged cells give: its products only reach windows past the
                // score map, which are never stored)
                bool ok = cell_wait(0);
                if (ok) pair_sums(slot_of(0), tid);
                for (int u = 0; u < n_blk; ++u) {
                    const uint32_t k = nrow + u;
                    ok = ok && cell_wait(u) && cell_wait(u + 1);
                    if (ok) pair_sums(slot_of(u + 1), tid);
                    producer_barrier();  // every producer warp, also after a failed wait
                    if (ok && k >= 2) ok = warp_wait(&S.aempty[k & 1], ((k >> 1) - 1) & 1u);
                    if (ok) {
                        tc_fence_after();
                        // this warp's TMEM lanes 32 (w % 4) .., A stage k % 2
                        const uint32_t a = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + kTmemA + (k & 1) * 96;
                        const Slot &s0 = slot_of(u), &s1 = slot_of(u + 1);
                        if (!is_lbp)
                            build_hog(s0, s1, S.tab, c, cl, clip, a);
                        else
                            build_lbp(s0, s1, S.tab, cl, a);
                        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                        tc_fence_before();
                    }
                    __syncwarp();
                    if (ok && lane == 0) {
                        arrive(&S.afull[k & 1]);
                        arrive(&S.cempty[(ncell + u) % kSlots]);
                        if (u == n_blk - 1) arrive(&S.cempty[(ncell + u + 1) % kSlots]);
                    }
                }
            } else {
                // ---- epilogue warps 8-11 (TMEM lanes 32 q .. 32 q + 31); lane 0 of
                // warp 8 also issues the cell loads and the MMAs of each row
                // before the epilogue of the row above it
                const int q = warp & 3;
                const bool ctrl = warp == kProducers && lane == 0;
                const int wl = kWinPerWarp * q + lane;
                const int wx = it.wx0 + wl;
                bool ok = true, cok = true;  // epilogue / control progress
                float acc[kWinBH];           // running scores of window rows r - i (a run starts afresh)
#pragma unroll
                for (int i = 0; i < kWinBH; ++i) acc[i] = 0.f;
                auto issue = [&](int u) {  // control: load cell row ra + u into its slot once free
                    const uint32_t idx = ncell + u;
                    if (idx >= kSlots)
                        cok = cok && bar_wait(S, &S.cempty[idx % kSlots], (idx / kSlots - 1) & 1u, err);
                    if (!cok) return;
                    Slot &sl = S.slot[idx % kSlots];
                    unsigned long long *bar = &S.cfull[idx % kSlots];
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                                 "r"((uint32_t)(sizeof(float) * HP * kHogX + kLbpBins * kLbpX))
                                 : "memory");
                    tma_3d(&sl.hog[0][0], level_maps ? level_maps + 2 * L.tc_map : &hog_map, bar, it.wx0,
                           L.cell_row + ra + u, 0);
                    tma_3d(&sl.lbp[0][0], level_maps ? level_maps + 2 * L.tc_map + 1 : &lbp_map, bar, xl,
                           L.cell_row + ra + u, 0);
                    issued = idx + 1;
                };
                if (ctrl)
                    for (int u = 0; u < min(kSlots, n_cell); ++u) issue(u);
                for (int u = 0; u <= n_blk; ++u) {
                    if (ctrl && u < n_blk && cok) {
                        const uint32_t k = nrow + u;
                        cok = bar_wait(S, &S.afull[k & 1], (k >> 1) & 1u, err);
                        if (cok && k >= 2) cok = bar_wait(S, &S.dempty[k & 1], ((k >> 1) - 1) & 1u, err);
                        if (cok) {
                            tc_fence_after();
                            const uint32_t d = tmem + (k & 1) * 128;
                            const uint32_t a0 = tmem + kTmemA + (k & 1) * 96;  // 8 columns per K step
#pragma unroll
                            for (int s = 0; s < 6; ++s)
                                umma_ts(d, a0 + 8 * s, umma_desc(b_base + 256 * s), s > 0);
#pragma unroll
                            for (int s = 0; s < 6; ++s)
                                umma_ts(d, a0 + 48 + 8 * s, umma_desc(b_base + 256 * s), 1);
#pragma unroll
                            for (int s = 0; s < 6; ++s)
                                umma_ts(d, a0 + 8 * s, umma_desc(b_base + 12 * 128 + 256 * s), 1);
                            umma_commit(&S.aempty[k & 1]);
                            umma_commit(&S.dfull[k & 1]);
                            committed = k + 1;
                            // cell row ra + u is released after this block row: its slot takes ra + u + 4
                            if (u + kSlots < n_cell) issue(u + kSlots);
                        }
                    }
                    __syncwarp();
                    if (u == 0) continue;
                    // epilogue of block row ra + u - 1
                    const uint32_t k = nrow + u - 1;
                    const int r = ra + u - 1;
                    ok = ok && warp_wait(&S.dfull[k & 1], (k >> 1) & 1u);
                    if (!ok) continue;
                    tc_fence_after();
                    const uint32_t t0 = tmem + ((uint32_t)(32 * q) << 16) + (k & 1) * 128;
                    // 105 columns in seven groups of 16
                    acc[0] = bias;
#pragma unroll
                    for (int g = 0; g < 7; ++g) {
                        float v[16];
                        PD_LD_X16(t0 + 16 * g, v, 0);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        if (g == 6) {
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) arrive(&S.dempty[k & 1]);  // the accumulators may be overwritten
                        }
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int n = 16 * g + e;  // (i, j) = (n / 7, n % 7)
                            if (n < kWinBH * kWinBW) {
                                const int i = n / kWinBW, j = n % kWinBW;
                                acc[i] += j ? __shfl_down_sync(0xffffffffu, v[e], j) : v[e];
                            }
                        }
                    }
                    const int wy = r - (kWinBH - 1);
                    if (wy >= it.wy0 && lane < kWinPerWarp && wx < wend) {
                        const bool keep = !sparse || ((S.win_ok[wy - it.wy0][wl >> 5] >> (wl & 31)) & 1u);
                        scores[L.score_off + (int64_t)wy * L.cols + wx] = keep ? acc[kWinBH - 1] : -INFINITY;
                    }
#pragma unroll
                    for (int i = kWinBH - 1; i > 0; --i) acc[i] = acc[i - 1];
                }
            }
            nrow += n_blk;
            ncell += n_cell;
            r_next = rb + 1;
        }
        __syncthreads();  // the item is done by every role (nothing in flight unless a wait failed)
        if (S.failed) break;
    }

    __syncthreads();
    if (S.failed && warp == kProducers && lane == 0) {
        // drain this CTA's copies and MMAs (bounded) before the tensor memory
        // is freed: the last load of every slot, the last commit
        for (uint32_t idx = issued > kSlots ? issued - kSlots : 0u; idx < issued; ++idx)
            drain_wait(&S.cfull[idx % kSlots], (idx / kSlots) & 1u);
        if (committed > 0) drain_wait(&S.dfull[(committed - 1) & 1], ((committed - 1) >> 1) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

#undef PD_LD_X16

}  // namespace

cudaError_t init_svm_tc() {
    cudaError_t e = cudaFuncSetAttribute(k_svm_tc<kHogBins>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(TcSmemT<kHogBins>));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_svm_tc<4 * kHogBins>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(TcSmemT<4 * kHogBins>));
}

int svm_tc_smem_bytes(int hog_planes) {
    return hog_planes == 4 * kHogBins ? (int)sizeof(TcSmemT<4 * kHogBins>) : (int)sizeof(TcSmemT<kHogBins>);
}

cudaError_t launch_svm_tc(cudaStream_t s, const CUtensorMap &hog_map, const CUtensorMap &lbp_map,
                          const LevelDesc *d_levels, const TcItem *d_items, int n_items, int *d_queue, int grid,
                          const float *d_w, float bias, float clip, float *scores, const uint32_t *c_flag,
                          unsigned *d_err, int hog_planes, const CUtensorMap *level_maps) {
    if (n_items <= 0) return cudaSuccess;
    if (reinterpret_cast<uintptr_t>(level_maps) & 63) return cudaErrorInvalidValue;
    grid = grid < n_items ? grid : n_items;
    if (hog_planes == 4 * kHogBins)
        k_svm_tc<4 * kHogBins><<<grid, kThreads, sizeof(TcSmemT<4 * kHogBins>), s>>>(
            hog_map, lbp_map, d_levels, d_items, n_items, d_queue, d_w, bias, clip, scores, c_flag, d_err,
            level_maps);
    else
        k_svm_tc<kHogBins><<<grid, kThreads, sizeof(TcSmemT<kHogBins>), s>>>(
            hog_map, lbp_map, d_levels, d_items, n_items, d_queue, d_w, bias, clip, scores, c_flag, d_err,
            level_maps);
    return cudaGetLastError();
}

}  // namespace pd
