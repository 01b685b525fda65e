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
// carry zero weights; mma.sync m16n8k16), giving 35x35x16 activations.
// Layer 2 (17x17x32, K = 9 taps x 16) and layer 3 (8x8x32, K = 9 x 32) are
// implicit GEMMs on the 5th-generation tensor cores: one thread issues
// tcgen05.mma with both operands in shared memory (no-swizzle K-major
// layout: the activation planes below are already that layout for every
// tap, a tap being a start-address offset) and fp32 accumulators in tensor
// memory; completion arrives on an mbarrier (bounded wait), and the
// epilogues read the accumulators with tcgen05.ld. Layer 2's 16x16 core runs
// as two M = 128 blocks; its 33 edge positions (row 16, column 16) run on
// mma.sync meanwhile. Layer 3 is one M = 64 block. The 1x1 head gives h.
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
constexpr int kRawW = kCnnBoxW;  // staged bytes per row: pixels x0-9 .. x0+86 (TMA box)
static_assert(XR == kCnnBoxH, "input box height");
static_assert((XR * kRawW) % 128 == 0, "second raw buffer stays 128-byte aligned");
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
constexpr float kInv255 = 1.0f / 255.0f;   // float32 nearest to 1/255

// Canonical (no-swizzle, K-major) UMMA B operands: per tap a 32 x 16 bf16
// matrix stored as [8-row group n/8][8-column chunk k/8][row n%8][k%8], so the
// K-chunk stride (LBO) is 128 bytes and the 8-row-group stride (SBO) 256.
constexpr int kBTapBytes = 1024;
constexpr int kL2Core = 16;       // layer-2 outputs [0,16)^2 on tcgen05; row 16 and column 16 on mma.sync
constexpr int kEdge = 2 * R2 - 1; // 33 edge positions
constexpr uint32_t kTmemCols = 128;  // L2 core accumulators in columns [0,64), L3 in [64,96)
constexpr uint64_t kWaitNs = 1000000000ull;

struct CnnSmem {
    uint8_t raw[2][XR][kRawW];   // input bytes, double buffered (TMA destinations: 128-byte aligned)
    uint4 a1[2 * 2 * PS1];       // [channel group 0..1][parity] planes of layer 1
    union {
        uint32_t xb[XR * XBW];   // bf16 pixel pairs (dead once layer 1 is done)
        uint4 a2[4 * 2 * PS2];   // [channel group 0..3][parity] planes of layer 2
    } u;
    uint8_t w2c[9 * kBTapBytes];      // layer-2 B operands, one per tap
    uint8_t w3c[9 * 2 * kBTapBytes];  // layer-3 B operands, per tap and input-channel half
    float b1[16];
    float b2[32];
    float b3[32];
    float wh[32];
    float hpart[2][64];
    unsigned long long bar;      // MMA completion (one phase per commit)
    unsigned long long inbar[2]; // input tile arrival, one per raw buffer
    uint32_t tmem;               // tensor-memory base of this CTA
    int failed;
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

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ---- tcgen05 (5th-generation tensor cores, accumulators in tensor memory)
// Shared-memory matrix descriptor, no swizzle, K-major: start, K-chunk
// stride (LBO) and 8-row-group stride (SBO) in 16-byte units; bit 46 is the
// descriptor version.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3fff) | ((uint64_t)((lbo >> 4) & 0x3fff) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fff) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: f32 accumulator, bf16 A and B, both
// K-major, N / 8 and M / 16.
__host__ __device__ constexpr uint32_t umma_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void umma_commit(unsigned long long *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 16 consecutive f32 columns of this thread's tensor-memory lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Every thread waits (bounded) for phase `parity` of the MMA barrier; a wait
// that gives up sets the error word and the CTA's failed flag.
__device__ __forceinline__ bool mma_wait(CnnSmem &S, uint32_t parity, unsigned *err) {
    const uint32_t a = smem_u32(&S.bar);
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
    if (!ok) {
        S.failed = 1;
        if (err) atomicOr(err, kErrTimeout);
    }
    return ok != 0;
}

// Issues the TMA load of an item's input box into a raw buffer: bytes
// [8 cx0 - 16, 8 cx0 + 80) of rows [8 cy0 - 7, 8 cy0 + 65) of its level (the
// x coordinate is a multiple of 16 bytes; outside the level the box reads
// zeros, and the conversion zeroes those pixels anyway).
__device__ __forceinline__ void load_input(uint8_t (*raw)[kRawW], unsigned long long *bar,
                                           const CUtensorMap *__restrict__ maps, const CnnItem &it) {
    const uint32_t b = smem_u32(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"((uint32_t)(kRawW * XR))
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(&raw[0][0])),
        "l"(reinterpret_cast<uint64_t>(maps + it.level)), "r"(8 * it.cx0 - 16), "r"(8 * it.cy0 - 7), "r"(b)
        : "memory");
}

// Bounded wait (every thread) for phase `parity` of a barrier.
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

// Position of layer-2 edge index e (row 16, then column 16): (r, c).
__device__ __forceinline__ int2 edge_pos(int e) {
    e = min(e, kEdge - 1);
    return e < R2 ? make_int2(kL2Core, e) : make_int2(e - R2, kL2Core);
}

__global__ void __launch_bounds__(kThreads, 2) k_cnn_fwd(const LevelDesc *__restrict__ levels,
                                                         const CUtensorMap *__restrict__ lvl_maps,
                                                         const CnnItem *__restrict__ items, int n_items,
                                                         const CnnWeights wts, float *__restrict__ hmap,
                                                         int32_t hmap_pitch, unsigned *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    CnnSmem &S = *reinterpret_cast<CnnSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    int item = blockIdx.x;
    if (item >= n_items) return;
    if (smem_u32(S.raw) & 127u) {  // TMA destinations need 128-byte alignment: never expected
        if (tid == 0 && err) atomicOr(err, kErrTimeout);
        return;
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.inbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.inbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        load_input(S.raw[0], &S.inbar[0], lvl_maps, items[item]);
    }
    // thread 0: loads issued and not yet consumed (bit b: raw buffer b) and their phase parities
    uint32_t pend = tid == 0 ? 1u : 0u, ppar = 0u;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.failed = 0;
    }
    // canonical B operands of layers 2 and 3 from the bf16-rounded weights
    for (int i = tid; i < 9 * 32 * 16; i += kThreads) {
        const int tap = i / 512, n = (i >> 4) & 31, k = i & 15;
        const uint32_t off = tap * kBTapBytes + (n >> 3) * 256 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16 *>(S.w2c + off) = __float2bfloat16_rn(wts.w2[(n * 16 + k) * 9 + tap]);
    }
    for (int i = tid; i < 9 * 2 * 32 * 16; i += kThreads) {
        const int tk = i / 512, n = (i >> 4) & 31, k = i & 15;  // tk = tap * 2 + k-half
        const int tap = tk >> 1, kh = tk & 1;
        const uint32_t off = tk * kBTapBytes + (n >> 3) * 256 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16 *>(S.w3c + off) =
            __float2bfloat16_rn(wts.w3[(n * 32 + 16 * kh + k) * 9 + tap]);
    }
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
    // layer-2 B fragments (9 taps x 4 n-tiles x 2 regs) for the edge positions on mma.sync
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
    const uint32_t a1_base = smem_u32(&S.a1[0]);
    const uint32_t a2_base = smem_u32(&S.u.a2[0]);
    const uint32_t w2c_base = smem_u32(S.w2c), w3c_base = smem_u32(S.w3c);
    async_proxy_fence();  // the B operands are read by the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    uint32_t phase = 0;  // parity of the next MMA barrier phase

    for (int iter = 0; item < n_items && !S.failed; ++iter, item += gridDim.x) {
        const int cur = iter & 1;
        const int next = item + gridDim.x;
        if (tid == 0 && next < n_items) {
            async_proxy_fence();  // the buffer's previous bytes were read by the generic proxy
            load_input(S.raw[cur ^ 1], &S.inbar[cur ^ 1], lvl_maps, items[next]);
            pend |= 1u << (cur ^ 1);
            ppar = (ppar & ~(1u << (cur ^ 1))) | ((((uint32_t)(iter + 1) >> 1) & 1u) << (cur ^ 1));
        }
        // this tile's input: phase iter / 2 of its buffer's barrier (CTA-uniform decision)
        const bool in_ok = bar_wait(&S.inbar[cur], (uint32_t)(iter >> 1) & 1u);
        if (tid == 0 && in_ok) pend &= ~(1u << cur);
        if (__syncthreads_or(!in_ok)) {
            if (tid == 0) {
                S.failed = 1;
                if (err) atomicOr(err, kErrTimeout);
            }
            break;
        }

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

        // ---- pixels -> bf16 x; xb[r][c] = x(y0 + r, x0 + c) = raw[r][c + 9].
        // x = bf16(L/255 - 0.5): one fma in float32 rounded once to bf16 equals
        // the correctly rounded value for all 256 inputs (checked exhaustively
        // against exact rational arithmetic when this path was written).
        for (int k = tid; k < XR * (XR / 4); k += kThreads) {
            const int r = k / (XR / 4), j = k - r * (XR / 4);
            const uint32_t *rw = reinterpret_cast<const uint32_t *>(S.raw[cur][r]);
            const uint32_t v = __byte_perm(rw[j + 2], rw[j + 3], 0x4321);  // bytes 4j + 9 .. 4j + 12
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
        // ---- layer 1 on tensor cores (mma.sync): 1225 positions x 16 channels, K = 16 (4x4 patch)
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
        async_proxy_fence();  // layer-1 planes are read by the tensor cores next
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- layer 2, outputs [0,16)^2 on tcgen05: two 16-row x 8-column blocks (M = 128),
        // N = 32, K = 16 per tap. A for tap (dy, dx), block c0: rows 2r + dy of the
        // parity-(dx & 1) plane, columns c0 + dx / 2 + 0..7; 8-row groups 2 plane rows apart.
        if (tid == 0) {
            constexpr uint32_t kIdesc = umma_idesc(128, 32);
#pragma unroll
            for (int cb = 0; cb < 2; ++cb)
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3, dx = tap % 3;
                    const uint32_t a = a1_base + (uint32_t)((((dx & 1) * PS1) + dy * C1P + 8 * cb + (dx >> 1)) << 4);
                    umma_bf16(tmem + 32 * cb, umma_desc(a, 2 * PS1 * 16, 2 * C1P * 16),
                              umma_desc(w2c_base + tap * kBTapBytes, 128, 256), kIdesc, tap > 0);
                }
            umma_commit(&S.bar);
        }
        // ---- layer 2 edges (row 16, column 16: 33 positions) on mma.sync, meanwhile
        if (warp < 3) {
            const int mt = warp;
            const int2 e0 = edge_pos(mt * 16 + g), e1 = edge_pos(mt * 16 + g + 8);
            const int2 le = edge_pos(mt * 16 + (lane & 15));
            const uint32_t src = a1_base + ((((lane >> 4) * 2) * PS1 + 2 * le.x * C1P + le.y) << 4);
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
            const bool in0 = interior2 || ((y2 + e0.x) >= 0 && (y2 + e0.x) < H2 && (x2 + e0.y) >= 0 && (x2 + e0.y) < W2);
            const bool in1 = interior2 || ((y2 + e1.x) >= 0 && (y2 + e1.x) < H2 && (x2 + e1.y) >= 0 && (x2 + e1.y) < W2);
            const uint32_t dst = a2_base + ((((lane >> 4) * 2 + (le.y & 1)) * PS2 + le.x * C2P + (le.y >> 1)) << 4);
#pragma unroll
            for (int h = 0; h < 2; ++h)
                stsm_x4(dst + ((4 * h * PS2) << 4),
                        in0 ? relu_pack_bf16(acc[2 * h][0], acc[2 * h][1]) : 0u,
                        in1 ? relu_pack_bf16(acc[2 * h][2], acc[2 * h][3]) : 0u,
                        in0 ? relu_pack_bf16(acc[2 * h + 1][0], acc[2 * h + 1][1]) : 0u,
                        in1 ? relu_pack_bf16(acc[2 * h + 1][2], acc[2 * h + 1][3]) : 0u);
        }
        if (__syncthreads_or(!mma_wait(S, phase, err))) break;  // CTA-uniform
        phase ^= 1u;
        tc_fence_after();
        // ---- layer-2 core epilogue: warp w reads lanes 32 (w % 4) .. + 31 of block w / 4:
        // lane m = 32 (w % 4) + l holds output (r, c) = (m / 8, 8 (w / 4) + m % 8), 32 channels
        {
            const int cb = warp >> 2, m = 32 * (warp & 3) + lane;
            const int r = m >> 3, c = 8 * cb + (m & 7);
            const bool in = interior2 || ((y2 + r) >= 0 && (y2 + r) < H2 && (x2 + c) >= 0 && (x2 + c) < W2);
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + 32 * cb + 16 * hf, v);
#pragma unroll
                for (int gg = 0; gg < 2; ++gg) {
                    const int grp = 2 * hf + gg;
                    const float *bb = &S.b2[8 * grp];
                    uint4 q;
                    q.x = in ? relu_pack_bf16(v[8 * gg + 0] + bb[0], v[8 * gg + 1] + bb[1]) : 0u;
                    q.y = in ? relu_pack_bf16(v[8 * gg + 2] + bb[2], v[8 * gg + 3] + bb[3]) : 0u;
                    q.z = in ? relu_pack_bf16(v[8 * gg + 4] + bb[4], v[8 * gg + 5] + bb[5]) : 0u;
                    q.w = in ? relu_pack_bf16(v[8 * gg + 6] + bb[6], v[8 * gg + 7] + bb[7]) : 0u;
                    S.u.a2[(grp * 2 + (c & 1)) * PS2 + r * C2P + (c >> 1)] = q;
                }
            }
        }
        async_proxy_fence();  // layer-2 planes are read by the tensor cores next
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- layer 3 on tcgen05: 8 x 8 outputs (M = 64), N = 32, K = 9 taps x 2 halves x 16
        if (tid == 0) {
            constexpr uint32_t kIdesc = umma_idesc(64, 32);
#pragma unroll
            for (int tap = 0; tap < 9; ++tap)
#pragma unroll
                for (int kh = 0; kh < 2; ++kh) {
                    const int dy = tap / 3, dx = tap % 3;
                    const uint32_t a =
                        a2_base + (uint32_t)((((2 * kh) * 2 + (dx & 1)) * PS2 + dy * C2P + (dx >> 1)) << 4);
                    umma_bf16(tmem + 64, umma_desc(a, 2 * PS2 * 16, 2 * C2P * 16),
                              umma_desc(w3c_base + (tap * 2 + kh) * kBTapBytes, 128, 256), kIdesc, tap + kh > 0);
                }
            umma_commit(&S.bar);
        }
        if (__syncthreads_or(!mma_wait(S, phase, err))) break;  // CTA-uniform
        phase ^= 1u;
        tc_fence_after();
        // ---- layer-3 epilogue and head: M = 64 rows sit in lanes 32 q + (0..15) of
        // quadrant q (rows 16 q .. 16 q + 15); warps 0-3 take channels 0-15, warps 4-7 16-31
        {
            const int q = warp & 3, half = warp >> 2;
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + 64 + 16 * half, v);
            float hp = 0.f;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int ch = 16 * half + i;
                hp = fmaf(fmaxf(v[i] + S.b3[ch], 0.f), S.wh[ch], hp);
            }
            if (lane < 16) S.hpart[half][16 * q + lane] = hp;
        }
        __syncthreads();
        if (tid < 64) {
            const int cy = y3 + (tid >> 3), cx = x3 + (tid & 7);
            if (cy < L.Hc && cx < L.Wc)
                hmap[(int64_t)(L.cell_row + cy) * hmap_pitch + cx] = bh + S.hpart[0][tid] + S.hpart[1][tid];
        }
    }
    // drain loads still in flight (bounded) before the CTA leaves
    if (tid == 0)
        for (int b = 0; b < 2; ++b)
            if ((pend >> b) & 1u) bar_wait(&S.inbar[b], (ppar >> b) & 1u);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// Window pooling z[wy][wx] = bv + sum_{r<16, s<8} V[r][s] h[wy+r][wx+s]: one
// CTA per (level, 64 x 16 window tile); the tile's 31 x 71 cells of h are
// staged in shared memory; each thread computes 4 consecutive windows of one
// row (8 taps x 4 windows per h row from 11 staged values), in a fixed order.
// With level groups a level's h is its group level's head map read at the
// cell holding each cell's centre: row min(floor((2 cy + 1) Hk_j / (2 Hk)),
// Hc_j - 1), column likewise (the identity for the group level itself).
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
    const LevelDesc J = levels[L.hsrc];
    const bool same = L.hsrc == (int)blockIdx.y;
    for (int i = threadIdx.x; i < 128; i += blockDim.x) V[i] = v[i];
    for (int i = threadIdx.x; i < kPoolHH * kPoolHW; i += blockDim.x) {
        const int r = i / kPoolHW, c = i - r * kPoolHW;
        const int cy = wy0 + r, cx = wx0 + c;
        float hv = 0.f;
        if (cy < L.Hc && cx < L.Wc) {
            const int sy = same ? cy : min((2 * cy + 1) * J.Hk / (2 * L.Hk), J.Hc - 1);
            const int sx = same ? cx : min((2 * cx + 1) * J.Wk / (2 * L.Wk), J.Wc - 1);
            hv = hmap[(int64_t)(J.cell_row + sy) * hmap_pitch + sx];
        }
        Hs[r][c] = hv;
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

cudaError_t launch_cnn(cudaStream_t s, const LevelDesc *d_levels, int n_levels, const CUtensorMap *lvl_maps,
                       const CnnItem *d_items, int n_items, const CnnWeights &w, float *hmap,
                       int32_t hmap_pitch, float *logits, int pool_tiles, unsigned *err) {
    if (n_items > 0) {
        const int grid = std::min(n_items, g_cnn_grid > 0 ? g_cnn_grid : n_items);
        k_cnn_fwd<<<grid, kThreads, sizeof(CnnSmem), s>>>(d_levels, lvl_maps, d_items, n_items, w, hmap,
                                                           hmap_pitch, err);
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
