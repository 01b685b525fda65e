// K4 -- block normalisation fused with the sliding-window linear SVM
// (Section 4.4, Algorithm 6; block features of Sections 4.2-4.3).
//
// score[wy][wx] = b + sum_{i<15, j<7, t<95} f[wy+i][wx+j][t] * w[i][j][t]
// where f[by][bx] is the 95-value block feature: the 4 HOG cells of the 2x2
// block (top-left, top-right, bottom-left, bottom-right; 36 values)
// normalised with L2-Hys, then the sum of the 4 LBP cell counts (59 values)
// normalised with L1-sqrt (every block holds 256 pixels, so f = sqrt(c/256)).
//
// This is a single-template correlation with 95 input channels, not a dense
// GEMM, so it runs on the FP32 CUDA cores (no tensor-core formulation).
//
// One CTA (8 warps) computes one TW x TH tile of windows of one level. The
// tile shape is chosen per level by the host planner among seven shapes
// (lanes along x LX, window rows per thread RY): 32x16, 64x8, 32x8, 64x4,
// 64x2, 32x12, 32x4 (the small ones keep the short top levels of the
// pyramid from computing windows past the score map).
//  1. Thread 0 issues TMA loads (cp.async.bulk.tensor.3d): the tile's cell
//     region of all 9 HOG planes (f32) at once, and the first two 8-plane
//     chunks of the 59 LBP planes (u8) into a double buffer; each buffer
//     completes on its own mbarrier (bounded waits: a 1 s limit, then the
//     error word is set and the CTA drains its copies and leaves).
//  2. The CTA computes the two L2-Hys scale factors of every block of the
//     region (|v| over the 36 HOG values, then over the clipped values).
//  3. The 95 channels go round by round, 8 per round, one per warp
//     (channel t = 8*round + warp). For its channel a warp loads the 15x7
//     template slice into registers (warp-uniform loads, issued first so
//     they overlap the next step), writes the channel's feature plane for
//     the whole region into its own shared-memory slice, and runs the
//     correlation: each lane owns 4 x RY windows and, for each block row it
//     touches, loads 12 consecutive features with three 128-bit shared loads
//     and issues up to RY x 7 x 4 FMAs. All loop indices are compile-time,
//     so the template slice stays in registers. LBP rounds read the 8-plane
//     chunk of their round; after each round the freed buffer is refilled
//     with the chunk two rounds ahead.
//  4. The 8 per-warp partial sums are added in warp order (deterministic),
//     the bias is added and the valid windows are stored.
#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kRounds = (kFeat + kWarps - 1) / kWarps;  // 12
constexpr int kLbpChunk = 8;                             // LBP planes per TMA chunk
constexpr int kFirstLbpRound = kHogDim / kWarps;         // 4: round 4 holds t = 32..39

template <int LX, int RY>
struct Shape {
    static constexpr int LY = 32 / LX;
    static constexpr int TW = 4 * LX;             // windows along x
    static constexpr int TH = RY * LY;            // windows along y
    static constexpr int RBY = TH + kWinBH - 1;   // block rows of the region
    static constexpr int RBX = TW + kWinBW - 1;   // block columns of the region
    static constexpr int CR = RBY + 1;            // cell rows of the region
    static constexpr int FP = TW + 8;             // feature-plane pitch (floats), >= 4*LX + 8
    static constexpr int HX = TW + 8;             // HOG box width (cells), 16-byte multiple
    static constexpr int LXB = (TW + 8 + 15) / 16 * 16;  // LBP box width (bytes)
    static constexpr uint32_t kHogBytes = 4u * kHogBins * CR * HX;
    static constexpr uint32_t kLbpBytes = 1u * kLbpChunk * CR * LXB;
    // shared-memory layout (byte offsets, 128-byte aligned pieces)
    static constexpr size_t oHog = 0;
    static constexpr size_t oLbp = (oHog + kHogBytes + 127) / 128 * 128;
    static constexpr size_t oInv = (oLbp + 2 * kLbpBytes + 127) / 128 * 128;
    static constexpr size_t oFeat = (oInv + 2 * 4 * RBY * FP + 127) / 128 * 128;
    static constexpr size_t oTab = oFeat + 4ull * kWarps * RBY * FP;
    static constexpr size_t oBar = (oTab + 4 * 260 + 15) / 16 * 16;
    static constexpr size_t kSmem = oBar + 64;
    static_assert(kWarps * RBY * FP >= kWarps * TW * TH, "reduction buffer fits in the planes");
    static_assert(FP % 4 == 0 && HX % 4 == 0, "alignment");
};

// The tile shapes, by index (the host planner uses the same order).
using S0 = Shape<8, 4>;   // 32 x 16
using S1 = Shape<16, 4>;  // 64 x 8
using S2 = Shape<8, 2>;   // 32 x 8
using S3 = Shape<16, 2>;  // 64 x 4
using S4 = Shape<16, 1>;  // 64 x 2
using S5 = Shape<8, 3>;   // 32 x 12
using S6 = Shape<8, 1>;   // 32 x 4
constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
constexpr size_t kSmemMax =
    cmax(cmax(cmax(S0::kSmem, S1::kSmem), cmax(S2::kSmem, S3::kSmem)), cmax(cmax(S4::kSmem, S5::kSmem), S6::kSmem)) +
    128;

struct SvmMaps {
    CUtensorMap hog[kSvmShapes];
    CUtensorMap lbp[kSvmShapes];
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on phase `parity`: gives up after limit_ns nanoseconds.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, uint32_t parity,
                                                  uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, unsigned long long *bar,
                                            int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s

template <class SH, int RY>
__device__ void svm_tile(const SvmItem &it, const LevelDesc &L, const CUtensorMap *hog_map,
                         const CUtensorMap *lbp_map, const float *__restrict__ wt, float bias,
                         float clip, float *__restrict__ scores, unsigned *__restrict__ err,
                         unsigned char *smem) {
    constexpr int LX = SH::TW / 4, TW = SH::TW, TH = SH::TH;
    constexpr int RBY = SH::RBY, RBX = SH::RBX, CR = SH::CR, FP = SH::FP, HX = SH::HX, LXB = SH::LXB;
    float(*hog)[CR][HX] = reinterpret_cast<float(*)[CR][HX]>(smem + SH::oHog);
    uint8_t(*lbp)[kLbpChunk][CR][LXB] = reinterpret_cast<uint8_t(*)[kLbpChunk][CR][LXB]>(smem + SH::oLbp);
    float(*inv1)[FP] = reinterpret_cast<float(*)[FP]>(smem + SH::oInv);
    float(*inv2)[FP] = inv1 + RBY;
    float(*feat)[RBY][FP] = reinterpret_cast<float(*)[RBY][FP]>(smem + SH::oFeat);
    float *sqrt_tab = reinterpret_cast<float *>(smem + SH::oTab);
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem + SH::oBar);  // hog, lbp0, lbp1
    volatile int *failed = reinterpret_cast<volatile int *>(bars + 4);  // a wait of this CTA gave up
    int *released = reinterpret_cast<int *>(bars + 4) + 1;             // [2] warps done with each LBP buffer
    int *issued = released + 2;                                        // [2] loads issued into each buffer
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cy = L.cell_row + it.wy0;

    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);
        *failed = 0;
        released[0] = released[1] = 0;
        issued[0] = issued[1] = 1;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&bars[0], SH::kHogBytes);
        tma_load_3d(&hog[0][0][0], hog_map, &bars[0], it.wx0, cy, 0);
        for (int b = 0; b < 2; ++b) {
            mbar_expect_tx(&bars[1 + b], SH::kLbpBytes);
            tma_load_3d(&lbp[b][0][0][0], lbp_map, &bars[1 + b], it.wx0, cy,
                        kWarps * (kFirstLbpRound + b) - kHogDim);
        }
    }
    for (int c = tid; c <= 256; c += kThreads) sqrt_tab[c] = sqrtf((float)c * (1.0f / 256.0f));
    // Every lane waits (bounded) so that it observes the completed phase and
    // thereby acquires the TMA-written data; a warp whose wait gave up marks
    // the CTA failed and skips to the end.
    auto warp_wait = [&](int b, uint32_t parity) -> bool {
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[b], parity, kWaitNs));
        if (!ok && lane == 0) {
            atomicOr(err, kErrTimeout);
            *failed = 1;
        }
        return ok;
    };
    const bool hog_ok = warp_wait(0, 0);

    // ---- 2. L2-Hys scale factors of every block of the region
    if (hog_ok) {
        for (int i = tid; i < RBY * FP; i += kThreads) {
            const int by = i / FP, bx = i - by * FP;
            float i1 = 0.f, i2 = 0.f;
            if (bx < RBX) {
                float s = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int b = 0; b < kHogBins; ++b) {
                        const float v = hog[b][by + (q >> 1)][bx + (q & 1)];
                        s = fmaf(v, v, s);
                    }
                i1 = 1.0f / sqrtf(s + 1.0f);
                float s2 = 0.f;
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int b = 0; b < kHogBins; ++b) {
                        const float u = fminf(hog[b][by + (q >> 1)][bx + (q & 1)] * i1, clip);
                        s2 = fmaf(u, u, s2);
                    }
                i2 = 1.0f / sqrtf(s2 + 1e-6f);
            }
            inv1[by][bx] = i1;
            inv2[by][bx] = i2;
        }
    }
    __syncthreads();

    // ---- 3. channel rounds. Warps are not kept in step: a warp waits only
    // for the LBP chunk of its round, and the last warp to finish with a
    // buffer refills it with the chunk two rounds ahead, so one warp's
    // plane building overlaps another's FMAs.
    const int lx = lane % LX, ly = lane / LX;
    float acc[RY][4];
#pragma unroll
    for (int q = 0; q < RY; ++q)
#pragma unroll
        for (int x = 0; x < 4; ++x) acc[q][x] = 0.f;
    float(*F)[FP] = feat[warp];

    for (int round = 0; round < kRounds && !*failed; ++round) {
        const int t = kWarps * round + warp;
        const int k = round - kFirstLbpRound, buf = k & 1;
        if (round >= kFirstLbpRound && !warp_wait(1 + buf, (k >> 1) & 1)) break;
        if (t < kFeat) {
            // template slice of channel t: w[t][i][0..7] (warp-uniform loads)
            float w[kWinBH][kWinBW];
            const float4 *wp = reinterpret_cast<const float4 *>(wt + (size_t)t * kWinBH * kWPad);
#pragma unroll
            for (int i = 0; i < kWinBH; ++i) {
                const float4 a = __ldg(wp + 2 * i), c = __ldg(wp + 2 * i + 1);
                w[i][0] = a.x; w[i][1] = a.y; w[i][2] = a.z; w[i][3] = a.w;
                w[i][4] = c.x; w[i][5] = c.y; w[i][6] = c.z;
            }
            // feature plane of channel t over the region, 4 blocks per step
            constexpr int Q = FP / 4;
            if (t < kHogDim) {
                const int q = t / kHogBins, b = t - q * kHogBins;
                const int oy = q >> 1, ox = q & 1;
                for (int i = lane; i < RBY * Q; i += 32) {
                    const int by = i / Q, bx = 4 * (i - by * Q);
                    const float4 s1 = *reinterpret_cast<const float4 *>(&inv1[by][bx]);
                    const float4 s2 = *reinterpret_cast<const float4 *>(&inv2[by][bx]);
                    const float *h = &hog[b][by + oy][bx + ox];
                    float4 v;  // s1 = s2 = 0 on the padding columns
                    v.x = fminf(h[0] * s1.x, clip) * s2.x;
                    v.y = fminf(h[1] * s1.y, clip) * s2.y;
                    v.z = fminf(h[2] * s1.z, clip) * s2.z;
                    v.w = ox + bx + 3 < HX ? fminf(h[3] * s1.w, clip) * s2.w : 0.f;
                    *reinterpret_cast<float4 *>(&F[by][bx]) = v;
                }
            } else {
                // LBP channel: this warp's plane of the round's chunk
                const uint8_t(*P)[LXB] = lbp[buf][warp];
                for (int i = lane; i < RBY * Q; i += 32) {
                    const int by = i / Q, bx = 4 * (i - by * Q);
                    const uint32_t r0 = *reinterpret_cast<const uint32_t *>(&P[by][bx]);
                    const uint32_t r1 = *reinterpret_cast<const uint32_t *>(&P[by + 1][bx]);
                    // counts <= 64, so the byte-wise vertical sums (<= 128) do not carry
                    const uint32_t sv = r0 + r1;
                    const uint32_t sn = (uint32_t)P[by][bx + 4] + (uint32_t)P[by + 1][bx + 4];
                    const uint32_t b0 = sv & 255u, b1 = (sv >> 8) & 255u, b2 = (sv >> 16) & 255u,
                                   b3 = sv >> 24;
                    float4 v;
                    // (indices clamped: counts above 64 are not valid input, but
                    // must not read past the table)
                    v.x = sqrt_tab[min(b0 + b1, 256u)];
                    v.y = sqrt_tab[min(b1 + b2, 256u)];
                    v.z = sqrt_tab[min(b2 + b3, 256u)];
                    v.w = sqrt_tab[min(b3 + sn, 256u)];
                    if (bx + 4 > RBX) {  // padding columns of the plane
                        if (bx + 0 >= RBX) v.x = 0.f;
                        if (bx + 1 >= RBX) v.y = 0.f;
                        if (bx + 2 >= RBX) v.z = 0.f;
                        if (bx + 3 >= RBX) v.w = 0.f;
                    }
                    *reinterpret_cast<float4 *>(&F[by][bx]) = v;
                }
            }
            __syncwarp();
            const float *base = &F[RY * ly][4 * lx];
#pragma unroll
            for (int r = 0; r < RY + kWinBH - 1; ++r) {
                const float4 f0 = *reinterpret_cast<const float4 *>(base + r * FP);
                const float4 f1 = *reinterpret_cast<const float4 *>(base + r * FP + 4);
                const float4 f2 = *reinterpret_cast<const float4 *>(base + r * FP + 8);
                const float f[12] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w, f2.x, f2.y, f2.z, f2.w};
#pragma unroll
                for (int q = 0; q < RY; ++q) {
                    const int i = r - q;
                    if (i < 0 || i >= kWinBH) continue;
#pragma unroll
                    for (int j = 0; j < kWinBW; ++j)
#pragma unroll
                        for (int x = 0; x < 4; ++x) acc[q][x] = fmaf(f[x + j], w[i][j], acc[q][x]);
                }
            }
        }
        __syncwarp();  // the plane and the LBP chunk are no longer read by this warp
        if (round >= kFirstLbpRound && lane == 0) {
            __threadfence_block();
            if (atomicAdd(&released[buf], 1) % kWarps == kWarps - 1 && round + 2 < kRounds) {
                // last warp out of this buffer: refill it with the chunk two rounds ahead
                __threadfence_block();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issued[buf] += 1;
                mbar_expect_tx(&bars[1 + buf], SH::kLbpBytes);
                tma_load_3d(&lbp[buf][0][0][0], lbp_map, &bars[1 + buf], it.wx0, cy,
                            kWarps * (round + 2) - kHogDim);
            }
        }
    }
    __syncthreads();
    if (*failed) {
        // drain the copies still in flight (bounded) before the CTA leaves
        if (tid == 0) {
            mbar_wait_bounded(&bars[0], 0, kWaitNs);
            for (int b = 0; b < 2; ++b) mbar_wait_bounded(&bars[1 + b], (issued[b] - 1) & 1, kWaitNs);
        }
        return;
    }

    // ---- 4. deterministic cross-warp reduction
    float *red = &feat[0][0][0];  // [kWarps][TH][TW]
#pragma unroll
    for (int q = 0; q < RY; ++q)
#pragma unroll
        for (int x = 0; x < 4; ++x) red[(warp * TH + RY * ly + q) * TW + 4 * lx + x] = acc[q][x];
    __syncthreads();
    for (int i = tid; i < TH * TW; i += kThreads) {
        const int wyl = i / TW, wxl = i - wyl * TW;
        const int wy = it.wy0 + wyl, wx = it.wx0 + wxl;
        if (wy >= L.rows || wx >= L.cols) continue;
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) s += red[k * TH * TW + i];
        scores[L.score_off + (int64_t)wy * L.cols + wx] = s + bias;
    }
}

__device__ __forceinline__ SvmShapeInfo svm_shape_dev(int s) {
    switch (s) {
        case 0: return {S0::TW, S0::TH, 0, 0, 0};
        case 1: return {S1::TW, S1::TH, 0, 0, 0};
        case 2: return {S2::TW, S2::TH, 0, 0, 0};
        case 3: return {S3::TW, S3::TH, 0, 0, 0};
        case 4: return {S4::TW, S4::TH, 0, 0, 0};
        case 5: return {S5::TW, S5::TH, 0, 0, 0};
        default: return {S6::TW, S6::TH, 0, 0, 0};
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    k_svm(const __grid_constant__ SvmMaps maps, const LevelDesc *__restrict__ levels,
          const float *__restrict__ wt, float bias, float clip, float *__restrict__ scores,
          const SvmItem *__restrict__ items, unsigned *__restrict__ err,
          const uint32_t *__restrict__ s_flag) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const SvmItem it = items[blockIdx.x];
    const LevelDesc L = levels[it.level];
    if (s_flag && !s_flag[blockIdx.x]) {
        // sparse path: no kept window in this tile; its windows are not scored
        const SvmShapeInfo sh = svm_shape_dev(it.shape);
        const int tw = sh.tw, th = sh.th;
        for (int i = threadIdx.x; i < tw * th; i += kThreads) {
            const int wy = it.wy0 + i / tw, wx = it.wx0 + i % tw;
            if (wy < L.rows && wx < L.cols) scores[L.score_off + (int64_t)wy * L.cols + wx] = -INFINITY;
        }
        return;
    }
    switch (it.shape) {
        case 0: svm_tile<S0, 4>(it, L, &maps.hog[0], &maps.lbp[0], wt, bias, clip, scores, err, smem); break;
        case 1: svm_tile<S1, 4>(it, L, &maps.hog[1], &maps.lbp[1], wt, bias, clip, scores, err, smem); break;
        case 2: svm_tile<S2, 2>(it, L, &maps.hog[2], &maps.lbp[2], wt, bias, clip, scores, err, smem); break;
        case 3: svm_tile<S3, 2>(it, L, &maps.hog[3], &maps.lbp[3], wt, bias, clip, scores, err, smem); break;
        case 4: svm_tile<S4, 1>(it, L, &maps.hog[4], &maps.lbp[4], wt, bias, clip, scores, err, smem); break;
        case 5: svm_tile<S5, 3>(it, L, &maps.hog[5], &maps.lbp[5], wt, bias, clip, scores, err, smem); break;
        default: svm_tile<S6, 1>(it, L, &maps.hog[6], &maps.lbp[6], wt, bias, clip, scores, err, smem); break;
    }
}

}  // namespace

SvmShapeInfo svm_shape(int s) {
    SvmShapeInfo r{};
    switch (s) {
        case 0: r = {S0::TW, S0::TH, S0::HX, S0::LXB, S0::CR}; break;
        case 1: r = {S1::TW, S1::TH, S1::HX, S1::LXB, S1::CR}; break;
        case 2: r = {S2::TW, S2::TH, S2::HX, S2::LXB, S2::CR}; break;
        case 3: r = {S3::TW, S3::TH, S3::HX, S3::LXB, S3::CR}; break;
        case 4: r = {S4::TW, S4::TH, S4::HX, S4::LXB, S4::CR}; break;
        case 5: r = {S5::TW, S5::TH, S5::HX, S5::LXB, S5::CR}; break;
        default: r = {S6::TW, S6::TH, S6::HX, S6::LXB, S6::CR}; break;
    }
    return r;
}

int svm_lbp_chunk() { return kLbpChunk; }

cudaError_t init_svm() {
    return cudaFuncSetAttribute(k_svm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
}

cudaError_t launch_svm(cudaStream_t s, const CUtensorMap *hog_maps, const CUtensorMap *lbp_maps,
                       const LevelDesc *d_levels, const float *d_w, float bias, float clip,
                       float *scores, const SvmItem *d_items, int n_items, unsigned *d_err,
                       const uint32_t *s_flag) {
    if (n_items <= 0) return cudaSuccess;
    SvmMaps m;
    for (int i = 0; i < kSvmShapes; ++i) {
        m.hog[i] = hog_maps[i];
        m.lbp[i] = lbp_maps[i];
    }
    k_svm<<<n_items, kThreads, kSmemMax, s>>>(m, d_levels, d_w, bias, clip, scores, d_items, d_err, s_flag);
    return cudaGetLastError();
}

}  // namespace pd
