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
// One CTA (8 warps) computes a 32 x 16 tile of windows of one level:
//  1. one thread issues two TMA loads (cp.async.bulk.tensor.3d) of the
//     tile's cell region -- 31 rows x 40 columns of the 9 HOG planes (f32)
//     and 31 x 48 of the 59 LBP planes (u8) -- completing on one mbarrier
//     (bounded wait: a 1 s limit, then the error word is set);
//  2. the CTA computes the two L2-Hys scale factors of each of the region's
//     30 x 38 blocks;
//  3. the 95 channels are split over the 8 warps (channel t goes to warp
//     t % 8). For each of its channels a warp writes the channel's feature
//     plane for the whole region into its own shared-memory slice, loads the
//     channel's 15x7 template slice into registers (warp-uniform loads) and
//     runs the correlation: each lane owns a 4 x 4 block of windows and, for
//     each of the 18 block rows it touches, loads 12 consecutive features
//     with three 128-bit shared loads and issues up to 4 x 7 x 4 FMAs per
//     kernel row. All loop indices are compile-time, so the template stays
//     in registers.
//  4. the 8 per-warp partial sums are added in warp order (deterministic),
//     the bias is added and the valid windows are stored.
#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kWarps = 8;
constexpr int kThreads = 32 * kWarps;
constexpr int kTW = kSvmTW;             // 32 windows
constexpr int kTH = kSvmTH;             // 16 windows
constexpr int kRegBY = kTH + kWinBH - 1;  // 30 block rows
constexpr int kRegBX = kTW + kWinBW - 1;  // 38 block columns
constexpr int kCellRows = kRegBY + 1;     // 31
constexpr int kHogBoxX = 40;              // >= 39 cell columns, 16-byte multiple
constexpr int kLbpBoxX = 48;              // >= 39 cell columns, 16-byte multiple
constexpr int kFP = 40;                   // feature-plane pitch (floats)

struct __align__(128) SvmSmem {
    alignas(128) float hog[kHogBins][kCellRows][kHogBoxX];    // 44,640 B (TMA destination)
    alignas(128) uint8_t lbp[kLbpBins][kCellRows][kLbpBoxX];  // 87,792 B (TMA destination)
    alignas(16) float inv1[kRegBY][kFP];                      // 1/sqrt(|v|^2 + 1)
    alignas(16) float inv2[kRegBY][kFP];                      // 1/sqrt(|u|^2 + 1e-6)
    alignas(16) float feat[kWarps][kRegBY][kFP];  // per-warp channel plane (also the reduction buffer)
    float sqrt_tab[260];                          // sqrt(c/256), c = 0..256
    unsigned long long bar;
    int ok;
};
static_assert(sizeof(float) * kWarps * kRegBY * kFP >= sizeof(float) * kWarps * kTW * kTH,
              "reduction buffer must fit in the feature planes");
constexpr uint32_t kHogBytes = sizeof(float) * kHogBins * kCellRows * kHogBoxX;
constexpr uint32_t kLbpBytes = kLbpBins * kCellRows * kLbpBoxX;

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

__global__ void __launch_bounds__(kThreads, 1)
    k_svm(const __grid_constant__ CUtensorMap hog_map, const __grid_constant__ CUtensorMap lbp_map,
          const LevelDesc *__restrict__ levels, const float *__restrict__ wt, float bias,
          float clip, float *__restrict__ scores, const SvmItem *__restrict__ items,
          unsigned *__restrict__ err) {
    extern __shared__ unsigned char smem_raw[];
    SvmSmem &S = *reinterpret_cast<SvmSmem *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const SvmItem it = items[blockIdx.x];
    const LevelDesc L = levels[it.level];

    if (tid == 0) {
        mbar_init(&S.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&S.bar, kHogBytes + kLbpBytes);
        tma_load_3d(&S.hog[0][0][0], &hog_map, &S.bar, it.wx0, L.cell_row + it.wy0, 0);
        tma_load_3d(&S.lbp[0][0][0], &lbp_map, &S.bar, it.wx0, L.cell_row + it.wy0, 0);
    }
    for (int c = tid; c <= 256; c += kThreads) S.sqrt_tab[c] = sqrtf((float)c * (1.0f / 256.0f));
    // One thread waits (1 s limit) so that the outcome is CTA-uniform.
    if (tid == 0) {
        int ok = mbar_wait_bounded(&S.bar, 0, 1000000000ull) ? 1 : 0;
        if (!ok) {
            // The copies never completed: flag it and give them one more
            // bounded chance to land, so that no TMA write outlives the CTA.
            atomicOr(err, kErrTimeout);
            mbar_wait_bounded(&S.bar, 0, 1000000000ull);
        }
        S.ok = ok;
    }
    __syncthreads();
    if (!S.ok) return;
    // The phase is complete, so this returns at once; it makes every thread
    // observe the completion (and so acquire the TMA-written data).
    if (!mbar_wait_bounded(&S.bar, 0, 1000000000ull)) atomicOr(err, kErrTimeout);

    // ---- 2. L2-Hys scale factors of every block of the region
    for (int i = tid; i < kRegBY * kFP; i += kThreads) {
        const int by = i / kFP, bx = i - by * kFP;
        float i1 = 0.f, i2 = 0.f;
        if (bx < kRegBX) {
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int b = 0; b < kHogBins; ++b) {
                    const float v = S.hog[b][by + (q >> 1)][bx + (q & 1)];
                    s = fmaf(v, v, s);
                }
            i1 = 1.0f / sqrtf(s + 1.0f);
            float s2 = 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int b = 0; b < kHogBins; ++b) {
                    const float u = fminf(S.hog[b][by + (q >> 1)][bx + (q & 1)] * i1, clip);
                    s2 = fmaf(u, u, s2);
                }
            i2 = 1.0f / sqrtf(s2 + 1e-6f);
        }
        S.inv1[by][bx] = i1;
        S.inv2[by][bx] = i2;
    }
    __syncthreads();

    // ---- 3. per-warp channels
    const int lx = lane & 7, ly = lane >> 3;
    float acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int x = 0; x < 4; ++x) acc[q][x] = 0.f;
    float(*F)[kFP] = S.feat[warp];

    for (int t = warp; t < kFeat; t += kWarps) {
        // feature plane of channel t over the region
        if (t < kHogDim) {
            const int q = t / kHogBins, b = t - q * kHogBins;
            const int oy = q >> 1, ox = q & 1;
            for (int i = lane; i < kRegBY * kFP; i += 32) {
                const int by = i / kFP, bx = i - by * kFP;
                float v = 0.f;
                if (bx < kRegBX)
                    v = fminf(S.hog[b][by + oy][bx + ox] * S.inv1[by][bx], clip) * S.inv2[by][bx];
                F[by][bx] = v;
            }
        } else {
            const int l = t - kHogDim;
            for (int i = lane; i < kRegBY * kFP; i += 32) {
                const int by = i / kFP, bx = i - by * kFP;
                float v = 0.f;
                if (bx < kRegBX) {
                    const int c = S.lbp[l][by][bx] + S.lbp[l][by][bx + 1] + S.lbp[l][by + 1][bx] +
                                  S.lbp[l][by + 1][bx + 1];
                    v = S.sqrt_tab[c];
                }
                F[by][bx] = v;
            }
        }
        // template slice of channel t: w[t][i][0..7] (warp-uniform loads)
        float w[kWinBH][kWinBW];
        const float4 *wp = reinterpret_cast<const float4 *>(wt + (size_t)t * kWinBH * kWPad);
#pragma unroll
        for (int i = 0; i < kWinBH; ++i) {
            const float4 a = __ldg(wp + 2 * i), c = __ldg(wp + 2 * i + 1);
            w[i][0] = a.x; w[i][1] = a.y; w[i][2] = a.z; w[i][3] = a.w;
            w[i][4] = c.x; w[i][5] = c.y; w[i][6] = c.z;
        }
        __syncwarp();
        const float *base = &F[4 * ly][4 * lx];
#pragma unroll
        for (int r = 0; r < 4 + kWinBH - 1; ++r) {
            const float4 f0 = *reinterpret_cast<const float4 *>(base + r * kFP);
            const float4 f1 = *reinterpret_cast<const float4 *>(base + r * kFP + 4);
            const float4 f2 = *reinterpret_cast<const float4 *>(base + r * kFP + 8);
            const float f[12] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w, f2.x, f2.y, f2.z, f2.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = r - q;
                if (i < 0 || i >= kWinBH) continue;
#pragma unroll
                for (int j = 0; j < kWinBW; ++j)
#pragma unroll
                    for (int x = 0; x < 4; ++x) acc[q][x] = fmaf(f[x + j], w[i][j], acc[q][x]);
            }
        }
        __syncwarp();
    }
    __syncthreads();

    // ---- 4. deterministic cross-warp reduction
    float *red = &S.feat[0][0][0];  // [kWarps][kTH][kTW]
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int x = 0; x < 4; ++x) red[(warp * kTH + 4 * ly + q) * kTW + 4 * lx + x] = acc[q][x];
    __syncthreads();
    for (int i = tid; i < kTH * kTW; i += kThreads) {
        const int wyl = i / kTW, wxl = i - wyl * kTW;
        const int wy = it.wy0 + wyl, wx = it.wx0 + wxl;
        if (wy >= L.rows || wx >= L.cols) continue;
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) s += red[k * kTH * kTW + i];
        scores[L.score_off + (int64_t)wy * L.cols + wx] = s + bias;
    }
}

}  // namespace

cudaError_t init_svm() {
    return cudaFuncSetAttribute(k_svm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(SvmSmem) + 128);
}

cudaError_t launch_svm(cudaStream_t s, const CUtensorMap *hog_map, const CUtensorMap *lbp_map,
                       const LevelDesc *d_levels, int32_t atlas_pitch, const float *d_w, float bias,
                       float clip, float *scores, const SvmItem *d_items, int n_items,
                       unsigned *d_err) {
    (void)atlas_pitch;
    if (n_items <= 0) return cudaSuccess;
    k_svm<<<n_items, kThreads, sizeof(SvmSmem) + 128, s>>>(*hog_map, *lbp_map, d_levels, d_w, bias,
                                                          clip, scores, d_items, d_err);
    return cudaGetLastError();
}

}  // namespace pd
