// K5 -- non-maximum suppression (refinement stage of Section 3, run on the
// host in the paper; greedy IoU suppression here, on the device).
//
// One CTA (1024 threads) per frame, or a thread-block cluster of 2-8 CTAs
// that share its collection, large sorts and suppression passes when the
// batch leaves SMs free. A batch of more frames than clusters that fit on the
// GPU at once runs on persistent clusters that draw frames from a ticket
// queue, most candidates first (a counting kernel and a one-CTA sort set the
// order), so the heaviest frames do not start last. Per frame:
//  1. collects every window of every level with score > threshold into a
//     shared-memory key list (64-bit keys: the float score mapped to an
//     order-reversing integer in the high word, level/wy/wx in the low word,
//     so ascending keys = score descending, then level, wy, wx ascending);
//     with a candidate cap above 16,384 the key list lives in the frame's
//     global scratch instead (same steps, slower sort);
//  2. sorts the keys: a bitonic sort in shared memory, or, for caps above
//     16,384, bitonic sorts of 16,384-key chunks in shared memory followed by
//     merge passes over the global key list (each thread merges its slice
//     of outputs after locating it by binary search on the two runs);
//  3. decodes every candidate's box once (exactly rounded float division)
//     into shared memory (over the no longer needed key array, whose keys
//     move to a per-frame global scratch array) or, for very many
//     candidates, into that global scratch;
//  4. walks the candidates in order in batches of the next 64 not yet
//     suppressed: all threads compute the batch's pairwise suppression bits,
//     warp 0 resolves the batch (kept iff no kept earlier member suppresses
//     it), and all threads then suppress the later candidates against the
//     batch's kept members (their boxes staged in shared memory). This
//     takes the same decisions as the one-at-a-time greedy walk (candidates
//     between batch members are already suppressed).
// The IoU test first evaluates the IoU in float. For boxes of this detector
// (width >= 64, height >= 128, coordinates < 8192) the float value is within
// 7e-5 of the exact one: each coordinate sum or difference is off by at most
// 3 float roundings of values < 8192 (1.5e-3 px), which moves the
// intersection by at most (w + h) * 1.5e-3 px^2 and the IoU by at most
// 1.5e-3 * (1/w + 1/h) <= 3.5e-5 through the intersection and as much again
// through the union. So a float IoU more than 2e-4 away from the threshold
// decides; otherwise the IoU is recomputed in double precision with
// explicitly rounded operations (no FMA contraction), which is the exact IEEE
// evaluation of the definition. Decisions are therefore the same as those of
// a plain double-precision implementation, and the slow double path runs
// only for the rare pairs in the band.
#include <cooperative_groups.h>

#include <algorithm>

#include "pd_internal.h"

namespace pd {
namespace {

constexpr int kThreads = 1024;
constexpr int kMaxCandidates = 16384;     // keys + flags + kept list fit in shared memory
constexpr int kMaxCandidatesBig = 65536;  // keys in global scratch
constexpr int kMaxBoxes = 16384;
constexpr int kBatch = 64;                // greedy walk: candidates resolved per block-wide step
constexpr int kGrid = 32;                 // culling grid: kGrid x kGrid cells over the frame
constexpr int kCountBlocks = 32;          // blocks per frame counting its candidates
static_assert(nms_sched_ints(1) == 2 + kCountBlocks,
              "scheduling scratch: the ticket, then per frame its order slot and counts");
constexpr int kOrderMax = 16384;          // frames the order kernel sorts (more: drawn in index order)
static_assert(kThreads == 16 * kBatch, "pairwise matrix: 16 threads per batch member");
static_assert(kThreads == kGrid * kGrid, "one culling cell per thread");

__device__ __forceinline__ unsigned long long make_key(float s, int level, int wy, int wx) {
    const uint32_t u = __float_as_uint(s);
    const uint32_t ord = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return ((unsigned long long)(~ord) << 32) |
           (uint32_t)((level << 24) | (wy << 12) | wx);
}

__device__ __forceinline__ bool suppresses(const float4 &a, const float4 &b, float thr);

__device__ __noinline__ void decode_f64(long long nx, long long ny, int W, int H, int2 d, pd_box &b) {
    b.x = (float)__ddiv_rn((double)nx, (double)d.x);
    b.y = (float)__ddiv_rn((double)ny, (double)d.y);
    b.w = (float)__ddiv_rn(64.0 * W, (double)d.x);
    b.h = (float)__ddiv_rn(128.0 * H, (double)d.y);
}

// Box of a key. x = 8*wx*W/Wk etc. are quotients of integers below 2^24, so
// the correctly rounded float quotient (__fdiv_rn) equals the double quotient
// rounded to float (a quotient of two such integers cannot lie within 2^-49
// of a float rounding midpoint without being on it): no double arithmetic.
__device__ __forceinline__ pd_box decode(unsigned long long key, int W, int H, const int2 *wkhk) {
    const uint32_t hi = (uint32_t)(key >> 32), lo = (uint32_t)key;
    const uint32_t ord = ~hi;
    const uint32_t u = (ord & 0x80000000u) ? (ord ^ 0x80000000u) : ~ord;
    pd_box b;
    b.score = __uint_as_float(u);
    b.level = (int)(lo >> 24);
    b.wy = (int)((lo >> 12) & 4095);
    b.wx = (int)(lo & 4095);
    const int2 d = wkhk[b.level];
    const long long nx = 8LL * b.wx * W, ny = 8LL * b.wy * H;
    if (nx < (1 << 24) && ny < (1 << 24) && 128LL * H < (1 << 24) && 64LL * W < (1 << 24) &&
        d.x < (1 << 24) && d.y < (1 << 24)) {
        b.x = __fdiv_rn((float)nx, (float)d.x);
        b.y = __fdiv_rn((float)ny, (float)d.y);
        b.w = __fdiv_rn((float)(64 * W), (float)d.x);
        b.h = __fdiv_rn((float)(128 * H), (float)d.y);
    } else {  // operands not exact in float: the double quotient, rounded
        decode_f64(nx, ny, W, H, d, b);
    }
    return b;
}

__device__ __forceinline__ double iou(const pd_box &a, const pd_box &b) {
    const double ax0 = a.x, ay0 = a.y, ax1 = __dadd_rn((double)a.x, (double)a.w),
                 ay1 = __dadd_rn((double)a.y, (double)a.h);
    const double bx0 = b.x, by0 = b.y, bx1 = __dadd_rn((double)b.x, (double)b.w),
                 by1 = __dadd_rn((double)b.y, (double)b.h);
    const double iw = __dsub_rn(fmin(ax1, bx1), fmax(ax0, bx0));
    const double ih = __dsub_rn(fmin(ay1, by1), fmax(ay0, by0));
    if (iw <= 0.0 || ih <= 0.0) return 0.0;
    const double inter = __dmul_rn(iw, ih);
    const double ua = __dsub_rn(__dadd_rn(__dmul_rn((double)a.w, (double)a.h),
                                          __dmul_rn((double)b.w, (double)b.h)),
                                inter);
    return __ddiv_rn(inter, ua);
}

// Out of line on purpose: the double-precision path is rare, and inlined it
// would be if-converted and executed for every pair.
__device__ __noinline__ double iou4(const float4 &a, const float4 &b) {
    pd_box x, y;
    x.x = a.x; x.y = a.y; x.w = a.z; x.h = a.w;
    y.x = b.x; y.y = b.y; y.w = b.z; y.h = b.w;
    return iou(x, y);
}

__device__ __forceinline__ bool suppresses(const float4 &a, const float4 &b, float thr) {
    const float iw = fminf(a.x + a.z, b.x + b.z) - fmaxf(a.x, b.x);
    const float ih = fminf(a.y + a.w, b.y + b.w) - fmaxf(a.y, b.y);
    float fi = 0.f;
    if (iw > 0.f && ih > 0.f) {
        const float inter = iw * ih;
        fi = __fdividef(inter, a.z * a.w + b.z * b.w - inter);
    }
    if (fi < thr - 2e-4f) return false;
    if (fi > thr + 2e-4f) return true;
    return iou4(a, b) > (double)thr;
}

constexpr int kSortChunk = 16384;  // keys per shared-memory chunk of the large-cap sort (128 KB)

// Ascending bitonic sort of m = R * kThreads keys in shared memory k, with
// each thread holding the R consecutive keys [tid R, tid R + R) in registers:
// compare-exchange steps of stride j < R run in registers, R <= j < 32 R with
// warp shuffles (the partner is lane ^ j / R, same register), and only
// j >= 32 R through shared memory with a block barrier per step. Same network
// (and result) as bitonic_smem, with log2(m / 32R)-many fewer barriers per
// stage.
// The register and shuffle steps of one stage (stride j and below) for the
// R keys a thread holds, whose global indices are g0 .. g0 + R - 1.
template <int R>
__device__ __forceinline__ void bitonic_reg_steps(unsigned long long (&v)[R], int g0, int j, int len, int lane) {
    for (; j >= R; j >>= 1) {
        // partner: lane ^ (j / R), same register
        const int lm = j / R;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, v[i], lm);
            const bool lower = (lane & lm) == 0, asc = ((g0 + i) & len) == 0;
            v[i] = (lower == asc) ? (v[i] < o ? v[i] : o) : (v[i] < o ? o : v[i]);
        }
    }
    // in registers: strides R/2 .. 1 (compile-time, so v stays in registers);
    // a stage of length len has only the strides below len
#pragma unroll
    for (int jj = R / 2; jj > 0; jj >>= 1) {
        if (jj >= len) continue;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int p = i ^ jj;
            if (p > i) {
                const bool asc = ((g0 + i) & len) == 0;
                const unsigned long long a = v[i], b = v[p];
                const bool sw = (a > b) == asc;
                v[i] = sw ? b : a;
                v[p] = sw ? a : b;
            }
        }
    }
}

// Compare-exchange steps of stride j .. jmin (>= jmin) over k[lo, lo + m) in
// shared memory, one block barrier per step (global indices lo + i).
__device__ __forceinline__ void bitonic_smem_steps(unsigned long long *k, int lo, int m, int j, int jmin, int len,
                                                   int tid) {
    for (; j >= jmin; j >>= 1) {
        for (int i = tid; i < m; i += kThreads) {
            const int ixj = i ^ j;
            if (ixj > i) {
                const unsigned long long a = k[lo + i], b = k[lo + ixj];
                if ((a > b) == (((lo + i) & len) == 0)) {
                    k[lo + i] = b;
                    k[lo + ixj] = a;
                }
            }
        }
        __syncthreads();
    }
}

// Ascending bitonic sort of m = R * kThreads keys k[lo, lo + m) in shared
// memory (as part of a larger network when lo > 0: directions follow the
// global index), each thread holding the R consecutive keys [lo + tid R,
// lo + tid R + R) in registers: compare-exchange steps of stride j < R run in
// registers, R <= j < 32 R with warp shuffles (the partner is lane ^ j / R,
// same register), and only j >= 32 R through shared memory with a block
// barrier per step. Same network (and result) as bitonic_smem, with
// log2(32R)-many fewer barriers per stage. Stages len = 2 .. len_max.
template <int R>
__device__ __forceinline__ void bitonic_hybrid(unsigned long long *k, int lo, int len_max, int tid) {
    constexpr int m = R * kThreads;
    unsigned long long v[R];
    const int base = lo + tid * R, lane = tid & 31;
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = k[base + i];
    for (int len = 2; len <= len_max; len <<= 1) {
        int j = len >> 1;
        if (j >= 32 * R) {
            // large strides: through shared memory
#pragma unroll
            for (int i = 0; i < R; ++i) k[base + i] = v[i];
            __syncthreads();
            bitonic_smem_steps(k, lo, m, j, 32 * R, len, tid);
            j = 16 * R;
#pragma unroll
            for (int i = 0; i < R; ++i) v[i] = k[base + i];
            __syncthreads();  // every thread has read its keys before the next stage writes
        }
        bitonic_reg_steps<R>(v, base, j, len, lane);
    }
#pragma unroll
    for (int i = 0; i < R; ++i) k[base + i] = v[i];
    __syncthreads();
}

// 16,384 keys: each 8,192-key half sorted by the hybrid network (the second
// half descending, as the bitonic network has it), then the last stage's
// large strides in shared memory and its small ones per half in registers.
__device__ __forceinline__ void bitonic_hybrid_16k(unsigned long long *k, int tid) {
    constexpr int R = 8, H = R * kThreads, M = 2 * H;
    bitonic_hybrid<R>(k, 0, H, tid);
    bitonic_hybrid<R>(k, H, H, tid);
    bitonic_smem_steps(k, 0, M, M / 2, 32 * R, M, tid);
    const int lane = tid & 31;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        unsigned long long v[R];
        const int base = h * H + tid * R;
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = k[base + i];
        bitonic_reg_steps<R>(v, base, 16 * R, M, lane);
#pragma unroll
        for (int i = 0; i < R; ++i) k[base + i] = v[i];
    }
    __syncthreads();
}

// Ascending sort of m (a power of two) keys in shared memory: the hybrid
// bitonic network for 1024 <= m <= 16384, the plain one otherwise.
__device__ __forceinline__ void bitonic_sort_smem(unsigned long long *k, int m, int tid);

// Ascending bitonic sort of m (a power of two) keys in shared memory.
__device__ __forceinline__ void bitonic_smem(unsigned long long *k, int m, int tid) {
    for (int len = 2; len <= m; len <<= 1) {
        for (int j = len >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < m; i += kThreads) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const unsigned long long a = k[i], b = k[ixj];
                    if ((a > b) == ((i & len) == 0)) {
                        k[i] = b;
                        k[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__device__ __forceinline__ void bitonic_sort_smem(unsigned long long *k, int m, int tid) {
    switch (m) {
        case 1024: bitonic_hybrid<1>(k, 0, m, tid); break;
        case 2048: bitonic_hybrid<2>(k, 0, m, tid); break;
        case 4096: bitonic_hybrid<4>(k, 0, m, tid); break;
        case 8192: bitonic_hybrid<8>(k, 0, m, tid); break;
        case 16384: bitonic_hybrid_16k(k, tid); break;
        default: bitonic_smem(k, m, tid);
    }
}

// Large caps: keys[0, np) (np a power of two >= n, padded with ~0) sorted
// ascending by the nr CTAs of a frame's cluster (rank = this CTA): chunks of
// up to kSortChunk keys sorted in each CTA's shared memory `sm` (chunk c by
// rank c mod nr), then merge passes doubling the run length, ping-ponging
// through `tmp` (np keys), each of the nr * kThreads threads merging its
// slice of the output; the result ends in keys. csync is the cluster-wide
// barrier (the keys are in global memory).
template <class Sync>
__device__ void sort_large(unsigned long long *keys, unsigned long long *tmp, int np, unsigned long long *sm,
                           int tid, int rank, int nr, Sync &&csync) {
    const int C = np < kSortChunk ? np : kSortChunk;
    for (int c0 = rank * C; c0 < np; c0 += nr * C) {
        for (int i = tid; i < C; i += kThreads) sm[i] = keys[c0 + i];
        __syncthreads();
        bitonic_sort_smem(sm, C, tid);
        for (int i = tid; i < C; i += kThreads) keys[c0 + i] = sm[i];
        __syncthreads();
    }
    csync();
    unsigned long long *src = keys, *dst = tmp;
    const int g = rank * kThreads + tid;
    const int per = np / (nr * kThreads);  // outputs per thread (np >= 2 C here, so per divides every pair)
    for (int w = C; w < np; w <<= 1) {
        const int o0 = g * per;
        const int base = o0 & ~(2 * w - 1), d = o0 - base;
        const unsigned long long *A = src + base, *B = src + base + w;
        // i = keys taken from A among the pair's first d outputs (A first on ties)
        int lo = d > w ? d - w : 0, hi = d < w ? d : w;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (A[mid] <= B[d - 1 - mid])
                lo = mid + 1;
            else
                hi = mid;
        }
        int i = lo, j = d - lo;
        unsigned long long a = i < w ? A[i] : ~0ull, b = j < w ? B[j] : ~0ull;
        for (int k = 0; k < per; ++k) {
            const bool take_a = j >= w || (i < w && a <= b);
            if (take_a) {
                dst[o0 + k] = a;
                ++i;
                a = i < w ? A[i] : ~0ull;
            } else {
                dst[o0 + k] = b;
                ++j;
                b = j < w ? B[j] : ~0ull;
            }
        }
        csync();
        unsigned long long *t = src;
        src = dst;
        dst = t;
    }
    if (src != keys) {
        for (int i = g; i < np; i += nr * kThreads) keys[i] = src[i];
        csync();
    }
}

__global__ void __launch_bounds__(kThreads) k_nms(const FrameDesc *__restrict__ frames,
                                                  const LevelDesc *__restrict__ levels,
                                                  const float *__restrict__ scores, float threshold,
                                                  float iou_thr, int cap, float4 *__restrict__ scratch,
                                                  pd_box *__restrict__ boxes, int max_boxes,
                                                  int32_t *__restrict__ counts, int n_frames,
                                                  const int *__restrict__ order, int *__restrict__ queue) {
    extern __shared__ unsigned long long skeys[];  // [cap_pow2] keys (small caps), cap bytes of flags, kept list
    __shared__ int n_cand;
    __shared__ int2 wkhk[PD_MAX_LEVELS];  // level sizes of this frame
    __shared__ int s_done, s_bx_smem;  // leader's state: walk over; boxes on chip
    __shared__ int s_frame;            // the frame this cluster works on (-1: none left)
    // A frame is one cluster of C CTAs (C = 1 without a cluster launch). Every
    // rank collects a share of the frame's candidates into the leader's list;
    // with large caps (keys in global memory) every rank also sorts and
    // decodes a share. Rank 0, the leader, sorts small lists and picks and
    // resolves the batches exactly as a lone CTA would; every rank takes a
    // 1/C share of each suppression pass, reading the leader's flags and
    // boxes through distributed shared memory. All ranks pass the same
    // cluster barriers: what comes next is read from the leader after one.
    // Without a queue, cluster i takes frame i. With one (more frames than
    // clusters that fit on the GPU), the clusters are persistent: the leader
    // draws the next ticket, takes that frame of `order` (heaviest first)
    // and writes it into every rank's s_frame before the barrier that starts
    // the frame, so all ranks work on the same frame and stop together.
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
    const bool leader = rank == 0;
    const int tid = threadIdx.x;
    int cap_pow2 = 1;
    while (cap_pow2 < cap) cap_pow2 <<= 1;
    const bool big = cap > kMaxCandidates;
    if (queue) cluster.sync();  // every CTA of the cluster runs before the leader writes into it
    for (int pass = 0;; ++pass) {
        if (queue) {
            if (leader && tid == 0) {
                const int t = atomicAdd(queue, 1);
                const int fr = t < n_frames ? (order ? order[t] : t) : -1;
                for (int r = 0; r < C; ++r) *cluster.map_shared_rank(&s_frame, r) = fr;
                n_cand = 0;
            }
        } else if (tid == 0) {
            s_frame = pass == 0 ? (int)(blockIdx.x / C) : -1;
            if (leader) n_cand = 0;
        }
        cluster.sync();  // every rank knows the frame; the leader's counter is zero
        const int f = s_frame;
        if (f < 0) return;  // the same value in every rank: all leave together
        const FrameDesc fd = frames[f];
        float4 *gbx = scratch + (size_t)f * nms_scratch_float4s(cap);
        unsigned long long *keys = big ? reinterpret_cast<unsigned long long *>(gbx + cap) : skeys;
        uint8_t *supp = reinterpret_cast<uint8_t *>(big ? skeys : skeys + cap_pow2);
        const float4 *bx = gbx;
        const unsigned long long *ksrc = keys;
        for (int k = tid; k < fd.n_levels; k += kThreads) {
            const LevelDesc L = levels[fd.first_level + k];
            wkhk[k] = make_int2(L.Wk, L.Hk);
        }
        {
            // every rank scans its share of the windows (every C-th run of
            // kThreads * kUnroll of a level) and appends to the leader's list
            int *cnt = leader ? &n_cand : cluster.map_shared_rank(&n_cand, 0);
            unsigned long long *kw = big ? keys : leader ? skeys : cluster.map_shared_rank(skeys, 0);
            for (int k = 0; k < fd.n_levels; ++k) {
                const LevelDesc L = levels[fd.first_level + k];
                const int n = L.rows * L.cols;
                const float *sc = scores + L.score_off;
                // warp-aggregated appends; kUnroll independent loads per thread are in
                // flight before any of them is used (the scan is latency-bound otherwise)
                constexpr int kUnroll = 8;
                for (int i0 = rank * kThreads * kUnroll; i0 < n; i0 += C * kThreads * kUnroll) {
                    float sv[kUnroll];
    #pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        const int i = i0 + u * kThreads + tid;
                        sv[u] = i < n ? __ldg(sc + i) : 0.f;
                    }
    #pragma unroll
                    for (int u = 0; u < kUnroll; ++u) {
                        const int i = i0 + u * kThreads + tid;
                        if (i0 + u * kThreads >= n) break;  // block-uniform
                        const float s = sv[u];
                        const bool hit = i < n && s > threshold;
                        const unsigned m = __ballot_sync(0xffffffffu, hit);
                        int base = 0;
                        if ((tid & 31) == 0 && m) base = atomicAdd(cnt, __popc(m));
                        base = __shfl_sync(0xffffffffu, base, 0);
                        if (hit) {
                            const int idx = base + __popc(m & ((1u << (tid & 31)) - 1u));
                            if (idx < cap) {
                                const int wy = i / L.cols;
                                kw[idx] = make_key(s, k, wy, i - wy * L.cols);
                            }
                        }
                    }
                }
            }
        }
        cluster.sync();  // every rank's candidates are in
        const int n = leader ? n_cand : *cluster.map_shared_rank(&n_cand, 0);
        if (n > cap) {
            if (leader && tid == 0) {
                counts[2 * f] = 0;
                counts[2 * f + 1] = -n;
            }
            cluster.sync();  // nobody moves on while another rank reads its shared memory
            continue;
        }
        int np = 1;
        while (np < n) np <<= 1;
        if (big) {
            // keys and boxes in global memory: every rank sorts and decodes a share
            for (int i = n + rank * kThreads + tid; i < np; i += C * kThreads) keys[i] = ~0ull;
            cluster.sync();
            // the boxes region (cap float4s) is free until the decode below
            sort_large(keys, reinterpret_cast<unsigned long long *>(gbx), np, skeys, tid, rank, C,
                       [&] { cluster.sync(); });
            for (int i = rank * kThreads + tid; i < n; i += C * kThreads) {
                const pd_box b = decode(keys[i], fd.W, fd.H, wkhk);
                gbx[i] = make_float4(b.x, b.y, b.w, b.h);
            }
            if (leader) {
                for (int i = tid; i < n; i += kThreads) supp[i] = 0;
                if (tid == 0) s_bx_smem = 0;
            }
        } else if (leader) {
            for (int i = n + tid; i < np; i += kThreads) keys[i] = ~0ull;
            __syncthreads();
            bitonic_sort_smem(keys, np, tid);
            for (int i = tid; i < n; i += kThreads) supp[i] = 0;
            __syncthreads();
            // Decoded boxes: in shared memory when they fit in the key region (the
            // keys then move to the global scratch, where only kept ones are read
            // again), otherwise in the global scratch. Each greedy pass reads every
            // remaining box, so keeping them on chip shortens every pass.
            if (2 * n <= cap_pow2) {
                unsigned long long *gkeys = reinterpret_cast<unsigned long long *>(gbx);
                for (int i = tid; i < n; i += kThreads) gkeys[i] = keys[i];
                __syncthreads();
                float4 *sbx = reinterpret_cast<float4 *>(keys);
                for (int i = tid; i < n; i += kThreads) {  // each thread re-reads only its own writes
                    const pd_box b = decode(gkeys[i], fd.W, fd.H, wkhk);
                    sbx[i] = make_float4(b.x, b.y, b.w, b.h);
                }
                bx = sbx;
                ksrc = gkeys;
            } else {
                for (int i = tid; i < n; i += kThreads) {
                    const pd_box b = decode(keys[i], fd.W, fd.H, wkhk);
                    gbx[i] = make_float4(b.x, b.y, b.w, b.h);
                }
            }
            if (tid == 0) s_bx_smem = bx != gbx;
        }
        cluster.sync();  // the leader's candidates, flags and boxes are in place
        // the flags and the boxes of the walk: the leader's own, or read remotely
        uint8_t *fl = leader ? supp : cluster.map_shared_rank(supp, 0);
        if (!leader && *cluster.map_shared_rank(&s_bx_smem, 0))
            bx = cluster.map_shared_rank(reinterpret_cast<float4 *>(keys), 0);
        // Greedy walk in batches. All threads find the next (up to) 64 candidates
        // not yet suppressed, in order (1024 positions per round), and copy their
        // boxes to shared memory; all threads compute the batch's pairwise
        // suppression bits (4 pairs each); warp 0 resolves the members (a member
        // is kept iff no kept member before it suppresses it: the candidates
        // between members are already suppressed) and copies the kept boxes to
        // shared memory; then every thread suppresses the later candidates against
        // them. Same decisions as the sequential definition, with ~64x fewer
        // block-wide barriers.
        //
        // Culling (IoU threshold >= 0.5): if IoU(A, B) > 0.5 then A's centre lies
        // in B (were it outside B on one axis, A and B would overlap on at most
        // half of A's extent there, so inter <= |A| / 2, and inter > (|A| + |B|)
        // / 3 would need |B| < |A| / 2 while inter <= |B| needs |B| > |A| / 2).
        // Each batch records, for every cell of a 32 x 32 grid over the frame,
        // which of its kept boxes cover the cell (one cell of margin for
        // rounding); a candidate is tested only against the kept boxes that cover
        // its centre's cell (no test at all when none does).
        __shared__ int batch[kBatch];
        __shared__ float4 bbx[kBatch], kbx[kBatch];
        __shared__ unsigned long long bcol[kBatch];  // member b: bit a set iff a < b and a suppresses b
        __shared__ int n_batch, n_keep, kept_total, scan_pos;
        __shared__ int wcnt[kThreads / 32];
        __shared__ unsigned long long cmask[kGrid * kGrid];  // culling grid: kept boxes covering each cell
        __shared__ int4 krect[kBatch];                       // kept boxes' cell ranges x0, x1, y0, y1
        int *kept_idx = reinterpret_cast<int *>(supp + ((cap + 15) & ~15));
        const int warp = tid >> 5, lane = tid & 31;
        const bool cull = iou_thr >= 0.5f;
        const float gsx = (float)kGrid / (float)fd.W, gsy = (float)kGrid / (float)fd.H;
        if (tid == 0 && leader) {
            kept_total = 0;
            scan_pos = 0;
        }
        __syncthreads();
        while (true) {
            if (leader) {
                // ---- the next batch: the first kBatch alive candidates at or after scan_pos
                {
                    int cnt = 0, pos = scan_pos;
                    while (cnt < kBatch && pos < n) {
                        const int j = pos + tid;
                        const bool alive = j < n && !fl[j];
                        const unsigned m = __ballot_sync(0xffffffffu, alive);
                        if (lane == 0) wcnt[warp] = __popc(m);
                        __syncthreads();
                        int before = 0, total = 0;
    #pragma unroll 8
                        for (int w = 0; w < kThreads / 32; ++w) {
                            const int c = wcnt[w];
                            before += w < warp ? c : 0;
                            total += c;
                        }
                        const int slot = cnt + before + __popc(m & ((1u << lane) - 1u));
                        if (alive && slot < kBatch) {
                            batch[slot] = j;
                            bbx[slot] = bx[j];
                            if (slot == kBatch - 1) scan_pos = j + 1;  // stop right after the last member
                        }
                        if (cnt + total < kBatch && tid == 0) scan_pos = min(pos + kThreads, n);
                        cnt = min(cnt + total, kBatch);
                        pos += kThreads;
                        __syncthreads();  // wcnt reused by the next round; scan_pos, batch visible
                    }
                    if (tid == 0) n_batch = cnt;
                }
                __syncthreads();
                const int nb = n_batch;
                if (nb > 0) {
                    {
                        // member b = tid / 16 is tested against members a = 4 (tid % 16) .. + 3
                        // (a < b); the 16 threads of a member OR their bits together
                        const int b = tid >> 4, a0 = (tid & 15) * 4;
                        unsigned long long bits = 0;
                        if (b < nb) {
                            const float4 bb = bbx[b];
    #pragma unroll
                            for (int q = 0; q < 4; ++q) {
                                const int a = a0 + q;
                                if (a < b && suppresses(bbx[a], bb, iou_thr)) bits |= 1ull << a;
                            }
                        }
    #pragma unroll
                        for (int o = 8; o > 0; o >>= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
                        if ((tid & 15) == 0 && b < kBatch) bcol[b] = bits;
                    }
                    __syncthreads();
                    if (warp == 0) {
                        // Resolve in rounds: a member is dropped once a kept member
                        // suppresses it, and kept once every member that could suppress it
                        // is decided and none of them is kept. This reaches the in-order
                        // result (induction on the member index) in as many rounds as the
                        // longest chain of suppressions.
                        const unsigned long long all = nb == 64 ? ~0ull : ((1ull << nb) - 1ull);
                        const unsigned long long c0 = bcol[lane], c1 = bcol[lane + 32];
                        unsigned long long keep = 0, decided = ~all;
                        while (decided != ~0ull) {
                            const bool k0 = !((decided >> lane) & 1ull) && !(c0 & keep) && !(c0 & ~decided);
                            const bool d0 = k0 || (!((decided >> lane) & 1ull) && (c0 & keep));
                            const bool k1 = !((decided >> (lane + 32)) & 1ull) && !(c1 & keep) && !(c1 & ~decided);
                            const bool d1 = k1 || (!((decided >> (lane + 32)) & 1ull) && (c1 & keep));
                            keep |= (unsigned long long)__ballot_sync(0xffffffffu, k0) |
                                    ((unsigned long long)__ballot_sync(0xffffffffu, k1) << 32);
                            decided |= (unsigned long long)__ballot_sync(0xffffffffu, d0) |
                                       ((unsigned long long)__ballot_sync(0xffffffffu, d1) << 32);
                        }
                        // the cap on kept boxes: only the first (max_boxes - kept so far) in order
                        const int kt = kept_total;
                        const int room = max_boxes - kt;
                        while (__popcll(keep) > room) keep &= ~(1ull << (63 - __clzll(keep)));
    #pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int m = lane + 32 * h;
                            if (m < nb && ((keep >> m) & 1ull)) {
                                const int r = __popcll(keep & ((1ull << m) - 1ull));
                                kept_idx[kt + r] = batch[m];
                                kbx[r] = bbx[m];
                            }
                        }
                        if (lane == 0) {
                            n_keep = __popcll(keep);
                            kept_total = kt + __popcll(keep);
                        }
                    }
                }
                __syncthreads();
                if (tid == 0) s_done = nb == 0 || kept_total >= max_boxes;
            }
            cluster.sync();  // the batch is resolved (or the walk is over)
            if (leader ? s_done : *cluster.map_shared_rank(&s_done, 0)) break;
            int nk, sp;
            if (leader) {
                nk = n_keep;
                sp = scan_pos;
            } else {  // the kept boxes of the batch and the scan start, from the leader
                nk = *cluster.map_shared_rank(&n_keep, 0);
                sp = *cluster.map_shared_rank(&scan_pos, 0);
                const float4 *lk = cluster.map_shared_rank(kbx, 0);
                for (int k = tid; k < nk; k += kThreads) kbx[k] = lk[k];
                __syncthreads();
            }
            if (cull) {
                // grid cells under each kept box, with one cell of margin; then per
                // cell (one per thread) the set of kept boxes that cover it
                if (tid < nk) {
                    const float4 b = kbx[tid];
                    krect[tid] = make_int4(max((int)floorf(b.x * gsx) - 1, 0),
                                           min((int)floorf((b.x + b.z) * gsx) + 1, kGrid - 1),
                                           max((int)floorf(b.y * gsy) - 1, 0),
                                           min((int)floorf((b.y + b.w) * gsy) + 1, kGrid - 1));
                }
                __syncthreads();
                const int cx = tid & (kGrid - 1), cy = tid / kGrid;
                unsigned long long m = 0ull;
                for (int k = 0; k < nk; ++k) {
                    const int4 r = krect[k];
                    if (cx >= r.x && cx <= r.y && cy >= r.z && cy <= r.w) m |= 1ull << k;
                }
                cmask[tid] = m;
                __syncthreads();
            }
            int j = sp + rank * kThreads + tid;  // this rank's share: every C-th run of kThreads
            float4 bnext = j < n ? bx[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            for (; j < n; j += C * kThreads) {
                // the next box is loaded while this one is tested (global for large caps)
                const float4 bj = bnext;
                if (j + C * kThreads < n) bnext = bx[j + C * kThreads];
                if (fl[j]) continue;
                bool hit = false;
                if (cull) {
                    // only the kept boxes that cover the centre's cell can suppress it
                    const int cx = min(max((int)floorf((bj.x + 0.5f * bj.z) * gsx), 0), kGrid - 1);
                    const int cy = min(max((int)floorf((bj.y + 0.5f * bj.w) * gsy), 0), kGrid - 1);
                    unsigned long long m = cmask[cy * kGrid + cx];
                    while (m && !hit) {
                        const int k = __ffsll((long long)m) - 1;
                        m &= m - 1ull;
                        hit = suppresses(kbx[k], bj, iou_thr);
                    }
                } else {
                    for (int k = 0; k < nk && !hit; k += 4) {
                        // four tests in flight (kept boxes past nk repeat the first one)
                        const bool h0 = suppresses(kbx[k], bj, iou_thr);
                        const bool h1 = suppresses(kbx[k + 1 < nk ? k + 1 : 0], bj, iou_thr);
                        const bool h2 = suppresses(kbx[k + 2 < nk ? k + 2 : 0], bj, iou_thr);
                        const bool h3 = suppresses(kbx[k + 3 < nk ? k + 3 : 0], bj, iou_thr);
                        hit = h0 || h1 || h2 || h3;
                    }
                }
                if (hit) fl[j] = 1;
            }
            cluster.sync();  // every rank's share of the pass is done
        }
        cluster.sync();  // nobody moves on while another rank reads its shared memory
        if (!leader) continue;
        const int kept = kept_total;
        pd_box *out = boxes + (size_t)f * max_boxes;
        for (int k = tid; k < kept; k += kThreads) {
            const int c = kept_idx[k];
            const unsigned long long key = ksrc[c];
            const float4 bc = bx[c];
            const uint32_t hi = (uint32_t)(key >> 32), lo = (uint32_t)key;
            const uint32_t ord = ~hi;
            pd_box b;
            b.x = bc.x;
            b.y = bc.y;
            b.w = bc.z;
            b.h = bc.w;
            b.score = __uint_as_float((ord & 0x80000000u) ? (ord ^ 0x80000000u) : ~ord);
            b.level = (int)(lo >> 24);
            b.wy = (int)((lo >> 12) & 4095);
            b.wx = (int)(lo & 4095);
            out[k] = b;
        }
        if (tid == 0) {
            counts[2 * f] = kept;
            counts[2 * f + 1] = n;
        }
    }
}

// Candidates per frame for the order of the persistent clusters. A frame's
// score maps lie back to back (its levels in order); block x of frame y
// counts the scores above the threshold in every kCountBlocks-th run of
// 4 x 256 of them, four loads in flight per thread.
__global__ void __launch_bounds__(256) k_nms_count(const FrameDesc *__restrict__ frames,
                                                   const LevelDesc *__restrict__ levels,
                                                   const float *__restrict__ scores, float threshold,
                                                   int *__restrict__ partial) {
    const int f = blockIdx.y;
    const FrameDesc fd = frames[f];
    int c = 0;
    if (fd.n_levels > 0) {
        const LevelDesc &a = levels[fd.first_level], &z = levels[fd.first_level + fd.n_levels - 1];
        const float *sc = scores + a.score_off;
        const int n = (int)(z.score_off + (int64_t)z.rows * z.cols - a.score_off);
        constexpr int kU = 4;
        for (int i0 = blockIdx.x * 256 * kU + threadIdx.x; i0 < n; i0 += kCountBlocks * 256 * kU) {
            float v[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) v[u] = i0 + u * 256 < n ? __ldg(sc + i0 + u * 256) : -INFINITY;
#pragma unroll
            for (int u = 0; u < kU; ++u) c += v[u] > threshold;
        }
    }
    c = __reduce_add_sync(0xffffffffu, c);
    __shared__ int ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < 8; ++w) t += ws[w];
        partial[f * kCountBlocks + blockIdx.x] = t;
    }
}

// The frames by candidates, most first (ties: lower frame first), and the
// ticket counter reset. One CTA, a bitonic sort of n_frames keys.
__global__ void __launch_bounds__(kThreads) k_nms_order(const int *__restrict__ partial, int n_frames,
                                                        int *__restrict__ order, int *__restrict__ queue) {
    extern __shared__ unsigned long long okeys[];
    const int tid = threadIdx.x;
    int np = 1;
    while (np < n_frames) np <<= 1;
    for (int i = tid; i < np; i += kThreads) {
        unsigned long long key = ~0ull;
        if (i < n_frames) {
            int c = 0;
            for (int b = 0; b < kCountBlocks; ++b) c += partial[i * kCountBlocks + b];
            key = ((unsigned long long)(uint32_t)(0x7fffffff - c) << 32) | (uint32_t)i;
        }
        okeys[i] = key;
    }
    __syncthreads();
    bitonic_sort_smem(okeys, np, tid);
    __syncthreads();
    for (int t = tid; t < n_frames; t += kThreads) order[t] = (int)(uint32_t)okeys[t];
    if (tid == 0) *queue = 0;
}

size_t nms_smem(int cap, int max_boxes) {
    int p = 1;
    while (p < cap) p <<= 1;
    const size_t keys = cap > kMaxCandidates ? 0 : (size_t)p * sizeof(unsigned long long);
    const size_t walk = keys + (size_t)((cap + 15) & ~15) + 4 * (size_t)max_boxes;
    // large caps: the sort's key chunks use the same shared memory first
    const size_t chunk = cap > kMaxCandidates ? (size_t)kSortChunk * sizeof(unsigned long long) : 0;
    return walk > chunk ? walk : chunk;
}

}  // namespace

namespace {
int g_nms_max_cluster = 1;  // largest cluster of k_nms CTAs the device can hold (1, 2, 4 or 8)
int g_nms_active[4] = {1, 0, 0, 0};  // clusters of 1, 2, 4, 8 CTAs that fit on the device at once

int log2_cluster(int c) { return c == 8 ? 3 : c == 4 ? 2 : c == 2 ? 1 : 0; }
}  // namespace

cudaError_t init_nms(bool occupancy) {
    const int smem = (int)nms_smem(kMaxCandidates, kMaxBoxes);
    cudaError_t e = cudaFuncSetAttribute(k_nms, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_nms_order, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kOrderMax * (int)sizeof(unsigned long long));
    if (e != cudaSuccess || !occupancy) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nms, kThreads, (size_t)smem)) != cudaSuccess)
        return e;
    g_nms_active[0] = std::max(sms * per_sm, 1);
    g_nms_max_cluster = 1;
    for (int c = 8; c >= 2; c >>= 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = (size_t)smem;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = c;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, k_nms, &cfg) == cudaSuccess && n > 0) {
            g_nms_active[log2_cluster(c)] = n;
            g_nms_max_cluster = std::max(g_nms_max_cluster, c);
        } else {
            g_nms_active[log2_cluster(c)] = 0;
            (void)cudaGetLastError();  // a refused size is not an error
        }
    }
    return cudaSuccess;
}

int nms_cluster_for(int n_frames, int sm_count, int max_cand) {
    // the CTAs of a frame share its suppression passes; only while every CTA
    // still gets an SM of its own (one 1024-thread CTA per SM), or, for large
    // candidate lists, while two rounds of clusters cover the frames (the
    // clusters then draw the frames heaviest first)
    const int64_t budget = (max_cand > kMaxCandidates ? 2 : 1) * (int64_t)sm_count;
    int c = 1;
    while (2 * c <= g_nms_max_cluster && g_nms_active[log2_cluster(2 * c)] > 0 && (int64_t)n_frames * 2 * c <= budget)
        c *= 2;
    return c;
}

bool nms_persistent(int n_frames, int cluster) { return n_frames > g_nms_active[log2_cluster(cluster)]; }

int nms_launches(int n_frames, int cluster) {
    if (n_frames <= 0) return 0;
    return nms_persistent(n_frames, cluster) && n_frames <= kOrderMax ? 3 : 1;
}

cudaError_t launch_nms(cudaStream_t s, const FrameDesc *d_frames, const LevelDesc *d_levels,
                       int n_frames, const float *scores, float threshold, float iou,
                       float4 *scratch, int max_cand, pd_box *boxes, int max_boxes,
                       int32_t *counts, int cluster, int *sched) {
    if (n_frames <= 0) return cudaSuccess;
    if (max_cand < 1 || max_cand > kMaxCandidatesBig || max_boxes < 1 || max_boxes > kMaxBoxes ||
        cluster < 1 || cluster > 8 || (cluster & (cluster - 1)))
        return cudaErrorInvalidValue;
    const size_t smem = nms_smem(max_cand, max_boxes);
    // more frames than clusters that fit at once: persistent clusters over a
    // ticket queue, frames ordered by their candidate counts (most first)
    int *queue = nullptr, *order = nullptr;
    int n_clusters = n_frames;
    if (sched && nms_persistent(n_frames, cluster)) {
        queue = sched;
        n_clusters = g_nms_active[log2_cluster(cluster)];
        if (n_frames <= kOrderMax) {
            order = sched + 1;
            int *partial = order + n_frames;
            k_nms_count<<<dim3(kCountBlocks, n_frames), 256, 0, s>>>(d_frames, d_levels, scores, threshold,
                                                                       partial);
            int np = 1;
            while (np < n_frames) np <<= 1;
            k_nms_order<<<1, kThreads, (size_t)np * sizeof(unsigned long long), s>>>(partial, n_frames, order,
                                                                                     queue);
        } else {
            const cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
            if (e != cudaSuccess) return e;
        }
    }
    if (cluster == 1) {
        k_nms<<<n_clusters, kThreads, smem, s>>>(d_frames, d_levels, scores, threshold, iou, max_cand, scratch,
                                                 boxes, max_boxes, counts, n_frames, order, queue);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(n_clusters * cluster);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = cluster;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_nms, d_frames, d_levels, scores, threshold, iou, max_cand, scratch, boxes,
                              max_boxes, counts, n_frames, (const int *)order, queue);
}

// ---------------------------------------------------------------------------
// Allocation-free NMS (pd_nms_noalloc). The kernel above needs device memory
// beyond its inputs and outputs: the frame / level descriptors it reads and
// the per-candidate decoded boxes. For callers that cannot allocate device
// memory, that scratch lives in one file-scope array that every GPU loading
// this library holds until the process exits. A small set-up kernel copies
// the level geometry (passed by value) into it before the unchanged NMS
// kernel runs.
namespace {

constexpr int kNoAllocMaxCandidates = 16384;
constexpr int kNoAllocMaxLevels = PD_MAX_LEVELS;

struct NoAllocScratch {
    FrameDesc frame;
    LevelDesc levels[kNoAllocMaxLevels];
    float4 boxes[kNoAllocMaxCandidates];  // decoded candidate boxes
};

struct NoAllocGeometry {
    int32_t W, H, n_levels, pad;
    int32_t Wk[kNoAllocMaxLevels], Hk[kNoAllocMaxLevels];
    int32_t rows[kNoAllocMaxLevels], cols[kNoAllocMaxLevels];
    int64_t score_off[kNoAllocMaxLevels];
};

}  // namespace

static __device__ __align__(256) unsigned char g_nms_scratch[sizeof(NoAllocScratch)];

namespace {

__global__ void k_nms_noalloc_setup(const __grid_constant__ NoAllocGeometry g, NoAllocScratch *s) {
    if (threadIdx.x == 0) {
        FrameDesc f{};
        f.W = g.W;
        f.H = g.H;
        f.first_level = 0;
        f.n_levels = g.n_levels;
        s->frame = f;
    }
    for (int k = threadIdx.x; k < g.n_levels; k += blockDim.x) {
        LevelDesc L{};
        L.W = g.W;
        L.H = g.H;
        L.Wk = g.Wk[k];
        L.Hk = g.Hk[k];
        L.rows = g.rows[k];
        L.cols = g.cols[k];
        L.score_off = g.score_off[k];
        s->levels[k] = L;
    }
}

}  // namespace

}  // namespace pd

extern "C" int pd_nms_noalloc(void *stream, const float *d_scores, int n_levels, const int32_t *rows,
                              const int32_t *cols, const int32_t *Wk, const int32_t *Hk, int W, int H,
                              float threshold, float nms_iou, int max_candidates, pd_box *d_boxes,
                              int max_boxes, int32_t *d_counts) {
    using namespace pd;
    if (!d_scores || !rows || !cols || !Wk || !Hk || !d_boxes || !d_counts || n_levels < 0 ||
        n_levels > kNoAllocMaxLevels || max_candidates < 1 || max_candidates > kNoAllocMaxCandidates ||
        max_boxes < 1 || max_boxes > kMaxBoxes || W < 1 || H < 1 || !(nms_iou >= 0.f))
        return PD_EINVAL;
    NoAllocGeometry g{};
    g.W = W;
    g.H = H;
    g.n_levels = n_levels;
    int64_t off = 0;
    for (int k = 0; k < n_levels; ++k) {
        if (rows[k] < 0 || cols[k] < 0 || rows[k] > 4096 || cols[k] > 4096 || Wk[k] < 1 || Hk[k] < 1)
            return PD_EINVAL;
        g.Wk[k] = Wk[k];
        g.Hk[k] = Hk[k];
        g.rows[k] = rows[k];
        g.cols[k] = cols[k];
        g.score_off[k] = off;
        off += (int64_t)rows[k] * cols[k];
    }
    // Every call: the current device's address of the scratch array (the
    // host-side symbol is only a stand-in) and the kernel's shared-memory
    // opt-in. Both are cheap host calls; doing them each time keeps the
    // address right after a device reset or on a new primary context.
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_nms_scratch) != cudaSuccess || !p) return PD_ECUDA;
    if (init_nms(false) != cudaSuccess) return PD_ECUDA;  // one cluster-less CTA: no occupancy table
    NoAllocScratch *scratch = reinterpret_cast<NoAllocScratch *>(p);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_nms_noalloc_setup<<<1, 128, 0, s>>>(g, scratch);
    if (cudaGetLastError() != cudaSuccess) return PD_ECUDA;
    if (launch_nms(s, &scratch->frame, scratch->levels, 1, d_scores, threshold, nms_iou, scratch->boxes,
                   max_candidates, d_boxes, max_boxes, d_counts) != cudaSuccess)
        return PD_ECUDA;
    return PD_OK;
}
