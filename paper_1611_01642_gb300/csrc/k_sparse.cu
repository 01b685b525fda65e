// Sparse path: which tiles the learned proposal keeps.
//
// A window is kept when its keep-logit exceeds the keep threshold. One warp
// per window tile of the FP32 K4's plan decides whether the tile holds a
// kept window. For the FP32 K4 a kept tile marks every K2+K3 cell tile its
// cell region overlaps, and K4 computes the kept tiles (their windows are all
// scored exactly; the others get -inf, which never becomes an NMS candidate).
// For the tensor-core K4 (per_window) each kept window marks only the cell
// tiles under its own 8 x 16 cells, and K4 scores every window whose cells
// were all computed. Flags are plain stores of 1, so they do not depend on
// the order of the warps. Either way every kept window is scored exactly, so
// the recall is at least that of the window-level proposal.
#include "pd_internal.h"

namespace pd {
namespace {

__constant__ int2 kShapeDims[kSvmShapes] = {{32, 16}, {64, 8}, {32, 8}, {64, 4}, {64, 2}, {32, 12}, {32, 4}};

__global__ void __launch_bounds__(256) k_proposal_flags(const LevelDesc *__restrict__ levels,
                                                        const SvmItem *__restrict__ s_items, int n_items,
                                                        const float *__restrict__ logits, float tau,
                                                        uint32_t *__restrict__ s_flag, uint32_t *__restrict__ c_flag,
                                                        int per_window) {
    const int lane = threadIdx.x & 31;
    const int item = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (item >= n_items) return;
    const SvmItem it = s_items[item];
    const LevelDesc L = levels[it.level];
    const int2 d = kShapeDims[it.shape];
    bool any = false;
    for (int i = lane; i < d.x * d.y; i += 32) {
        const int wy = it.wy0 + i / d.x, wx = it.wx0 + i % d.x;
        if (wy < L.rows && wx < L.cols && logits[L.score_off + (int64_t)wy * L.cols + wx] > tau) {
            any = true;
            if (per_window)  // cell tiles under cell rows wy .. wy+15, columns wx .. wx+7
                for (int ty = wy / kCellTH; ty <= (wy + kWinBH) / kCellTH; ++ty)
                    for (int tx = wx / kCellTW; tx <= (wx + kWinBW) / kCellTW; ++tx)
                        c_flag[L.citem0 + ty * L.ctx + tx] = 1u;
        }
    }
    any = __any_sync(0xffffffffu, any);
    if (lane == 0) s_flag[item] = any ? 1u : 0u;
    if (!any || per_window) return;
    // cells of the tile's windows: rows wy0 .. wy0+TH+14, columns wx0 .. wx0+TW+6
    const int cy_end = min(it.wy0 + d.y + kWinBH, L.Hc), cx_end = min(it.wx0 + d.x + kWinBW, L.Wc);
    const int ty0 = it.wy0 / kCellTH, ty1 = (cy_end - 1) / kCellTH;
    const int tx0 = it.wx0 / kCellTW, tx1 = (cx_end - 1) / kCellTW;
    const int ntx = tx1 - tx0 + 1, n = (ty1 - ty0 + 1) * ntx;
    for (int k = lane; k < n; k += 32) {
        const int ty = ty0 + k / ntx, tx = tx0 + k % ntx;
        c_flag[L.citem0 + ty * L.ctx + tx] = 1u;
    }
}

}  // namespace

cudaError_t launch_proposal_flags(cudaStream_t s, const LevelDesc *d_levels, const SvmItem *d_items, int n_items,
                                  const float *logits, float tau, uint32_t *s_flag, uint32_t *c_flag,
                                  bool per_window) {
    if (n_items <= 0) return cudaSuccess;
    k_proposal_flags<<<(n_items + 7) / 8, 256, 0, s>>>(d_levels, d_items, n_items, logits, tau, s_flag, c_flag,
                                                       per_window ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace pd
