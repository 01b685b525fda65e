// Host runtime of the detector library: parameter checks, batch planning,
// the device arena, TMA tensor maps and the C ABI of include/pd.h.
//
// A batch plan lists, for every frame, its pyramid levels (Section 4.4) and
// lays out every intermediate in one device arena allocated at pd_create:
//   pyramid images      u8, level k of frame f at img_off, pitch round16(Wk)
//   HOG cell atlas      f32 [9][atlas_rows][P]
//   LBP cell atlas      u8  [59][atlas_rows][P]   (P = round16(max cells_x))
//   score maps          f32, map of (f, k) at score_off, rows x cols
//   boxes / counts      per frame
// Every level owns a band of atlas rows, so one pair of tensor maps (encoded
// once) covers all levels of all frames. The plan also carries the work
// lists of the four kernels and the Q11 resample tables; it is packed into a
// pinned host buffer and sent with one asynchronous copy per pd_detect.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "pd_internal.h"

using namespace pd;

namespace {

constexpr int64_t kAlign = 256;
// relative time of one K4 tile per shape (model; the autotuner replaces it)
// Relative per-tile costs of the dense path, from timings on GB300: a tile
// costs about 1 (512 windows) or 0.6 (256 windows); the three small shapes
// are priced so that dense plans never take them (measured whole-plan times
// were no better with them); the sparse path, where small tiles skip more,
// prices them itself.
const float kDefaultTileCost[kSvmShapes] = {1.0f, 1.0f, 0.6f, 0.6f, 1.0f, 1.0f, 1.0f};
// Sparse path: a tile is computed only if it holds a kept window, so narrow
// tiles skip more; the 64-wide shapes and the smallest ones lost on GB300
// (whole-path timings of the proposal workload).
const float kSparseTileCost[kSvmShapes] = {1.0f, 1e3f, 0.6f, 1e3f, 1e3f, 0.82f, 1e3f};

int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// Cell features a pipeline uses (Section 4.1: HOG-SVM, LBP-SVM or HOGLBP-SVM).
// Per-block HOG (Algorithm 5 read per block) adds kFeatHogBlock.
int features_of(int32_t flags) {
    const int blk = (flags & PD_FLAG_HOG_PER_BLOCK) ? kFeatHogBlock : 0;
    if (flags & PD_FLAG_HOG_ONLY) return kFeatHog | blk;
    if (flags & PD_FLAG_LBP_ONLY) return kFeatLbp;
    return kFeatHog | kFeatLbp | blk;
}

// HOG planes of the cell atlas: 9 bins, or 4 places x 9 bins per cell.
int hog_planes_of(int32_t flags) { return (flags & PD_FLAG_HOG_PER_BLOCK) ? 4 * kHogBins : kHogBins; }

struct Plan {
    std::vector<FrameDesc> frames;
    std::vector<LevelDesc> levels;
    std::vector<ResizeItem> r_items;
    std::vector<CellItem> c_items;
    std::vector<StripItem> strips;
    std::vector<SvmItem> s_items;
    std::vector<TcItem> t_items;
    std::vector<CnnItem> cnn_items;
    std::vector<int32_t> tabs;
    std::vector<int32_t> tc_widths;  // tensor-core K4: level widths (cells) with a pair of maps
    int tc_rows = kTcChunk;  // tensor-core K4 window rows per item (tuning; kept by clear())
    int64_t pyr_bytes = 0;
    int64_t score_floats = 0;
    int32_t atlas_rows = 0;
    int32_t max_wc = 0;
    // frames of equal size share their Q11 tables: (W, H) -> first level index
    std::map<std::pair<int, int>, int> tab_owner;

    void clear() {
        tab_owner.clear();
        frames.clear();
        levels.clear();
        r_items.clear();
        c_items.clear();
        strips.clear();
        s_items.clear();
        t_items.clear();
        cnn_items.clear();
        tabs.clear();
        tc_widths.clear();
        pyr_bytes = score_floats = 0;
        atlas_rows = max_wc = 0;
    }
};

// Byte offsets of the plan's sections inside the packed descriptor block.
struct Packed {
    int64_t frames, levels, r_items, c_items, strips, s_items, t_items, cnn_items, tabs, tmaps, tc_maps, total;
};

Packed pack_layout(const Plan &p) {
    Packed o;
    int64_t off = 0;
    auto take = [&](int64_t bytes) {
        int64_t at = off;
        off = round_up(off + bytes, 16);
        return at;
    };
    o.frames = take((int64_t)p.frames.size() * sizeof(FrameDesc));
    o.levels = take((int64_t)p.levels.size() * sizeof(LevelDesc));
    o.r_items = take((int64_t)p.r_items.size() * sizeof(ResizeItem));
    o.c_items = take((int64_t)p.c_items.size() * sizeof(CellItem));
    o.strips = take((int64_t)p.strips.size() * sizeof(StripItem));
    o.s_items = take((int64_t)p.s_items.size() * sizeof(SvmItem));
    o.t_items = take((int64_t)p.t_items.size() * sizeof(TcItem));
    o.cnn_items = take((int64_t)p.cnn_items.size() * sizeof(CnnItem));
    o.tabs = take((int64_t)p.tabs.size() * sizeof(int32_t));
    off = round_up(off, 64);  // tensor maps: 64-byte aligned
    o.tmaps = take(p.cnn_items.empty() ? 0 : (int64_t)p.levels.size() * sizeof(CUtensorMap));
    off = round_up(off, 64);
    o.tc_maps = take(2 * (int64_t)p.tc_widths.size() * sizeof(CUtensorMap));
    o.total = off;
    return o;
}

// Q11 source index and weight of destination coordinate x for a resize of
// n source samples to m: round-half-up of ((x + 0.5) * n / m - 0.5) * 2048,
// clamped to the first / last sample. Packed as index << 11 | weight.
int32_t q11_entry(int x, int n, int m) {
    const int64_t num = ((int64_t)(2 * x + 1) * n - m) * 2048 + m;
    const int64_t den = 2 * (int64_t)m;
    int64_t q = num / den;
    if (num % den != 0 && num < 0) q -= 1;
    int32_t idx, a;
    if (q < 0) {
        idx = 0;
        a = 0;
    } else {
        idx = (int32_t)(q >> 11);
        a = (int32_t)(q & 2047);
        if (idx >= n - 1) {
            idx = n - 1;
            a = 0;
        }
    }
    return (idx << 11) | a;
}

// Pyramid level sizes: the `upscale` upsampled levels k = -upscale .. -1
// first (most upsampled first), then k = 0, 1, ... while a 64x128 window
// fits; level k is floor(W / factor^k + 1e-9) x floor(H / factor^k + 1e-9).
int level_sizes(int W, int H, double factor, int upscale, int max_levels, int32_t *Wk, int32_t *Hk) {
    if (!(factor > 1.0) || W < 0 || H < 0 || upscale < 0) return PD_EINVAL;
    int n = 0;
    for (int k = -upscale; k < 0 && n < max_levels; ++k) {
        const double s = std::pow(factor, (double)k);
        const int wk = (int)std::floor((double)W / s + 1e-9);
        const int hk = (int)std::floor((double)H / s + 1e-9);
        if (wk < 64 || hk < 128) continue;
        Wk[n] = wk;
        Hk[n] = hk;
        ++n;
    }
    for (int k = 0; n < max_levels; ++k) {
        const double s = std::pow(factor, (double)k);
        const int wk = (int)std::floor((double)W / s + 1e-9);
        const int hk = (int)std::floor((double)H / s + 1e-9);
        if (wk < 64 || hk < 128) break;
        Wk[n] = wk;
        Hk[n] = hk;
        ++n;
    }
    return n;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

}  // namespace

namespace pd {

void build_lbp_bin_table(uint8_t table[256]) {
    // uniform = at most two 0/1 transitions around the 8-bit circle; uniform
    // codes are numbered in increasing order, all others share the last bin
    int rank = 0;
    for (int c = 0; c < 256; ++c) {
        const int rot = ((c >> 1) | (c << 7)) & 255;
        const int transitions = __builtin_popcount((unsigned)(c ^ rot));
        table[c] = transitions <= 2 ? (uint8_t)rank++ : (uint8_t)(kLbpBins - 1);
    }
}

int encode_plane_map(CUtensorMap *map, void *base, CUtensorMapDataType dtype, int elem_bytes,
                     int64_t pitch, int64_t rows, int64_t planes, int64_t plane_stride_elems,
                     uint32_t box_x, uint32_t box_y, uint32_t box_planes, int64_t width) {
    auto fn = get_encode();
    if (!fn) return PD_ECUDA;
    cuuint64_t dims[3] = {(cuuint64_t)(width > 0 ? width : pitch), (cuuint64_t)rows, (cuuint64_t)planes};
    cuuint64_t strides[2] = {(cuuint64_t)(pitch * elem_bytes), (cuuint64_t)(plane_stride_elems * elem_bytes)};
    cuuint32_t box[3] = {box_x, box_y, box_planes};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, dtype, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? PD_OK : PD_ECUDA;
}

// 2D map over one pyramid level (u8 [Hk][pitch]) for the proposal network's
// input tiles.
int encode_level_map(CUtensorMap *map, const uint8_t *base, int Wk, int Hk, int pitch) {
    auto fn = get_encode();
    if (!fn) return PD_ECUDA;
    cuuint64_t dims[2] = {(cuuint64_t)Wk, (cuuint64_t)Hk};
    cuuint64_t strides[1] = {(cuuint64_t)pitch};
    cuuint32_t box[2] = {(cuuint32_t)kCnnBoxW, (cuuint32_t)kCnnBoxH};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? PD_OK : PD_ECUDA;
}

}  // namespace pd

struct pd_handle {
    pd_params p{};
    int device = 0;
    float bias = 0.f;
    // arena
    unsigned char *arena = nullptr;
    size_t arena_bytes = 0;
    float *d_w = nullptr;          // [95][15][8]
    uint8_t *d_lbp_map = nullptr;  // [256]
    unsigned char *d_desc = nullptr;
    int64_t desc_cap = 0;
    uint8_t *d_pyr = nullptr;
    int64_t pyr_cap = 0;
    CellAtlas atlas{};
    float *d_scores = nullptr;
    int64_t score_cap = 0;
    pd_box *d_boxes = nullptr;
    int32_t *d_counts = nullptr;  // [2 * max_frames]
    float4 *d_nms_scratch = nullptr;  // [max_frames][max_candidates] decoded candidate boxes
    unsigned *d_err = nullptr;
    uint8_t *d_frames = nullptr;  // host-input staging for pd_detect_host
    int64_t frames_cap = 0;
    int64_t level_cap = 0, r_cap = 0, c_cap = 0, s_cap = 0, tab_cap = 0;
    // pinned host
    unsigned char *h_desc = nullptr;
    pd_box *h_boxes = nullptr;     // mapped: written by the NMS kernel
    int32_t *h_counts = nullptr;   // mapped: [2 * max_frames] kept / candidates
    pd_box *m_boxes = nullptr;     // device views of the two mapped buffers
    int32_t *m_counts = nullptr;
    unsigned *h_err = nullptr;
    cudaEvent_t desc_done = nullptr;
    cudaEvent_t stage_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool timed = false;
    // learned proposal: parameters (fp32 master + Adam state + rounded copy),
    // inference fragments, per-cell head values, window logits
    float *cnn = nullptr;           // [5][kCnnParams]: master, m, v, grad, rounded
    float *in_tab = nullptr;        // [256]
    uint32_t *w2frag = nullptr;     // [2304]
    float *hmap = nullptr;          // one f32 plane over the cell atlas
    float *logits = nullptr;        // window logits, score-map layout
    bool cnn_loaded = false, frag_stale = false;
    bool proposal = false;          // sparse path on
    bool ran_proposal = false;      // the last pd_detect ran the sparse path
    float tau = 0.f;                // keep-logit threshold
    uint32_t *s_flag = nullptr;     // per K4 item: holds a kept window
    uint32_t *c_flag = nullptr;     // per K2+K3 item: needed by a kept tile
    int64_t flag_cap = 0;
    int adam_t = 0;
    // training workspace (allocated on first use, grown with the batch)
    unsigned char *train_ws = nullptr;
    unsigned char *scheme_ws = nullptr;  // scratch of the paper's kernel schemes (grown on demand)
    size_t scheme_ws_bytes = 0;
    size_t train_ws_bytes = 0;
    int train_levels = 0;
    float *train_loss_ptr = nullptr;
    // tensor maps over the atlases, one pair per K4 tile shape
    CUtensorMap hog_map[kSvmShapes]{}, lbp_map[kSvmShapes]{};
    CUtensorMap tc_hog_map{}, tc_lbp_map{};  // the same planes for the tensor-core K4
    int *d_queue = nullptr;                  // [2]: K4's and K2+K3's item counters (zeroed before each launch)
    int *d_nms_sched = nullptr;              // NMS ticket counter, frame order and candidate counts
    int sm_count = 1;
    float tile_cost[kSvmShapes] = {kDefaultTileCost[0], kDefaultTileCost[1], kDefaultTileCost[2],
                                   kDefaultTileCost[3], kDefaultTileCost[4], kDefaultTileCost[5],
                                   kDefaultTileCost[6]};
    pd_tuning tuning{8, kTcChunk};  // launch shapes of the default path (autotuner output)
    // last batch
    Plan plan;
    // cached plan + captured graph for a repeated batch shape
    std::vector<int32_t> sig;        // n_frames, then (W, H, pitch) per frame
    bool cache_valid = false;        // plan + full descriptors on the device match `sig`
    Packed packed{};
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t graph_done = nullptr;
    cudaStream_t stream = nullptr;
    bool detected = false, synced = false;
    int last_launches = 0;
    std::string err;
};

namespace {

int fail(pd_handle *h, int code, const char *fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return code;
}

#define PD_CUDA(h, call)                                                                     \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) return fail((h), PD_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// K4 tiling of a rows x cols score map: bands of rows, each band one tile
// height, each band a sequence of tiles of that height whose widths may
// differ; chosen by dynamic programming to minimise the summed per-tile
// cost (cost[s] = relative time of one tile of shape s). The last band and
// the last tile of a band may reach past the map (their extra windows are
// computed and not stored).
void plan_windows(std::vector<SvmItem> &out, int li, int rows, int cols, const float *cost) {
    if (rows <= 0 || cols <= 0) return;
    int heights[kSvmShapes], nh = 0;
    for (int s = 0; s < kSvmShapes; ++s) {
        const int th = svm_shape(s).th;
        bool seen = false;
        for (int i = 0; i < nh; ++i) seen |= heights[i] == th;
        if (!seen) heights[nh++] = th;
    }
    // per height: cheapest left-to-right covering of the columns
    std::vector<double> band_cost(nh);
    std::vector<std::vector<int>> band_shapes(nh);
    std::vector<double> best(cols + 1);
    std::vector<int> pick(cols + 1);
    for (int hi = 0; hi < nh; ++hi) {
        best[cols] = 0.0;
        for (int x = cols - 1; x >= 0; --x) {
            best[x] = 1e300;
            pick[x] = -1;
            for (int s = 0; s < kSvmShapes; ++s) {
                const SvmShapeInfo sh = svm_shape(s);
                if (sh.th != heights[hi]) continue;
                const double c = (double)cost[s] + best[std::min(cols, x + sh.tw)];
                if (c < best[x] - 1e-12) {
                    best[x] = c;
                    pick[x] = s;
                }
            }
        }
        band_cost[hi] = best[0];
        for (int x = 0; x < cols; x += svm_shape(pick[x]).tw) band_shapes[hi].push_back(pick[x]);
    }
    // rows: cheapest top-to-bottom sequence of bands
    std::vector<double> rbest(rows + 1);
    std::vector<int> rpick(rows + 1);
    rbest[rows] = 0.0;
    for (int y = rows - 1; y >= 0; --y) {
        rbest[y] = 1e300;
        rpick[y] = -1;
        for (int hi = 0; hi < nh; ++hi) {
            const double c = band_cost[hi] + rbest[std::min(rows, y + heights[hi])];
            if (c < rbest[y] - 1e-12) {
                rbest[y] = c;
                rpick[y] = hi;
            }
        }
    }
    for (int y = 0; y < rows; y += heights[rpick[y]]) {
        const int hi = rpick[y];
        int x = 0;
        for (int s : band_shapes[hi]) {
            out.push_back({li, x, y, s});
            x += svm_shape(s).tw;
        }
    }
}

// Tensor-core K4 items of a rows x cols score map: strips of kTcStrip window
// columns, each cut into near-equal pieces of at most `chunk` window rows
// (a piece also reads the 14 block rows below its last window row).
void plan_tc(std::vector<TcItem> &out, int li, int rows, int cols, int chunk) {
    if (rows <= 0 || cols <= 0) return;
    const int pieces = (rows + chunk - 1) / chunk;
    for (int x = 0; x < cols; x += kTcStrip)
        for (int k = 0; k < pieces; ++k)
            out.push_back({li, x, (int)((int64_t)rows * k / pieces), (int)((int64_t)rows * (k + 1) / pieces)});
}

// K2+K3 strips of every level of a plan, tallest first (the warps take them
// in this order, so the queue ends with the short ones). A strip is
// kStripTiles cell tiles tall, or shorter (down to 2 cell rows) when a
// small plan would otherwise leave warps idle in its last round. The strip
// height does not change the result (every cell row sums its votes in the
// same order).
void plan_strips(Plan &p, int resident_warps) {
    // A strip of r cell rows costs r + 1 bands of 8 pixel rows (one band of
    // halo), and the persistent warps take strips, tallest first, until none
    // is left. Of the heights 32, 16, ..., 2 the planner takes the one whose
    // schedule ends first, a shorter one only if it ends at least 3% sooner:
    // with many rounds of strips per warp that is 32 (least halo); with few,
    // a shorter height evens out the last round. The schedule (each strip to
    // the warp that is free first) is simulated when 32-row strips make fewer
    // than 16 rounds, from the histogram of strip heights with warps counted
    // per integer time (strips of one height go to the free warps in bulk).
    constexpr int kMaxRows = kCellTH * kStripTiles;
    const int64_t R = std::max(resident_warps, 1);
    auto histogram = [&](int rows, int64_t (&n)[kMaxRows + 1]) {
        int64_t total = 0;
        for (int r = 0; r <= kMaxRows; ++r) n[r] = 0;
        for (const LevelDesc &L : p.levels) {
            if (L.Hc <= 0) continue;
            n[rows] += (int64_t)L.ctx * (L.Hc / rows);
            n[L.Hc % rows] += L.Hc % rows ? L.ctx : 0;
            total += (int64_t)L.ctx * ((L.Hc + rows - 1) / rows);
        }
        return total;
    };
    auto makespan = [&](int rows) {
        int64_t n[kMaxRows + 1];
        histogram(rows, n);
        std::vector<int64_t> free_at(1, R);  // free_at[t]: warps that become free at time t
        size_t t = 0, end = 0;
        for (int r = kMaxRows; r >= 1; --r) {
            for (int64_t left = n[r]; left > 0;) {
                while (free_at[t] == 0) ++t;
                const int64_t k = std::min(free_at[t], left);
                const size_t e = t + (size_t)r + 1;
                if (e >= free_at.size()) free_at.resize(e + 1, 0);
                free_at[t] -= k;
                free_at[e] += k;
                left -= k;
                end = std::max(end, e);
            }
        }
        return (int64_t)end;
    };
    int rows = kMaxRows;
    int64_t n32[kMaxRows + 1];
    if (histogram(rows, n32) < 16 * R) {
        int64_t best = makespan(rows);
        for (int r = rows / 2; r >= 2; r /= 2) {
            const int64_t t = makespan(r);
            if (100 * t <= 97 * best) {
                best = t;
                rows = r;
            }
        }
    }
    p.strips.clear();
    for (int li = 0; li < (int)p.levels.size(); ++li) {
        const LevelDesc &L = p.levels[li];
        for (int cx = 0; cx < L.Wc; cx += kCellTW)
            for (int cy = 0; cy < L.Hc; cy += rows) p.strips.push_back({li, cx, cy, std::min(cy + rows, L.Hc)});
    }
    std::stable_sort(p.strips.begin(), p.strips.end(),
                     [](const StripItem &a, const StripItem &b) { return a.cy1 - a.cy0 > b.cy1 - b.cy0; });
}

// Largest items first (block rows walked: window rows + 14), so that the
// persistent CTAs' queue ends with the small ones.
void order_tc(std::vector<TcItem> &t) {
    std::stable_sort(t.begin(), t.end(),
                     [](const TcItem &a, const TcItem &b) { return a.wy1 - a.wy0 > b.wy1 - b.wy0; });
}

// K1 tables of one level (Section 4.4 resample, reading Q).
//   ytab: per output row an int2: the byte offset of its top source row's
//         quad row (source row * 4 * kResizeQP; the kernel subtracts the
//         tile's first row) and its scaled row weights (8192 - 4 a) | 4 a << 16;
//   ybnd: per source-tile row t, the first output row whose source row is >= 32 t;
//   xtab: per group of G output columns (G = 4; G = 1 when a group of 4
//         would reach more than kResizeBW - 2 source columns past the left
//         edge of the tile that owns it), an int4 of the packed column
//         weights (2048 - a) | a << 16 (lanes past G are 0);
//   xq:   per group one word: byte i = index of column i's source quad in the
//         owner tile's shared-memory quad row (resize_quad_index of its source
//         column relative to the tile). Columns past the level's width repeat
//         its last column;
//   xbnd: per source-tile column t, the first group whose first column's
//         source index is >= 128 t (the owner of a group is that tile).
void k1_tables(Plan &p, LevelDesc &L, int W, int H, int Wk, int Hk) {
    std::vector<int32_t> ex(Wk);
    for (int x = 0; x < Wk; ++x) ex[x] = q11_entry(x, W, Wk);
    auto src = [&](int x) { return ex[std::min(x, Wk - 1)] >> 11; };
    auto span_of = [&](int G) {
        int span = 0;
        for (int g = 0; g * G < Wk; ++g) {
            const int owner = src(g * G) / kResizeTW;
            for (int i = 0; i < G; ++i) span = std::max(span, src(g * G + i) - owner * kResizeTW + 2);
        }
        return span;
    };
    int G = 4, span = span_of(4);
    if (span > kResizeBW) {
        G = 1;
        span = span_of(1);
    }
    L.rgroup = G;
    L.rspan = span;
    const int groups = (Wk + G - 1) / G;
    while (p.tabs.size() % 4) p.tabs.push_back(0);
    L.xtab_off = (int32_t)p.tabs.size();
    for (int g = 0; g < groups; ++g)
        for (int i = 0; i < 4; ++i) {
            const int a = ex[std::min(g * G + i, Wk - 1)] & 2047;
            p.tabs.push_back(i < G ? (int32_t)((uint32_t)(2048 - a) | ((uint32_t)a << 16)) : 0);
        }
    L.xq_off = (int32_t)p.tabs.size();
    for (int g = 0; g < groups; ++g) {
        const int owner = src(g * G) / kResizeTW;
        uint32_t w = 0;
        for (int i = 0; i < G; ++i)
            w |= (uint32_t)resize_quad_index(src(g * G + i) - owner * kResizeTW) << (8 * i);
        p.tabs.push_back((int32_t)w);
    }
    std::vector<int32_t> ey(Hk);
    for (int y = 0; y < Hk; ++y) ey[y] = q11_entry(y, H, Hk);
    while (p.tabs.size() % 2) p.tabs.push_back(0);
    L.ytab_off = (int32_t)p.tabs.size();
    for (int y = 0; y < Hk; ++y) {
        const uint32_t a = (uint32_t)ey[y] & 2047u;
        p.tabs.push_back((ey[y] >> 11) * 4 * kResizeQP);
        p.tabs.push_back((int32_t)((8192u - 4u * a) | ((4u * a) << 16)));
    }
    L.xbnd_off = (int32_t)p.tabs.size();
    {
        int g = 0;
        for (int t = 0; t <= (W + kResizeTW - 1) / kResizeTW; ++t) {
            while (g < groups && src(g * G) < t * kResizeTW) ++g;
            p.tabs.push_back(g);
        }
    }
    L.ybnd_off = (int32_t)p.tabs.size();
    {
        int y = 0;
        for (int t = 0; t <= (H + kResizeTH - 1) / kResizeTH; ++t) {
            while (y < Hk && (ey[y] >> 11) < t * kResizeTH) ++y;
            p.tabs.push_back(y);
        }
    }
}

// Adds one level to the plan (tables, descriptor, work items).
void plan_level(Plan &p, int frame, int level, int W, int H, int Wk, int Hk, int64_t img_off,
                int32_t img_pitch, const LevelDesc *share = nullptr,
                const float *tile_cost = kDefaultTileCost) {
    LevelDesc L{};
    L.tc_map = -1;
    L.img_off = img_off;
    L.img_pitch = img_pitch;
    L.frame = frame;
    L.level = level;
    L.W = W;
    L.H = H;
    L.Wk = Wk;
    L.Hk = Hk;
    L.Wc = Wk / 8;
    L.Hc = Hk / 8;
    L.cell_row = p.atlas_rows;
    L.rows = std::max(L.Hc - kWinBH, 0);  // block rows Hc-1, window height 15 blocks
    L.cols = std::max(L.Wc - kWinBW, 0);
    if (L.rows == 0 || L.cols == 0) L.rows = L.cols = 0;
    L.score_off = p.score_floats;
    if (share) {
        L.xtab_off = share->xtab_off;
        L.ytab_off = share->ytab_off;
        L.xbnd_off = share->xbnd_off;
        L.ybnd_off = share->ybnd_off;
        L.rgroup = share->rgroup;
        L.rspan = share->rspan;
        L.xq_off = share->xq_off;
    } else {
        k1_tables(p, L, W, H, Wk, Hk);
    }
    const int li = (int)p.levels.size();
    L.hsrc = li;
    L.citem0 = (int32_t)p.c_items.size();
    L.ctx = (L.Wc + kCellTW - 1) / kCellTW;
    for (int cy = 0; cy < L.Hc; cy += kCellTH)
        for (int cx = 0; cx < L.Wc; cx += kCellTW) p.c_items.push_back({li, cx, cy, 0});
    plan_windows(p.s_items, li, L.rows, L.cols, tile_cost);
    plan_tc(p.t_items, li, L.rows, L.cols, p.tc_rows);
    p.atlas_rows += L.Hc;
    p.score_floats += (int64_t)L.rows * L.cols;
    p.max_wc = std::max(p.max_wc, L.Wc);
    p.levels.push_back(L);
}

// Source bytes K1 stages per tile row of a frame: what its levels need.
int32_t staged_bytes(const Plan &p, const FrameDesc &fd) {
    int32_t bw = 2;
    for (int k = 0; k < fd.n_levels; ++k) bw = std::max(bw, p.levels[fd.first_level + k].rspan);
    return bw;
}

// Plans one frame with the pyramid rule; returns PD_OK or an error.
int plan_frame(Plan &p, const pd_params &prm, const uint8_t *ptr, int W, int H, int pitch,
               const float *tile_cost = kDefaultTileCost, bool proposal = false) {
    int32_t Wk[PD_MAX_LEVELS], Hk[PD_MAX_LEVELS];
    int n = level_sizes(W, H, prm.pyr_factor, prm.upscale_levels, PD_MAX_LEVELS, Wk, Hk);
    if (n < 0) return n;
    FrameDesc fd{};
    fd.ptr = ptr;
    fd.W = W;
    fd.H = H;
    fd.pitch = pitch;
    fd.first_level = (int32_t)p.levels.size();
    fd.n_levels = n;
    const int f = (int)p.frames.size();
    auto owner = p.tab_owner.find({W, H});
    const int first_shared = owner == p.tab_owner.end() ? -1 : owner->second;
    if (first_shared < 0 && n > 0) p.tab_owner[{W, H}] = (int)p.levels.size();
    for (int k = 0; k < n; ++k) {
        const int32_t lp = (int32_t)round_up(Wk[k], 16);
        const LevelDesc share = first_shared >= 0 ? p.levels[first_shared + k] : LevelDesc{};
        plan_level(p, f, k, W, H, Wk[k], Hk[k], p.pyr_bytes, lp, first_shared >= 0 ? &share : nullptr,
                   tile_cost);
        p.pyr_bytes += (int64_t)lp * Hk[k];
        if (proposal) {
            // level groups: the network runs on levels 0, m, 2m, ...; level k uses the head
            // map of level m floor(k / m) (its first level, the largest)
            LevelDesc &L = p.levels.back();
            const int li = (int)p.levels.size() - 1;
            const int m = prm.proposal_level_step;
            L.hsrc = fd.first_level + m * (k / m);
            if (L.rows > 0 && k % m == 0)
                for (int cy = 0; cy < L.Hc; cy += kCnnTile)
                    for (int cx = 0; cx < L.Wc; cx += kCnnTile) p.cnn_items.push_back({li, cy, cx, 0});
        }
    }
    fd.rbw = staged_bytes(p, fd);
    if (n > 0)
        for (int y = 0; y < H; y += kResizeTH)
            for (int x = 0; x < W; x += kResizeTW) p.r_items.push_back({f, x, y, 0});
    p.frames.push_back(fd);
    return PD_OK;
}

bool params_ok(const pd_params *p) {
    return p && p->struct_size == sizeof(pd_params) && p->pyr_factor > 1.0f && p->l2hys_clip > 0.f &&
           !std::isnan(p->keep_logit_threshold) && p->upscale_levels >= 0 && p->upscale_levels <= 64 &&
           p->proposal_level_step >= 1 && p->proposal_level_step <= 16 &&
           p->nms_iou >= 0.f && p->max_boxes_per_frame > 0 && p->max_boxes_per_frame <= 16384 &&
           p->max_candidates_per_frame > 0 &&
           p->max_candidates_per_frame <= 65536 && p->max_frames > 0 && p->max_width > 0 &&
           p->max_height > 0 &&
           (p->flags & (PD_FLAG_HOG_ONLY | PD_FLAG_LBP_ONLY)) != (PD_FLAG_HOG_ONLY | PD_FLAG_LBP_ONLY) &&
           !((p->flags & PD_FLAG_HOG_PER_BLOCK) && (p->flags & (PD_FLAG_SVM_FP32 | PD_FLAG_LBP_ONLY)));
}

int encode_tc_maps(CUtensorMap *hog_map, CUtensorMap *lbp_map, const float *hog, const uint8_t *lbp, int64_t pitch,
                   int64_t rows, int64_t hog_plane, int64_t lbp_plane, int hog_planes = kHogBins,
                   int64_t width = 0) {
    if (encode_plane_map(hog_map, const_cast<float *>(hog), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, pitch, rows,
                         hog_planes, hog_plane, 112, 1, hog_planes, width) != PD_OK ||
        encode_plane_map(lbp_map, const_cast<uint8_t *>(lbp), CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, pitch, rows,
                         kLbpBins, lbp_plane, 128, 1, kLbpBins, width) != PD_OK)
        return PD_ECUDA;
    return PD_OK;
}

// Tensor-core K4: one pair of cell-plane maps per distinct level width, so
// that a box reaching past a level's right edge reads zeros (TMA fill) and
// not the atlas row's padding from memory (the windows that use those cells
// are not stored).
void assign_tc_maps(Plan &p) {
    p.tc_widths.clear();
    std::map<int32_t, int32_t> index;
    for (LevelDesc &L : p.levels) {
        auto it = index.find(L.Wc);
        if (it == index.end()) {
            it = index.emplace(L.Wc, (int32_t)p.tc_widths.size()).first;
            p.tc_widths.push_back(L.Wc);
        }
        L.tc_map = it->second;
    }
}

// Packs the plan into the pinned staging buffer and sends it to the device.
int upload_plan(pd_handle *h, cudaStream_t s, const Plan &p, Packed &o, const uint8_t *pyr_base = nullptr) {
    o = pack_layout(p);
    if (o.total > h->desc_cap) return fail(h, PD_EINVAL, "plan descriptors exceed the arena");
    PD_CUDA(h, cudaEventSynchronize(h->desc_done));  // previous copy has left the staging buffer
    auto put = [&](int64_t off, const void *src, size_t bytes) {
        if (bytes) std::memcpy(h->h_desc + off, src, bytes);
    };
    put(o.frames, p.frames.data(), p.frames.size() * sizeof(FrameDesc));
    put(o.levels, p.levels.data(), p.levels.size() * sizeof(LevelDesc));
    put(o.r_items, p.r_items.data(), p.r_items.size() * sizeof(ResizeItem));
    put(o.c_items, p.c_items.data(), p.c_items.size() * sizeof(CellItem));
    put(o.strips, p.strips.data(), p.strips.size() * sizeof(StripItem));
    put(o.s_items, p.s_items.data(), p.s_items.size() * sizeof(SvmItem));
    put(o.t_items, p.t_items.data(), p.t_items.size() * sizeof(TcItem));
    put(o.cnn_items, p.cnn_items.data(), p.cnn_items.size() * sizeof(CnnItem));
    put(o.tabs, p.tabs.data(), p.tabs.size() * sizeof(int32_t));
    for (size_t k = 0; k < p.tc_widths.size(); ++k) {
        CUtensorMap *maps = reinterpret_cast<CUtensorMap *>(h->h_desc + o.tc_maps) + 2 * k;
        if (encode_tc_maps(&maps[0], &maps[1], h->atlas.hog, h->atlas.lbp, h->atlas.pitch, h->atlas.rows,
                           h->atlas.hog_plane, h->atlas.lbp_plane, hog_planes_of(h->p.flags), p.tc_widths[k]) != PD_OK)
            return fail(h, PD_ECUDA, "cell-plane tensor map");
    }
    if (!p.cnn_items.empty()) {
        CUtensorMap *maps = reinterpret_cast<CUtensorMap *>(h->h_desc + o.tmaps);
        for (size_t k = 0; k < p.levels.size(); ++k) {
            const LevelDesc &L = p.levels[k];
            if (encode_level_map(&maps[k], pyr_base + L.img_off, L.Wk, L.Hk, L.img_pitch) != PD_OK)
                return fail(h, PD_ECUDA, "level tensor map");
        }
    }
    if (o.total) PD_CUDA(h, cudaMemcpyAsync(h->d_desc, h->h_desc, o.total, cudaMemcpyHostToDevice, s));
    PD_CUDA(h, cudaEventRecord(h->desc_done, s));
    return PD_OK;
}

// One HOG and one LBP tensor map per K4 tile shape over plane-major cell
// planes [planes][rows][pitch].
int encode_svm_maps(CUtensorMap *hog_maps, CUtensorMap *lbp_maps, const float *hog, const uint8_t *lbp,
                    int64_t pitch, int64_t rows, int64_t hog_plane, int64_t lbp_plane) {
    for (int s = 0; s < kSvmShapes; ++s) {
        const SvmShapeInfo sh = svm_shape(s);
        if (encode_plane_map(&hog_maps[s], const_cast<float *>(hog), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                             pitch, rows, kHogBins, hog_plane, sh.hog_box_x, sh.cell_rows, kHogBins) != PD_OK ||
            encode_plane_map(&lbp_maps[s], const_cast<uint8_t *>(lbp), CU_TENSOR_MAP_DATA_TYPE_UINT8, 1,
                             pitch, rows, kLbpBins, lbp_plane, sh.lbp_box_x, sh.cell_rows,
                             svm_lbp_chunk()) != PD_OK)
            return PD_ECUDA;
    }
    return PD_OK;
}

// The tensor-core K4's maps: one cell row of a 112-cell strip of the 9 (or,
// per-block HOG, 36) HOG planes, and of a 128-cell strip of the 59 LBP planes.
// Round to the nearest bfloat16 (ties to even): 8 significant bits of the
// exact value, as a float.
float bf16_round_host(double a) {
    if (a == 0.0 || !std::isfinite(a)) return (float)a;
    int e = 0;
    const double m = std::frexp(a, &e);      // a = m 2^e, 0.5 <= |m| < 1
    return (float)std::ldexp(std::nearbyint(m * 256.0) / 256.0, e);
}

uint32_t bf16_bits(float f) {  // f is already a bf16 value: its top 16 bits
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u >> 16;
}

// mma.sync m16n8k16 B fragments (B = K x N): lane (g = lane/4, t = lane%4)
// holds B[2t][g], B[2t+1][g] in register 0 and B[2t+8][g], B[2t+9][g] in
// register 1 (first element in the low half).
void pack_frag(const float *W, int cin, int ci0, int tap, int nt, uint32_t *out /* [32][2] */) {
    for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, t = lane & 3, co = nt * 8 + g;
        auto w = [&](int ci) { return bf16_bits(bf16_round_host(W[((size_t)co * cin + ci) * 9 + tap])); };
        out[2 * lane] = w(ci0 + 2 * t) | (w(ci0 + 2 * t + 1) << 16);
        out[2 * lane + 1] = w(ci0 + 2 * t + 8) | (w(ci0 + 2 * t + 9) << 16);
    }
}

void invalidate_cache(pd_handle *h) {
    h->cache_valid = false;
    h->sig.clear();
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
}

int max_pool_tiles(const Plan &p) {
    int m = 0;
    for (const LevelDesc &L : p.levels) m = std::max(m, pool_tiles_of(L.rows, L.cols));
    return m;
}

template <class T>
const T *dptr(pd_handle *h, int64_t off) {
    return reinterpret_cast<const T *>(h->d_desc + off);
}

// K2+K3 of a plan: the warp-per-strip kernel, or for per-block HOG the
// CTA-per-tile kernel.
cudaError_t launch_cell_stage(pd_handle *h, cudaStream_t s, const LevelDesc *dl, const uint8_t *pyr,
                              const CellAtlas &atlas, const Plan &p, const Packed &o, const uint32_t *c_flag,
                              int feat) {
    if (feat & kFeatHogBlock)
        return launch_cells(s, dl, pyr, atlas, dptr<CellItem>(h, o.c_items), (int)p.c_items.size(), h->d_lbp_map,
                            c_flag, feat);
    int *queue = h->d_queue + 1;  // the strip counter (K4's is d_queue[0])
    const cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    return launch_cells_warp(s, dl, pyr, atlas, dptr<StripItem>(h, o.strips), (int)p.strips.size(), queue,
                             h->sm_count, h->d_lbp_map, c_flag, feat);
}

}  // namespace

namespace {

CnnWeights cnn_weights(const pd_handle *h) {
    const float *wr = h->cnn + 4 * kCnnParams;
    CnnWeights w;
    w.in_tab = h->in_tab;
    w.w1 = wr + kOffW1;
    w.b1 = wr + kOffB1;
    w.w2frag = h->w2frag;
    w.w2 = wr + kOffW2;
    w.w3 = wr + kOffW3;
    w.b2 = wr + kOffB2;
    w.b3 = wr + kOffB3;
    w.wh = wr + kOffWh;
    w.bh = wr + kOffBh;
    w.v = wr + kOffV;
    w.bv = wr + kOffBv;
    return w;
}

// Inference fragments from the master weights (after set_params or training).
// Waits for the device first: training steps may still be writing the
// master weights on a stream that the copy below does not order after.
int refresh_fragments(pd_handle *h) {
    PD_CUDA(h, cudaDeviceSynchronize());
    std::vector<float> p(kCnnParams);
    PD_CUDA(h, cudaMemcpy(p.data(), h->cnn, kCnnParams * 4, cudaMemcpyDeviceToHost));
    // layer 2's mma.sync B fragments (its edge positions); the tcgen05 operands
    // are built by the kernel from the rounded weights
    std::vector<uint32_t> f2(2304);
    for (int tap = 0; tap < 9; ++tap)
        for (int nt = 0; nt < 4; ++nt) pack_frag(p.data() + kOffW2, 16, 0, tap, nt, &f2[(tap * 4 + nt) * 64]);
    PD_CUDA(h, cudaMemcpy(h->w2frag, f2.data(), f2.size() * 4, cudaMemcpyHostToDevice));
    h->frag_stale = false;
    return PD_OK;
}

}  // namespace

extern "C" {

int pd_params_default(pd_params *p) {
    if (!p) return PD_EINVAL;
    std::memset(p, 0, sizeof *p);
    p->struct_size = sizeof(pd_params);
    p->pyr_factor = 1.05f;
    p->l2hys_clip = 0.2f;
    p->threshold = 0.0f;
    p->nms_iou = 0.5f;
    p->max_boxes_per_frame = 4096;
    p->max_candidates_per_frame = 16384;
    p->max_frames = 1;
    p->max_width = 1242;
    p->max_height = 375;
    p->flags = 0;
    p->proposal_level_step = 1;
    return PD_OK;
}

int pd_pyramid(int W, int H, float factor, int max_levels, int32_t *Wk, int32_t *Hk) {
    if (!Wk || !Hk || max_levels < 0) return PD_EINVAL;
    return level_sizes(W, H, factor, 0, max_levels, Wk, Hk);
}

int pd_pyramid_ex(int W, int H, float factor, int upscale_levels, int max_levels, int32_t *Wk, int32_t *Hk) {
    if (!Wk || !Hk || max_levels < 0) return PD_EINVAL;
    return level_sizes(W, H, factor, upscale_levels, max_levels, Wk, Hk);
}

const char *pd_last_error(const pd_handle *h) { return h ? h->err.c_str() : "null handle"; }

int pd_last_launch_count(const pd_handle *h) { return h ? h->last_launches : 0; }

void pd_destroy(pd_handle *h) {
    if (!h) return;
    cudaDeviceSynchronize();
    if (h->arena) cudaFree(h->arena);
    if (h->h_desc) cudaFreeHost(h->h_desc);
    if (h->h_boxes) cudaFreeHost(h->h_boxes);
    if (h->h_counts) cudaFreeHost(h->h_counts);
    if (h->desc_done) cudaEventDestroy(h->desc_done);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    if (h->train_ws) cudaFree(h->train_ws);
    if (h->scheme_ws) cudaFree(h->scheme_ws);
    if (h->graph_done) cudaEventDestroy(h->graph_done);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (auto &e : h->stage_ev)
        if (e) cudaEventDestroy(e);
    delete h;
}

int pd_create(const pd_params *params, const float *svm_w, float svm_b, pd_handle **out) {
    if (!out) return PD_EINVAL;
    *out = nullptr;
    if (!params_ok(params) || !svm_w) return PD_EINVAL;
    pd_handle *h = new pd_handle();
    h->p = *params;
    h->bias = svm_b;
    auto bail = [&](int code) {
        pd_destroy(h);
        return code;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) return bail(PD_ECUDA);
    if (init_resize() != cudaSuccess || init_cells() != cudaSuccess || init_cells_warp() != cudaSuccess ||
        init_svm() != cudaSuccess || init_svm_tc() != cudaSuccess ||
        init_nms() != cudaSuccess ||
        init_cnn() != cudaSuccess)
        return bail(PD_ECUDA);

    // Worst-case plan: max_frames frames of max_width x max_height.
    Plan worst;
    for (int f = 0; f < params->max_frames; ++f)
        if (plan_frame(worst, *params, nullptr, params->max_width, params->max_height,
                       params->max_width) != PD_OK)
            return bail(PD_EINVAL);
    if (worst.levels.empty()) {
        // frames too small for any window still get a valid (tiny) arena
        worst.max_wc = std::max(params->max_width / 8, 1);
    }
    // Descriptor capacity: per frame, the largest frame's levels, work items
    // (K4 tiles counted for the shape with the most tiles) and its own Q11
    // tables (frames of different sizes do not share them).
    {
        Plan one;
        one.tc_rows = kTcMinChunk;  // the most tensor-core K4 items any tuning can ask for
        plan_frame(one, *params, nullptr, params->max_width, params->max_height, params->max_width);
        int64_t s_bound = 0;
        for (const LevelDesc &L : one.levels) {
            int64_t most = 0;
            // any band / width mix has at most (rows / smallest height + 1) bands of at
            // most (cols / smallest width + 1) tiles
            int min_th = 1 << 30, min_tw = 1 << 30;
            for (int sh = 0; sh < kSvmShapes; ++sh) {
                min_th = std::min(min_th, svm_shape(sh).th);
                min_tw = std::min(min_tw, svm_shape(sh).tw);
            }
            if (L.rows > 0) most = (int64_t)(L.rows / min_th + 1) * (L.cols / min_tw + 1);
            s_bound += most;
        }
        const int64_t F = params->max_frames;
        int64_t cnn_bound = 0;
        for (const LevelDesc &L : one.levels)
            cnn_bound += (int64_t)((L.Hc + kCnnTile - 1) / kCnnTile) * ((L.Wc + kCnnTile - 1) / kCnnTile);
        h->flag_cap = F * std::max<int64_t>(s_bound, (int64_t)one.c_items.size()) + 64;
        h->desc_cap = round_up(F * (int64_t)one.levels.size() * (int64_t)sizeof(CUtensorMap), 64) + 128 +
                      round_up(2 * (int64_t)std::max(worst.max_wc, 1) * (int64_t)sizeof(CUtensorMap), 64) + 64 +
                      round_up(F * cnn_bound * (int64_t)sizeof(CnnItem), 16) +
                      round_up(F * (int64_t)sizeof(FrameDesc), 16) +
                      round_up(F * (int64_t)one.levels.size() * (int64_t)sizeof(LevelDesc), 16) +
                      round_up(F * (int64_t)one.r_items.size() * (int64_t)sizeof(ResizeItem), 16) +
                      round_up(F * (int64_t)one.c_items.size() * (int64_t)sizeof(CellItem), 16) +
                      round_up(4 * F * (int64_t)one.c_items.size() * (int64_t)sizeof(StripItem), 16) +  // 2-row strips
                      round_up(F * s_bound * (int64_t)sizeof(SvmItem), 16) +
                      round_up(F * (int64_t)one.t_items.size() * (int64_t)sizeof(TcItem), 16) +
                      round_up(F * (int64_t)one.tabs.size() * 4, 16) + 4096;
        h->desc_cap = round_up(h->desc_cap, kAlign);
    }
    h->pyr_cap = round_up(std::max<int64_t>(worst.pyr_bytes, 16), kAlign);
    const int32_t P = (int32_t)std::max<int64_t>(round_up(std::max(worst.max_wc, 1), 16), 48);
    const int32_t rows = std::max(worst.atlas_rows, 1);
    h->atlas.pitch = P;
    h->atlas.rows = rows;
    h->atlas.hog_plane = (int64_t)rows * P;
    h->atlas.lbp_plane = (int64_t)rows * P;
    h->score_cap = std::max<int64_t>(worst.score_floats, 1);
    h->frames_cap = (int64_t)params->max_frames * round_up(params->max_width, 16) * params->max_height;

    struct Part {
        int64_t bytes;
        int64_t off;
    };
    std::vector<Part> parts = {
        {(int64_t)kFeat * kWinBH * kWPad * 4, 0},                  // 0 template
        {256, 0},                                                  // 1 lbp map
        {h->desc_cap, 0},                                          // 2 descriptors
        {h->pyr_cap, 0},                                           // 3 pyramid
        {(int64_t)hog_planes_of(params->flags) * h->atlas.hog_plane * 4, 0},  // 4 hog atlas
        {(int64_t)kLbpBins * h->atlas.lbp_plane, 0},               // 5 lbp atlas
        {h->score_cap * 4, 0},                                     // 6 scores
        {(int64_t)params->max_frames * params->max_boxes_per_frame * (int64_t)sizeof(pd_box), 0},  // 7
        {(int64_t)params->max_frames * 2 * 4 + 16, 0},             // 8 counts + error word + item counters
        {h->frames_cap, 0},                                        // 9 host-input frames
        {(int64_t)params->max_frames * (int64_t)nms_scratch_float4s(params->max_candidates_per_frame) * 16,
         0},                                                                        // 10 NMS scratch
        {(int64_t)5 * kCnnParams * 4 + 1024 + 2304 * 4, 0},                        // 11 CNN parameters
        {(int64_t)rows * P * 4, 0},                                                 // 12 head values
        {h->score_cap * 4, 0},                                                      // 13 window logits
        {2 * h->flag_cap * 4, 0},                                                   // 14 tile flags
        {(int64_t)nms_sched_ints(params->max_frames) * 4, 0},                       // 15 NMS frame order
    };
    int64_t total = 0;
    for (auto &pt : parts) {
        pt.off = total;
        total = round_up(total + pt.bytes, kAlign);
    }
    h->arena_bytes = (size_t)total;
    if (cudaMalloc(&h->arena, h->arena_bytes) != cudaSuccess) return bail(PD_ENOMEM);
    if (cudaMemset(h->arena, 0, h->arena_bytes) != cudaSuccess) return bail(PD_ECUDA);
    h->d_w = reinterpret_cast<float *>(h->arena + parts[0].off);
    h->d_lbp_map = h->arena + parts[1].off;
    h->d_desc = h->arena + parts[2].off;
    h->d_pyr = h->arena + parts[3].off;
    h->atlas.hog = reinterpret_cast<float *>(h->arena + parts[4].off);
    h->atlas.lbp = h->arena + parts[5].off;
    h->d_scores = reinterpret_cast<float *>(h->arena + parts[6].off);
    h->d_boxes = reinterpret_cast<pd_box *>(h->arena + parts[7].off);
    h->d_counts = reinterpret_cast<int32_t *>(h->arena + parts[8].off);
    h->d_err = reinterpret_cast<unsigned *>(h->d_counts + 2 * params->max_frames);
    h->d_queue = reinterpret_cast<int *>(h->d_err + 1);
    h->d_frames = h->arena + parts[9].off;
    h->d_nms_scratch = reinterpret_cast<float4 *>(h->arena + parts[10].off);
    h->cnn = reinterpret_cast<float *>(h->arena + parts[11].off);
    h->in_tab = h->cnn + 5 * kCnnParams;
    h->w2frag = reinterpret_cast<uint32_t *>(h->in_tab + 256);
    h->hmap = reinterpret_cast<float *>(h->arena + parts[12].off);
    h->logits = reinterpret_cast<float *>(h->arena + parts[13].off);
    h->s_flag = reinterpret_cast<uint32_t *>(h->arena + parts[14].off);
    h->c_flag = h->s_flag + h->flag_cap;
    h->d_nms_sched = reinterpret_cast<int *>(h->arena + parts[15].off);
    h->proposal = params->use_proposal != 0;
    h->tau = params->keep_logit_threshold;

    if (cudaMallocHost(&h->h_desc, h->desc_cap) != cudaSuccess) return bail(PD_ENOMEM);
    // Results land in mapped pinned host memory: NMS writes the kept boxes and
    // counts there directly, so pd_sync needs no device-to-host copies.
    if (cudaHostAlloc(&h->h_boxes, (size_t)params->max_frames * params->max_boxes_per_frame * sizeof(pd_box),
                      cudaHostAllocMapped) != cudaSuccess)
        return bail(PD_ENOMEM);
    if (cudaHostAlloc(&h->h_counts, (size_t)params->max_frames * 2 * 4 + 16, cudaHostAllocMapped) != cudaSuccess)
        return bail(PD_ENOMEM);
    h->h_err = reinterpret_cast<unsigned *>(h->h_counts + 2 * params->max_frames);
    if (cudaHostGetDevicePointer(reinterpret_cast<void **>(&h->m_boxes), h->h_boxes, 0) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&h->m_counts), h->h_counts, 0) != cudaSuccess)
        return bail(PD_ECUDA);
    if (cudaEventCreateWithFlags(&h->desc_done, cudaEventDisableTiming) != cudaSuccess)
        return bail(PD_ECUDA);
    if (cudaEventRecord(h->desc_done, 0) != cudaSuccess) return bail(PD_ECUDA);
    if (params->flags & PD_FLAG_STAGE_TIMING)
        for (auto &e : h->stage_ev)
            if (cudaEventCreate(&e) != cudaSuccess) return bail(PD_ECUDA);
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->graph_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(h->graph_done, 0) != cudaSuccess)
        return bail(PD_ECUDA);

    // template -> [t][i][8] (j padded), lbp map; a HOG-only or LBP-only
    // pipeline scores with the other features' weights at zero (its cells
    // are not computed)
    std::vector<float> wt((size_t)kFeat * kWinBH * kWPad, 0.f);
    const int feat = features_of(params->flags);
    for (int i = 0; i < kWinBH; ++i)
        for (int j = 0; j < kWinBW; ++j)
            for (int t = 0; t < kFeat; ++t) {
                const bool used = t < kHogDim ? (feat & kFeatHog) != 0 : (feat & kFeatLbp) != 0;
                wt[((size_t)t * kWinBH + i) * kWPad + j] = used ? svm_w[((size_t)i * kWinBW + j) * kFeat + t] : 0.f;
            }
    float tab[256];
    for (int v = 0; v < 256; ++v) tab[v] = bf16_round_host((double)v / 255.0 - 0.5);
    if (cudaMemcpy(h->in_tab, tab, sizeof tab, cudaMemcpyHostToDevice) != cudaSuccess) return bail(PD_ECUDA);
    uint8_t map[256];
    build_lbp_bin_table(map);
    if (cudaMemcpy(h->d_w, wt.data(), wt.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->d_lbp_map, map, 256, cudaMemcpyHostToDevice) != cudaSuccess)
        return bail(PD_ECUDA);
    if (encode_svm_maps(h->hog_map, h->lbp_map, h->atlas.hog, h->atlas.lbp, P, rows, h->atlas.hog_plane,
                        h->atlas.lbp_plane) != PD_OK ||
        encode_tc_maps(&h->tc_hog_map, &h->tc_lbp_map, h->atlas.hog, h->atlas.lbp, P, rows, h->atlas.hog_plane,
                       h->atlas.lbp_plane, hog_planes_of(params->flags)) != PD_OK)
        return bail(PD_ECUDA);
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
        return bail(PD_ECUDA);
    *out = h;
    return PD_OK;
}

int pd_detect(pd_handle *h, void *stream, int n_frames, const uint8_t *const *d_frames,
              const int32_t *widths, const int32_t *heights, const int32_t *pitches) {
    if (!h) return PD_EINVAL;
    h->detected = h->synced = false;
    h->last_launches = 0;
    if (n_frames < 0 || n_frames > h->p.max_frames)
        return fail(h, PD_EINVAL, "n_frames %d outside [0, %d]", n_frames, h->p.max_frames);
    if (n_frames > 0 && (!d_frames || !widths || !heights || !pitches))
        return fail(h, PD_EINVAL, "null argument");
    std::vector<int32_t> sig;
    sig.reserve(1 + 3 * (size_t)n_frames);
    sig.push_back(n_frames);
    for (int f = 0; f < n_frames; ++f) {
        const int W = widths[f], H = heights[f], pitch = pitches[f];
        if (W < 1 || H < 1 || W > h->p.max_width || H > h->p.max_height || pitch < W || !d_frames[f])
            return fail(h, PD_EINVAL, "frame %d: bad size %dx%d pitch %d", f, W, H, pitch);
        sig.push_back(W);
        sig.push_back(H);
        sig.push_back(pitch);
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    h->stream = s;
    if (h->proposal && !h->cnn_loaded) return fail(h, PD_ESTATE, "proposal on but no parameters loaded");
    if (h->proposal && h->frag_stale) {
        int rr = refresh_fragments(h);
        if (rr != PD_OK) return rr;
    }
    Plan &p = h->plan;
    const bool reuse = h->cache_valid && sig == h->sig;
    if (!reuse) {
        invalidate_cache(h);
        p.clear();
        p.tc_rows = h->tuning.tc_item_rows;
        for (int f = 0; f < n_frames; ++f) {
            int r = plan_frame(p, h->p, d_frames[f], widths[f], heights[f], pitches[f],
                               h->proposal ? kSparseTileCost : h->tile_cost, h->proposal);
            if (r != PD_OK) return fail(h, r, "frame %d: planning failed", f);
        }
        order_tc(p.t_items);
        plan_strips(p, h->sm_count * kStripWarpsPerSm);
        if (!(h->p.flags & PD_FLAG_SVM_FP32)) assign_tc_maps(p);
        if (p.atlas_rows > h->atlas.rows || p.pyr_bytes > h->pyr_cap || p.score_floats > h->score_cap ||
            (int64_t)p.s_items.size() > h->flag_cap || (int64_t)p.c_items.size() > h->flag_cap)
            return fail(h, PD_EINVAL, "batch exceeds the arena");
        // full descriptor upload, once per batch shape
        int r = upload_plan(h, s, p, h->packed, h->d_pyr);
        if (r != PD_OK) return r;
        h->sig = sig;
        h->cache_valid = true;
    }
    // frame pointers change from call to call: rewrite only that section
    PD_CUDA(h, cudaEventSynchronize(h->graph_done));
    PD_CUDA(h, cudaEventSynchronize(h->desc_done));
    for (int f = 0; f < n_frames; ++f) p.frames[f].ptr = d_frames[f];
    const Packed &o = h->packed;
    if (n_frames) std::memcpy(h->h_desc + o.frames, p.frames.data(), p.frames.size() * sizeof(FrameDesc));
    const FrameDesc *df = dptr<FrameDesc>(h, o.frames);
    const LevelDesc *dl = dptr<LevelDesc>(h, o.levels);
    const bool timed = (h->p.flags & PD_FLAG_STAGE_TIMING) != 0;
    h->timed = timed;
    // inside a capture an event record must be an external node to be timed
    bool capturing = false;
    auto record = [&](cudaEvent_t e, cudaStream_t q) {
        return capturing ? cudaEventRecordWithFlags(e, q, cudaEventRecordExternal) : cudaEventRecord(e, q);
    };
    auto enqueue = [&](cudaStream_t q) -> int {
        if (n_frames)
            PD_CUDA(h, cudaMemcpyAsync(h->d_desc + o.frames, h->h_desc + o.frames,
                                       p.frames.size() * sizeof(FrameDesc), cudaMemcpyHostToDevice, q));
        PD_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), q));
        if (timed) PD_CUDA(h, record(h->stage_ev[0], q));
        PD_CUDA(h, launch_resize(q, df, dl, dptr<int32_t>(h, o.tabs), h->d_pyr, dptr<ResizeItem>(h, o.r_items),
                                 (int)p.r_items.size(), h->tuning.k1_groups));
        if (timed) PD_CUDA(h, record(h->stage_ev[5], q));
        const uint32_t *cf = nullptr, *sf = nullptr;
        if (h->proposal) {
            // learned proposal: keep-logits of every window, then the tiles to score
            PD_CUDA(h, launch_cnn(q, dl, (int)p.levels.size(), dptr<CUtensorMap>(h, o.tmaps),
                                  dptr<CnnItem>(h, o.cnn_items),
                                  (int)p.cnn_items.size(), cnn_weights(h), h->hmap, h->atlas.pitch, h->logits,
                                  max_pool_tiles(p), h->d_err));
            PD_CUDA(h, cudaMemsetAsync(h->c_flag, 0, p.c_items.size() * 4 + 4, q));
            PD_CUDA(h, launch_proposal_flags(q, dl, dptr<SvmItem>(h, o.s_items), (int)p.s_items.size(), h->logits,
                                             h->tau, h->s_flag, h->c_flag, !(h->p.flags & PD_FLAG_SVM_FP32)));
            cf = h->c_flag;
            sf = h->s_flag;
        }
        if (timed) PD_CUDA(h, record(h->stage_ev[1], q));
        PD_CUDA(h, launch_cell_stage(h, q, dl, h->d_pyr, h->atlas, p, o, cf, features_of(h->p.flags)));
        if (timed) PD_CUDA(h, record(h->stage_ev[2], q));
        if (h->p.flags & PD_FLAG_SVM_FP32) {
            PD_CUDA(h, launch_svm(q, h->hog_map, h->lbp_map, dl, h->d_w, h->bias, h->p.l2hys_clip, h->d_scores,
                                  dptr<SvmItem>(h, o.s_items), (int)p.s_items.size(), h->d_err, sf));
        } else {
            PD_CUDA(h, cudaMemsetAsync(h->d_queue, 0, sizeof(int), q));
            PD_CUDA(h, launch_svm_tc(q, h->tc_hog_map, h->tc_lbp_map, dl, dptr<TcItem>(h, o.t_items),
                                     (int)p.t_items.size(), h->d_queue, h->sm_count, h->d_w, h->bias,
                                     h->p.l2hys_clip, h->d_scores, cf, h->d_err, hog_planes_of(h->p.flags),
                                     p.tc_widths.empty() ? nullptr : dptr<CUtensorMap>(h, o.tc_maps)));
        }
        if (timed) PD_CUDA(h, record(h->stage_ev[3], q));
        PD_CUDA(h, launch_nms(q, df, dl, n_frames, h->d_scores, h->p.threshold, h->p.nms_iou,
                              h->d_nms_scratch, h->p.max_candidates_per_frame, h->m_boxes,
                              h->p.max_boxes_per_frame, h->m_counts,
                              nms_cluster_for(n_frames, h->sm_count, h->p.max_candidates_per_frame),
                              h->d_nms_sched));
        if (timed) PD_CUDA(h, record(h->stage_ev[4], q));
        return PD_OK;
    };
    if (reuse && !h->graph) {
        // second call with this batch shape: capture the step once
        PD_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
        capturing = true;
        int r = enqueue(h->cap_stream);
        capturing = false;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
        if (r != PD_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess) return fail(h, PD_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&h->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->graph = nullptr;
            return fail(h, PD_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
    }
    if (h->graph) {
        PD_CUDA(h, cudaGraphLaunch(h->graph, s));
    } else {
        int r = enqueue(s);
        if (r != PD_OK) return r;
    }
    PD_CUDA(h, cudaEventRecord(h->graph_done, s));
    h->last_launches = (p.r_items.empty() ? 0 : 1) + (p.c_items.empty() ? 0 : 1) +
                       (p.s_items.empty() ? 0 : 1) +
                       nms_launches(n_frames, nms_cluster_for(n_frames, h->sm_count, h->p.max_candidates_per_frame)) +
                       (h->proposal ? (p.cnn_items.empty() ? 0 : 1) + (p.levels.empty() ? 0 : 1) +
                                          (p.s_items.empty() ? 0 : 1)
                                    : 0);
    h->detected = true;
    h->ran_proposal = h->proposal;
    return PD_OK;
}

int pd_detect_host(pd_handle *h, void *stream, int n_frames, const uint8_t *const *h_frames,
                   const int32_t *widths, const int32_t *heights, const int32_t *pitches) {
    if (!h) return PD_EINVAL;
    if (n_frames < 0 || n_frames > h->p.max_frames)
        return fail(h, PD_EINVAL, "n_frames %d outside [0, %d]", n_frames, h->p.max_frames);
    if (n_frames > 0 && (!h_frames || !widths || !heights || !pitches))
        return fail(h, PD_EINVAL, "null argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<const uint8_t *> dev((size_t)n_frames);
    std::vector<int32_t> dp((size_t)n_frames);
    int64_t off = 0;
    for (int f = 0; f < n_frames; ++f) {
        const int W = widths[f], H = heights[f];
        if (W < 1 || H < 1 || W > h->p.max_width || H > h->p.max_height || pitches[f] < W || !h_frames[f])
            return fail(h, PD_EINVAL, "frame %d: bad size %dx%d pitch %d", f, W, H, pitches[f]);
        // Pinned (page-locked) host frames are read by the pyramid kernel in
        // place, over the host link; other host memory is copied first.
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, h_frames[f]) == cudaSuccess && a.type == cudaMemoryTypeHost &&
            a.devicePointer) {
            dev[f] = reinterpret_cast<const uint8_t *>(a.devicePointer);
            dp[f] = pitches[f];
            continue;
        }
        cudaGetLastError();  // clear a failed query on unregistered memory
        dp[f] = (int32_t)round_up(W, 16);
        dev[f] = h->d_frames + off;
        PD_CUDA(h, cudaMemcpy2DAsync(h->d_frames + off, dp[f], h_frames[f], pitches[f], W, H,
                                     cudaMemcpyHostToDevice, s));
        off += (int64_t)dp[f] * H;
    }
    return pd_detect(h, stream, n_frames, dev.data(), widths, heights, dp.data());
}

int pd_sync(pd_handle *h) {
    if (!h) return PD_EINVAL;
    if (!h->detected) return fail(h, PD_ESTATE, "pd_sync without pd_detect");
    const int nf = (int)h->plan.frames.size();
    PD_CUDA(h, cudaMemcpyAsync(h->h_err, h->d_err, 4, cudaMemcpyDeviceToHost, h->stream));
    PD_CUDA(h, cudaStreamSynchronize(h->stream));  // boxes and counts are already in host memory
    int status = PD_OK;
    if (*h->h_err & kErrTimeout) status = fail(h, PD_ETIMEOUT, "device wait timed out");
    else if (*h->h_err & kErrBounds) status = fail(h, PD_EBOUNDS, "device bounds check fired");
    for (int f = 0; f < nf && status == PD_OK; ++f)
        if (h->h_counts[2 * f + 1] < 0)
            status = fail(h, PD_EOVERFLOW, "frame %d: %d candidates > %d", f, -h->h_counts[2 * f + 1],
                          h->p.max_candidates_per_frame);
    h->synced = true;
    return status;
}

int pd_frame_candidates(const pd_handle *h, int frame, int *n) {
    if (!h || !n) return PD_EINVAL;
    if (!h->synced) return PD_ESTATE;
    if (frame < 0 || frame >= (int)h->plan.frames.size()) return PD_EINVAL;
    *n = h->h_counts[2 * frame + 1];
    return PD_OK;
}

int pd_set_tile_costs(pd_handle *h, const float *cost) {
    if (!h || !cost) return PD_EINVAL;
    for (int s = 0; s < kSvmShapes; ++s)
        if (!(cost[s] > 0.f)) return fail(h, PD_EINVAL, "tile cost %d must be > 0", s);
    for (int s = 0; s < kSvmShapes; ++s) h->tile_cost[s] = cost[s];
    invalidate_cache(h);
    return PD_OK;
}

int pd_get_tile_costs(const pd_handle *h, float *cost) {
    if (!h || !cost) return PD_EINVAL;
    for (int s = 0; s < kSvmShapes; ++s) cost[s] = h->tile_cost[s];
    return PD_OK;
}

// ----------------------------------------------------------------------------- learned proposal

int pd_cnn_set_params(pd_handle *h, const float *params, int n) {
    if (!h || !params || n != kCnnParams)
        return h ? fail(h, PD_EINVAL, "expected %d parameters", kCnnParams) : PD_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(params[i])) return fail(h, PD_EINVAL, "parameter %d is not finite", i);
    PD_CUDA(h, cudaDeviceSynchronize());
    PD_CUDA(h, cudaMemcpy(h->cnn, params, kCnnParams * 4, cudaMemcpyHostToDevice));
    PD_CUDA(h, cudaMemset(h->cnn + kCnnParams, 0, 3 * kCnnParams * 4));  // Adam m, v and grad
    PD_CUDA(h, launch_round_params(0, h->cnn, h->cnn + 4 * kCnnParams));
    PD_CUDA(h, cudaDeviceSynchronize());
    h->adam_t = 0;
    h->cnn_loaded = true;
    return refresh_fragments(h);
}

int pd_cnn_get_params(pd_handle *h, float *params, float *grad, int n) {
    if (!h || n != kCnnParams) return PD_EINVAL;
    PD_CUDA(h, cudaDeviceSynchronize());
    if (params) PD_CUDA(h, cudaMemcpy(params, h->cnn, kCnnParams * 4, cudaMemcpyDeviceToHost));
    if (grad) PD_CUDA(h, cudaMemcpy(grad, h->cnn + 3 * kCnnParams, kCnnParams * 4, cudaMemcpyDeviceToHost));
    return PD_OK;
}

int pd_cnn_forward(pd_handle *h, void *stream, const uint8_t *d_level, int Wk, int Hk, int pitch, float *d_h,
                   int h_pitch, float *d_logits) {
    if (!h) return PD_EINVAL;
    invalidate_cache(h);  // the descriptor region is reused below
    const int Wc = Wk / 8, Hc = Hk / 8;
    if (!d_level || !d_h || !d_logits || Wk < 1 || Hk < 1 || pitch < Wk || h_pitch < Wc)
        return fail(h, PD_EINVAL, "pd_cnn_forward: bad argument");
    if (!h->cnn_loaded) return fail(h, PD_ESTATE, "no proposal parameters (pd_cnn_set_params)");
    if (h->frag_stale) {
        int r = refresh_fragments(h);
        if (r != PD_OK) return r;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the kernel's TMA needs 16-byte aligned rows: other layouts go through the pyramid buffer
    if (((uintptr_t)d_level | (uintptr_t)pitch) & 15u) {
        const int lp = (int)round_up(Wk, 16);
        if ((int64_t)lp * Hk > h->pyr_cap) return fail(h, PD_EINVAL, "pd_cnn_forward: level larger than the arena");
        PD_CUDA(h, cudaMemcpy2DAsync(h->d_pyr, lp, d_level, pitch, Wk, Hk, cudaMemcpyDeviceToDevice, s));
        d_level = h->d_pyr;
        pitch = lp;
    }
    Plan p;
    plan_level(p, 0, 0, Wk, Hk, Wk, Hk, 0, pitch);
    p.c_items.clear();
    p.strips.clear();
    p.s_items.clear();
    p.t_items.clear();
    p.tabs.clear();
    for (int cy = 0; cy < Hc; cy += kCnnTile)
        for (int cx = 0; cx < Wc; cx += kCnnTile) p.cnn_items.push_back({0, cy, cx, 0});
    Packed o;
    int r = upload_plan(h, s, p, o, d_level);
    if (r != PD_OK) return r;
    PD_CUDA(h, launch_cnn(s, dptr<LevelDesc>(h, o.levels), p.levels[0].rows > 0 ? 1 : 0,
                          dptr<CUtensorMap>(h, o.tmaps), dptr<CnnItem>(h, o.cnn_items), (int)p.cnn_items.size(),
                          cnn_weights(h), d_h, h_pitch, d_logits, max_pool_tiles(p), h->d_err));
    return PD_OK;
}

int pd_cnn_train_step(pd_handle *h, void *stream, float pos_weight, float label_threshold, float lr) {
    if (!h) return PD_EINVAL;
    if (!h->detected || !h->cache_valid) return fail(h, PD_ESTATE, "pd_cnn_train_step needs a pd_detect batch");
    if (h->ran_proposal) return fail(h, PD_ESTATE, "labels need a pd_detect batch with the proposal off");
    if (!h->cnn_loaded) return fail(h, PD_ESTATE, "no proposal parameters (pd_cnn_set_params)");
    if (!(pos_weight > 0.f) || !(lr >= 0.f)) return fail(h, PD_EINVAL, "bad pos_weight / lr");
    const Plan &p = h->plan;
    const int nl = (int)p.levels.size();
    std::vector<TrainLevel> tl(nl);
    int64_t n16 = 0, n32 = 0, nwin = 0;
    for (int k = 0; k < nl; ++k) {
        const LevelDesc &L = p.levels[k];
        TrainLevel &T = tl[k];
        T.level = k;
        T.H1 = (L.Hk + 1) / 2; T.W1 = (L.Wk + 1) / 2;
        T.H2 = (T.H1 + 1) / 2; T.W2 = (T.W1 + 1) / 2;
        T.H3 = (T.H2 + 1) / 2; T.W3 = (T.W2 + 1) / 2;
        T.pad = 0;
        T.a1 = n16; n16 += (int64_t)16 * T.H1 * T.W1;
        T.a2 = n16; n16 += (int64_t)32 * T.H2 * T.W2;
        T.a3 = n32; n32 += (int64_t)32 * T.H3 * T.W3;
        nwin += (int64_t)L.rows * L.cols;
    }
    if (nwin == 0) return fail(h, PD_EINVAL, "batch has no window");
    // workspace: tl | act16 (bf16) | act32 | dz16 | dz32 | dh plane | dz | level losses
    const int64_t rows = h->atlas.rows, P = h->atlas.pitch;
    const size_t need = round_up((int64_t)nl * sizeof(TrainLevel), 256) + round_up(n16 * 2, 256) +
                        round_up(n32 * 4, 256) + round_up(n16 * 4, 256) + round_up(n32 * 4, 256) +
                        round_up(rows * P * 4, 256) + round_up(h->score_cap * 4, 256) + round_up((int64_t)nl * 4, 256);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (need > h->train_ws_bytes) {
        PD_CUDA(h, cudaStreamSynchronize(s));
        if (h->train_ws) cudaFree(h->train_ws);
        h->train_ws = nullptr;
        h->train_ws_bytes = 0;
        if (cudaMalloc(&h->train_ws, need) != cudaSuccess) return fail(h, PD_ENOMEM, "training workspace");
        h->train_ws_bytes = need;
    }
    unsigned char *w = h->train_ws;
    auto take = [&](int64_t bytes) {
        unsigned char *at = w;
        w += round_up(bytes, 256);
        return at;
    };
    TrainArgs a{};
    a.tl = reinterpret_cast<TrainLevel *>(take((int64_t)nl * sizeof(TrainLevel)));
    a.act16 = reinterpret_cast<__nv_bfloat16 *>(take(n16 * 2));
    a.act32 = reinterpret_cast<float *>(take(n32 * 4));
    a.dz16 = reinterpret_cast<float *>(take(n16 * 4));
    a.dz32 = reinterpret_cast<float *>(take(n32 * 4));
    a.dh = reinterpret_cast<float *>(take(rows * P * 4));
    a.dz = reinterpret_cast<float *>(take(h->score_cap * 4));
    a.level_loss = reinterpret_cast<float *>(take((int64_t)nl * 4));
    PD_CUDA(h, cudaMemcpyAsync((void *)a.tl, tl.data(), tl.size() * sizeof(TrainLevel), cudaMemcpyHostToDevice, s));
    PD_CUDA(h, cudaStreamSynchronize(s));  // the host vector goes out of scope
    a.n_levels = nl;
    a.levels = dptr<LevelDesc>(h, h->packed.levels);
    a.pyr = h->d_pyr;
    a.w = cnn_weights(h);
    a.master = h->cnn;
    a.m = h->cnn + kCnnParams;
    a.v = h->cnn + 2 * kCnnParams;
    a.grad = h->cnn + 3 * kCnnParams;
    a.wr = h->cnn + 4 * kCnnParams;
    a.hmap = h->hmap;
    a.hp = (int32_t)P;
    a.logits = h->logits;
    a.scores = h->d_scores;
    a.label_thr = label_threshold;
    a.pos_weight = pos_weight;
    a.inv_n = 1.0f / (float)nwin;
    a.pool_tiles = max_pool_tiles(p);
    a.lr = lr;
    a.beta1 = 0.9f;
    a.beta2 = 0.999f;
    a.eps = 1e-8f;
    if (lr > 0.f) {
        ++h->adam_t;
        a.c1 = 1.0f - (float)std::pow(0.9, h->adam_t);
        a.c2 = 1.0f - (float)std::pow(0.999, h->adam_t);
        h->frag_stale = true;
    }
    h->train_levels = nl;
    h->train_loss_ptr = a.level_loss;
    PD_CUDA(h, launch_train_step(s, a));
    return PD_OK;
}

int pd_cnn_train_loss(pd_handle *h, void *stream, float *loss) {
    if (!h || !loss) return PD_EINVAL;
    if (!h->train_ws || h->train_levels <= 0) return fail(h, PD_ESTATE, "no training step yet");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    PD_CUDA(h, cudaStreamSynchronize(s));
    // one partial loss per level (already weighted by its share of the windows)
    std::vector<float> ll(h->train_levels);
    PD_CUDA(h, cudaMemcpy(ll.data(), h->train_loss_ptr, ll.size() * 4, cudaMemcpyDeviceToHost));
    double sum = 0;
    for (float v : ll) sum += v;
    *loss = (float)sum;
    return PD_OK;
}

int pd_set_proposal(pd_handle *h, int enable, float keep_logit_threshold) {
    if (!h) return PD_EINVAL;
    if (enable && !h->cnn_loaded) return fail(h, PD_ESTATE, "no proposal parameters (pd_cnn_set_params)");
    if (std::isnan(keep_logit_threshold)) return fail(h, PD_EINVAL, "threshold is NaN");
    h->proposal = enable != 0;
    h->tau = keep_logit_threshold;
    invalidate_cache(h);
    return PD_OK;
}

int pd_set_tuning(pd_handle *h, const pd_tuning *t) {
    if (!h || !t) return PD_EINVAL;
    if ((t->k1_groups != 4 && t->k1_groups != 8 && t->k1_groups != 16) || t->tc_item_rows < kTcMinChunk ||
        t->tc_item_rows > kTcChunk)
        return fail(h, PD_EINVAL, "tuning: k1_groups %d, tc_item_rows %d", t->k1_groups, t->tc_item_rows);
    h->tuning = *t;
    invalidate_cache(h);
    return PD_OK;
}

int pd_get_tuning(const pd_handle *h, pd_tuning *t) {
    if (!h || !t) return PD_EINVAL;
    *t = h->tuning;
    return PD_OK;
}

int pd_set_proposal_levels(pd_handle *h, int level_step) {
    if (!h) return PD_EINVAL;
    if (level_step < 1 || level_step > 16) return fail(h, PD_EINVAL, "level step %d outside [1, 16]", level_step);
    h->p.proposal_level_step = level_step;
    invalidate_cache(h);
    return PD_OK;
}

int pd_logits(const pd_handle *h, const float **d_logits, int64_t *total) {
    if (!h || !d_logits || !total) return PD_EINVAL;
    *d_logits = h->logits;
    *total = h->detected && h->ran_proposal ? h->plan.score_floats : 0;
    return PD_OK;
}

int pd_stage_times(const pd_handle *h, float *ms) {
    if (!h || !ms) return PD_EINVAL;
    if (!h->timed || !h->synced) return PD_ESTATE;
    // events: 0 pyramid 5 proposal 1 cells 2 scores 3 nms 4
    static const int from[5] = {0, 1, 2, 3, 5}, to[5] = {5, 2, 3, 4, 1};
    for (int i = 0; i < 5; ++i)
        if (cudaEventElapsedTime(&ms[i], h->stage_ev[from[i]], h->stage_ev[to[i]]) != cudaSuccess) return PD_ECUDA;
    return PD_OK;
}

int pd_frame_levels(const pd_handle *h, int frame, int *n_levels, pd_level_info *info) {
    if (!h || !n_levels || !info || !h->detected) return PD_EINVAL;
    if (frame < 0 || frame >= (int)h->plan.frames.size()) return PD_EINVAL;
    const FrameDesc &fd = h->plan.frames[frame];
    *n_levels = fd.n_levels;
    for (int k = 0; k < fd.n_levels; ++k) {
        const LevelDesc &L = h->plan.levels[fd.first_level + k];
        info[k].width = L.Wk;
        info[k].height = L.Hk;
        info[k].cells_x = L.Wc;
        info[k].cells_y = L.Hc;
        info[k].rows = L.rows;
        info[k].cols = L.cols;
        info[k].score_offset = L.score_off;
    }
    return PD_OK;
}

int pd_scores(const pd_handle *h, const float **d_scores, int64_t *total) {
    if (!h || !d_scores || !total) return PD_EINVAL;
    *d_scores = h->d_scores;
    *total = h->detected ? h->plan.score_floats : 0;
    return PD_OK;
}

int pd_boxes(const pd_handle *h, int frame, pd_box *out, int cap, int *count) {
    if (!h || !count || (cap > 0 && !out)) return PD_EINVAL;
    if (!h->synced) return PD_ESTATE;
    if (frame < 0 || frame >= (int)h->plan.frames.size()) return PD_EINVAL;
    const int kept = h->h_counts[2 * frame];
    *count = kept;
    const int n = std::min(kept, cap);
    if (n > 0)
        std::memcpy(out, h->h_boxes + (size_t)frame * h->p.max_boxes_per_frame, (size_t)n * sizeof(pd_box));
    return PD_OK;
}

// ----------------------------------------------------------------------------- stage entry points
int pd_resize_levels(pd_handle *h, void *stream, const uint8_t *d_frame, int W, int H, int pitch,
                     int n_levels, const int32_t *Wk, const int32_t *Hk, uint8_t *d_levels,
                     const int64_t *level_offsets, const int32_t *level_pitches) {
    if (!h) return PD_EINVAL;
    invalidate_cache(h);  // the descriptor region is reused below
    if (!d_frame || !d_levels || !Wk || !Hk || !level_offsets || !level_pitches || W < 1 || H < 1 ||
        pitch < W || n_levels < 0 || n_levels > PD_MAX_LEVELS)
        return fail(h, PD_EINVAL, "pd_resize_levels: bad argument");
    Plan p;
    FrameDesc fd{};
    fd.ptr = d_frame;
    fd.W = W;
    fd.H = H;
    fd.pitch = pitch;
    fd.first_level = 0;
    fd.n_levels = n_levels;
    for (int k = 0; k < n_levels; ++k) {
        if (Wk[k] < 1 || Hk[k] < 1 || Wk[k] > 4 * W || Hk[k] > 4 * H || level_pitches[k] < Wk[k])
            return fail(h, PD_EINVAL, "pd_resize_levels: level %d size %dx%d", k, Wk[k], Hk[k]);
        plan_level(p, 0, k, W, H, Wk[k], Hk[k], level_offsets[k], level_pitches[k]);
    }
    fd.rbw = staged_bytes(p, fd);
    for (int y = 0; y < H; y += kResizeTH)
        for (int x = 0; x < W; x += kResizeTW) p.r_items.push_back({0, x, y, 0});
    p.frames.push_back(fd);
    p.c_items.clear();
    p.strips.clear();
    p.s_items.clear();
    p.t_items.clear();
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Packed o;
    int r = upload_plan(h, s, p, o);
    if (r != PD_OK) return r;
    PD_CUDA(h, launch_resize(s, dptr<FrameDesc>(h, o.frames), dptr<LevelDesc>(h, o.levels),
                             dptr<int32_t>(h, o.tabs), d_levels, dptr<ResizeItem>(h, o.r_items),
                             (int)p.r_items.size(), h->tuning.k1_groups));
    return PD_OK;
}

int pd_cell_features(pd_handle *h, void *stream, const uint8_t *d_level, int Wk, int Hk, int pitch,
                     float *d_hog, int64_t hog_plane, uint8_t *d_lbp, int64_t lbp_plane, int cell_pitch) {
    if (!h) return PD_EINVAL;
    invalidate_cache(h);  // the descriptor region is reused below
    const int Wc = Wk / 8, Hc = Hk / 8;
    if (!d_level || !d_hog || !d_lbp || Wk < 1 || Hk < 1 || pitch < Wk || cell_pitch < Wc ||
        cell_pitch % 16 != 0 || hog_plane < (int64_t)Hc * cell_pitch || lbp_plane < (int64_t)Hc * cell_pitch)
        return fail(h, PD_EINVAL, "pd_cell_features: bad argument");
    Plan p;
    plan_level(p, 0, 0, Wk, Hk, Wk, Hk, 0, pitch);
    plan_strips(p, h->sm_count * kStripWarpsPerSm);
    p.s_items.clear();
    p.t_items.clear();
    p.tabs.clear();
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Packed o;
    int r = upload_plan(h, s, p, o);
    if (r != PD_OK) return r;
    CellAtlas a{};
    a.hog = d_hog;
    a.lbp = d_lbp;
    a.hog_plane = hog_plane;
    a.lbp_plane = lbp_plane;
    a.pitch = cell_pitch;
    a.rows = Hc;
    PD_CUDA(h, launch_cell_stage(h, s, dptr<LevelDesc>(h, o.levels), d_level, a, p, o, nullptr,
                                 kFeatHog | kFeatLbp | (features_of(h->p.flags) & kFeatHogBlock)));
    return PD_OK;
}

int pd_window_scores(pd_handle *h, void *stream, const float *d_hog, int64_t hog_plane,
                     const uint8_t *d_lbp, int64_t lbp_plane, int cell_pitch, int cells_x, int cells_y,
                     float *d_scores) {
    if (!h) return PD_EINVAL;
    invalidate_cache(h);  // the descriptor region is reused below
    if (!d_hog || !d_lbp || !d_scores || cells_x < 0 || cells_y < 0 || cell_pitch < cells_x ||
        cell_pitch % 16 != 0 || hog_plane % 4 != 0 || lbp_plane % 16 != 0 ||
        hog_plane < (int64_t)cells_y * cell_pitch || lbp_plane < (int64_t)cells_y * cell_pitch ||
        (reinterpret_cast<uintptr_t>(d_hog) & 15) || (reinterpret_cast<uintptr_t>(d_lbp) & 15))
        return fail(h, PD_EINVAL, "pd_window_scores: bad argument");
    Plan p;
    p.tc_rows = h->tuning.tc_item_rows;
    plan_level(p, 0, 0, 8 * cells_x, 8 * cells_y, 8 * cells_x, 8 * cells_y, 0, 8 * cells_x, nullptr,
               h->tile_cost);
    p.c_items.clear();
    p.strips.clear();
    p.tabs.clear();
    if (p.s_items.empty()) return PD_OK;
    const bool fp32 = (h->p.flags & PD_FLAG_SVM_FP32) != 0;
    if (fp32)
        p.t_items.clear();
    else
        p.s_items.clear();
    order_tc(p.t_items);
    CUtensorMap hm[kSvmShapes], lm[kSvmShapes], th, tl;
    const int64_t rows = std::max(cells_y, 1);
    if (encode_svm_maps(hm, lm, d_hog, d_lbp, cell_pitch, rows, hog_plane, lbp_plane) != PD_OK ||
        encode_tc_maps(&th, &tl, d_hog, d_lbp, cell_pitch, rows, hog_plane, lbp_plane,
                       hog_planes_of(h->p.flags)) != PD_OK)
        return fail(h, PD_ECUDA, "pd_window_scores: tensor map encoding failed");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Packed o;
    int r = upload_plan(h, s, p, o);
    if (r != PD_OK) return r;
    PD_CUDA(h, cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), s));
    if (fp32) {
        PD_CUDA(h, launch_svm(s, hm, lm, dptr<LevelDesc>(h, o.levels), h->d_w, h->bias, h->p.l2hys_clip,
                              d_scores, dptr<SvmItem>(h, o.s_items), (int)p.s_items.size(), h->d_err));
    } else {
        PD_CUDA(h, cudaMemsetAsync(h->d_queue, 0, sizeof(int), s));
        PD_CUDA(h, launch_svm_tc(s, th, tl, dptr<LevelDesc>(h, o.levels), dptr<TcItem>(h, o.t_items),
                                 (int)p.t_items.size(), h->d_queue, h->sm_count, h->d_w, h->bias,
                                 h->p.l2hys_clip, d_scores, nullptr, h->d_err, hog_planes_of(h->p.flags)));
    }
    return PD_OK;
}

int pd_nms_maps(pd_handle *h, void *stream, const float *d_scores, int n_levels, const int32_t *rows,
                const int32_t *cols, const int32_t *Wk, const int32_t *Hk, int W, int H, pd_box *d_boxes,
                int max_boxes, int32_t *d_counts) {
    if (!h) return PD_EINVAL;
    invalidate_cache(h);  // the descriptor region is reused below
    if (!d_scores || !rows || !cols || !Wk || !Hk || !d_boxes || !d_counts || n_levels < 0 ||
        n_levels > PD_MAX_LEVELS || max_boxes < 1 || max_boxes > 16384 || W < 1 || H < 1)
        return fail(h, PD_EINVAL, "pd_nms_maps: bad argument");
    Plan p;
    FrameDesc fd{};
    fd.W = W;
    fd.H = H;
    fd.first_level = 0;
    fd.n_levels = n_levels;
    int64_t off = 0;
    for (int k = 0; k < n_levels; ++k) {
        if (rows[k] < 0 || cols[k] < 0 || rows[k] > 4096 || cols[k] > 4096 || Wk[k] < 1 || Hk[k] < 1)
            return fail(h, PD_EINVAL, "pd_nms_maps: level %d", k);
        LevelDesc L{};
        L.W = W;
        L.H = H;
        L.Wk = Wk[k];
        L.Hk = Hk[k];
        L.rows = rows[k];
        L.cols = cols[k];
        L.score_off = off;
        off += (int64_t)rows[k] * cols[k];
        p.levels.push_back(L);
    }
    p.frames.push_back(fd);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Packed o;
    int r = upload_plan(h, s, p, o);
    if (r != PD_OK) return r;
    PD_CUDA(h, launch_nms(s, dptr<FrameDesc>(h, o.frames), dptr<LevelDesc>(h, o.levels), 1, d_scores,
                          h->p.threshold, h->p.nms_iou, h->d_nms_scratch, h->p.max_candidates_per_frame,
                          d_boxes, max_boxes, d_counts,
                          nms_cluster_for(1, h->sm_count, h->p.max_candidates_per_frame)));
    return PD_OK;
}

namespace {
// Scratch of the kernel-scheme entries, grown on demand (the stream is
// synchronised first: earlier work on it may still use the old buffer).
int scheme_scratch(pd_handle *h, cudaStream_t s, size_t need) {
    if (need <= h->scheme_ws_bytes) return PD_OK;
    PD_CUDA(h, cudaStreamSynchronize(s));
    if (h->scheme_ws) cudaFree(h->scheme_ws);
    h->scheme_ws = nullptr;
    h->scheme_ws_bytes = 0;
    if (cudaMalloc(&h->scheme_ws, need) != cudaSuccess) return fail(h, PD_ENOMEM, "scheme scratch");
    h->scheme_ws_bytes = need;
    return PD_OK;
}
}  // namespace

int pd_scheme_cells(pd_handle *h, void *stream, int scheme, const uint8_t *d_level, int Wk, int Hk, int pitch,
                    float *d_hog, int64_t hog_plane, uint8_t *d_lbp, int64_t lbp_plane, int cell_pitch) {
    if (!h) return PD_EINVAL;
    const int Wc = Wk / 8, Hc = Hk / 8;
    const bool lbp_s = scheme == PD_SCHEME_LBP_NAIVE || scheme == PD_SCHEME_LBP_SCALABLE;
    const bool hog_s =
        scheme == PD_SCHEME_HOG_GLOBAL || scheme == PD_SCHEME_HOG_LOCAL || scheme == PD_SCHEME_HOG_SHARED;
    if (!(lbp_s || hog_s) || !d_level || Wk < 1 || Hk < 1 || pitch < Wk || cell_pitch < Wc ||
        (lbp_s && (!d_lbp || lbp_plane < (int64_t)Hc * cell_pitch)) ||
        (hog_s && (!d_hog || hog_plane < (int64_t)Hc * cell_pitch)))
        return fail(h, PD_EINVAL, "pd_scheme_cells: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int r = scheme_scratch(h, s, scheme_cells_scratch(Wk, Hk));
    if (r != PD_OK) return r;
    PD_CUDA(h, launch_scheme_cells(s, scheme, d_level, Wk, Hk, pitch, d_hog, hog_plane, d_lbp, lbp_plane,
                                   cell_pitch, h->d_lbp_map, h->scheme_ws,
                                   (h->p.flags & PD_FLAG_HOG_PER_BLOCK) != 0));
    return PD_OK;
}

int pd_scheme_window_scores(pd_handle *h, void *stream, int scheme, const float *d_hog, int64_t hog_plane,
                            const uint8_t *d_lbp, int64_t lbp_plane, int cell_pitch, int cells_x, int cells_y,
                            float *d_scores) {
    if (!h) return PD_EINVAL;
    if ((scheme != PD_SCHEME_SVM_NAIVE && scheme != PD_SCHEME_SVM_WARP) || !d_hog || !d_lbp || !d_scores ||
        cells_x < 0 || cells_y < 0 || cell_pitch < cells_x || hog_plane < (int64_t)cells_y * cell_pitch ||
        lbp_plane < (int64_t)cells_y * cell_pitch)
        return fail(h, PD_EINVAL, "pd_scheme_window_scores: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int r = scheme_scratch(h, s, scheme_scores_scratch(cells_x, cells_y));
    if (r != PD_OK) return r;
    PD_CUDA(h, launch_scheme_scores(s, scheme, d_hog, hog_plane, d_lbp, lbp_plane, cell_pitch, cells_x, cells_y,
                                    h->d_w, h->bias, h->p.l2hys_clip, d_scores, h->scheme_ws,
                                    (h->p.flags & PD_FLAG_HOG_PER_BLOCK) != 0));
    return PD_OK;
}

}  // extern "C"
