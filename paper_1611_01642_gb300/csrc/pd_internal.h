// Internal declarations shared by the CUDA translation units of the detector
// library: work descriptors, arena layout constants and kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pd.h"

namespace pd {

constexpr int kHogBins = PD_HOG_BINS;
constexpr int kLbpBins = PD_LBP_BINS;
constexpr int kHogDim = 36;
constexpr int kFeat = PD_FEAT;
constexpr int kWinBW = PD_WIN_BW;
constexpr int kWinBH = PD_WIN_BH;
constexpr int kWPad = 8;  // template row j padded from 7 to 8 floats (two float4)

// Device error word bits (OR-ed by kernels, read by pd_sync).
constexpr unsigned kErrTimeout = 1u;
constexpr unsigned kErrBounds = 2u;

// One frame of a batch.
struct FrameDesc {
    const uint8_t *ptr;
    int32_t W, H, pitch;
    int32_t first_level, n_levels;  // range in the LevelDesc table
    int32_t rbw;                    // K1: source bytes staged per tile row (max of the levels' rspan)
};

// One (frame, level).
struct LevelDesc {
    int64_t img_off;    // byte offset of the level image in the pyramid buffer
    int64_t score_off;  // float offset of the score map in the score buffer
    int32_t frame;      // index in the FrameDesc table
    int32_t level;      // level number within the frame
    int32_t W, H;       // frame size
    int32_t Wk, Hk;     // level size
    int32_t Wc, Hc;     // cells
    int32_t img_pitch;  // bytes
    int32_t cell_row;   // first row of this level in the cell atlas
    int32_t rows, cols; // score map size (0 when no window fits)
    int32_t xtab_off;   // K1 column weights: per group of rgroup output columns an int4 of packed
                        // weights (2048 - a) | a << 16 (16-byte aligned; unused lanes 0)
    int32_t ytab_off;   // K1 row table: per output row an int2 {byte offset of its top source row's
                        // quad row (source row * 4 * kResizeQP), (8192 - 4 a) | 4 a << 16}
    int32_t citem0;     // index of this level's first K2+K3 item
    int32_t ctx;        // K2+K3 tiles per row of cells
    int32_t xbnd_off;   // per K1 source-tile column t: first column group whose first source is >= 128 t
    int32_t ybnd_off;   // per K1 source-tile row t: first output row whose source is >= 32 t
    int32_t rgroup;     // K1 output columns per group: 4, or 1 when a group of 4 reaches past the halo
    int32_t rspan;      // K1 source bytes a tile row needs for this level (<= kResizeBW)
    int32_t xq_off;     // K1 column quads: per group one word, byte i = quad index of column i
    int32_t hsrc;       // proposal: index (in this table) of the level whose head map this level uses
    int32_t tc_map;     // tensor-core K4: pair (HOG, LBP) of cell-plane maps whose x extent is this
                        // level's width (index into the plan's map table; -1: none)
};

// Work items (one CTA each).
struct ResizeItem { int32_t frame, x0, y0, pad; };   // source tile of a frame
struct CellItem { int32_t level, cx0, cy0, pad; };   // cell tile of a level
struct SvmItem { int32_t level, wx0, wy0, shape; };  // window tile of a level, tile shape index
struct TcItem { int32_t level, wx0, wy0, wy1; };     // tensor-core K4: window columns [wx0, wx0 + 104), rows [wy0, wy1)
struct StripItem { int32_t level, cx0, cy0, cy1; };  // K2+K3 warp: cells [cx0, cx0 + 15) x rows [cy0, cy1)

// Tiles.
constexpr int kResizeTW = 128;  // source tile width  (pixels)
constexpr int kResizeTH = 32;   // source tile height (pixels)
constexpr int kResizeBW = 160;  // source bytes staged per tile row at most (tile + right halo)
// K1 shared-memory quad word of source column d of a tile row (skewed by d / 32)
__host__ __device__ inline int resize_quad_index(int d) { return d + (d >> 5); }
// K1 quad row pitch in words: > resize_quad_index(kResizeBW - 2) and 1 mod 32, so that
// quad rows sy and sy + 1 start one bank apart
constexpr int kResizeQP = 193;
constexpr int kCellTW = 15;     // cells per cell tile along x (8*15+8 = 128 columns: 128 threads, or 32 lanes x 4)
constexpr int kCellTH = 8;      // cells per cell tile along y
constexpr int kStripTiles = 4;  // cell tiles per K2+K3 strip (one warp each), top to bottom, at most
constexpr int kStripWarpsPerSm = 16;  // K2+K3 warps resident per SM (4 CTAs of 4)
constexpr int kSvmShapes = 7;   // K4 tile shapes: 32x16, 64x8, 32x8, 64x4, 64x2, 32x12, 32x4 windows
constexpr int kTcStrip = 104;   // tensor-core K4: window columns per item
constexpr int kTcChunk = 64;    // tensor-core K4: window rows per item at most (tunable down to kTcMinChunk)
constexpr int kTcMinChunk = 8;

struct SvmShapeInfo {
    int tw, th;     // windows per tile along x / y
    int hog_box_x;  // TMA box width of the HOG cell planes (cells)
    int lbp_box_x;  // TMA box width of the LBP cell planes (cells)
    int cell_rows;  // TMA box height (cell rows)
};
SvmShapeInfo svm_shape(int s);
int svm_lbp_chunk();  // LBP planes per TMA box

// Cell atlas: plane-major [plane][atlas_rows][pitch]; pitch in elements.
struct CellAtlas {
    float *hog;        // 9 planes (36 for per-block HOG)
    uint8_t *lbp;      // 59 planes
    int64_t hog_plane; // elements per HOG plane
    int64_t lbp_plane; // elements per LBP plane
    int32_t pitch;     // elements per row (multiple of 16)
    int32_t rows;      // rows per plane
};

// One-time per-device kernel attribute set-up (dynamic shared memory opt-in).
cudaError_t init_cells();
cudaError_t init_svm();
cudaError_t init_nms(bool occupancy = true);  // occupancy: also the clusters that fit (for the launch policy)
cudaError_t init_resize();

// Kernel launchers (host functions defined next to their kernels).
// k1_groups: column groups per warp task (4, 8 or 16)
cudaError_t launch_resize(cudaStream_t s, const FrameDesc *d_frames, const LevelDesc *d_levels,
                          const int32_t *d_tabs, uint8_t *pyr, const ResizeItem *d_items,
                          int n_items, int k1_groups = 8);
// CTA-per-tile K2+K3 for per-block HOG: feat = kFeatHogBlock | kFeatHog
// (| kFeatLbp); 36 HOG planes, the 4 block-restricted histograms of every
// cell, plane 9 q + bin. Other feature sets: cudaErrorInvalidValue (they
// run on launch_cells_warp).
constexpr int kFeatHog = 1, kFeatLbp = 2, kFeatHogBlock = 4;
cudaError_t launch_cells(cudaStream_t s, const LevelDesc *d_levels, const uint8_t *pyr,
                         CellAtlas atlas, const CellItem *d_items, int n_items, const uint8_t *d_lbp_map,
                         const uint32_t *c_flag = nullptr, int feat = kFeatHog | kFeatLbp);
// Default K2+K3 (HOG and / or LBP without per-block HOG): one warp per strip.
cudaError_t init_cells_warp();
// Persistent warps over a strip queue (*d_queue must be 0 at launch).
cudaError_t launch_cells_warp(cudaStream_t s, const LevelDesc *d_levels, const uint8_t *pyr, CellAtlas atlas,
                              const StripItem *d_items, int n_items, int *d_queue, int sm_count,
                              const uint8_t *d_lbp_map, const uint32_t *c_flag, int feat);
cudaError_t launch_proposal_flags(cudaStream_t s, const LevelDesc *d_levels, const SvmItem *d_items, int n_items,
                                  const float *logits, float tau, uint32_t *s_flag, uint32_t *c_flag,
                                  bool per_window);
cudaError_t launch_svm(cudaStream_t s, const CUtensorMap *hog_maps, const CUtensorMap *lbp_maps,
                       const LevelDesc *d_levels, const float *d_w, float bias, float clip,
                       float *scores, const SvmItem *d_items, int n_items, unsigned *d_err,
                       const uint32_t *s_flag = nullptr);
// Tensor-core K4: persistent CTAs (grid at most one per SM) over an item
// queue (*d_queue must be 0 at launch); c_flag non-null selects the sparse
// path. hog_map / lbp_map: 3-D maps over the cell planes with boxes of
// 112 x 1 x hog_planes (f32; 9, or 36 for per-block HOG) and 128 x 1 x 59 (u8).
cudaError_t init_svm_tc();
int svm_tc_smem_bytes(int hog_planes = kHogBins);
// level_maps: null, or 2 maps per entry of LevelDesc::tc_map (HOG, LBP) in device
// memory (64-byte aligned) whose x extent is the level's width, so that a box
// reaching past it reads zeros instead of the atlas row's padding.
cudaError_t launch_svm_tc(cudaStream_t s, const CUtensorMap &hog_map, const CUtensorMap &lbp_map,
                          const LevelDesc *d_levels, const TcItem *d_items, int n_items, int *d_queue, int grid,
                          const float *d_w, float bias, float clip, float *scores, const uint32_t *c_flag,
                          unsigned *d_err, int hog_planes = kHogBins, const CUtensorMap *level_maps = nullptr);
// Per-frame NMS scratch (float4 units) for a candidate cap: the decoded
// boxes, plus the sort keys when the cap is above 16,384 (shared memory
// holds them below).
__host__ __device__ inline size_t nms_scratch_float4s(int cap) {
    size_t p = 1;
    while (p < (size_t)cap) p <<= 1;
    return cap > 16384 ? (size_t)cap + p / 2 : (size_t)cap;
}
// cluster: CTAs per frame (1, 2, 4 or 8; a thread-block cluster that shares
// the frame's suppression passes); nms_cluster_for picks it for a batch.
// sched: nms_sched_ints(n_frames) ints of device scratch, or null. With it,
// a batch of more frames than clusters that fit on the GPU at once runs on
// persistent clusters that take the frames by a ticket queue, most
// candidates first (two more kernels count and order them); without it,
// one cluster per frame.
cudaError_t launch_nms(cudaStream_t s, const FrameDesc *d_frames, const LevelDesc *d_levels,
                       int n_frames, const float *scores, float threshold, float iou,
                       float4 *scratch, int max_cand, pd_box *boxes, int max_boxes,
                       int32_t *counts, int cluster = 1, int *sched = nullptr);
int nms_cluster_for(int n_frames, int sm_count, int max_cand);
// launch_nms with sched runs the persistent form (count, order, NMS kernels)
bool nms_persistent(int n_frames, int cluster);
int nms_launches(int n_frames, int cluster);  // kernels launch_nms with sched starts
constexpr size_t nms_sched_ints(int n_frames) { return 1 + 33 * (size_t)n_frames; }

// ---- the paper's kernel schemes (comparison with the fused kernels)
size_t scheme_cells_scratch(int Wk, int Hk);
cudaError_t launch_scheme_cells(cudaStream_t s, int scheme, const uint8_t *img, int Wk, int Hk, int pitch, float *hog,
                                int64_t hog_plane, uint8_t *lbp, int64_t lbp_plane, int cell_pitch,
                                const uint8_t *bin_of, unsigned char *scratch, bool per_block);
size_t scheme_scores_scratch(int cells_x, int cells_y);
cudaError_t launch_scheme_scores(cudaStream_t s, int scheme, const float *hog, int64_t hog_plane,
                                 const uint8_t *lbp, int64_t lbp_plane, int cell_pitch, int cells_x, int cells_y,
                                 const float *wt, float bias, float clip, float *scores, unsigned char *scratch,
                                 bool per_block);

// ---- learned window proposal
constexpr int kCnnParams = 14210;  // flat order: w1 b1 w2 b2 w3 b3 wh bh v bv
constexpr int kOffW1 = 0, kOffB1 = 144, kOffW2 = 160, kOffB2 = 4768, kOffW3 = 4800, kOffB3 = 14016;
constexpr int kOffWh = 14048, kOffBh = 14080, kOffV = 14081, kOffBv = 14209;
constexpr int kCnnTile = 8;        // cells per side of an inference tile

struct CnnItem { int32_t level, cy0, cx0, pad; };

// Device pointers of the inference weights.
struct CnnWeights {
    const float *in_tab;      // [256] bf16(L/255 - 0.5) as float
    const float *w1, *b1;     // [16][9] (bf16-rounded), [16]
    const uint32_t *w2frag;   // layer-2 mma B fragments [9 taps][4 n-tiles][32 lanes][2]
    const float *b2;          // [32]
    const float *w2, *w3;     // [32][16][3][3], [32][32][3][3] (bf16-rounded)
    const float *b3, *wh;     // [32], [32]
    const float *bh;          // [1]
    const float *v, *bv;      // [16][8], [1]
};

struct TrainLevel {
    int32_t level;            // index in the LevelDesc table
    int32_t H1, W1, H2, W2, H3, W3;
    int32_t pad;
    int64_t a1, a2, a3;       // element offsets: a1, a2 in the bf16 buffer, a3 in the f32 buffer
};

struct TrainArgs {
    const TrainLevel *tl;
    int n_levels;
    const LevelDesc *levels;
    const uint8_t *pyr;
    CnnWeights w;             // in_tab used; other fields refreshed from wr
    float *wr;                // rounded working copy [kCnnParams]
    float *master, *m, *v, *grad;
    __nv_bfloat16 *act16;
    float *act32, *dz16, *dz32;
    float *hmap, *dh;
    int32_t hp;
    float *logits;
    const float *scores;
    float *dz, *level_loss;
    float label_thr, pos_weight, inv_n;
    float lr, beta1, beta2, eps, c1, c2;
    int pool_tiles;           // window-pooling tiles of the largest level
};

cudaError_t init_cnn();
// Window pooling tiles: 64 x 16 windows per CTA; pool_tiles = the largest
// level's tile count (ceil(cols / 64) * ceil(rows / 16)).
constexpr int kPoolTW = 64, kPoolTH = 16;
inline int pool_tiles_of(int rows, int cols) {
    return rows > 0 && cols > 0 ? ((cols + kPoolTW - 1) / kPoolTW) * ((rows + kPoolTH - 1) / kPoolTH) : 0;
}
// Input tile of one proposal-network item: bytes [8 cx0 - 16, 8 cx0 + 80) of
// level rows [8 cy0 - 7, 8 cy0 + 65), fetched by TMA through one 2D tensor
// map per level (u8, box 96 x 72, zero fill outside the level).
constexpr int kCnnBoxW = 96, kCnnBoxH = 72;
cudaError_t launch_cnn(cudaStream_t s, const LevelDesc *d_levels, int n_levels, const CUtensorMap *lvl_maps,
                       const CnnItem *d_items, int n_items, const CnnWeights &w, float *hmap,
                       int32_t hmap_pitch, float *logits, int pool_tiles, unsigned *err);
cudaError_t launch_train_step(cudaStream_t s, const TrainArgs &a);
cudaError_t launch_round_params(cudaStream_t s, const float *master, float *wr);

// Encodes a 3-D tiled tensor map over plane-major cell planes; x extent: the
// row pitch, or width when it is positive (boxes reaching past it read zeros).
int encode_plane_map(CUtensorMap *map, void *base, CUtensorMapDataType dtype, int elem_bytes,
                     int64_t pitch, int64_t rows, int64_t planes, int64_t plane_stride_elems,
                     uint32_t box_x, uint32_t box_y, uint32_t box_planes, int64_t width = 0);

// Host-side tables.
void build_lbp_bin_table(uint8_t table[256]);

}  // namespace pd
