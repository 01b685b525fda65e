// Internal declarations shared by the CUDA translation units of the detector
// library: work descriptors, arena layout constants and kernel launchers.
#pragma once

#include <cuda.h>
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
    int32_t pad;
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
    int32_t xtab_off;   // Q11 source-column table of this level (Wk entries)
    int32_t ytab_off;   // Q11 source-row table of this level (Hk entries)
};

// Work items (one CTA each).
struct ResizeItem { int32_t frame, x0, y0, pad; };   // source tile of a frame
struct CellItem { int32_t level, cx0, cy0, pad; };   // cell tile of a level
struct SvmItem { int32_t level, wx0, wy0, shape; };  // window tile of a level, tile shape index

// Tiles.
constexpr int kResizeTW = 128;  // source tile width  (pixels)
constexpr int kResizeTH = 32;   // source tile height (pixels)
constexpr int kCellTW = 15;     // cells per cell tile along x (128 threads = 8*15+8 columns)
constexpr int kCellTH = 8;      // cells per cell tile along y
constexpr int kSvmShapes = 4;   // K4 tile shapes: 32x16, 64x8, 32x8, 64x4 windows

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
    float *hog;        // 9 planes
    uint8_t *lbp;      // 59 planes
    int64_t hog_plane; // elements per HOG plane
    int64_t lbp_plane; // elements per LBP plane
    int32_t pitch;     // elements per row (multiple of 16)
    int32_t rows;      // rows per plane
};

// One-time per-device kernel attribute set-up (dynamic shared memory opt-in).
cudaError_t init_cells();
cudaError_t init_svm();
cudaError_t init_nms();

// Kernel launchers (host functions defined next to their kernels).
cudaError_t launch_resize(cudaStream_t s, const FrameDesc *d_frames, const LevelDesc *d_levels,
                          const int32_t *d_tabs, uint8_t *pyr, const ResizeItem *d_items,
                          int n_items);
cudaError_t launch_cells(cudaStream_t s, const LevelDesc *d_levels, const uint8_t *pyr,
                         CellAtlas atlas, const CellItem *d_items, int n_items, const uint8_t *d_lbp_map);
cudaError_t launch_svm(cudaStream_t s, const CUtensorMap *hog_maps, const CUtensorMap *lbp_maps,
                       const LevelDesc *d_levels, const float *d_w, float bias, float clip,
                       float *scores, const SvmItem *d_items, int n_items, unsigned *d_err);
cudaError_t launch_nms(cudaStream_t s, const FrameDesc *d_frames, const LevelDesc *d_levels,
                       int n_frames, const float *scores, float threshold, float iou,
                       float4 *scratch, int max_cand, pd_box *boxes, int max_boxes,
                       int32_t *counts);

// Encodes a 3-D tiled tensor map over plane-major cell planes.
int encode_plane_map(CUtensorMap *map, void *base, CUtensorMapDataType dtype, int elem_bytes,
                     int64_t pitch, int64_t rows, int64_t planes, int64_t plane_stride_elems,
                     uint32_t box_x, uint32_t box_y, uint32_t box_planes);

// Host-side tables.
void build_lbp_bin_table(uint8_t table[256]);

}  // namespace pd
