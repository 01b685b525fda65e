/*
 * pd.h -- C ABI of the GB300 (sm_103a) HOG+LBP sliding-window SVM pedestrian
 * detector (arXiv 1611.01642, "GPU-based pedestrian detection for autonomous
 * driving").
 *
 * The detector (Section 4.1, steps 2-5) builds an image pyramid of every
 * frame, extracts uniform-LBP and HOG cell histograms on every level,
 * normalises 2x2-cell blocks, scores every 64x128 window (stride 8) with a
 * linear SVM and finishes with non-maximum suppression. All of it runs in
 * this library's CUDA kernels; there is no CPU fallback.
 *
 * Conventions
 *  - Every call returns an int status: PD_OK (0) or a negative PD_E* code.
 *    No C++ exception crosses this boundary. Calls that take a handle record
 *    a message retrievable with pd_last_error().
 *  - "device" pointers are CUDA global-memory addresses of the current
 *    device; "host" pointers are ordinary CPU memory. The caller owns every
 *    pointer it passes; the library never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Device work is stream-ordered and asynchronous unless a
 *    function says it synchronises.
 *  - Images are 8-bit grayscale, row-major, `pitch` bytes between rows.
 *
 * Method constants (Sections 4.2-4.4): 8x8-pixel cells, 2x2-cell blocks at
 * a one-cell stride, 64x128-pixel windows = 7x15 blocks at an 8-pixel
 * stride, 9 unsigned orientation bins, 59 uniform-LBP bins, a 95-value
 * block feature (36 HOG then 59 LBP).
 */
#ifndef PD_H
#define PD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PD_ABI_VERSION 1

#define PD_OK 0
#define PD_EINVAL (-1)    /* bad argument, size or layout */
#define PD_ENOMEM (-2)    /* device or pinned-host allocation failed */
#define PD_ECUDA (-3)     /* a CUDA runtime call or kernel launch failed */
#define PD_ETIMEOUT (-4)  /* a bounded device-side wait ran out; results invalid */
#define PD_EBOUNDS (-5)   /* a device-side bounds check fired; results invalid */
#define PD_ESTATE (-6)    /* call out of order (e.g. results before pd_sync) */
#define PD_EOVERFLOW (-7) /* more NMS candidates in a frame than max_candidates */

#define PD_HOG_BINS 9
#define PD_LBP_BINS 59
#define PD_FEAT 95
#define PD_WIN_BW 7   /* window width in blocks  (64 px) */
#define PD_WIN_BH 15  /* window height in blocks (128 px) */
#define PD_TEMPLATE_SIZE (PD_WIN_BH * PD_WIN_BW * PD_FEAT) /* 9975 */
#define PD_MAX_LEVELS 96

/* pd_params.flags */
#define PD_FLAG_STAGE_TIMING 1 /* record CUDA events around each kernel of pd_detect */
/* K4 on the FP32 CUDA cores (tiled direct correlation) instead of the default
 * tensor-core kernel (one bf16-split GEMM per block row, fp32 accumulation).
 * Both stay within the score tolerance of the float64 definition; scores of
 * one kernel do not depend on how it tiles a level, and the sparse path
 * reproduces the dense path's scores of the same kernel bit for bit. */
#define PD_FLAG_SVM_FP32 2
/* The HOG-SVM and LBP-SVM pipelines of Section 4.1 (default: HOGLBP-SVM):
 * only that feature's cell histograms are computed, and windows are scored
 * with the template's weights of that feature (the others are taken as 0),
 * so a score is b + sum over the 15 x 7 blocks of the 36 HOG (or 59 LBP)
 * block features times their weights. At most one of the two. */
#define PD_FLAG_HOG_ONLY 4
#define PD_FLAG_LBP_ONLY 8
/* Per-block HOG (Section 4.3, Algorithm 5 read per block): each 16x16 block's
 * 4 cell histograms are filled by the block's own 256 pixels only. A pixel
 * votes bilinearly towards the two nearest of the block's cell centres (local
 * 3.5 and 11.5) on each axis, and votes towards a cell outside the block are
 * dropped, so it lands in 2, 4 or 8 bins. Neighbouring blocks then do not
 * share cell histograms. The default instead bins every pixel on one shared
 * cell grid, with clamped borders. The cell planes then hold 36 HOG planes
 * (see pd_cell_features). Tensor-core K4 only: not with PD_FLAG_SVM_FP32 or
 * PD_FLAG_LBP_ONLY (PD_EINVAL). */
#define PD_FLAG_HOG_PER_BLOCK 16

typedef struct pd_handle pd_handle;

/* Detector parameters. Fill with pd_params_default() and then override.
 * struct_size must be sizeof(pd_params) (ABI versioning). */
typedef struct pd_params {
    uint32_t struct_size;
    float pyr_factor;        /* scale step between pyramid levels, > 1 (1.05 or 1.2) */
    float l2hys_clip;        /* HOG L2-Hys clipping value, 0.2 */
    float threshold;         /* a window is a detection iff score > threshold (0) */
    float nms_iou;           /* NMS suppresses when IoU > nms_iou (0.5) */
    int32_t max_boxes_per_frame;      /* NMS output cap per frame (4096), <= 16384 */
    int32_t max_candidates_per_frame; /* windows above threshold per frame, <= 65536 (default 16384;
                                       * above 16384 the NMS sorts in global memory, slower) */
    int32_t max_frames;      /* frames per pd_detect call (arena sizing) */
    int32_t max_width;       /* largest frame width  (arena sizing) */
    int32_t max_height;      /* largest frame height (arena sizing) */
    int32_t flags;           /* PD_FLAG_* bits, 0 by default */
    int32_t use_proposal;    /* 1: sparse path gated by the learned proposal (needs pd_cnn_set_params) */
    float keep_logit_threshold; /* a window is kept iff its keep-logit > this */
    int32_t upscale_levels;  /* 0..64 upsampled levels (scale pyr_factor^-j, j = upscale..1) placed
                                before the frame's level 0; 0 by default (the stop rule alone) */
    int32_t proposal_level_step; /* 1..16: the proposal network runs on levels 0, m, 2m, ... of each
                                    frame (m = this value) and every level's head map is taken from
                                    the first level of its group; 1 (every level) by default */
} pd_params;

/* One detection: a window in frame coordinates. */
typedef struct pd_box {
    float x, y, w, h;  /* top-left and size in frame pixels */
    float score;       /* SVM score (float32) */
    int32_t level;     /* pyramid level */
    int32_t wx, wy;    /* window position in cells on that level */
} pd_box;

/* Geometry of one pyramid level of one frame. */
typedef struct pd_level_info {
    int32_t width, height;   /* level size in pixels */
    int32_t cells_x, cells_y;/* floor(width/8), floor(height/8) */
    int32_t rows, cols;      /* score map size: cells_y-15 by cells_x-7 (0 if none) */
    int64_t score_offset;    /* float offset of this map in the handle's score buffer */
} pd_level_info;

/* Defaults: factor 1.05, clip 0.2, threshold 0, IoU 0.5, 4096 boxes,
 * 16384 candidates, 1 frame of 1242x375. */
int pd_params_default(pd_params *p);

/* Pyramid level sizes of a W x H frame (Section 4.4, pyramidal sliding
 * window; the level rule is this library's reading: level k has scale
 * factor^k, size floor(W/factor^k) x floor(H/factor^k), and levels are kept
 * while a 64x128 window fits). Host only. Wk/Hk: host arrays of max_levels
 * entries. Returns the number of levels (>= 0) or PD_EINVAL. */
int pd_pyramid(int W, int H, float factor, int max_levels, int32_t *Wk, int32_t *Hk);

/* Same with `upscale_levels` upsampled levels first (most upsampled first):
 * level j of those is floor(W f^(upscale-j) + 1e-9) x floor(H f^(upscale-j)
 * + 1e-9), each kept if a 64x128 window fits (Section 4.4 pyramid; the
 * upsampled levels reach pedestrians shorter than the window). Returns the
 * number of levels or PD_EINVAL. */
int pd_pyramid_ex(int W, int H, float factor, int upscale_levels, int max_levels, int32_t *Wk, int32_t *Hk);

/* Creates a detector. svm_w: host float[15][7][95] template in window order
 * (block row i, block column j, feature t: 36 HOG values = 4 cells x 9 bins
 * in the order top-left, top-right, bottom-left, bottom-right, then 59 LBP
 * values); svm_b: bias (Section 4.4: distance to the SVM hyper-plane). The
 * handle allocates its device arena (cudaMalloc) sized by params, on the
 * current device, and owns it until pd_destroy. Errors: PD_EINVAL,
 * PD_ENOMEM, PD_ECUDA; *out is NULL on error. */
int pd_create(const pd_params *params, const float *svm_w, float svm_b, pd_handle **out);

/* Frees the arena and the handle (synchronises the device first). NULL is a no-op. */
void pd_destroy(pd_handle *h);

/* Last error message recorded on the handle ("" if none). Valid until the next call. */
const char *pd_last_error(const pd_handle *h);

/* Runs the whole plain path on n_frames frames (Section 4.1 steps 2-5):
 * pyramid (K1), LBP and HOG cell histograms (K2/K3), block normalisation fused
 * with the window scores (K4), NMS (K5). d_frames: host array of n_frames
 * DEVICE pointers to u8 frames; widths/heights/pitches: host arrays. Frames
 * smaller than 64x128 have no level and no detection (not an error).
 * Asynchronous on `stream`; the frames must stay valid until pd_sync
 * returns. Results live in the handle until the next pd_detect.
 * Errors: PD_EINVAL (n_frames > max_frames, a frame larger than
 * max_width x max_height, NULL pointer, pitch < width), PD_ECUDA. */
int pd_detect(pd_handle *h, void *stream, int n_frames, const uint8_t *const *d_frames,
              const int32_t *widths, const int32_t *heights, const int32_t *pitches);

/* Waits for the last pd_detect, then surfaces device-side status: PD_OK,
 * PD_EOVERFLOW (a frame had more candidates than max_candidates_per_frame;
 * its boxes are invalid), PD_ETIMEOUT / PD_EBOUNDS (results invalid), or
 * PD_ECUDA. The NMS kernel writes the kept boxes and counts straight into
 * mapped pinned host memory owned by the handle. Synchronous. */
int pd_sync(pd_handle *h);

/* Number of windows above threshold (NMS candidates) of frame `frame` of the
 * last detect; negative if it exceeded max_candidates_per_frame. Requires
 * pd_sync (else PD_ESTATE). */
int pd_frame_candidates(const pd_handle *h, int frame, int *n);

/* Level geometry of frame `frame` of the last pd_detect (host). info: host
 * array of PD_MAX_LEVELS entries. Available right after pd_detect. */
int pd_frame_levels(const pd_handle *h, int frame, int *n_levels, pd_level_info *info);

/* Device pointer to all score maps of the last pd_detect (float32; map of
 * (frame, level) at pd_level_info.score_offset, row-major rows x cols;
 * window (wx, wy) scores the 64x128 window whose top-left pixel is
 * (8wx, 8wy) on that level). Valid until the next pd_detect / pd_destroy;
 * read it after pd_sync or on the same stream. *total = number of floats. */
int pd_scores(const pd_handle *h, const float **d_scores, int64_t *total);

/* Host copy of frame `frame`'s kept boxes, in NMS order (score descending,
 * ties by level, wy, wx ascending). Requires pd_sync first (else PD_ESTATE).
 * out: host array of cap entries; *count = number of boxes (may exceed cap;
 * only min(count, cap) are written). */
int pd_boxes(const pd_handle *h, int frame, pd_box *out, int cap, int *count);

/* Number of this library's kernel launches issued by the last pd_detect. */
int pd_last_launch_count(const pd_handle *h);

/* Launch shapes of the default path (this library's addition), chosen by an
 * autotuner that times them on the caller's workload:
 *   k1_groups     column groups (of 4 output pixels) per warp task of the
 *                 pyramid kernel: 4, 8 or 16; a warp's 32 lanes are
 *                 k1_groups groups x 32 / k1_groups row slices (default 8);
 *   tc_item_rows  window rows per work item of the tensor-core score kernel,
 *                 8 .. 64: a 104-window strip is cut into near-equal pieces
 *                 of at most this many rows, each piece also reading the 14
 *                 block rows below its last window row (default 64).
 * Results do not depend on them: every output is the same sum in the same
 * order. Errors: PD_EINVAL. Affects the next pd_detect. */
typedef struct pd_tuning {
    int32_t k1_groups;
    int32_t tc_item_rows;
} pd_tuning;
int pd_set_tuning(pd_handle *h, const pd_tuning *t);
int pd_get_tuning(const pd_handle *h, pd_tuning *t);

/* Tile shapes of the FP32 K4 (PD_FLAG_SVM_FP32; windows per CTA tile, x by y): 0 = 32x16, 1 = 64x8,
 * 2 = 32x8, 3 = 64x4, 4 = 64x2, 5 = 32x12, 6 = 32x4. For each level the
 * planner takes the shape with the least (number of tiles x cost[shape]).
 * The default costs come from an instruction-count model of one tile
 * (FMAs of its windows, feature planes of its block region, a fixed part);
 * the autotuner measures them on the running GPU and sets them here. The
 * table applies to the dense path; with the proposal on, the planner uses a
 * fixed table of its own that favours narrow tiles. cost: host array of PD_TILE_SHAPES positive floats. Affects the
 * next pd_detect / pd_window_scores; results are identical for any costs up
 * to float rounding (the same sums in a different tiling). */
#define PD_TILE_SHAPES 7
int pd_set_tile_costs(pd_handle *h, const float *cost);
int pd_get_tile_costs(const pd_handle *h, float *cost);

/* Device time in milliseconds of each stage of the last pd_detect, from CUDA
 * events recorded on its stream around each launch (ms has 5 entries):
 * ms[0] pyramid (K1), ms[1] cell histograms (K2/K3), ms[2] block norm +
 * window scores (K4), ms[3] NMS (K5), ms[4] the proposal network and the
 * tile flags of the sparse path (about 0 with the proposal off). Needs
 * PD_FLAG_STAGE_TIMING at pd_create and a pd_sync after the detect (else
 * PD_ESTATE). */
int pd_stage_times(const pd_handle *h, float *ms);

/* Same as pd_detect with frames in HOST memory (h_frames: host array of host
 * pointers; Section 4.1 step 1, the host-to-device transfer). Page-locked
 * frames (cudaMallocHost / cudaHostRegister / pinned tensors) are read in
 * place by the pyramid kernel over the host link, once; other host frames are
 * first copied into the arena on `stream`. The host frames may be reused once
 * pd_sync returns. Errors as pd_detect. */
int pd_detect_host(pd_handle *h, void *stream, int n_frames, const uint8_t *const *h_frames,
                   const int32_t *widths, const int32_t *heights, const int32_t *pitches);

/* ---------------------------------------------------------------------------
 * Stage entry points (the same kernels pd_detect runs, one level at a time),
 * for parity tests and for callers that keep intermediates. All pointers are
 * DEVICE pointers owned by the caller; all calls are asynchronous on `stream`.
 * They use the handle's small descriptor scratch, so calls on one handle must
 * not overlap on the GPU with each other or with pd_detect.
 * ------------------------------------------------------------------------- */

/* K1, Section 4.4 pyramid: writes levels 0..n_levels-1 of one W x H frame
 * (fixed-point bilinear, 11-bit weights, each level resampled straight from
 * the frame; the frame is read once). Level k is Wk[k] x Hk[k] (host arrays;
 * 1 .. 4W x 1 .. 4H, so upsampled levels too) at d_levels + level_offsets[k]
 * (host array, bytes) with pitch
 * level_pitches[k] (host array, >= Wk[k]). n_levels <= PD_MAX_LEVELS.
 * Errors: PD_EINVAL, PD_ECUDA. */
int pd_resize_levels(pd_handle *h, void *stream, const uint8_t *d_frame, int W, int H, int pitch, int n_levels,
                     const int32_t *Wk, const int32_t *Hk, uint8_t *d_levels,
                     const int64_t *level_offsets, const int32_t *level_pitches);

/* K2 + K3, Sections 4.2-4.3 (Algorithms 1, 2, 4, 5): uniform-LBP cell counts
 * and soft-binned HOG cell histograms of one Wk x Hk level image.
 * Outputs are plane-major with `cell_pitch` elements per row
 * (cell_pitch >= floor(Wk/8), a multiple of 16):
 *   d_hog  float32 [9][cells_y][cell_pitch]   (plane stride hog_plane elems)
 *   d_lbp  uint8   [59][cells_y][cell_pitch]  (plane stride lbp_plane elems)
 * hog_plane / lbp_plane >= cells_y * cell_pitch. With PD_FLAG_HOG_PER_BLOCK
 * d_hog holds 36 planes: plane 9 q + bin of cell (cy, cx) is its histogram
 * restricted to the block in which it sits at place q (0 top-left, 1
 * top-right, 2 bottom-left, 3 bottom-right), so block (by, bx) is planes
 * 0-8 of cell (by, bx), 9-17 of (by, bx+1), 18-26 of (by+1, bx) and 27-35 of
 * (by+1, bx+1) (values at places no block uses are unspecified).
 * Errors: PD_EINVAL, PD_ECUDA. */
int pd_cell_features(pd_handle *h, void *stream, const uint8_t *d_level, int Wk, int Hk, int pitch, float *d_hog,
                     int64_t hog_plane, uint8_t *d_lbp, int64_t lbp_plane, int cell_pitch);

/* K4, Section 4.4 (Algorithm 6) with block normalisation: the score map of
 * one level from its cell planes (layouts of pd_cell_features, 36 HOG planes
 * with PD_FLAG_HOG_PER_BLOCK; LBP counts
 * must be <= 64, as a cell has 64 pixels), using the handle's template and
 * bias and its K4 kernel (tensor cores, or FP32 with PD_FLAG_SVM_FP32):
 * d_scores float32 [cells_y-15][cells_x-7], row pitch cells_x-7. The
 * cell planes are read through TMA: d_hog and d_lbp must be 16-byte aligned,
 * cell_pitch a multiple of 16, hog_plane a multiple of 4 and lbp_plane a
 * multiple of 16 elements. Errors: PD_EINVAL, PD_ECUDA. */
int pd_window_scores(pd_handle *h, void *stream, const float *d_hog, int64_t hog_plane,
                     const uint8_t *d_lbp, int64_t lbp_plane, int cell_pitch, int cells_x,
                     int cells_y, float *d_scores);

/* K5 (refinement stage, Section 3; greedy NMS) on caller score maps of ONE
 * frame: n_levels maps laid back to back from d_scores (float32, level k
 * rows[k] x cols[k], host arrays), level sizes Wk/Hk (host), frame W x H.
 * Writes the kept boxes in NMS order to d_boxes (device, cap max_boxes) and
 * the kept / candidate counts to d_counts[0] / d_counts[1] (device int32).
 * Uses the handle's threshold, nms_iou and caps and its scratch buffers.
 * Errors: PD_EINVAL, PD_ECUDA; a candidate overflow sets d_counts[1] to
 * -(number of candidates). */
int pd_nms_maps(pd_handle *h, void *stream, const float *d_scores, int n_levels, const int32_t *rows,
                const int32_t *cols, const int32_t *Wk, const int32_t *Hk, int W, int H,
                pd_box *d_boxes, int max_boxes, int32_t *d_counts);

/* ---------------------------------------------------------------------------
 * Learned window proposal (not in the paper; a small network that predicts
 * which windows of a pyramid level can score above the SVM threshold, so that
 * the detector can skip the others). Per level image L:
 *   x = bf16(L/255 - 0.5); a1 = relu(conv3x3 stride 2 (1 -> 16));
 *   a2 = relu(conv3x3 s2 (16 -> 32)); a3 = relu(conv3x3 s2 (32 -> 32)), one
 *   vector per 8x8 cell; h = wh . a3 + bh (1x1 head, one value per cell);
 *   z[wy][wx] = bv + sum_{r<16, s<8} V[r][s] h[wy+r][wx+s], one keep-logit per
 *   window (the window pooling lets the logit see the whole 64x128 window).
 * bf16 inputs, weights and stored activations, fp32 accumulation.
 * Parameters: PD_CNN_PARAMS floats in the order w1[16][1][3][3], b1[16],
 * w2[32][16][3][3], b2[32], w3[32][32][3][3], b3[32], wh[32], bh, V[16][8], bv.
 * ------------------------------------------------------------------------- */
#define PD_CNN_PARAMS 14210

/* Loads the proposal parameters (host, fp32 master copy) and resets the
 * optimiser state. Synchronous. Errors: PD_EINVAL, PD_ECUDA. */
int pd_cnn_set_params(pd_handle *h, const float *params, int n);

/* Host copies of the master parameters and of the gradient of the last
 * training step (either pointer may be NULL). Synchronous. */
int pd_cnn_get_params(pd_handle *h, float *params, float *grad, int n);

/* Proposal forward on one level image (device, u8, Wk x Hk, pitch): writes
 * the per-cell head values to d_h (float, cells_y rows of h_pitch) and the
 * window keep-logits to d_logits (float [cells_y-15][cells_x-7]). */
int pd_cnn_forward(pd_handle *h, void *stream, const uint8_t *d_level, int Wk, int Hk, int pitch, float *d_h,
                   int h_pitch, float *d_logits);

/* One training step on the last pd_detect batch (same stream): every window
 * of every level is an example, labelled positive iff its SVM score (already
 * computed by that pd_detect) is > label_threshold; the loss is the mean
 * binary cross-entropy with logits with positive weight pos_weight over all
 * windows of the batch; the gradient is computed by this library's backward
 * kernels (fixed-order reductions: deterministic) and, if lr > 0, Adam
 * (beta 0.9 / 0.999, eps 1e-8) updates the master parameters. The first call
 * allocates a training workspace (cudaMalloc). */
int pd_cnn_train_step(pd_handle *h, void *stream, float pos_weight, float label_threshold, float lr);

/* Loss of the last training step (synchronises the stream). */
int pd_cnn_train_loss(pd_handle *h, void *stream, float *loss);

/* Sparse path on (enable = 1) or off. When on, pd_detect also runs the
 * proposal network on every level after the pyramid. A window is kept when
 * its keep-logit exceeds keep_logit_threshold; the window tiles of the FP32
 * score kernel's plan that hold a kept window mark the cell tiles under them,
 * and only marked cell tiles are computed. The tensor-core score kernel then
 * scores every window whose cell tiles are all marked (a superset of the kept
 * windows: every window of a kept tile); the FP32 kernel scores the windows
 * of kept tiles. Scored windows get exactly the plain path's score, the
 * others -inf. With the threshold at -inf every window is scored. Needs
 * parameters (pd_cnn_set_params) to enable. Affects the next pd_detect. */
int pd_set_proposal(pd_handle *h, int enable, float keep_logit_threshold);

/* Level groups of the learned proposal (this library's addition; the
 * paper has no learned stage). With m = level_step the network runs on the
 * frame's levels 0, m, 2m, ... only; level k takes its head map from level
 * j = m * floor(k / m) by nearest cell: cell (cy, cx) of level k reads cell
 * (min(floor((2 cy + 1) Hk_j / (2 Hk_k)), cells_y_j - 1),
 *  min(floor((2 cx + 1) Wk_j / (2 Wk_k)), cells_x_j - 1)) of level j, the
 * cell holding its centre; the window pooling then runs on every level as
 * before. m = 1 is the network on every level. 1 <= level_step <= 16, else
 * PD_EINVAL. Affects the next pd_detect (the batch plan is rebuilt). */
int pd_set_proposal_levels(pd_handle *h, int level_step);

/* Device pointer to the window keep-logits of the last pd_detect with the
 * proposal on (same layout and offsets as pd_scores; *total = 0 when off). */
int pd_logits(const pd_handle *h, const float **d_logits, int64_t *total);

/* Allocation-free NMS. The paper has no counterpart: this exists for
 * callers that must not allocate device memory at run time -- a real-time
 * frame loop whose coding rules forbid allocation after start-up, a plugin
 * inside a host framework that owns all GPU memory, or code that only has a
 * fixed memory budget -- and so cannot create a pd_handle (pd_create calls
 * cudaMalloc). It computes exactly what pd_nms_maps computes, with the
 * threshold, IoU and caps passed as arguments, and needs no handle.
 * The scratch memory it needs (level descriptors and the decoded box of
 * every candidate) is one static array inside the library, about 270 KB,
 * that every GPU which loads the library holds until the process exits; it
 * limits a call to max_candidates <= 16384 and n_levels <= PD_MAX_LEVELS
 * (larger values, or max_boxes > 16384, return PD_EINVAL). The caller passes inputs and outputs as
 * for pd_nms_maps: d_scores, d_boxes (cap max_boxes) and d_counts (kept,
 * candidates; a candidate overflow writes 0 and -candidates). Every call
 * looks up the array's device address on the current device and sets the
 * kernel's shared-memory limit (host calls that allocate nothing); make the
 * first call on a device outside any stream capture.
 * All calls share the one array and it keeps the last call's contents, so
 * calls that overlap on the GPU (two streams, two threads) race: serialise
 * them. Errors: PD_EINVAL, PD_ECUDA. Asynchronous on `stream`. */
int pd_nms_noalloc(void *stream, const float *d_scores, int n_levels, const int32_t *rows,
                   const int32_t *cols, const int32_t *Wk, const int32_t *Hk, int W, int H, float threshold,
                   float nms_iou, int max_candidates, pd_box *d_boxes, int max_boxes, int32_t *d_counts);

/* ---------------------------------------------------------------------------
 * The paper's own kernel schemes (Section 4.2-4.4 and its per-algorithm
 * results, Section 5.3), re-expressed on this GPU for comparison with the
 * fused kernels above. They compute the same cell histograms and window
 * scores (same readings, same parity bars), with the paper's work
 * decompositions:
 *   PD_SCHEME_LBP_NAIVE     LBP code stencil (one thread per pixel), then one
 *                           thread per cell histogram (Map pattern);
 *   PD_SCHEME_LBP_SCALABLE  LBP code stencil, then one thread per pixel adding
 *                           to its cell histogram with atomics (Scatter);
 *   PD_SCHEME_HOG_GLOBAL / _LOCAL / _SHARED
 *                           gradient stencil (magnitude and orientation per
 *                           pixel), then one thread per cell histogram
 *                           (large-grain) accumulating its votes in global
 *                           memory, in a local array, or in shared memory;
 *   PD_SCHEME_SVM_NAIVE     block features materialised (one thread per
 *                           block), then one thread per window dot product;
 *   PD_SCHEME_SVM_WARP      the same features, one warp per window (lanes
 *                           split the products, shuffle reduction).
 * pd_scheme_cells writes the LBP planes (LBP schemes) or the HOG planes (HOG
 * schemes) in the layout of pd_cell_features; pd_scheme_window_scores takes
 * and returns what pd_window_scores does. With PD_FLAG_HOG_PER_BLOCK the HOG
 * schemes are Algorithm 5 as laid out in Section 4.3: one thread per 16x16
 * block (Global / Local / Shared: where its 36-bin histogram lives), writing
 * the 36-plane per-block layout, which the SVM schemes then read. Both
 * allocate a scratch buffer on first use (cudaMalloc; grown when a larger
 * level comes, freed by pd_destroy). Errors: PD_EINVAL (bad argument or scheme), PD_ENOMEM, PD_ECUDA. */
#define PD_SCHEME_LBP_NAIVE 1
#define PD_SCHEME_LBP_SCALABLE 2
#define PD_SCHEME_HOG_GLOBAL 3
#define PD_SCHEME_HOG_LOCAL 4
#define PD_SCHEME_HOG_SHARED 5
#define PD_SCHEME_SVM_NAIVE 6
#define PD_SCHEME_SVM_WARP 7
int pd_scheme_cells(pd_handle *h, void *stream, int scheme, const uint8_t *d_level, int Wk, int Hk, int pitch,
                    float *d_hog, int64_t hog_plane, uint8_t *d_lbp, int64_t lbp_plane, int cell_pitch);
int pd_scheme_window_scores(pd_handle *h, void *stream, int scheme, const float *d_hog, int64_t hog_plane,
                            const uint8_t *d_lbp, int64_t lbp_plane, int cell_pitch, int cells_x, int cells_y,
                            float *d_scores);

#ifdef __cplusplus
}
#endif

#endif /* PD_H */
