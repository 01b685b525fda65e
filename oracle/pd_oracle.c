/*
 * pd_oracle.c -- plain, slow, obviously-correct CPU oracle of the HOG+LBP
 * sliding-window SVM pedestrian detector of arXiv 1611.01642.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the bench's CPU-baseline
 * leg use it. It shares no code, header, table or constant generator with the
 * CUDA library; both sides read the same seeded inputs and nothing else.
 *
 * Every floating-point quantity is evaluated in IEEE double precision, in the
 * order the definitions below state it, one pixel / cell / block / window at a
 * time. Integer quantities (resized pixels, LBP codes and counts) are exact.
 * Build with -ffp-contract=off so that a*b+c is never fused behind our back.
 *
 * Layouts (row-major, innermost last):
 *   image / level      u8  [H][pitch]
 *   LBP cell counts    u8  [Hc][Wc][59]
 *   HOG cell histogram f64 [Hc][Wc][9]
 *   HOG block histogram f64 [Hb][Wb][36]  (per-block reading, cells TL TR BL BR)
 *   block feature      f64 [Hb][Wb][95]   (36 HOG values then 59 LBP values)
 *   SVM template       f64 [15][7][95]
 *   score map          f64 [Hc-15][Wc-7]
 * with Wc = floor(Wk/8), Hc = floor(Hk/8), Wb = Wc-1, Hb = Hc-1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PDO_HOG_BINS 9
#define PDO_LBP_BINS 59
#define PDO_HOG_DIM 36
#define PDO_FEAT 95
#define PDO_WIN_BW 7
#define PDO_WIN_BH 15
#define PDO_PI 3.14159265358979323846

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static long long floor_div(long long a, long long b) /* b > 0 */
{
    long long q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

/* ---------------------------------------------------------------------------
 * Pyramid levels (Section 4.4, pyramidal sliding window: downscaled copies of
 * the frame, each scanned with 128x64 windows). The paper fixes neither the
 * level sizes nor the stop rule. Reading: level k has scale s_k = factor^k,
 * Wk = floor(W/s_k + 1e-9), Hk = floor(H/s_k + 1e-9), and levels are kept
 * while a 64x128 window still fits. Returns the number of levels.
 * ------------------------------------------------------------------------- */
int pdo_pyramid_up(int W, int H, double factor, int upscale, int max_levels, int *Wk, int *Hk);

int pdo_pyramid(int W, int H, double factor, int max_levels, int *Wk, int *Hk)
{
    return pdo_pyramid_up(W, H, factor, 0, max_levels, Wk, Hk);
}

/* With `upscale` > 0 the pyramid also holds the upsampled levels k = -upscale
 * .. -1 (scale factor^k < 1, the same size rule), first, most upsampled
 * first; they reach pedestrians shorter than the 128-pixel window (the
 * 1242x375 workload's "about 40 levels" at factor 1.05 are 23 levels of the
 * stop rule plus 17 upsampled ones). Every level must still hold a window. */
int pdo_pyramid_up(int W, int H, double factor, int upscale, int max_levels, int *Wk, int *Hk)
{
    int n = 0;
    if (!(factor > 1.0) || upscale < 0) return -1;
    for (int k = -upscale; k < 0 && n < max_levels; ++k) {
        double s = pow(factor, (double)k);
        int wk = (int)floor((double)W / s + 1e-9);
        int hk = (int)floor((double)H / s + 1e-9);
        if (wk < 64 || hk < 128) continue;
        Wk[n] = wk;
        Hk[n] = hk;
        ++n;
    }
    for (int k = 0; n < max_levels; ++k) {
        double s = pow(factor, (double)k);
        int wk = (int)floor((double)W / s + 1e-9);
        int hk = (int)floor((double)H / s + 1e-9);
        if (wk < 64 || hk < 128) break;
        Wk[n] = wk;
        Hk[n] = hk;
        ++n;
    }
    return n;
}

/* ---------------------------------------------------------------------------
 * Fixed-point bilinear resample with 11-bit weights (one pyramid level,
 * straight from the frame). Source coordinate of destination x is the
 * half-pixel-centre mapping (x + 0.5) * W / Wk - 0.5, scaled by 2048 and
 * rounded half up; the integer part selects x0, the 11 low bits are the
 * weight of x0+1. Coordinates left of 0 clamp to pixel 0, right of W-1 to
 * pixel W-1. Same for y. The result is
 *   (((2048-ay)((2048-ax)I00 + ax I01) + ay((2048-ax)I10 + ax I11)) + 2^21) >> 22.
 * ------------------------------------------------------------------------- */
static void q11_coord(int x, int W, int Wk, int *x0, int *x1, int *a)
{
    long long num = ((long long)(2 * x + 1) * W - Wk) * 2048 + Wk;
    long long q = floor_div(num, 2LL * Wk);
    if (q < 0) {
        *x0 = 0;
        *a = 0;
    } else {
        *x0 = (int)(q >> 11);
        *a = (int)(q & 2047);
        if (*x0 >= W - 1) {
            *x0 = W - 1;
            *a = 0;
        }
    }
    *x1 = (*x0 + 1 < W - 1) ? *x0 + 1 : W - 1;
}

void pdo_resize(const uint8_t *img, int W, int H, int pitch,
                uint8_t *out, int Wk, int Hk, int out_pitch)
{
    for (int y = 0; y < Hk; ++y) {
        int y0, y1, ay;
        q11_coord(y, H, Hk, &y0, &y1, &ay);
        for (int x = 0; x < Wk; ++x) {
            int x0, x1, ax;
            q11_coord(x, W, Wk, &x0, &x1, &ax);
            long long i00 = img[(size_t)y0 * pitch + x0], i01 = img[(size_t)y0 * pitch + x1];
            long long i10 = img[(size_t)y1 * pitch + x0], i11 = img[(size_t)y1 * pitch + x1];
            long long top = (2048 - ax) * i00 + ax * i01;
            long long bot = (2048 - ax) * i10 + ax * i11;
            long long v = ((2048 - ay) * top + ay * bot + (1LL << 21)) >> 22;
            out[(size_t)y * out_pitch + x] = (uint8_t)v;
        }
    }
}

/* ---------------------------------------------------------------------------
 * LBP map (Section 4.2, Algorithm 1): the centre pixel is compared with each
 * of its 8 nearest neighbours; a neighbour lower than the centre gives 0,
 * otherwise 1; the 8 bits read as a number are the code. Neighbour k (bit
 * weight 2^k) walks clockwise from the top-left: (-1,-1) (-1,0) (-1,+1)
 * (0,+1) (+1,+1) (+1,0) (+1,-1) (0,-1) as (dy,dx). Borders clamp to the edge.
 * ------------------------------------------------------------------------- */
static const int LBP_DY[8] = {-1, -1, -1, 0, 1, 1, 1, 0};
static const int LBP_DX[8] = {-1, 0, 1, 1, 1, 0, -1, -1};

int pdo_lbp_code(const uint8_t *L, int Wk, int Hk, int pitch, int x, int y)
{
    int c = L[(size_t)y * pitch + x];
    int code = 0;
    for (int k = 0; k < 8; ++k) {
        int yy = clampi(y + LBP_DY[k], 0, Hk - 1);
        int xx = clampi(x + LBP_DX[k], 0, Wk - 1);
        int n = L[(size_t)yy * pitch + xx];
        if (n >= c) code |= 1 << k;
    }
    return code;
}

/* Uniform patterns: at most two 0/1 transitions around the circle (58 codes).
 * Bin = rank of the code among uniform codes in ascending order; every
 * non-uniform code goes to bin 58 (59 bins in all). */
int pdo_lbp_transitions(int code)
{
    int t = 0;
    for (int k = 0; k < 8; ++k) {
        int a = (code >> k) & 1;
        int b = (code >> ((k + 1) % 8)) & 1;
        if (a != b) ++t;
    }
    return t;
}

int pdo_lbp_bin(int code)
{
    if (pdo_lbp_transitions(code) > 2) return 58;
    int rank = 0;
    for (int c = 0; c < code; ++c)
        if (pdo_lbp_transitions(c) <= 2) ++rank;
    return rank;
}

/* LBP cell histograms (Section 4.2, Algorithm 2): every pixel of the 8x8 cell
 * grid adds one to the bin of its code in its own cell. Pixels beyond
 * 8*Wc x 8*Hc are not counted. */
void pdo_lbp_cells(const uint8_t *L, int Wk, int Hk, int pitch, uint8_t *cells)
{
    int Wc = Wk / 8, Hc = Hk / 8;
    int table[256];
    for (int c = 0; c < 256; ++c) table[c] = pdo_lbp_bin(c);
    memset(cells, 0, (size_t)Hc * Wc * PDO_LBP_BINS);
    for (int y = 0; y < 8 * Hc; ++y)
        for (int x = 0; x < 8 * Wc; ++x) {
            int bin = table[pdo_lbp_code(L, Wk, Hk, pitch, x, y)];
            cells[((size_t)(y / 8) * Wc + (x / 8)) * PDO_LBP_BINS + bin] += 1;
        }
}

/* ---------------------------------------------------------------------------
 * Gradient (Section 4.3, Algorithm 4). The printed magnitude/orientation
 * formulas are garbled; reading: gx = L[y][x+1]-L[y][x-1],
 * gy = L[y+1][x]-L[y-1][x] with clamped borders, magnitude sqrt(gx^2+gy^2),
 * orientation atan2(gy, gx) in degrees folded into [0,180) (unsigned).
 * ------------------------------------------------------------------------- */
void pdo_gradient(const uint8_t *L, int Wk, int Hk, int pitch, int x, int y,
                  double *mag, double *theta_deg)
{
    int xl = clampi(x - 1, 0, Wk - 1), xr = clampi(x + 1, 0, Wk - 1);
    int yu = clampi(y - 1, 0, Hk - 1), yd = clampi(y + 1, 0, Hk - 1);
    int gx = (int)L[(size_t)y * pitch + xr] - (int)L[(size_t)y * pitch + xl];
    int gy = (int)L[(size_t)yd * pitch + x] - (int)L[(size_t)yu * pitch + x];
    *mag = sqrt((double)gx * gx + (double)gy * gy);
    double th = atan2((double)gy, (double)gx) * (180.0 / PDO_PI);
    if (th < 0.0) th += 180.0;
    if (th >= 180.0) th -= 180.0;
    *theta_deg = th;
}

/* Orientation vote: 9 bins of 20 degrees with centres at 10, 30, ... 170.
 * b = theta/20 - 0.5; bins floor(b) and floor(b)+1 (mod 9) get 1-frac and
 * frac, which is linear interpolation between the two nearest bin centres. */
void pdo_orientation_vote(double theta_deg, int *bin0, int *bin1, double *w0, double *w1)
{
    double b = theta_deg / 20.0 - 0.5;
    double f = floor(b);
    double fr = b - f;
    int b0 = (int)f;
    *bin0 = ((b0 % 9) + 9) % 9;
    *bin1 = (((b0 + 1) % 9) + 9) % 9;
    *w0 = 1.0 - fr;
    *w1 = fr;
}

/* Spatial vote along one axis: cell centres at 8c + 3.5; coordinate p votes
 * into cells floor(u) and floor(u)+1 with u = (p - 3.5)/8 and linear weights;
 * a cell index outside [0, n-1] is clamped to the nearest cell. */
void pdo_spatial_vote(int p, int n, int *c0, int *c1, double *w0, double *w1)
{
    double u = ((double)p - 3.5) / 8.0;
    double f = floor(u);
    double fr = u - f;
    *c0 = clampi((int)f, 0, n - 1);
    *c1 = clampi((int)f + 1, 0, n - 1);
    *w0 = 1.0 - fr;
    *w1 = fr;
}

/* HOG cell histograms (Section 4.3, Algorithm 5, interpolation of Dalal and
 * Triggs): every pixel of the 8*Wc x 8*Hc grid adds magnitude x orientation
 * weight x horizontal weight x vertical weight to 2 orientation bins of 2x2
 * cells, i.e. to 2, 4 or 8 bins. The cells live on one global grid (read of
 * the paper's 8x8 cell split), so a 16x16 block is 4 concatenated cells. */
void pdo_hog_cells(const uint8_t *L, int Wk, int Hk, int pitch, double *cells)
{
    int Wc = Wk / 8, Hc = Hk / 8;
    for (size_t i = 0; i < (size_t)Hc * Wc * PDO_HOG_BINS; ++i) cells[i] = 0.0;
    for (int y = 0; y < 8 * Hc; ++y)
        for (int x = 0; x < 8 * Wc; ++x) {
            double mag, th;
            pdo_gradient(L, Wk, Hk, pitch, x, y, &mag, &th);
            int ob[2], cx[2], cy[2];
            double ow[2], wx[2], wy[2];
            pdo_orientation_vote(th, &ob[0], &ob[1], &ow[0], &ow[1]);
            pdo_spatial_vote(x, Wc, &cx[0], &cx[1], &wx[0], &wx[1]);
            pdo_spatial_vote(y, Hc, &cy[0], &cy[1], &wy[0], &wy[1]);
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b)
                    for (int o = 0; o < 2; ++o)
                        cells[((size_t)cy[a] * Wc + cx[b]) * PDO_HOG_BINS + ob[o]] +=
                            mag * ow[o] * wx[b] * wy[a];
        }
}

/* Spatial vote inside one 16x16 block along one axis (per-block reading of
 * Algorithm 5): the block's two cell centres sit at local coordinates 3.5 and
 * 11.5; local coordinate l (0..15) votes into cells floor(u) and floor(u)+1,
 * u = (l - 3.5)/8, with weights 1-frac and frac. Cells -1 and 2 lie outside
 * the block and their votes are dropped by the caller, so a pixel lands in
 * one or two cells per axis. */
void pdo_block_spatial_vote(int l, int *c0, int *c1, double *w0, double *w1)
{
    double u = ((double)l - 3.5) / 8.0;
    double f = floor(u);
    *c0 = (int)f;
    *c1 = (int)f + 1;
    *w1 = u - f;
    *w0 = 1.0 - *w1;
}

/* HOG block histograms, per-block reading (Section 4.3, Algorithm 5): one
 * histogram of 4 cells x 9 bins per 16x16 block (stride 8, Hb = Hc-1 by
 * Wb = Wc-1), filled by the block's own 256 pixels only. Each pixel
 * (Algorithm 4 gradient) adds magnitude x orientation weight x spatial
 * weights to the cells of the block its vote reaches, i.e. to 2, 4 or 8 bins
 * depending on where it sits in the block (Section 4.3). Votes towards cells
 * outside the block are not kept, so neighbouring blocks do not share cell
 * histograms. Output f64 [Hb][Wb][36], cell q = 2 a + b (a row, b column of
 * the cell in the block) at q*9. */
void pdo_hog_blocks(const uint8_t *L, int Wk, int Hk, int pitch, double *blocks)
{
    int Hb = Hk / 8 - 1, Wb = Wk / 8 - 1;
    if (Hb <= 0 || Wb <= 0) return;
    for (int by = 0; by < Hb; ++by)
        for (int bx = 0; bx < Wb; ++bx) {
            double *f = blocks + ((size_t)by * Wb + bx) * PDO_HOG_DIM;
            for (int t = 0; t < PDO_HOG_DIM; ++t) f[t] = 0.0;
            for (int i = 0; i < 16; ++i)
                for (int j = 0; j < 16; ++j) {
                    double mag, th;
                    pdo_gradient(L, Wk, Hk, pitch, 8 * bx + j, 8 * by + i, &mag, &th);
                    int ob[2], cy[2], cx[2];
                    double ow[2], wy[2], wx[2];
                    pdo_orientation_vote(th, &ob[0], &ob[1], &ow[0], &ow[1]);
                    pdo_block_spatial_vote(i, &cy[0], &cy[1], &wy[0], &wy[1]);
                    pdo_block_spatial_vote(j, &cx[0], &cx[1], &wx[0], &wx[1]);
                    for (int a = 0; a < 2; ++a) {
                        if (cy[a] < 0 || cy[a] > 1) continue;
                        for (int b = 0; b < 2; ++b) {
                            if (cx[b] < 0 || cx[b] > 1) continue;
                            for (int o = 0; o < 2; ++o)
                                f[(2 * cy[a] + cx[b]) * PDO_HOG_BINS + ob[o]] += mag * ow[o] * wx[b] * wy[a];
                        }
                    }
                }
        }
}

/* ---------------------------------------------------------------------------
 * Block features (Section 4.2, Algorithm 3; Section 4.3). A block is 2x2
 * cells (16x16 pixels) at a stride of one cell (50% overlap), Hb = Hc-1,
 * Wb = Wc-1. HOG part: the 4 cell histograms concatenated (top-left,
 * top-right, bottom-left, bottom-right) and normalised with L2-Hys:
 * v /= sqrt(|v|^2 + 1), clip at 0.2, v /= sqrt(|v|^2 + 1e-6). LBP part: the
 * sum of the 4 cell histograms (the histogram reduction of Algorithm 3)
 * normalised with L1-sqrt: f = sqrt(h / sum(h)).
 * ------------------------------------------------------------------------- */
void pdo_l2hys(double *v, int n, double clip)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += v[i] * v[i];
    double d = sqrt(s + 1.0);
    for (int i = 0; i < n; ++i) {
        v[i] = v[i] / d;
        if (v[i] > clip) v[i] = clip;
    }
    s = 0.0;
    for (int i = 0; i < n; ++i) s += v[i] * v[i];
    d = sqrt(s + 1e-6);
    for (int i = 0; i < n; ++i) v[i] = v[i] / d;
}

void pdo_block_features(const double *hog, const uint8_t *lbp, int Hc, int Wc,
                        double clip, double *feat)
{
    int Hb = Hc - 1, Wb = Wc - 1;
    for (int by = 0; by < Hb; ++by)
        for (int bx = 0; bx < Wb; ++bx) {
            double *f = feat + ((size_t)by * Wb + bx) * PDO_FEAT;
            for (int q = 0; q < 4; ++q) {
                int cy = by + q / 2, cx = bx + q % 2;
                for (int b = 0; b < PDO_HOG_BINS; ++b)
                    f[q * PDO_HOG_BINS + b] = hog[((size_t)cy * Wc + cx) * PDO_HOG_BINS + b];
            }
            pdo_l2hys(f, PDO_HOG_DIM, clip);
            double h[PDO_LBP_BINS], tot = 0.0;
            for (int t = 0; t < PDO_LBP_BINS; ++t) {
                h[t] = 0.0;
                for (int q = 0; q < 4; ++q) {
                    int cy = by + q / 2, cx = bx + q % 2;
                    h[t] += (double)lbp[((size_t)cy * Wc + cx) * PDO_LBP_BINS + t];
                }
                tot += h[t];
            }
            for (int t = 0; t < PDO_LBP_BINS; ++t)
                f[PDO_HOG_DIM + t] = tot > 0.0 ? sqrt(h[t] / tot) : 0.0;
        }
}

/* Block features with the per-block HOG histograms: the block's own 36 HOG
 * values (pdo_hog_blocks) L2-Hys normalised, then the LBP part as in
 * pdo_block_features. */
void pdo_block_features_pb(const double *hogb, const uint8_t *lbp, int Hc, int Wc,
                           double clip, double *feat)
{
    int Hb = Hc - 1, Wb = Wc - 1;
    for (int by = 0; by < Hb; ++by)
        for (int bx = 0; bx < Wb; ++bx) {
            double *f = feat + ((size_t)by * Wb + bx) * PDO_FEAT;
            const double *hb = hogb + ((size_t)by * Wb + bx) * PDO_HOG_DIM;
            for (int t = 0; t < PDO_HOG_DIM; ++t) f[t] = hb[t];
            pdo_l2hys(f, PDO_HOG_DIM, clip);
            double h[PDO_LBP_BINS], tot = 0.0;
            for (int t = 0; t < PDO_LBP_BINS; ++t) {
                h[t] = 0.0;
                for (int q = 0; q < 4; ++q) {
                    int cy = by + q / 2, cx = bx + q % 2;
                    h[t] += (double)lbp[((size_t)cy * Wc + cx) * PDO_LBP_BINS + t];
                }
                tot += h[t];
            }
            for (int t = 0; t < PDO_LBP_BINS; ++t)
                f[PDO_HOG_DIM + t] = tot > 0.0 ? sqrt(h[t] / tot) : 0.0;
        }
}

/* ---------------------------------------------------------------------------
 * Sliding-window linear SVM (Section 4.4, Algorithm 6): the window whose
 * top-left block is (wx, wy) covers 15x7 blocks; its descriptor is those
 * blocks' 95-d features concatenated; the score is the dot product with the
 * template plus the bias. Algorithm 6 multiplies the LBP and HOG parts by one
 * shared model array; reading: one template w[15][7][95] over the
 * concatenated 95-d block feature.
 * ------------------------------------------------------------------------- */
void pdo_scores(const double *feat, int Hb, int Wb, const double *w, double bias,
                double *scores)
{
    int rows = Hb - PDO_WIN_BH + 1, cols = Wb - PDO_WIN_BW + 1;
    for (int wy = 0; wy < rows; ++wy)
        for (int wx = 0; wx < cols; ++wx) {
            double s = 0.0;
            for (int i = 0; i < PDO_WIN_BH; ++i)
                for (int j = 0; j < PDO_WIN_BW; ++j)
                    for (int t = 0; t < PDO_FEAT; ++t)
                        s += feat[((size_t)(wy + i) * Wb + (wx + j)) * PDO_FEAT + t] *
                             w[((size_t)i * PDO_WIN_BW + j) * PDO_FEAT + t];
            scores[(size_t)wy * cols + wx] = s + bias;
        }
}

/* Whole level: cells, block features and scores of one pyramid level image.
 * hog/lbp/feat are caller scratch of the sizes given in the file header;
 * with per_block the HOG part comes from pdo_hog_blocks and hog must hold
 * Hb*Wb*36 values. */
void pdo_level_scores_ex(const uint8_t *L, int Wk, int Hk, int pitch, const double *w,
                         double bias, double clip, int per_block, double *hog, uint8_t *lbp,
                         double *feat, double *scores)
{
    int Wc = Wk / 8, Hc = Hk / 8;
    pdo_lbp_cells(L, Wk, Hk, pitch, lbp);
    if (per_block) {
        pdo_hog_blocks(L, Wk, Hk, pitch, hog);
        pdo_block_features_pb(hog, lbp, Hc, Wc, clip, feat);
    } else {
        pdo_hog_cells(L, Wk, Hk, pitch, hog);
        pdo_block_features(hog, lbp, Hc, Wc, clip, feat);
    }
    pdo_scores(feat, Hc - 1, Wc - 1, w, bias, scores);
}

void pdo_level_scores(const uint8_t *L, int Wk, int Hk, int pitch, const double *w,
                      double bias, double clip, double *hog, uint8_t *lbp, double *feat,
                      double *scores)
{
    pdo_level_scores_ex(L, Wk, Hk, pitch, w, bias, clip, 0, hog, lbp, feat, scores);
}

/* ---------------------------------------------------------------------------
 * Brute-force window descriptor, computed straight from the pixels with no
 * shared cell map: each cell histogram is GATHERED from the pixels whose
 * votes reach it (the scatter in pdo_hog_cells, turned around), and each
 * block is built from its own 4 cells. Used only to cross-check the map
 * based path. phi has 15*7*95 entries in template order.
 * ------------------------------------------------------------------------- */
static void bf_hog_cell(const uint8_t *L, int Wk, int Hk, int pitch, int cy, int cx, double *h)
{
    int Wc = Wk / 8, Hc = Hk / 8;
    for (int b = 0; b < PDO_HOG_BINS; ++b) h[b] = 0.0;
    for (int y = 8 * cy - 8; y < 8 * cy + 16; ++y) {
        if (y < 0 || y >= 8 * Hc) continue;
        for (int x = 8 * cx - 8; x < 8 * cx + 16; ++x) {
            if (x < 0 || x >= 8 * Wc) continue;
            int c0, c1;
            double a0, a1, wy = 0.0, wx = 0.0;
            pdo_spatial_vote(y, Hc, &c0, &c1, &a0, &a1);
            if (c0 == cy) wy += a0;
            if (c1 == cy) wy += a1;
            pdo_spatial_vote(x, Wc, &c0, &c1, &a0, &a1);
            if (c0 == cx) wx += a0;
            if (c1 == cx) wx += a1;
            if (wy == 0.0 || wx == 0.0) continue;
            double mag, th, o0, o1;
            int b0, b1;
            pdo_gradient(L, Wk, Hk, pitch, x, y, &mag, &th);
            pdo_orientation_vote(th, &b0, &b1, &o0, &o1);
            h[b0] += mag * o0 * wx * wy;
            h[b1] += mag * o1 * wx * wy;
        }
    }
}

void pdo_window_descriptor_bruteforce(const uint8_t *L, int Wk, int Hk, int pitch,
                                      int wx, int wy, double clip, double *phi)
{
    int table[256];
    for (int c = 0; c < 256; ++c) table[c] = pdo_lbp_bin(c);
    for (int i = 0; i < PDO_WIN_BH; ++i)
        for (int j = 0; j < PDO_WIN_BW; ++j) {
            double *f = phi + ((size_t)i * PDO_WIN_BW + j) * PDO_FEAT;
            int by = wy + i, bx = wx + j;
            double h[PDO_LBP_BINS];
            for (int t = 0; t < PDO_LBP_BINS; ++t) h[t] = 0.0;
            for (int q = 0; q < 4; ++q) {
                int cy = by + q / 2, cx = bx + q % 2;
                bf_hog_cell(L, Wk, Hk, pitch, cy, cx, f + q * PDO_HOG_BINS);
                for (int y = 8 * cy; y < 8 * cy + 8; ++y)
                    for (int x = 8 * cx; x < 8 * cx + 8; ++x)
                        h[table[pdo_lbp_code(L, Wk, Hk, pitch, x, y)]] += 1.0;
            }
            pdo_l2hys(f, PDO_HOG_DIM, clip);
            double tot = 0.0;
            for (int t = 0; t < PDO_LBP_BINS; ++t) tot += h[t];
            for (int t = 0; t < PDO_LBP_BINS; ++t)
                f[PDO_HOG_DIM + t] = tot > 0.0 ? sqrt(h[t] / tot) : 0.0;
        }
}

/* ---------------------------------------------------------------------------
 * Detections and non-maximum suppression (Section 3 refinement stage; the
 * paper cites Laptev and runs it on the host). Reading: every window with
 * score > threshold is a candidate; its box in frame coordinates is
 * x = 8 wx W/Wk, y = 8 wy H/Hk, w = 64 W/Wk, h = 128 H/Hk (double, stored as
 * float). Greedy: candidates in order of score (descending), ties by level,
 * then wy, then wx (ascending); a candidate is kept unless its IoU with an
 * already kept box exceeds iou_thr; at most max_boxes are kept.
 * ------------------------------------------------------------------------- */
typedef struct {
    float x, y, w, h, score;
    int32_t level, wx, wy;
} pdo_box;

void pdo_window_box(int W, int H, int Wk, int Hk, int wx, int wy, float *bx, float *by,
                    float *bw, float *bh)
{
    *bx = (float)((double)(8 * wx) * (double)W / (double)Wk);
    *by = (float)((double)(8 * wy) * (double)H / (double)Hk);
    *bw = (float)(64.0 * (double)W / (double)Wk);
    *bh = (float)(128.0 * (double)H / (double)Hk);
}

double pdo_iou(const pdo_box *a, const pdo_box *b)
{
    double ax0 = a->x, ay0 = a->y, ax1 = (double)a->x + (double)a->w, ay1 = (double)a->y + (double)a->h;
    double bx0 = b->x, by0 = b->y, bx1 = (double)b->x + (double)b->w, by1 = (double)b->y + (double)b->h;
    double iw = (ax1 < bx1 ? ax1 : bx1) - (ax0 > bx0 ? ax0 : bx0);
    double ih = (ay1 < by1 ? ay1 : by1) - (ay0 > by0 ? ay0 : by0);
    if (iw <= 0.0 || ih <= 0.0) return 0.0;
    double inter = iw * ih;
    double ua = (double)a->w * (double)a->h + (double)b->w * (double)b->h - inter;
    return inter / ua;
}

static int box_order(const void *pa, const void *pb)
{
    const pdo_box *a = (const pdo_box *)pa, *b = (const pdo_box *)pb;
    if (a->score != b->score) return a->score > b->score ? -1 : 1;
    if (a->level != b->level) return a->level < b->level ? -1 : 1;
    if (a->wy != b->wy) return a->wy < b->wy ? -1 : 1;
    if (a->wx != b->wx) return a->wx < b->wx ? -1 : 1;
    return 0;
}

/* score maps of n_levels levels laid out back to back (level k has
 * rows[k] x cols[k] entries, level sizes Wk/Hk). Scores are float (the
 * values the detector produced) and are compared exactly. Returns the
 * number of kept boxes (<= max_boxes), or -1 on allocation failure;
 * *n_candidates receives the number of windows above threshold. */
int pdo_nms(const float *scores, int n_levels, const int *rows, const int *cols,
            const int *Wk, const int *Hk, int W, int H, float threshold, double iou_thr,
            int max_boxes, pdo_box *out, int *n_candidates)
{
    size_t total = 0, off = 0;
    for (int k = 0; k < n_levels; ++k) total += (size_t)rows[k] * cols[k];
    pdo_box *cand = (pdo_box *)malloc((total ? total : 1) * sizeof(pdo_box));
    if (!cand) return -1;
    size_t n = 0;
    for (int k = 0; k < n_levels; ++k) {
        for (int wy = 0; wy < rows[k]; ++wy)
            for (int wx = 0; wx < cols[k]; ++wx) {
                float s = scores[off + (size_t)wy * cols[k] + wx];
                if (!(s > threshold)) continue;
                pdo_box b;
                pdo_window_box(W, H, Wk[k], Hk[k], wx, wy, &b.x, &b.y, &b.w, &b.h);
                b.score = s;
                b.level = k;
                b.wx = wx;
                b.wy = wy;
                cand[n++] = b;
            }
        off += (size_t)rows[k] * cols[k];
    }
    *n_candidates = (int)n;
    qsort(cand, n, sizeof(pdo_box), box_order);
    int kept = 0;
    for (size_t i = 0; i < n && kept < max_boxes; ++i) {
        int keep = 1;
        for (int j = 0; j < kept; ++j)
            if (pdo_iou(&cand[i], &out[j]) > iou_thr) {
                keep = 0;
                break;
            }
        if (keep) out[kept++] = cand[i];
    }
    free(cand);
    return kept;
}

/* ---------------------------------------------------------------------------
 * The whole plain path for one frame (Section 4.1 steps 2-5): pyramid,
 * per-level features and scores, NMS. Scores of all levels are written back
 * to back into `scores` (double) and, rounded, used for NMS. Returns the
 * number of boxes, or -1 on allocation failure. per_block selects the
 * per-block HOG histograms (pdo_hog_blocks) instead of the shared cells.
 * ------------------------------------------------------------------------- */
int pdo_detect_ex(const uint8_t *img, int W, int H, int pitch, double factor, int upscale, int per_block,
                  const double *w, double bias, double clip, float threshold, double iou_thr, int max_boxes,
                  int max_levels, int *n_levels_out, int *Wk, int *Hk, double *scores,
                  pdo_box *boxes, int *n_candidates);

int pdo_detect(const uint8_t *img, int W, int H, int pitch, double factor, const double *w,
               double bias, double clip, float threshold, double iou_thr, int max_boxes,
               int max_levels, int *n_levels_out, int *Wk, int *Hk, double *scores,
               pdo_box *boxes, int *n_candidates)
{
    return pdo_detect_ex(img, W, H, pitch, factor, 0, 0, w, bias, clip, threshold, iou_thr, max_boxes, max_levels,
                         n_levels_out, Wk, Hk, scores, boxes, n_candidates);
}

int pdo_detect_up(const uint8_t *img, int W, int H, int pitch, double factor, int upscale, const double *w,
                  double bias, double clip, float threshold, double iou_thr, int max_boxes,
                  int max_levels, int *n_levels_out, int *Wk, int *Hk, double *scores,
                  pdo_box *boxes, int *n_candidates)
{
    return pdo_detect_ex(img, W, H, pitch, factor, upscale, 0, w, bias, clip, threshold, iou_thr, max_boxes,
                         max_levels, n_levels_out, Wk, Hk, scores, boxes, n_candidates);
}

int pdo_detect_ex(const uint8_t *img, int W, int H, int pitch, double factor, int upscale, int per_block,
                  const double *w,
                  double bias, double clip, float threshold, double iou_thr, int max_boxes,
                  int max_levels, int *n_levels_out, int *Wk, int *Hk, double *scores,
                  pdo_box *boxes, int *n_candidates)
{
    int nl = pdo_pyramid_up(W, H, factor, upscale, max_levels, Wk, Hk);
    *n_levels_out = nl < 0 ? 0 : nl;
    if (nl <= 0) {
        *n_candidates = 0;
        return 0;
    }
    int rows[1024], cols[1024];
    size_t total = 0, maxpx = 0;
    for (int k = 0; k < nl; ++k) {
        rows[k] = Hk[k] / 8 - PDO_WIN_BH;
        cols[k] = Wk[k] / 8 - PDO_WIN_BW;
        total += (size_t)rows[k] * cols[k];
        if ((size_t)Wk[k] * Hk[k] > maxpx) maxpx = (size_t)Wk[k] * Hk[k];
    }
    size_t maxcells = maxpx / 64 + 1;
    uint8_t *L = (uint8_t *)malloc(maxpx);
    double *hog = (double *)malloc(maxcells * PDO_HOG_DIM * sizeof(double));
    uint8_t *lbp = (uint8_t *)malloc(maxcells * PDO_LBP_BINS);
    double *feat = (double *)malloc(maxcells * PDO_FEAT * sizeof(double));
    float *fs = (float *)malloc((total ? total : 1) * sizeof(float));
    if (!L || !hog || !lbp || !feat || !fs) {
        free(L); free(hog); free(lbp); free(feat); free(fs);
        return -1;
    }
    size_t off = 0;
    for (int k = 0; k < nl; ++k) {
        pdo_resize(img, W, H, pitch, L, Wk[k], Hk[k], Wk[k]);
        pdo_level_scores_ex(L, Wk[k], Hk[k], Wk[k], w, bias, clip, per_block, hog, lbp, feat, scores + off);
        for (size_t i = 0; i < (size_t)rows[k] * cols[k]; ++i) fs[off + i] = (float)scores[off + i];
        off += (size_t)rows[k] * cols[k];
    }
    int kept = pdo_nms(fs, nl, rows, cols, Wk, Hk, W, H, threshold, iou_thr, max_boxes, boxes,
                       n_candidates);
    free(L); free(hog); free(lbp); free(feat); free(fs);
    return kept;
}
