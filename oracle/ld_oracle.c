/*
 * ld_oracle.c -- plain, slow CPU oracle for the lane-detection hot path of
 * "Hardware Acceleration of Lane Detection Algorithm: A GPU Versus FPGA
 * Comparison" (arXiv 2212.09460).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  The CUDA library never
 * links, calls or includes it, and it shares no code, header or table with
 * the CUDA path.
 *
 * Every function is the direct definition of one step, written as plain
 * loops in the paper's order:
 *   Step 1  Sobel gradient magnitude |G| = |Sx*Img| + |Sy*Img|   (Sec. 2.1, Eq. 1)
 *           on the zero-padded image                            (Sec. 3.1, Sec. 4.1)
 *   Step 2  binarization to 0/255                               (Sec. 2.2, Sec. 3.2, Sec. 4.2)
 *   Step 3  Hough voting r = x cos(theta) + y sin(theta)        (Sec. 2.3, Eq. 3, Sec. 4.3)
 *           with the cos/sin symmetry of Eqs. 4-5               (Sec. 3.3)
 *   Step 4  Hough peaks (done in MATLAB in the paper)           (Sec. 2.3, Sec. 5)
 *
 * Readings where the paper is silent (each one is also listed with its pin in
 * the design notes):
 *   - Sobel pair: the standard 3x3 pair; |Gx|+|Gy| does not depend on sign,
 *     transpose, flip or correlation-vs-convolution conventions.
 *   - magnitude saturated to 255 (8-bit output); threshold T, test M >= T.
 *   - x = column (0..w-1, rightwards), y = row (0..h-1, downwards).
 *   - theta_k = k*180/n_theta degrees, k = 0..n_theta-1 (half-open [0,180)).
 *   - cos/sin in Q16: c_k = llround(cos(k*pi/n_theta)*65536) for
 *     k <= n_theta/2, and the mirror c_k = -c_{n-k}, s_k = s_{n-k} (Eqs. 4-5).
 *   - rho = floor((x*c_k + y*s_k + 32768) / 65536), accumulator index rho+D,
 *     D = ceil(sqrt(w^2+h^2)); a vote whose rho falls outside [-D, D] is not
 *     counted (it is reported in the return value).
 *   - peaks: greedy in the order votes desc, theta_idx asc, rho_idx asc,
 *     each pick suppresses a window of nms_theta x nms_rho cells (no wrap).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define LDO_BORDER_ZERO 0
#define LDO_BORDER_CLEAR 1

/* Smallest integer D with D*D >= w*w + h*h, i.e. ceil(sqrt(w^2+h^2)). */
int ldo_rho_max(int w, int h)
{
    int64_t r2 = (int64_t)w * w + (int64_t)h * h;
    int64_t d = 0;
    while (d * d < r2) d++;
    return (int)d;
}

/* Padded pixel P(x, y): the image inside, 0 outside (Sec. 3.1, Sec. 4.1). */
static int pix(const uint8_t *img, int w, int h, int pitch, int x, int y)
{
    if (x < 0 || y < 0 || x >= w || y >= h) return 0;
    return img[(size_t)y * pitch + x];
}

/*
 * Step 1 (Eq. 1): mag[y*w+x] = min(|Gx| + |Gy|, 255) with
 *   Gx = P(x+1,y-1) + 2P(x+1,y) + P(x+1,y+1) - P(x-1,y-1) - 2P(x-1,y) - P(x-1,y+1)
 *   Gy = P(x-1,y+1) + 2P(x,y+1) + P(x+1,y+1) - P(x-1,y-1) - 2P(x,y-1) - P(x+1,y-1)
 * written as the two 3x3 kernels applied tap by tap.  With border ==
 * LDO_BORDER_CLEAR the 1-pixel frame of the output is forced to 0.
 * variant (0..7) picks one of the eight sign/transpose conventions of the
 * kernel pair: bit0 negates Sx, bit1 negates Sy, bit2 swaps Sx and Sy.  All
 * give the same magnitude; the tests use this to pin convention independence.
 */
void ldo_sobel_mag(const uint8_t *img, int w, int h, int pitch, int border,
                   int variant, uint8_t *mag)
{
    static const int SX[3][3] = {{-1, 0, 1}, {-2, 0, 2}, {-1, 0, 1}};
    static const int SY[3][3] = {{-1, -2, -1}, {0, 0, 0}, {1, 2, 1}};
    int kx[3][3], ky[3][3];
    int sx = (variant & 1) ? -1 : 1, sy = (variant & 2) ? -1 : 1;
    for (int j = 0; j < 3; j++)
        for (int i = 0; i < 3; i++) {
            int a = sx * SX[j][i], b = sy * SY[j][i];
            if (variant & 4) { kx[j][i] = b; ky[j][i] = a; }
            else { kx[j][i] = a; ky[j][i] = b; }
        }
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            int gx = 0, gy = 0;
            for (int j = -1; j <= 1; j++)
                for (int i = -1; i <= 1; i++) {
                    int p = pix(img, w, h, pitch, x + i, y + j);
                    gx += kx[j + 1][i + 1] * p;
                    gy += ky[j + 1][i + 1] * p;
                }
            int m = abs(gx) + abs(gy);
            if (m > 255) m = 255;
            if (border == LDO_BORDER_CLEAR &&
                (x == 0 || y == 0 || x == w - 1 || y == h - 1))
                m = 0;
            mag[(size_t)y * w + x] = (uint8_t)m;
        }
}

/* Step 2 (Sec. 2.2): every pixel becomes 255 if mag >= T, else 0. */
void ldo_binarize(const uint8_t *mag, int w, int h, int threshold, uint8_t *bin)
{
    for (size_t i = 0; i < (size_t)w * h; i++)
        bin[i] = (mag[i] >= threshold) ? 255 : 0;
}

/*
 * Coordinates of the 255 pixels, row-major, packed as (y << 16) | x
 * (the edge list the GPU voting stage reads, Sec. 4.3).  Writes at most
 * `capacity` entries; returns the true count.
 */
int64_t ldo_edge_list(const uint8_t *bin, int w, int h, uint32_t *edges,
                      int64_t capacity)
{
    int64_t n = 0;
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++)
            if (bin[(size_t)y * w + x] == 255) {
                if (n < capacity) edges[n] = ((uint32_t)y << 16) | (uint32_t)x;
                n++;
            }
    return n;
}

/*
 * Q16 cos/sin table over theta_k = k*pi/n_theta (Sec. 3.3).  Entries for
 * k <= n_theta/2 are rounded from fp64 cos/sin; the rest follow from
 * Eq. 4 (sin t = sin(180-t)) and Eq. 5 (cos t = -cos(180-t)).
 */
void ldo_trig_q16(int n_theta, int32_t *c, int32_t *s)
{
    for (int k = 0; k <= n_theta / 2; k++) {
        double t = (double)k * M_PI / (double)n_theta;
        c[k] = (int32_t)llround(cos(t) * 65536.0);
        s[k] = (int32_t)llround(sin(t) * 65536.0);
    }
    for (int k = n_theta / 2 + 1; k < n_theta; k++) {
        c[k] = -c[n_theta - k];
        s[k] = s[n_theta - k];
    }
}

static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

/*
 * Step 3 (Eq. 3): acc[k*(2D+1) + rho + D] += 1 for every edge (x, y) and
 * every k, with rho = floor((x*c_k + y*s_k + 32768) / 65536) in int64.
 * acc holds n_theta*(2D+1) int32 cells and is overwritten.  Returns the
 * number of votes that fell outside [-D, D] (not counted).
 */
int64_t ldo_hough(const uint32_t *edges, int64_t n_edges, int w, int h,
                  int n_theta, int32_t *acc)
{
    int D = ldo_rho_max(w, h);
    int n_rho = 2 * D + 1;
    int32_t *c = (int32_t *)malloc(sizeof(int32_t) * n_theta);
    int32_t *s = (int32_t *)malloc(sizeof(int32_t) * n_theta);
    ldo_trig_q16(n_theta, c, s);
    memset(acc, 0, sizeof(int32_t) * (size_t)n_theta * n_rho);
    int64_t dropped = 0;
    for (int64_t e = 0; e < n_edges; e++) {
        int64_t x = edges[e] & 0xFFFF, y = edges[e] >> 16;
        for (int k = 0; k < n_theta; k++) {
            int64_t rho = floor_div(x * c[k] + y * s[k] + 32768, 65536);
            if (rho < -D || rho > D) { dropped++; continue; }
            acc[(size_t)k * n_rho + (size_t)(rho + D)] += 1;
        }
    }
    free(c);
    free(s);
    return dropped;
}

/* a precedes b in the peak order: votes desc, theta asc, rho asc. */
static int before(int32_t va, int ta, int ra, int32_t vb, int tb, int rb)
{
    if (va != vb) return va > vb;
    if (ta != tb) return ta < tb;
    return ra < rb;
}

/*
 * Step 4 (Sec. 2.3 "Hough Peak"): greedy non-maximum suppression.  Up to
 * top_k times: take the first cell in peak order that is not suppressed and
 * has votes >= min_votes; emit (theta_idx, rho_idx, votes); suppress every
 * cell with |dtheta| <= nms_theta/2 and |drho| <= nms_rho/2 (clipped, no
 * wrap).  out holds 3*top_k int32.  Returns the number of peaks emitted.
 */
int ldo_peaks(const int32_t *acc, int n_theta, int n_rho, int top_k,
              int nms_theta, int nms_rho, int min_votes, int32_t *out)
{
    uint8_t *sup = (uint8_t *)calloc((size_t)n_theta * n_rho, 1);
    int ht = nms_theta / 2, hr = nms_rho / 2, n = 0;
    for (int p = 0; p < top_k; p++) {
        int bt = -1, br = -1;
        int32_t bv = 0;
        for (int t = 0; t < n_theta; t++)
            for (int r = 0; r < n_rho; r++) {
                size_t i = (size_t)t * n_rho + r;
                if (sup[i] || acc[i] < min_votes) continue;
                if (bt < 0 || before(acc[i], t, r, bv, bt, br)) {
                    bt = t; br = r; bv = acc[i];
                }
            }
        if (bt < 0) break;
        out[3 * n + 0] = bt;
        out[3 * n + 1] = br;
        out[3 * n + 2] = bv;
        n++;
        for (int t = bt - ht; t <= bt + ht; t++)
            for (int r = br - hr; r <= br + hr; r++)
                if (t >= 0 && t < n_theta && r >= 0 && r < n_rho)
                    sup[(size_t)t * n_rho + r] = 1;
    }
    free(sup);
    return n;
}

/*
 * The whole path for one frame, Steps 1-4 in order; used by the CPU baseline.
 * mag/bin are w*h scratch, edges has capacity w*h, acc n_theta*(2D+1).
 * Returns the peak count (>= 0).
 */
int ldo_detect(const uint8_t *img, int w, int h, int pitch, int border,
               int threshold, int n_theta, int top_k, int nms_theta,
               int nms_rho, int min_votes, uint8_t *mag, uint8_t *bin,
               uint32_t *edges, int32_t *acc, int32_t *peaks)
{
    ldo_sobel_mag(img, w, h, pitch, border, 0, mag);
    ldo_binarize(mag, w, h, threshold, bin);
    int64_t n = ldo_edge_list(bin, w, h, edges, (int64_t)w * h);
    ldo_hough(edges, n, w, h, n_theta, acc);
    int D = ldo_rho_max(w, h);
    return ldo_peaks(acc, n_theta, 2 * D + 1, top_k, nms_theta, nms_rho,
                     min_votes, peaks);
}

/* Sort key of a supporting pixel: along x (then y) for a line closer to
 * horizontal than to vertical, along y (then x) otherwise. */
typedef struct { int x, y; } ldo_pt;
static int g_lines_by_x;
static int cmp_pt(const void *pa, const void *pb)
{
    const ldo_pt *a = (const ldo_pt *)pa, *b = (const ldo_pt *)pb;
    int a1 = g_lines_by_x ? a->x : a->y, b1 = g_lines_by_x ? b->x : b->y;
    int a2 = g_lines_by_x ? a->y : a->x, b2 = g_lines_by_x ? b->y : b->x;
    if (a1 != b1) return a1 < b1 ? -1 : 1;
    if (a2 != b2) return a2 < b2 ? -1 : 1;
    return 0;
}

/*
 * Hough lines: the line segments behind each peak (Step 4 of Sec. 1 without
 * the drawing; the paper hands the peaks to MATLAB's "Hough lines", Sec. 5,
 * Fig. 12, and states no parameters).  For peak p = (theta_idx k, rho_idx r):
 *   - its supporting pixels are the edges whose Q16 rho at theta_k (the vote's
 *     own rounding, Eq. 3 with Eqs. 4-5) equals r - D, so their number is the
 *     peak's vote count;
 *   - they are ordered along the line: by x (then y) when |c_k| <= |s_k| (the
 *     line is at most 45 degrees from horizontal), else by y (then x);
 *   - consecutive pixels more than fill_gap apart (squared Euclidean distance
 *     > fill_gap^2) start a new segment;
 *   - a segment is kept when its first and last pixel are at least min_length
 *     apart (squared distance >= min_length^2).
 * segs receives, per peak, up to max_segments kept segments in line order as
 * (x1, y1, x2, y2, theta_idx, rho_idx) with (x1, y1) the first pixel:
 * segs[(p * max_segments + i) * 6 + field].  counts[p] = the number of kept
 * segments (may exceed max_segments; only max_segments are written),
 * support[p] = the number of supporting pixels.
 */
void ldo_hough_lines(const uint32_t *edges, int64_t n_edges, int w, int h,
                     int n_theta, const int32_t *peaks, int n_peaks,
                     int fill_gap, int min_length, int max_segments,
                     int32_t *segs, int32_t *counts, int32_t *support)
{
    int D = ldo_rho_max(w, h);
    int32_t *c = (int32_t *)malloc(sizeof(int32_t) * n_theta);
    int32_t *s = (int32_t *)malloc(sizeof(int32_t) * n_theta);
    ldo_trig_q16(n_theta, c, s);
    ldo_pt *pts = (ldo_pt *)malloc(sizeof(ldo_pt) * (size_t)(n_edges > 0 ? n_edges : 1));
    int64_t gap2 = (int64_t)fill_gap * fill_gap, len2 = (int64_t)min_length * min_length;
    for (int p = 0; p < n_peaks; p++) {
        int k = peaks[3 * p + 0], r = peaks[3 * p + 1];
        int64_t n = 0;
        for (int64_t e = 0; e < n_edges; e++) {
            int64_t x = edges[e] & 0xFFFF, y = edges[e] >> 16;
            int64_t rho = floor_div(x * c[k] + y * s[k] + 32768, 65536);
            if (rho == (int64_t)r - D) {
                pts[n].x = (int)x;
                pts[n].y = (int)y;
                n++;
            }
        }
        support[p] = (int32_t)n;
        g_lines_by_x = abs(c[k]) <= abs(s[k]);
        qsort(pts, (size_t)n, sizeof(ldo_pt), cmp_pt);
        int kept = 0;
        int64_t a = 0;
        while (a < n) {
            int64_t b = a;   /* the segment is pts[a..b] */
            while (b + 1 < n) {
                int64_t dx = pts[b + 1].x - pts[b].x, dy = pts[b + 1].y - pts[b].y;
                if (dx * dx + dy * dy > gap2) break;
                b++;
            }
            int64_t dx = pts[b].x - pts[a].x, dy = pts[b].y - pts[a].y;
            if (dx * dx + dy * dy >= len2) {
                if (kept < max_segments) {
                    int32_t *o = segs + ((size_t)p * max_segments + kept) * 6;
                    o[0] = pts[a].x; o[1] = pts[a].y; o[2] = pts[b].x; o[3] = pts[b].y;
                    o[4] = k; o[5] = r;
                }
                kept++;
            }
            a = b + 1;
        }
        counts[p] = kept;
    }
    free(pts);
    free(c);
    free(s);
}

/*
 * Canny edge detection in place of Steps 1-2 (the paper's future work, Sec. 7),
 * producing the same 0/255 map and edge list the Hough vote reads.  Every stage
 * works on the image domain with zero outside it (the padding of Sec. 3.1),
 * in integers:
 *   1. Gaussian blur with the 5x5 binomial kernel b b^T, b = (1 4 6 4 1) (sum
 *      256), rounded: G = (sum K I + 128) >> 8, 0..255.
 *   2. Sobel on G (the kernels of Step 1): gx, gy, magnitude M = |gx| + |gy|
 *      (Eq. 1, not saturated, 0..2040).
 *   3. Direction sector from tan(22.5 deg) = 27146 / 65536 and tan(67.5 deg) =
 *      158218 / 65536 (rounded): |gy| 65536 <= 27146 |gx| compares along x,
 *      |gy| 65536 >= 158218 |gx| along y, otherwise along the diagonal
 *      (x-1, y-1)-(x+1, y+1) when gx gy > 0, else (x+1, y-1)-(x-1, y+1).
 *   4. Non-maximum suppression: a pixel stays if M > 0, M > M(n1) and
 *      M >= M(n2), where n1 is the neighbour of the pair with the smaller y (the
 *      smaller x along x): a ridge two pixels wide keeps one pixel.
 *   5. Hysteresis: a kept pixel is strong if M >= t_high, weak if t_low <= M <
 *      t_high; the edges are the strong pixels and every weak pixel joined to a
 *      strong one by an 8-connected chain of weak or strong pixels.
 * bin receives 0/255 [h][w]; mag (nullable) M [h][w] as int32.
 */
static int ldo_g_at(const uint8_t *g, int w, int h, int x, int y)
{
    return (x < 0 || y < 0 || x >= w || y >= h) ? 0 : g[(size_t)y * w + x];
}

void ldo_canny(const uint8_t *img, int w, int h, int pitch, int t_low, int t_high,
               uint8_t *bin, int32_t *mag_out)
{
    static const int B5[5] = {1, 4, 6, 4, 1};
    size_t n = (size_t)w * h;
    uint8_t *g = (uint8_t *)malloc(n);
    int32_t *m = (int32_t *)malloc(n * sizeof(int32_t));
    uint8_t *sec = (uint8_t *)malloc(n);
    uint8_t *cls = (uint8_t *)malloc(n);
    int32_t *queue = (int32_t *)malloc(n * sizeof(int32_t));
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            int s = 0;
            for (int j = -2; j <= 2; j++)
                for (int i = -2; i <= 2; i++)
                    s += B5[j + 2] * B5[i + 2] * pix(img, w, h, pitch, x + i, y + j);
            g[(size_t)y * w + x] = (uint8_t)((s + 128) >> 8);
        }
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            int gx = (ldo_g_at(g, w, h, x + 1, y - 1) + 2 * ldo_g_at(g, w, h, x + 1, y) + ldo_g_at(g, w, h, x + 1, y + 1))
                   - (ldo_g_at(g, w, h, x - 1, y - 1) + 2 * ldo_g_at(g, w, h, x - 1, y) + ldo_g_at(g, w, h, x - 1, y + 1));
            int gy = (ldo_g_at(g, w, h, x - 1, y + 1) + 2 * ldo_g_at(g, w, h, x, y + 1) + ldo_g_at(g, w, h, x + 1, y + 1))
                   - (ldo_g_at(g, w, h, x - 1, y - 1) + 2 * ldo_g_at(g, w, h, x, y - 1) + ldo_g_at(g, w, h, x + 1, y - 1));
            int64_t ax = abs(gx), ay = abs(gy);
            m[(size_t)y * w + x] = (int32_t)(ax + ay);
            int sc;
            if (ay * 65536 <= 27146 * ax) sc = 0;
            else if (ay * 65536 >= 158218 * ax) sc = 2;
            else sc = ((int64_t)gx * gy > 0) ? 1 : 3;
            sec[(size_t)y * w + x] = (uint8_t)sc;
        }
    /* neighbour offsets (n1, n2) per sector: n1 has the smaller y (smaller x along x) */
    static const int DX1[4] = {-1, -1, 0, 1}, DY1[4] = {0, -1, -1, -1};
    static const int DX2[4] = {1, 1, 0, -1}, DY2[4] = {0, 1, 1, 1};
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            size_t i = (size_t)y * w + x;
            int sc = sec[i], v = m[i];
            int x1 = x + DX1[sc], y1 = y + DY1[sc], x2 = x + DX2[sc], y2 = y + DY2[sc];
            int v1 = (x1 < 0 || y1 < 0 || x1 >= w || y1 >= h) ? 0 : m[(size_t)y1 * w + x1];
            int v2 = (x2 < 0 || y2 < 0 || x2 >= w || y2 >= h) ? 0 : m[(size_t)y2 * w + x2];
            int keep = v > 0 && v > v1 && v >= v2;
            cls[i] = !keep ? 0 : (v >= t_high ? 2 : (v >= t_low ? 1 : 0));
        }
    /* flood fill from the strong pixels through weak ones (8-connected) */
    size_t qh = 0, qt = 0;
    memset(bin, 0, n);
    for (size_t i = 0; i < n; i++)
        if (cls[i] == 2) { bin[i] = 255; queue[qt++] = (int32_t)i; }
    while (qh < qt) {
        int i = queue[qh++], x = i % w, y = i / w;
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int xx = x + dx, yy = y + dy;
                if (xx < 0 || yy < 0 || xx >= w || yy >= h) continue;
                size_t j = (size_t)yy * w + xx;
                if (cls[j] && !bin[j]) { bin[j] = 255; queue[qt++] = (int32_t)j; }
            }
    }
    if (mag_out) memcpy(mag_out, m, n * sizeof(int32_t));
    free(g); free(m); free(sec); free(cls); free(queue);
}

/* Gaussian stage alone (step 1 above), for pinning: out [h][w]. */
void ldo_canny_blur(const uint8_t *img, int w, int h, int pitch, uint8_t *out)
{
    static const int B5[5] = {1, 4, 6, 4, 1};
    for (int y = 0; y < h; y++)
        for (int x = 0; x < w; x++) {
            int s = 0;
            for (int j = -2; j <= 2; j++)
                for (int i = -2; i <= 2; i++)
                    s += B5[j + 2] * B5[i + 2] * pix(img, w, h, pitch, x + i, y + j);
            out[(size_t)y * w + x] = (uint8_t)((s + 128) >> 8);
        }
}
