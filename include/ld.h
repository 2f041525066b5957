/*
 * ld.h -- C ABI of the GB300 lane-detection hot path (libld.so).
 *
 * The library computes, on one CUDA GPU, the data-parallel steps of the
 * lane-detection pipeline of "Hardware Acceleration of Lane Detection
 * Algorithm: A GPU Versus FPGA Comparison" (arXiv 2212.09460):
 *
 *   Step 1  Sobel gradient magnitude |G| = |Sx*Img| + |Sy*Img|  (Sec. 2.1, Eq. 1)
 *           on the zero-padded image                           (Sec. 3.1, Sec. 4.1)
 *   Step 2  binarization to 0 / 255                            (Sec. 2.2, Sec. 4.2)
 *   Step 3  Hough voting r = x cos(theta) + y sin(theta)       (Sec. 2.3, Eq. 3, Sec. 4.3)
 *           with sin/cos symmetry                              (Sec. 3.3, Eqs. 4-5)
 *   Step 4  Hough peaks, which the paper leaves to MATLAB      (Sec. 2.3, Sec. 5)
 *
 * Conventions shared by every entry point:
 *   - Images are uint8, row-major, row stride `pitch` bytes.  x is the column
 *     (0..w-1, rightwards), y the row (0..h-1, downwards).
 *   - theta_idx k in [0, n_theta) means theta = k * 180 / n_theta degrees.
 *   - D = ceil(sqrt(w^2 + h^2)); rho lies in [-D, D] and is stored at
 *     rho_idx = rho + D, so an accumulator has n_rho = 2D + 1 columns.
 *   - The accumulator is int32, theta-major: acc[theta_idx * n_rho + rho_idx].
 *   - rho = floor((x * c_k + y * s_k + 32768) / 65536) with the Q16 table
 *     c_k = round(65536 cos(k pi / n_theta)), s_k = round(65536 sin(k pi / n_theta))
 *     for k <= n_theta / 2 and c_k = -c_{n-k}, s_k = s_{n-k} above (Eqs. 4-5).
 *   - An edge pixel is packed as (y << 16) | x in a uint32.
 *   - Pointers named d_* are device pointers, h_* host pointers.  The caller
 *     owns every buffer passed in; the library keeps only its context.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it; argument errors are
 *     returned synchronously and enqueue nothing.
 *   - Every call returns an ld_status; ld_last_error() gives the message of
 *     the calling thread's last failure.
 */
#ifndef LD_H
#define LD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LD_API __attribute__((visibility("default")))
#else
#define LD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LD_OK = 0,
    LD_ERR_INVALID = 1,   /* bad argument; nothing was enqueued */
    LD_ERR_CUDA = 2,      /* a CUDA runtime call failed */
    LD_ERR_NOMEM = 3,     /* device allocation of context scratch failed */
    LD_ERR_CAPACITY = 4,  /* an edge list overflowed its capacity */
    LD_ERR_TIMEOUT = 5    /* a bounded device wait gave up */
} ld_status;

typedef enum {
    LD_BORDER_ZERO = 0,   /* zero padding, output size = input size (Sec. 3.1, 4.1) */
    LD_BORDER_CLEAR = 1   /* as ZERO, then the 1-pixel output frame is forced to 0 */
} ld_border;

/* Method parameters.  ld_params_default() fills the values in brackets. */
typedef struct {
    int32_t n_theta;       /* theta bins over [0, 180) deg, even, 2..4096   [180] */
    int32_t threshold;     /* binarization: 255 if |G| >= threshold, 1..255  [128] */
    int32_t border;        /* ld_border                                      [ZERO] */
    int32_t top_k;         /* peaks to return, 1..16                         [4]   */
    int32_t nms_theta;     /* suppression window height (theta), odd >= 1    [5]   */
    int32_t nms_rho;       /* suppression window width (rho), odd >= 1       [5]   */
    int32_t min_votes;     /* a peak needs votes >= min_votes                [1]   */
    int32_t reserved;      /* must be 0                                            */
    int64_t edge_capacity; /* slots in a caller edge list; 0 = w*h           [0]   */
} ld_params;

/* One Hough peak: theta = theta_idx*180/n_theta deg, rho = rho_idx - D. */
typedef struct {
    int32_t theta_idx;
    int32_t rho_idx;
    int32_t votes;
} ld_peak;

/* One frame of a batch: device image, its size and row pitch in bytes. */
typedef struct {
    const uint8_t *img;
    int32_t w, h, pitch;
    int32_t reserved;      /* must be 0 */
} ld_frame;

typedef struct ld_ctx ld_ctx;

/* Fill *p with the defaults listed in ld_params. */
LD_API ld_status ld_params_default(ld_params *p);

/* Create a context on CUDA device `device`: Q16 tables and scratch for
 * ld_hough_peaks and ld_detect_batch are allocated lazily and kept until
 * ld_ctx_destroy.  A context may be used from one host thread at a time, and
 * the device work of two calls on one context must not overlap (they share
 * its scratch): use one stream per context, or one context per stream. */
LD_API ld_status ld_ctx_create(ld_ctx **out, int device);
LD_API ld_status ld_ctx_destroy(ld_ctx *ctx);

/* Pre-size the context scratch so that later ld_detect_batch calls with at
 * most `max_frames` frames totalling `max_pixels` pixels, and ld_hough_peaks
 * calls on at most `max_acc_cells` cells, allocate nothing (needed before
 * capturing those calls in a CUDA graph).  With max_frames > 0 this includes
 * the partial accumulators of split voting tiles (one per SM at the largest
 * interleaved accumulator, about 30 MB on a 152-SM GPU). */
LD_API ld_status ld_ctx_reserve(ld_ctx *ctx, int64_t max_pixels, int32_t max_frames,
                         int64_t max_acc_cells, const ld_params *p);

/* Sizes for a w x h image: *acc_elems = n_theta * (2D+1) int32 cells,
 * *edge_elems = w*h (worst-case edge count), *D = ceil(sqrt(w^2+h^2)).
 * Validates the size: 3 <= w, h and w + h <= 32767 (so the packed edge and
 * the Q16 rho fit 32 bits), and p (may be NULL for the defaults). */
LD_API ld_status ld_query_sizes(int32_t w, int32_t h, const ld_params *p,
                         size_t *acc_elems, size_t *edge_elems, int32_t *D);

/*
 * Steps 1-2 fused (Eq. 1, Sec. 2.2, Sec. 3.1, Sec. 4.1-4.2) plus the edge list
 * the voting stage reads (Sec. 4.3).
 *   d_img        uint8 [h][pitch]; pitch % 16 == 0, pitch >= w, d_img 16-byte
 *                aligned.  Bytes beyond w in a row are never read into the result.
 *   d_bin        optional (NULL to skip) uint8 [h][pitch] output, 0 or 255 per
 *                pixel, 16-byte aligned; the padding bytes w..pitch-1 of each row
 *                are unspecified on return.
 *   d_edges      uint32 [p->edge_capacity] (or [w*h] when that is 0) output:
 *                the (y << 16) | x of every 255 pixel, in unspecified order.
 *   d_edge_count int32 [1] output: the true number of edge pixels.  If it
 *                exceeds the capacity, only `capacity` entries were written
 *                (the caller checks after synchronising; LD_ERR_CAPACITY).
 */
LD_API ld_status ld_sobel_binarize(ld_ctx *ctx, const uint8_t *d_img, int32_t w,
                            int32_t h, int32_t pitch, const ld_params *p,
                            uint8_t *d_bin, uint32_t *d_edges,
                            int32_t *d_edge_count, void *stream);

/*
 * Step 3 (Eq. 3, Eqs. 4-5, Sec. 4.3): for every edge pixel and every theta bin,
 * acc[k][rho + D] += 1.
 *   d_edges      uint32 edge list, 16-byte aligned, as written by ld_sobel_binarize:
 *                distinct pixels.  Entries with x >= w or y >= h are skipped.  (The
 *                kernel counts in 16 bits per cell, exact for distinct pixels since
 *                a rho strip of width 1 holds at most 2*max(w, h) <= 65528 of them.)
 *   d_edge_count int32 [1] device count; min(count, capacity) edges are read,
 *                capacity = p->edge_capacity or w*h when 0.
 *   d_acc        int32 [n_theta][2D+1] output, fully overwritten.
 */
LD_API ld_status ld_hough_vote(ld_ctx *ctx, const uint32_t *d_edges,
                        const int32_t *d_edge_count, int32_t w, int32_t h,
                        const ld_params *p, int32_t *d_acc, void *stream);

/*
 * Step 4 (Sec. 2.3 "Hough Peak", Sec. 5): greedy non-maximum suppression.
 * Up to top_k times: take the cell first in the order (votes desc, theta_idx
 * asc, rho_idx asc) that is not suppressed and has votes >= min_votes, emit
 * it, and suppress the nms_theta x nms_rho window around it (clipped at the
 * grid edges, theta does not wrap).
 *   d_acc        int32 [n_theta][n_rho] input (any values).
 *   d_peaks      ld_peak [top_k] output, in emission order.
 *   d_n_peaks    int32 [1] output, the number of peaks emitted (<= top_k).
 */
LD_API ld_status ld_hough_peaks(ld_ctx *ctx, const int32_t *d_acc, int32_t n_theta,
                         int32_t n_rho, const ld_params *p, ld_peak *d_peaks,
                         int32_t *d_n_peaks, void *stream);

/*
 * Steps 1-4 for a batch of frames of possibly different sizes, each as in the
 * calls above (border, threshold, theta bins and peaks from *p).
 *   h_frames     host array of n frame descriptors (device images); 1 <= n.
 *   d_peaks      ld_peak [n][top_k] output.
 *   d_n_peaks    int32 [n] output.
 *   d_status     int32 [n] output, per-frame ld_status of the device work
 *                (LD_OK, or LD_ERR_TIMEOUT if a bounded wait gave up).
 * Edge lists and candidate buffers live in the context scratch, sized for
 * the worst case (every pixel an edge), so no capacity error can occur.
 * Step 3 runs in one of two voting kernels, per launch group of up to 128
 * frames: with min_votes >= 1, frames whose theta windows fit shared memory
 * in tiles of 16 or 8 theta pairs (windows up to about 6100 rows: every size
 * up to 3840x2160 and beyond; 8 pairs for windows over about 3000 rows, and
 * for launches whose 16-pair tiles would occupy at most half the SMs) take
 * the interleaved-column kernel, the others
 * the packed-pair kernel; a group with both kinds takes one launch per kernel
 * when each part fills the GPU, else the packed-pair kernel for all.  The
 * results never depend on the kernel, the tile sizes or the edge-range
 * splits.
 */
LD_API ld_status ld_detect_batch(ld_ctx *ctx, const ld_frame *h_frames, int32_t n,
                          const ld_params *p, ld_peak *d_peaks,
                          int32_t *d_n_peaks, int32_t *d_status, void *stream);

/*
 * Steps 1-4 as ld_detect_batch for frames and results in HOST memory: the
 * end-to-end call of a camera pipeline.
 *   h_frames     host array of n frame descriptors whose img are HOST
 *                pointers ([h][pitch] uint8, pitch a multiple of 16); page-
 *                locked memory lets the upload overlap other work.
 *   h_peaks      host ld_peak [n][top_k], h_n_peaks and h_status host int32
 *                [n]: the outputs of ld_detect_batch, copied back.
 * The call enqueues work and returns; the outputs are valid once `stream`'s
 * work up to this call has completed (e.g. after cudaStreamSynchronize).
 * The frames are copied (one cudaMemcpyAsync per run of frames adjacent in
 * host memory) into one of two device staging areas owned by the context,
 * used by alternate calls, on a copy stream of the context; detection waits
 * for the upload on `stream`, and an upload waits for the outputs of the
 * call before last (same area) to be read back.  So the upload of one call
 * overlaps the detection of the previous one.  The host buffers must stay
 * valid and unchanged until the call's work has completed.  An area grows
 * (waiting for its previous call) when a call needs more room.  Not
 * capturable in a CUDA graph (it uses the context's copy stream).  Argument
 * errors are reported before anything is enqueued.
 */
LD_API ld_status ld_detect_batch_host(ld_ctx *ctx, const ld_frame *h_frames, int32_t n,
                               const ld_params *p, ld_peak *h_peaks,
                               int32_t *h_n_peaks, int32_t *h_status, void *stream);

/*
 * Step 4 as ld_hough_peaks, for callers that may not allocate device memory.
 * The paper has no counterpart; this is a property of the library.
 *
 * ld_hough_peaks grows its candidate buffer inside the context with cudaMalloc.
 * A camera loop with a per-frame deadline or a host thread that must never
 * block cannot call cudaMalloc while running (it may synchronise the device and
 * its latency is unbounded), and a process whose device memory is fixed at
 * start-up may not grow it.  This entry point takes no context and allocates
 * nothing: the candidates live in a 1 MiB array of the library's own device
 * memory (131072 keys), present on every GPU that loads the library until the
 * process exits.  Arguments, results and errors are those of ld_hough_peaks,
 * on the calling thread's current device, plus one limit: ceil(n_theta*n_rho /
 * 16384) * (nms_theta*nms_rho*(top_k-1)+1) <= 131072 (a 360 x 4407
 * accumulator with 5x5 windows and top_k 4 needs 7372), else LD_ERR_INVALID.
 * The first call on a device looks up the array's device address and keeps
 * it; make that first call before any stream capture, and do not call this
 * entry point on a device after cudaDeviceReset (or another teardown of its
 * primary context) in the same process, since the kept address is then stale.
 * All calls on a device share the array (each call rewrites every slot it
 * reads, nothing needs clearing), so calls whose work overlaps on the GPU
 * race: serialise them.  p may be NULL for the defaults.
 */
LD_API ld_status ld_hough_peaks_static(const int32_t *d_acc, int32_t n_theta,
                                       int32_t n_rho, const ld_params *p,
                                       ld_peak *d_peaks, int32_t *d_n_peaks,
                                       void *stream);

/*
 * Hough lines: the line segments behind each peak (Step 4 of Sec. 1 without
 * the drawing; the paper hands the peaks to MATLAB's "Hough lines", Sec. 5,
 * Fig. 12, with no parameters stated).  For a peak (theta_idx k, rho_idx r)
 * the supporting pixels are the edges whose Q16 rho at theta_k is cell r (the
 * vote's own rounding, so their number is the peak's vote count).  They are
 * ordered along the line -- by x then y when |c_k| <= |s_k| (the line is at
 * most 45 degrees from horizontal), else by y then x -- and split wherever two
 * consecutive pixels are farther apart than fill_gap (squared Euclidean
 * distance > fill_gap^2); a piece is kept when its end pixels are at least
 * min_length apart (squared distance >= min_length^2).  A segment runs from
 * its first pixel (x1, y1) to its last (x2, y2) in that order.
 */
typedef struct {
    int32_t fill_gap;      /* largest gap inside a segment, pixels, 0..65535     [20] */
    int32_t min_length;    /* shortest kept segment, pixels, 0..65535            [40] */
    int32_t max_segments;  /* segments stored per peak, 1..4096                   [16] */
    int32_t reserved;      /* must be 0 */
} ld_lines_params;

typedef struct {
    int32_t x1, y1, x2, y2;     /* first and last supporting pixel */
    int32_t theta_idx, rho_idx; /* the peak's cell */
} ld_segment;

/* Fill *lp with the defaults listed in ld_lines_params. */
LD_API ld_status ld_lines_params_default(ld_lines_params *lp);

/*
 * Hough lines of one frame from its edge list and peaks.
 *   d_edges      uint32 edge list as for ld_hough_vote (16-byte aligned,
 *                distinct in-image pixels; entries outside the image are skipped).
 *   d_edge_count int32 [1]: min(count, capacity) edges are read (capacity =
 *                p->edge_capacity or w*h when 0).
 *   d_peaks      ld_peak [p->top_k] and d_n_peaks int32 [1], as ld_hough_peaks
 *                writes them (theta_idx < p->n_theta, rho_idx < 2D+1).
 *   d_segments   ld_segment [top_k][lp->max_segments] output: peak j's kept
 *                segments in line order (the first max_segments of them).
 *   d_n_segments int32 [top_k] output: kept segments per peak (may exceed
 *                max_segments; 0 for j >= *d_n_peaks).
 *   d_support    int32 [top_k] output (nullable): supporting pixels per peak.
 * Sizes: as ld_hough_vote, and max(w, h) <= 8192 (a peak's supporting pixels,
 * at most 2 max(w, h), are sorted in shared memory), else LD_ERR_INVALID.
 * p and lp may be NULL for the defaults.
 */
LD_API ld_status ld_hough_lines(ld_ctx *ctx, const uint32_t *d_edges, const int32_t *d_edge_count,
                                int32_t w, int32_t h, const ld_params *p, const ld_peak *d_peaks,
                                const int32_t *d_n_peaks, const ld_lines_params *lp,
                                ld_segment *d_segments, int32_t *d_n_segments, int32_t *d_support,
                                void *stream);

/*
 * Steps 1-4 with the Hough lines: ld_detect_batch, then the segments of every
 * frame's peaks from the frame's edge list (kept in the context scratch).
 * Outputs as ld_detect_batch plus d_segments [n][top_k][max_segments],
 * d_n_segments [n][top_k] and d_support [n][top_k] (nullable), laid out per
 * frame as ld_hough_lines writes them.  Frames need max(w, h) <= 8192.
 * The segments of a frame are meaningful when its d_status is LD_OK.
 */
LD_API ld_status ld_detect_lines_batch(ld_ctx *ctx, const ld_frame *h_frames, int32_t n,
                                       const ld_params *p, const ld_lines_params *lp,
                                       ld_peak *d_peaks, int32_t *d_n_peaks, int32_t *d_status,
                                       ld_segment *d_segments, int32_t *d_n_segments,
                                       int32_t *d_support, void *stream);

/*
 * Steps 1-3 without an edge list, in the spirit of the paper's FPGA dataflow
 * (Sec. 3.3: pixels stream through one unit per theta; Table 1): each CTA
 * finds the edge pixels of a 32 x 32 block of the image (Steps 1-2 as in
 * ld_sobel_binarize) and votes them into a shared-memory accumulator over
 * every theta and the rho cells the block reaches, then adds its non-zero
 * cells into d_acc.  The result equals ld_sobel_binarize followed by
 * ld_hough_vote.
 *   d_img   as for ld_sobel_binarize.
 *   d_acc   int32 [n_theta][2D+1] output, fully overwritten (zeroed here first).
 * Sizes: as ld_sobel_binarize, and p->n_theta <= 1024.
 */
LD_API ld_status ld_sobel_hough_fused(ld_ctx *ctx, const uint8_t *d_img, int32_t w, int32_t h,
                                      int32_t pitch, const ld_params *p, int32_t *d_acc, void *stream);

/* Steps 1-4 as ld_detect_batch, with Steps 1-3 fused as in
 * ld_sobel_hough_fused into per-frame accumulators in the context scratch
 * (n_theta * (2D+1) int32 cells per frame), then the peaks of each.
 * p->n_theta <= 1024. */
LD_API ld_status ld_detect_fused_batch(ld_ctx *ctx, const ld_frame *h_frames, int32_t n,
                                       const ld_params *p, ld_peak *d_peaks, int32_t *d_n_peaks,
                                       int32_t *d_status, void *stream);

/*
 * Canny edge detection in place of Steps 1-2 (the paper's future work, Sec. 7),
 * behind the same edge-list boundary as ld_sobel_binarize.  Integer stages, each
 * with zero outside the image (the padding of Sec. 3.1): a 5x5 binomial blur
 * G = (sum b_i b_j I + 128) >> 8 with b = (1 4 6 4 1); the Sobel magnitude
 * M = |gx| + |gy| of G (Eq. 1, not saturated); the gradient sector from
 * tan(22.5) = 27146/65536 and tan(67.5) = 158218/65536 (|gy| 65536 <= 27146 |gx|:
 * along x; >= 158218 |gx|: along y; else the diagonal of the sign of gx gy);
 * non-maximum suppression keeping M > 0, M > M(n1), M >= M(n2) with n1 the
 * neighbour with the smaller y (smaller x along x); hysteresis: the edges are
 * the 8-connected components of kept pixels with M >= t_low that hold one with
 * M >= t_high.  p->border = LD_BORDER_CLEAR also zeroes the 1-pixel frame;
 * p->threshold is not used.
 */
typedef struct {
    int32_t t_low;         /* weak edge threshold on M, 1..2040    [100] */
    int32_t t_high;        /* strong edge threshold on M, t_low..2040 [200] */
    int32_t reserved0, reserved1;   /* must be 0 */
} ld_canny_params;

/* Fill *cp with the defaults listed in ld_canny_params. */
LD_API ld_status ld_canny_params_default(ld_canny_params *cp);

/* Canny edges of one frame: arguments and outputs as ld_sobel_binarize (the
 * edge list in unspecified order, the true count, optional 0/255 map); the
 * context holds 6 bytes of scratch per pixel.  cp may be NULL for the defaults. */
LD_API ld_status ld_canny(ld_ctx *ctx, const uint8_t *d_img, int32_t w, int32_t h, int32_t pitch,
                          const ld_params *p, const ld_canny_params *cp, uint8_t *d_bin,
                          uint32_t *d_edges, int32_t *d_edge_count, void *stream);

/* Steps 1-4 as ld_detect_batch with Canny edges in place of Steps 1-2. */
LD_API ld_status ld_detect_canny_batch(ld_ctx *ctx, const ld_frame *h_frames, int32_t n,
                                       const ld_params *p, const ld_canny_params *cp,
                                       ld_peak *d_peaks, int32_t *d_n_peaks, int32_t *d_status,
                                       void *stream);

/*
 * Autotuner for ld_detect_batch.  For every distinct frame size among
 * h_frames (device images, as in ld_detect_batch), it times ld_detect_batch
 * on the frames of that size, `iters` calls per candidate: first the voting
 * stage for each candidate voting tile size (theta pairs per CTA: the
 * compiled sizes from 1/8 of the largest that fits shared memory up to it,
 * and the interleaved-column kernel where it fits and min_votes >= 1),
 * then the Sobel stage for each run length (1, 2 or 4 groups of 8 rows per
 * warp), and keeps the fastest of each in the context; later ld_detect_batch
 * calls on frames of that size and n_theta use them.  Results do not depend
 * on the choice.  Stage timings recorded before the call are discarded.  Runs
 * and synchronises `stream`; allocates scratch like ld_detect_batch; must not
 * be captured.  iters >= 1.
 */
LD_API ld_status ld_autotune(ld_ctx *ctx, const ld_frame *h_frames, int32_t n,
                             const ld_params *p, int32_t iters, void *stream);

/* The voting tile size (theta pairs per CTA) and the Sobel run length (in
 * groups of 8 rows per warp) that ld_detect_batch uses for w x h frames with
 * p->n_theta (tuned or default).  *pairs_per_tile is negative (minus the
 * pairs per tile) when the interleaved-column voting kernel votes (tiles of
 * up to 16 pairs; a launch group uses it only if every frame's plan does). */
LD_API ld_status ld_ctx_plan(ld_ctx *ctx, int32_t w, int32_t h, const ld_params *p,
                             int32_t *pairs_per_tile, int32_t *sobel_rows);

/* Fault-injection knob for the bounded waits of the voting kernels (not a
 * step of the method).  Later calls on ctx give up a wait for a streamed edge
 * chunk after `polls` polls of its mbarrier: 0 gives up at once, a negative
 * value restores the default 2^26 (polls <= 2^26, else LD_ERR_INVALID).  A CTA
 * whose wait gave up flags its frame, waits (with the default limit) for the
 * copies it issued itself, and stops; the frame's status stays LD_ERR_TIMEOUT
 * and its peaks are unspecified.  Lets a test make a wait run out without any
 * copy that fails to complete. */
LD_API ld_status ld_ctx_set_wait_limit(ld_ctx *ctx, int64_t polls);

/* Stage timing.  After ld_ctx_enable_timing(ctx, 1), every ld_detect_batch
 * call (and ld_detect_canny_batch, ld_detect_lines_batch and
 * ld_detect_fused_batch) also records CUDA events on its stream around its
 * launches: before Steps 1-2, between Steps 1-2 and Steps 3-4 (the voting
 * launch also merges the peaks), and after Steps 3-4 (batches of more than
 * 128 frames: the first launch group).  In ld_detect_fused_batch the first
 * stage is Steps 1-3 (the accumulator clear and the fused vote) and the second
 * Step 4; the segment search of ld_detect_lines_batch runs after the last
 * event.  ld_ctx_stage_ms waits for every call timed since its previous use
 * (at most 1024) and returns, summed over them, the device time of the first
 * stage (ms[0]) and the second (ms[1]) in milliseconds and the number of calls
 * in ms[2].  enable = 0 switches recording off. */
LD_API ld_status ld_ctx_enable_timing(ld_ctx *ctx, int enable);
LD_API ld_status ld_ctx_stage_ms(ld_ctx *ctx, float ms[3]);

/*
 * Input of the proposal network: for each frame, Steps 1-2 as in
 * ld_detect_batch, then the 8x8 box-downsampled binary map: d_pool[f] is a
 * uint8 [ceil(h/8)][ceil(w/8)] map (frames packed back to back, in order)
 * holding the number of edge pixels (0..64) in each 8x8 block (clipped at
 * the frame edge).
 */
LD_API ld_status ld_edge_pool_batch(ld_ctx *ctx, const ld_frame *h_frames, int32_t n,
                                    const ld_params *p, uint8_t *d_pool, void *stream);

/*
 * Learned theta-band proposal network: its layers as separate calls (the
 * caller's training loop or inference orders them).  The paper has no learned
 * stage; this network predicts, from the 8x8 edge-count map (read as
 * count / 64 by the first layer), which
 * 5-degree theta bands hold the top Hough peaks (36 logits) and which of 8
 * row bands their lines cross (8 logits), so that voting can skip bands.
 * Layout: activations NHWC, bf16 (uint8 counts 0..64 for the first layer's
 * input, scaled by 1/64);
 * conv weights bf16 [Cout][3][3][Cin]; biases, head, losses and gradients
 * fp32; "dy" is the gradient with respect to a layer's ReLU output.
 * Supported convs: 1->16 (stride 1), 16->32 and 32->32 (stride 1 or 2), all
 * 3x3 with zero padding 1; output size (h + 2 - 3) / stride + 1.  Sizes:
 * w >= 2 and h * w * w < 2^32 (else LD_ERR_INVALID).
 */
/* y = relu(conv(x, w) + b). */
LD_API ld_status ld_conv3x3_forward(const void *d_x, int32_t n, int32_t h, int32_t w,
                                    int32_t cin, int32_t cout, int32_t stride,
                                    const void *d_w, const float *d_b, void *d_y, void *stream);
/* Faults recorded on CUDA device `device` by the tensor-core forward
 * convolutions (16->32 and 32->32) since the previous call: a bounded wait
 * for the tensor cores that gave up, after which that layer's output is
 * unspecified.  Reads and clears; *flags = 0 when there was none. */
LD_API ld_status ld_conv_faults(int32_t device, int32_t *flags);
/* From dy (bf16, w.r.t. the ReLU output y): dw += dL/dw, db += dL/db (fp32,
 * accumulated: zero them first) and, if d_dx != NULL, dx = dL/dx (bf16).  The
 * 1-channel layer takes d_dx = NULL.  Partial sums are reduced in a fixed
 * order (a stream-ordered workspace), so the results are bitwise
 * reproducible. */
LD_API ld_status ld_conv3x3_backward(const void *d_x, int32_t n, int32_t h, int32_t w,
                                     int32_t cin, int32_t cout, int32_t stride,
                                     const void *d_w, const void *d_y, const void *d_dy,
                                     void *d_dx, float *d_dw, float *d_db, void *stream);
/* Adaptive average pool of conv4's output y4 [n][h4][w4][32] to 4x8 ->
 * feat [n][1024] ((bin row, bin col, channel) order), logits [n][44] =
 * feat . wh^T + bh, wh [44][1024]. */
LD_API ld_status ld_pool_head_forward(const void *d_y4, int32_t n, int32_t h4, int32_t w4,
                                      const float *d_wh, const float *d_bh, float *d_feat,
                                      float *d_logits, void *stream);
/* dwh += dlogits^T feat, dbh += sum dlogits (accumulated), dy4 = dL/dy4 (bf16). */
LD_API ld_status ld_pool_head_backward(const float *d_feat, const float *d_dlogits,
                                       const float *d_wh, int32_t n, int32_t h4, int32_t w4,
                                       float *d_dwh, float *d_dbh, void *d_dy4, void *stream);
/* Mean binary cross-entropy with logits over n*k outputs -> *d_loss, and
 * d_dlogits = dloss/dlogits. */
LD_API ld_status ld_bce_loss(const float *d_logits, const float *d_target, int32_t n, int32_t k,
                             float *d_loss, float *d_dlogits, void *stream);
/* One Adam step (bias-corrected, step >= 1) on fp32 params; if d_param_bf16
 * is not NULL it receives the bf16 copy used by the forward pass. */
LD_API ld_status ld_adam_step(float *d_param, const float *d_grad, float *d_m, float *d_v,
                              int64_t count, float lr, float beta1, float beta2, float eps,
                              int32_t step, void *d_param_bf16, void *stream);

/* Training targets [n][44] for the network from a batch's peaks (as written
 * by ld_detect_batch, top_k per frame).  A peak counts if it is among the
 * first always_k or has at least rel_votes times the first peak's votes.
 * Targets: 1 for the 5-degree theta band of each counted peak (n_theta a
 * multiple of 36), and 1 for each of the 8 row bands (h/8 rows each) holding
 * a row where a counted peak's line crosses the w x h frame. */
LD_API ld_status ld_proposal_targets(const ld_peak *d_peaks, const int32_t *d_n_peaks,
                                     int32_t n, int32_t top_k, int32_t w, int32_t h,
                                     int32_t n_theta, int32_t always_k, float rel_votes,
                                     float *d_targets, void *stream);

/* Device pointers of a trained network (layouts as above). */
typedef struct {
    const void *w[4];       /* bf16 conv weights */
    const float *b[4];
    const float *wh;        /* [44][1024] */
    const float *bh;        /* [44] */
} ld_proposal_net;

typedef struct {
    float p_band;           /* vote a band if sigmoid(logit) >= p_band              [0.2]  */
    float p_fallback;       /* full vote if every band's probability < p_fallback  [0.5]
                               (or < p_band: a frame always votes some pair)           */
    int32_t margin;         /* extra theta bins voted on each side of a kept band  [2]   */
    int32_t reserved;       /* must be 0 */
} ld_proposal_params;

/*
 * Steps 1-4 with the learned proposal in front of the vote, for a batch of
 * frames of one size: Steps 1-2 plus the 8x8 edge-count map, the network,
 * band selection, then Hough voting only over the theta pairs {k, n-k} that
 * hold a kept bin (Eqs. 3-5), and the peak greedy over the voted cells.  The
 * peaks equal those of ld_detect_batch whenever the kept bins contain every
 * peak of the full vote (each cell's count is exact, and a cell outside the
 * kept bins can only precede a full-vote peak in the order if an earlier pick
 * suppresses it).  Outputs as ld_detect_batch, plus per frame: d_fallback[f]
 * = 1 if the full vote ran, d_active_pairs[f] = theta pairs voted (both
 * nullable).  pp may be NULL for the defaults.  p->n_theta must be a
 * multiple of 36; the frame size must leave conv4 at least 4 x 8 (about
 * w >= 450, h >= 200).
 */
LD_API ld_status ld_detect_batch_proposal(ld_ctx *ctx, const ld_frame *h_frames, int32_t n,
                                          const ld_params *p, const ld_proposal_net *net,
                                          const ld_proposal_params *pp, ld_peak *d_peaks,
                                          int32_t *d_n_peaks, int32_t *d_status,
                                          int32_t *d_fallback, int32_t *d_active_pairs,
                                          void *stream);

/* Inference of the proposal network on n edge-count maps d_pool [n][ph][pw]
 * (uint8 counts 0..64 as ld_edge_pool_batch writes them): the network of the
 * layer calls here, with conv1 fused into conv2 on the tensor cores (its
 * output never leaves the SM; the logits are bit-identical to the layer calls),
 * then conv3, conv4 and pool + head.  d_logits: fp32 [n][44].  Scratch lives in
 * the context.  The map must leave conv4's output at least 4 x 8. */
LD_API ld_status ld_proposal_logits(ld_ctx *ctx, const uint8_t *d_pool, int32_t n, int32_t ph,
                                    int32_t pw, const ld_proposal_net *net, float *d_logits,
                                    void *stream);


/*
 * Synthetic input frames, generated on the device (for training the proposal
 * network and feeding the serving loop).  Not a step of the method: the
 * paper's test image is not available, so seeded synthetic road frames stand
 * in for it.  A frame is the integer function of its descriptor described in
 * synth.py (background gradient, Q16 stripes with dashes, Irwin-Hall noise
 * from SplitMix64 streams, salt); both generators give the same bytes.
 */
typedef struct {
    int64_t nx, ny, c;      /* inside if |x*nx + y*ny - c| < 3*65536 (Q16 unit normal) */
    int64_t tx, ty, t0;     /* dash phase t = floor((x*tx + y*ty - t0) / 65536) */
    int32_t dash, gap;      /* dash if t mod (dash+gap) < dash; dash = 0: solid */
    int32_t value;          /* stripe intensity */
    int32_t reserved;
} ld_synth_stripe;

typedef struct {
    uint8_t *img;           /* device output [h][pitch] */
    int32_t w, h, pitch;
    int32_t n_stripes;      /* 0..4 */
    uint64_t base[3];       /* SplitMix64 stream bases: noise a, noise b, salt */
    int64_t k_top, k_road;  /* Q32 noise scale above / below the horizon y = h/2 */
    uint64_t salt_thr;      /* salt where the draw's low 32 bits < salt_thr (0: none) */
    ld_synth_stripe stripes[4];
} ld_synth_frame;

/* Generate n frames; d_frames is a DEVICE array of n descriptors. */
LD_API ld_status ld_synth_frames(const ld_synth_frame *d_frames, int32_t n, void *stream);

/* Measurement probe (not part of the path): n_ctas CTAs of 1024 threads each
 * perform `iters` 32-bit shared-memory reductions per thread (red.shared.add)
 * into a 16 KB shared array: pattern 0 puts the 32 lanes of every
 * instruction on 32 distinct banks (the conflict-free rate that bounds Step
 * 3's voting, Sec. 4.3), pattern 1 on pseudo-random words (32 unrelated
 * votes).  Each CTA writes its array's sum (n_ctas * 1024 * iters in all) to
 * d_sink[blockIdx] (device, n_ctas uint32).  The caller times the call on
 * `stream`.  iters: a positive multiple of 8. */
LD_API ld_status ld_probe_smem_red(int32_t n_ctas, int32_t iters, int32_t pattern, uint32_t *d_sink,
                                   void *stream);

/* Message of the calling thread's last failed call ("" if none). */
LD_API const char *ld_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LD_H */
