// ld_internal.cuh -- declarations shared by the CUDA translation units of
// libld.so (kernels, launch descriptors, small device helpers).  Nothing here
// is part of the public C ABI, which lives in include/ld.h.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/ld.h"

namespace ld {

// ---------------------------------------------------------------- limits
constexpr int kMaxLaunchFrames = 128;   // frame descriptors passed by value per launch
constexpr int kMaxTopK = 16;
constexpr int kMaxTheta = 4096;
constexpr int kSmemLimit = 232448;      // 227 KB opt-in dynamic shared memory per CTA

// Device-side error bits (OR-ed into a per-frame flag word).
constexpr int32_t kFlagTimeout = 1;

// Bounded spin: polls of an mbarrier before a wait gives up.
constexpr uint32_t kSpinLimit = 1u << 26;

// ---------------------------------------------------------------- Sobel
constexpr int kSobelThreads = 256;      // 8 warps, each an independent task
constexpr int kSobelWarps = kSobelThreads / 32;
constexpr int kSobelStripW = 480;       // output pixels of a warp row (lanes 1..30 x 16)

// Sobel geometry: a warp task is a strip of kSobelStripW columns by a run of
// 8 * groups rows; a CTA takes kSobelWarps consecutive tasks of one frame.
inline int sobel_strips(int w) { return (w + kSobelStripW - 1) / kSobelStripW; }
inline int sobel_frame_ctas(int w, int h, int groups) {
    const int run = 8 * groups;
    const int tasks = sobel_strips(w) * ((h + run - 1) / run);
    return (tasks + kSobelWarps - 1) / kSobelWarps;
}

struct SobelFrame {
    const uint8_t *img;
    uint8_t *bin;          // nullable
    uint32_t *edges;
    int32_t *count;
    int32_t *status_init;  // nullable: set to LD_ERR_TIMEOUT until the frame's peaks are merged
    int32_t *npeaks_init;  // nullable: set to 0 likewise
    uint8_t *pool;         // nullable: 8x8 edge counts [ceil(h/8)][ceil(w/8)] (0..64)
    int64_t cap;
    int32_t w, h, pitch;
    int32_t tile_begin;    // first CTA of this frame (host bookkeeping)
    int32_t tiles_x;       // column strips (sobel_strips(w))
    int32_t pad_;
    int64_t group_begin;   // first 8-row group of this frame in the launch (set by launch_sobel)
};

struct SobelLaunch {
    int32_t n;
    int32_t threshold;
    int32_t border;
    int32_t groups;        // 8-row groups per warp task (host bookkeeping: caps the grid)
    int64_t total_groups;  // set by launch_sobel
    SobelFrame f[kMaxLaunchFrames];
};

// ---------------------------------------------------------------- Hough
constexpr int kHoughThreads = 512;      // 16 warps (up to 128 registers per thread)
constexpr int kHoughWarps = kHoughThreads / 32;
// Edge chunk streamed per stage: 32 lane segments of odd length S, so that the
// 32 lanes of a warp read 32 distinct shared-memory banks (index l*S + o).
constexpr int kChunkSeg = 5 * kHoughWarps - 1;   // S = 79
constexpr int kChunkEdges = 32 * kChunkSeg;      // 2528 edges = 10112 bytes
constexpr int kStages = 3;

enum HoughMode : int32_t {
    kHoughFullAcc = 0,      // write the int32 accumulator (store or atomic add)
    kHoughCandidates = 1,   // emit per-tile top-M candidate keys instead
};

struct HoughFrame {
    const uint32_t *edges;
    const int32_t *count;
    int64_t cap;
    int32_t *acc;          // [n_theta][n_rho] (full-acc mode)
    uint64_t *cand;        // [n_tiles][M] keys (candidate mode)
    int32_t *flags;        // nullable per-frame error flags
    int32_t *done;         // candidate mode: tiles finished (zeroed before the launch)
    ld_peak *peaks;        // candidate mode: merged peaks [top_k]
    int32_t *n_peaks;
    int32_t *status;       // nullable
    const int32_t *pair_list;   // nullable: restricted vote, ascending active pair indices (device)
    const int32_t *pair_count;  // with pair_list: number of active pairs (device)
    int32_t w, h, D, n_rho;
    int32_t unit_begin;    // first work unit of this frame
    int32_t n_splits;      // units sharing one theta tile (edge ranges)
    int32_t pairs_per_tile;
    int32_t n_tiles;
    int32_t rows;          // interleaved-column kernel: rows of the tile accumulator
    int32_t split_base;    // interleaved-column kernel, n_splits > 1: the frame's first tile
                           // in the launch's split-tile arrays (tile_cnt, part)
    int32_t col_width;     // interleaved-column kernel: slots per tile (16, or 8 for long windows)
    int32_t pad_;
};

struct HoughLaunch {
    int32_t n;
    int32_t n_theta;
    int32_t mode;
    int32_t cand_m;        // M per tile (candidate mode)
    int32_t min_votes;
    int32_t total_units;   // work units over all frames
    int32_t top_k, nms_theta, nms_rho;   // candidate mode: the merge
    int32_t col_chunk;     // interleaved-column kernel: edges per streamed chunk
    int32_t part_stride;   // interleaved-column kernel: words per partial accumulator
    uint32_t wait_polls;   // a consumer-side wait for an edge chunk gives up after this
                           // many polls (kSpinLimit normally; 0 gives up at once)
    uint32_t *part;        // interleaved-column kernel: partial accumulators of split tiles
    int32_t *tile_cnt;     // interleaved-column kernel: finished pieces per split tile (zeroed)
    int32_t *queue;        // work-queue head (zeroed before the launch)
    const int32_t *unit_begin_dev;   // nullable: device [n + 1] unit offsets (restricted vote)
    const int32_t *col_plan;         // interleaved kernel with unit_begin_dev: device [n][3]
                                     // (tiles, n_splits, split_base) per frame
    const int32_t *trig;   // [(n_theta/2 + 1) * 2] Q16 (c_k, s_k), k <= n_theta/2
    HoughFrame f[kMaxLaunchFrames];
};

// ---------------------------------------------------------------- peaks
constexpr int kSelectThreads = 512;
constexpr int kMergeThreads = 512;
constexpr int kSelectChunk = 16384;     // accumulator cells per candidate CTA

struct SelectJob {          // candidates from a full accumulator
    const int32_t *acc;
    uint64_t *cand;         // [n_chunks][M]
    int64_t cells;
    int32_t n_rho;
    int32_t n_chunks;
    int32_t chunk_begin;    // first CTA of this accumulator
    int32_t pad_;
};

struct SelectLaunch {
    int32_t n;
    int32_t cand_m;
    int32_t min_votes;
    int32_t pad_;
    SelectJob j[kMaxLaunchFrames];
};

struct MergeJob {
    const uint64_t *cand;
    int64_t n_cand;
    ld_peak *peaks;
    int32_t *n_peaks;
    int32_t *status;        // nullable: per-frame ld_status output
    const int32_t *flags;   // nullable: per-frame device error flags
};

struct MergeLaunch {
    int32_t n;
    int32_t top_k;
    int32_t nms_theta;
    int32_t nms_rho;
    MergeJob j[kMaxLaunchFrames];
};

// Candidate key: votes desc, theta asc, rho asc  <=>  key desc.  The theta
// field is 0xFFFF - theta >= 0xF000 (theta < 4096), so a valid key is never 0.
__host__ __device__ inline uint64_t peak_key(int32_t votes, int32_t theta, int32_t rho) {
    return (uint64_t(uint32_t(votes) ^ 0x80000000u) << 32) |
           (uint64_t(0xFFFFu - uint32_t(theta)) << 16) | uint64_t(0xFFFFu - uint32_t(rho));
}

// ---------------------------------------------------------------- Hough lines
constexpr int kLinesKeys = 16384;      // supporting pixels one CTA holds (2 max(w, h))
constexpr int kLinesMaxSide = kLinesKeys / 2;

struct LinesFrame {
    const uint32_t *edges;  // 16-byte aligned edge list
    const int32_t *count;
    int64_t cap;
    const ld_peak *peaks;   // [top_k]
    const int32_t *n_peaks;
    ld_segment *segs;       // [top_k][max_segments]
    int32_t *n_segs;        // [top_k]
    int32_t *support;       // nullable [top_k]
    int32_t w, h, D, pad_;
};

struct LinesLaunch {
    int32_t n, top_k, n_theta, fill_gap, min_length, max_segments;
    int32_t keys_cap, pad_;   // shared-memory keys per CTA (set by launch_lines)
    const int32_t *trig;    // [(n_theta/2 + 1) * 2] Q16 (c_k, s_k), k <= n_theta/2
    LinesFrame f[kMaxLaunchFrames];
};

// ---------------------------------------------------------------- Canny
struct CannyFrame {
    const uint8_t *img;
    uint8_t *bin;          // nullable 0/255 map [h][pitch]
    uint32_t *edges;
    int32_t *count;
    int32_t *status_init;  // nullable: set to LD_ERR_TIMEOUT until the frame's peaks are merged
    int32_t *npeaks_init;  // nullable: set to 0 likewise
    uint8_t *cls;          // scratch [h][w]: 0, 1 weak, 2 strong
    int32_t *parent;       // scratch [h][w]: union-find forest
    uint8_t *strong;       // scratch [h][w]: root holds a strong pixel
    int64_t cap;
    int64_t px_begin;      // first pixel of this frame in the launch's pixel range
    int64_t chunk_begin;   // first 16-pixel row chunk of this frame (set by launch_canny)
    int32_t w, h, pitch;
    int32_t tile_begin;    // first 32 x 32 tile of this frame
};

struct CannyLaunch {
    int32_t n, t_low, t_high, border;
    int64_t total_px;
    int64_t total_chunks;  // set by launch_canny
    CannyFrame f[kMaxLaunchFrames];
};

// ---------------------------------------------------------------- fused Steps 1-3
constexpr int kFusedBlock = 32;        // block side (pixels) of the smaller blocks
constexpr int kFusedMaxTheta = 1024;   // the block's accumulator fits shared memory

struct FusedFrame {
    const uint8_t *img;
    int32_t *acc;          // [n_theta][n_rho], zeroed before the launch
    int32_t *status_init;  // nullable: LD_ERR_TIMEOUT until the frame's peaks are merged
    int32_t *npeaks_init;  // nullable: 0 likewise
    int32_t w, h, pitch, D, n_rho;
    int32_t tile_begin;    // first block of this frame
    int32_t tiles_x;       // blocks per row
    int32_t pad_;
};

struct FusedLaunch {
    int32_t n, n_theta, threshold, border;
    const int32_t *trig;   // [(n_theta/2 + 1) * 2] Q16 (c_k, s_k), k <= n_theta/2
    FusedFrame f[kMaxLaunchFrames];
};

// ---------------------------------------------------------------- launchers
// Fused Steps 1-3 (no edge list): one CTA per 64 x 64 block when its
// accumulator fits shared memory (n_theta <= 512) and the launch has at least
// two such blocks per SM, else per 32 x 32 block; the launch sets the frames'
// block layout itself (n_blocks is not used).
cudaError_t launch_fused_vote(const FusedLaunch &L, int n_blocks, cudaStream_t s);
size_t fused_smem_bytes(int n_theta);
int fused_blocks(int w, int h);
// Canny edges of a launch's frames (four launches on the stream); n_tiles =
// the sum of canny_tiles over the frames.
cudaError_t launch_canny(const CannyLaunch &L, int n_tiles, cudaStream_t s);
int canny_tiles(int w, int h);
// One CTA per (frame, peak slot).
cudaError_t launch_lines(const LinesLaunch &L, cudaStream_t s);
cudaError_t launch_sobel(const SobelLaunch &L, int n_ctas, cudaStream_t s);
// Persistent launch: n_ctas CTAs (at most one per SM) pull L.total_units
// work units from L.queue.  acc_words_max: the largest pairs_per_tile * n_rho
// over the launch's frames.
cudaError_t launch_hough(const HoughLaunch &L, int n_ctas, int pairs_max, int64_t acc_words_max,
                         cudaStream_t s);
cudaError_t launch_select(const SelectLaunch &L, int n_ctas, cudaStream_t s);
cudaError_t launch_merge(const MergeLaunch &L, cudaStream_t s);

// Largest pairs-per-tile whose packed accumulator fits shared memory.
int hough_max_pairs(int n_rho);

// Interleaved-column voting kernel (candidate mode, min_votes >= 1, full
// pair ranges): tiles of up to kHoughColPairs theta pairs, one per lane of a
// half-warp; the accumulator holds `rows` rows of kHoughColPairs words.  A
// frame's tiles may be split into n_splits edge ranges whose partial
// accumulators meet in L.part.
constexpr int kHoughColPairs = 16;
// Tiles of frames whose windows are too long for 16 slots use 8 slots (rows
// twice as long), one per lane of a quarter-warp (HoughFrame::col_width).
// Largest accumulator (rows x slots words) that fits shared memory with the
// smallest edge ring, and the largest `rows` for a tile width.
int hough_cols_max_words();
int hough_cols_max_rows(int width);
// Edges per streamed chunk for an accumulator of words_max words (the
// largest ring that fits).
int hough_cols_chunk(int words_max);
cudaError_t launch_hough_cols(const HoughLaunch &L, int n_ctas, int words_max, cudaStream_t s);

// Compiled tile sizes (theta pairs per CTA) of the voting kernel; a tile of
// exactly one of these sizes runs without per-pair predicates.
#define LD_HOUGH_PAIR_SIZES(X) X(2) X(3) X(4) X(5) X(6) X(8) X(9) X(10) X(12) X(15) X(16) X(18) X(20) X(24) X(30)
// Smallest compiled tile size >= pairs (0 if none).
int hough_template_pairs(int pairs);

// Proposal network: forward 3x3 convolution on the tcgen05 tensor cores
// (cin 16 or 32 -> 32 channels, NHWC bf16, + bias, ReLU).
struct ConvTcGeom {
    int n, h, w, oh, ow, stride;
};
cudaError_t launch_conv_fwd_tc(const void *x, const ConvTcGeom &G, int cin, const void *w, const float *b, void *y,
                               cudaStream_t s);
// Backward of conv2..4 on tcgen05 (ld_conv_tc.cu).  Weight gradient: per CTA
// (chunk of output pixels of one image) the partial sums of dw [32][9][cin]
// and db [32] into part / part_b (as many rows as CTAs: ceil(oh*ow/chunk) x n,
// image-major), to be summed in CTA order.  Input gradient: dx [n][h][w][cin]
// bf16 from dy masked by the ReLU of y (both [n][oh][ow][32]).
cudaError_t launch_conv_wgrad_tc(const void *x, const void *y, const void *dy, const ConvTcGeom &G, int cin,
                                 int chunk, float *part, float *part_b, cudaStream_t s);
cudaError_t launch_conv_dgrad_tc(const void *y, const void *dy, const ConvTcGeom &G, int cin, const void *w, void *dx,
                                 cudaStream_t s);
// Inference: conv1 (1->16, from the uint8 edge counts x0 [n][h][w]) fused into
// conv2 (16->32, stride 2); G describes conv2 (input h x w = conv1's output).
cudaError_t launch_conv12_fused_tc(const uint8_t *x0, const ConvTcGeom &G, const void *w1, const float *b1,
                                   const void *w2, const float *b2, void *y2, cudaStream_t s);

// Proposal: band logits -> per-frame ascending active-pair lists, counts,
// fallback flags, tile counts (at most pmax pairs and tile_cap tiles a frame,
// sized to fill waves of `slots` persistent CTAs) and the device prefix
// unit_begin [n + 1].  1 <= n <= kMaxLaunchFrames.
cudaError_t launch_select_bands(const float *logits, int n, int n_theta, float p_band, float p_fallback, int margin,
                                int pmax, int tile_cap, int slots, int32_t *pair_list, int32_t *pair_count,
                                int32_t *fallback, int32_t *tiles, int32_t *unit_begin, cudaStream_t s);
// The same band selection, planned for the interleaved-column kernel: tiles
// of at most kHoughColPairs pairs, and when the launch's last wave (of
// `slots` CTAs) would be at most half full, the tiles of the last frames split
// into edge-range pieces (at most `slots` pieces); with fewer tiles than
// slots and `fill`, every tile splits.  Writes col_plan [n][3] (tiles,
// n_splits, split_base), unit_begin [n + 1], and zeroes the split tiles'
// counters tile_cnt [slots].
cudaError_t launch_select_bands_cols(const float *logits, int n, int n_theta, float p_band, float p_fallback,
                                     int margin, int slots, bool fill, int32_t *pair_list, int32_t *pair_count,
                                     int32_t *fallback, int32_t *col_plan, int32_t *unit_begin, int32_t *tile_cnt,
                                     cudaStream_t s);

// Set the calling thread's ld_last_error() message.
void set_last_error(const char *msg);

// Parameters of a peak search on an accumulator with n_theta rows: *pp (or the
// defaults when pp is NULL) checked as ld_hough_peaks checks them; LD_OK and
// *out filled, or an error with ld_last_error() set.
ld_status peak_params(const ld_params *pp, int32_t n_theta, ld_params *out);

// One-time per-device setup of a kernel (function attributes): `done` holds
// one bit per device 0..63, set after `setup(device)` succeeded; later calls
// on that device skip it (devices >= 64 run it every time).  Launch paths
// call this instead of setting attributes on every launch, which costs driver
// calls and can wait on driver locks that other host threads hold.
template <class F>
cudaError_t once_per_device(std::atomic<uint64_t> &done, F &&setup) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 64 && ((done.load(std::memory_order_acquire) >> dev) & 1u)) return cudaSuccess;
    e = setup(dev);
    if (e == cudaSuccess && dev < 64) done.fetch_or(uint64_t(1) << dev, std::memory_order_acq_rel);
    return e;
}

}  // namespace ld
