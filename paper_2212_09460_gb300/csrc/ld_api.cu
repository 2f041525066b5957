// ld_api.cu -- host side of the C ABI declared in include/ld.h: argument
// validation, the context (Q16 cos/sin tables, scratch), launch planning.
// All computation runs in the kernels of ld_sobel.cu, ld_hough.cu and
// ld_peaks.cu; nothing here computes a result on the host.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <mutex>
#include <string>
#include <vector>

#include "ld_internal.cuh"
#include "ld_plan.h"

using namespace ld;
static_assert(kPlanColPairs == kHoughColPairs, "planning and kernel tile widths differ");

namespace {

thread_local std::string g_err;

ld_status fail(ld_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

ld_status cuda_fail(cudaError_t e, const char *what) {
    return fail(LD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    // Grow-only device buffer; false on allocation failure.
    bool ensure(size_t need) {
        if (need <= bytes) return true;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        if (cudaMalloc(&p, need) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        bytes = need;
        return true;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

// Keeps the calling thread's current device, switching to the context's.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

void ld::set_last_error(const char *msg) { g_err = msg; }

struct ld_ctx {
    int device = 0;
    int num_sms = 148;
    std::map<int, int32_t *> trig;        // n_theta -> device Q16 table
    std::map<int, std::vector<int32_t>> trig_host;
    DevBuf edges, small, cand;            // detect_batch / hough_peaks scratch
    DevBuf prop;                          // proposal path: edge-count maps, activations, pair lists
    DevBuf part;                          // interleaved voting: split tiles' partial accumulators + counters
    DevBuf canny;                         // Canny: class map, union-find forest, strong marks
    DevBuf fused;                         // fused Steps 1-3: per-frame accumulators
    std::vector<cudaEvent_t> ev;   // 3 events per timed call, reused in order
    int timed_calls = 0;           // timed calls since the last ld_ctx_stage_ms
    bool timing = false;
    // autotuned plans: (w, h, n_theta) -> (theta pairs per tile, Sobel rows per
    // warp); pairs -1 selects the interleaved-column voting kernel
    std::map<std::tuple<int, int, int>, std::pair<int, int>> tuned;
    int force_pairs = 0, force_rows = 0;   // set while the autotuner times candidates
    uint32_t wait_polls = kSpinLimit;      // consumer-side chunk waits of the voting kernels
    // (w, h, n_theta) -> rows of the interleaved-column accumulator
    mutable std::map<std::tuple<int, int, int>, int> col_rows;
    // ld_detect_batch_host: two device staging areas (frames, then the outputs)
    // used by alternate calls, the copy stream and, per area, the events that
    // mark its frames copied and its outputs read back
    DevBuf stage[2];
    cudaStream_t hcopy = nullptr;
    cudaEvent_t hev_copied[2] = {nullptr, nullptr}, hev_free[2] = {nullptr, nullptr};
    bool hev_used[2] = {false, false};
    uint64_t host_calls = 0;
    std::mutex mu;
};

namespace {

ld_status check_params(const ld_params *p) {
    if (!p) return LD_OK;
    if (p->n_theta < 2 || p->n_theta > kMaxTheta || (p->n_theta & 1))
        return fail(LD_ERR_INVALID, "n_theta must be even in [2, %d], got %d", kMaxTheta, p->n_theta);
    if (p->threshold < 1 || p->threshold > 255)
        return fail(LD_ERR_INVALID, "threshold must be in [1, 255], got %d", p->threshold);
    if (p->border != LD_BORDER_ZERO && p->border != LD_BORDER_CLEAR)
        return fail(LD_ERR_INVALID, "border must be LD_BORDER_ZERO or LD_BORDER_CLEAR");
    if (p->top_k < 1 || p->top_k > kMaxTopK)
        return fail(LD_ERR_INVALID, "top_k must be in [1, %d], got %d", kMaxTopK, p->top_k);
    if (p->nms_theta < 1 || !(p->nms_theta & 1) || p->nms_rho < 1 || !(p->nms_rho & 1) ||
        p->nms_theta > 255 || p->nms_rho > 255)
        return fail(LD_ERR_INVALID, "nms_theta and nms_rho must be odd in [1, 255]");
    if ((int64_t)p->nms_theta * p->nms_rho * (p->top_k - 1) + 1 > 4096)
        return fail(LD_ERR_INVALID, "nms_theta*nms_rho*(top_k-1)+1 must be <= 4096");
    if (p->reserved != 0) return fail(LD_ERR_INVALID, "ld_params.reserved must be 0");
    if (p->edge_capacity < 0) return fail(LD_ERR_INVALID, "edge_capacity must be >= 0");
    return LD_OK;
}

int cand_m(const ld_params &p) { return p.nms_theta * p.nms_rho * (p.top_k - 1) + 1; }

// Image size rules plus the guarantee the voting kernel relies on: every
// pixel's Q16 rho lies in [-D, D].  rho is linear in (x, y), so checking the
// four corners for every table entry is exact.
ld_status check_size(int w, int h, const ld_params &p, const std::vector<int32_t> *trig) {
    if (w < 3 || h < 3 || (int64_t)w + h > 32767)
        return fail(LD_ERR_INVALID, "image size %dx%d: need w, h >= 3 and w + h <= 32767", w, h);
    const int64_t D = rho_max_of(w, h);
    const int64_t n_rho = 2 * D + 1;
    if (hough_max_pairs((int)n_rho) < 1)
        return fail(LD_ERR_INVALID, "image %dx%d: accumulator row of %lld cells does not fit shared memory",
                    w, h, (long long)n_rho);
    if (trig) {
        const int half = p.n_theta / 2;
        const int64_t xs[2] = {0, w - 1}, ys[2] = {0, h - 1};
        for (int k = 0; k < p.n_theta; ++k) {
            const int kk = k <= half ? k : p.n_theta - k;
            const int64_t c = k <= half ? (*trig)[2 * kk] : -(*trig)[2 * kk];
            const int64_t s = (*trig)[2 * kk + 1];
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    const int64_t v = xs[a] * c + ys[b] * s + 32768;
                    const int64_t r = v >= 0 ? v / 65536 : -((-v + 65535) / 65536);
                    if (r < -D || r > D)
                        return fail(LD_ERR_INVALID, "image %dx%d with %d theta bins: rho leaves [-D, D]", w,
                                    h, p.n_theta);
                }
        }
    }
    return LD_OK;
}

ld_status get_trig(ld_ctx *ctx, int n_theta, const int32_t **dev, const std::vector<int32_t> **host) {
    auto it = ctx->trig.find(n_theta);
    if (it == ctx->trig.end()) {
        std::vector<int32_t> t = make_trig(n_theta);
        int32_t *d = nullptr;
        cudaError_t e = cudaMalloc(&d, t.size() * sizeof(int32_t));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(trig)");
        e = cudaMemcpy(d, t.data(), t.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(d);
            return cuda_fail(e, "cudaMemcpy(trig)");
        }
        ctx->trig_host[n_theta] = std::move(t);
        it = ctx->trig.emplace(n_theta, d).first;
    }
    *dev = it->second;
    if (host) *host = &ctx->trig_host[n_theta];
    return LD_OK;
}

ld_params defaults() {
    ld_params p;
    p.n_theta = 180;
    p.threshold = 128;
    p.border = LD_BORDER_ZERO;
    p.top_k = 4;
    p.nms_theta = 5;
    p.nms_rho = 5;
    p.min_votes = 1;
    p.reserved = 0;
    p.edge_capacity = 0;
    return p;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Sobel 8-row groups per warp task: the longest runs (4 groups) that still
// give at least 3 CTAs per SM for the launch group, else shorter ones (small
// frames need the CTAs more than the longer runs).  ctas_at_g1 is the CTA
// count with 1 group per task.
int pick_sobel_groups(int64_t ctas_at_g1, int num_sms) {
    if (ctas_at_g1 / 4 >= 3 * num_sms) return 4;
    if (ctas_at_g1 / 2 >= 3 * num_sms) return 2;
    return 1;
}

// Small per-context scratch: per-frame edge counts, error flags and finished
// tile counts of one launch group, and the work-queue head.
constexpr size_t kSmallInts = 3 * kMaxLaunchFrames + 32;
struct Small {
    int32_t *counts, *flags, *done, *queue;
};
Small small_of(void *p) {
    int32_t *b = (int32_t *)p;
    return {b, b + kMaxLaunchFrames, b + 2 * kMaxLaunchFrames, b + 3 * kMaxLaunchFrames};
}

// Split tiles of the interleaved voting kernel: at most num_sms pieces in a
// launch; scratch = the pieces' arrival counters (one per tile, 256-byte
// padded) then their partial accumulators.
size_t split_scratch_bytes(int pieces, int words) {
    return ((size_t)pieces * 4 + 255) / 256 * 256 + (size_t)pieces * words * 4;
}

HoughPlan plan_with_pairs(int w, int h, int n_theta, int pairs) {
    HoughPlan hp;
    hp.D = (int)rho_max_of(w, h);
    hp.n_rho = 2 * hp.D + 1;
    const int n_pairs = n_theta / 2;
    const int pmax = hough_max_pairs(hp.n_rho);
    hp.pairs = pairs < 1 ? 1 : (pairs > pmax ? pmax : pairs);
    if (hp.pairs > n_pairs) hp.pairs = n_pairs;
    hp.n_tiles = (n_pairs + hp.pairs - 1) / hp.pairs;
    hp.pairs = (n_pairs + hp.n_tiles - 1) / hp.n_tiles;   // pairs are split evenly over the tiles
    return hp;
}

HoughPlan plan_hough(int w, int h, int n_theta) {
    HoughPlan hp;
    hp.D = (int)rho_max_of(w, h);
    hp.n_rho = 2 * hp.D + 1;
    const int n_pairs = n_theta / 2;
    const int pmax = hough_max_pairs(hp.n_rho);
    // Prefer a compiled tile size that divides the pairs exactly (every tile
    // runs the predicate-free loop) unless it is much smaller than what fits.
    int best_div = 0;
#define LD_DIV(P) if (P <= pmax && n_pairs % P == 0 && P > best_div) best_div = P;
    LD_HOUGH_PAIR_SIZES(LD_DIV)
#undef LD_DIV
    if (best_div > 0 && 10 * best_div >= 7 * (pmax < n_pairs ? pmax : n_pairs)) {
        hp.pairs = best_div;
        hp.n_tiles = n_pairs / best_div;
        return hp;
    }
    hp.n_tiles = (n_pairs + pmax - 1) / pmax;
    hp.pairs = (n_pairs + hp.n_tiles - 1) / hp.n_tiles;
    return hp;
}

// Rows of the interleaved-column accumulator for w x h frames (window_rows,
// cached in the context).
int interleaved_rows(const ld_ctx *ctx, int w, int h, int n_theta) {
    const auto key = std::make_tuple(w, h, n_theta);
    auto it = ctx->col_rows.find(key);
    if (it != ctx->col_rows.end()) return it->second;
    const int r = window_rows(w, h, n_theta, make_trig(n_theta));
    ctx->col_rows[key] = r;
    return r;
}

// The interleaved-column plan (tiles of at most `width` pairs, split evenly:
// 16 slots, or 8 when the frame's window rows do not fit 16 columns), or a
// plan with cols == false if even 8 columns do not fit.
HoughPlan plan_cols(const ld_ctx *ctx, int w, int h, int n_theta) {
    HoughPlan hp;
    hp.D = (int)rho_max_of(w, h);
    hp.n_rho = 2 * hp.D + 1;
    const int n_pairs = n_theta / 2;
    hp.rows = interleaved_rows(ctx, w, h, n_theta);
    hp.width = hp.rows <= hough_cols_max_rows(kHoughColPairs) ? kHoughColPairs : 8;
    hp.n_tiles = (n_pairs + hp.width - 1) / hp.width;
    hp.pairs = (n_pairs + hp.n_tiles - 1) / hp.n_tiles;
    hp.cols = hp.rows <= hough_cols_max_rows(hp.width);
    return hp;
}

// An interleaved-kernel plan with `width` pairs per tile (its rows fit).
HoughPlan plan_cols_width(HoughPlan hp, int n_theta, int width) {
    const int n_pairs = n_theta / 2;
    hp.width = width;
    hp.n_tiles = (n_pairs + width - 1) / width;
    hp.pairs = (n_pairs + hp.n_tiles - 1) / hp.n_tiles;
    return hp;
}

// The voting plan of w x h frames.  allow_cols: the launch may use the
// interleaved-column kernel (full vote in candidate mode with min_votes >= 1,
// where cells outside a theta's window, which it does not hold, cannot be
// candidates).  Forced (autotuner), else tuned, else the interleaved kernel
// when it fits and its tiles are at least 3/4 full on average (a lane per
// pair: emptier tiles leave lanes idle), else the packed-pair plan.
HoughPlan plan_for(const ld_ctx *ctx, int w, int h, int n_theta, bool allow_cols) {
    int pairs = ctx->force_pairs;
    if (pairs == 0) {
        auto it = ctx->tuned.find(std::make_tuple(w, h, n_theta));
        if (it != ctx->tuned.end()) pairs = it->second.first;
    }
    if (pairs > 0) return plan_with_pairs(w, h, n_theta, pairs);
    if (allow_cols) {
        const HoughPlan hc = plan_cols(ctx, w, h, n_theta);
        // tiles at least 3/4 full on average (n_pairs / n_tiles >= 0.75 width)
        if (hc.cols && (pairs == -1 || 2 * n_theta >= 3 * hc.width * hc.n_tiles)) return hc;
    }
    return plan_hough(w, h, n_theta);
}

// Sobel 8-row groups per warp task for a launch group: forced, else the tuned
// value of the group's largest frame size, else the default heuristic.
int rows_for(const ld_ctx *ctx, const ld_frame *fr, int g0, int g1, int n_theta) {
    if (ctx->force_rows > 0) return ctx->force_rows;
    int64_t best_px = -1;
    int rows = 0;
    for (int i = g0; i < g1; ++i) {
        auto it = ctx->tuned.find(std::make_tuple(fr[i].w, fr[i].h, n_theta));
        const int64_t px = (int64_t)fr[i].w * fr[i].h;
        if (it != ctx->tuned.end() && px > best_px) {
            best_px = px;
            rows = it->second.second;
        }
    }
    if (rows > 0) return rows;
    int64_t ctas_g1 = 0;
    for (int i = g0; i < g1; ++i) ctas_g1 += sobel_frame_ctas(fr[i].w, fr[i].h, 1);
    return pick_sobel_groups(ctas_g1, ctx->num_sms);
}

// Hough-lines request riding on a detection call (ld_detect_lines_batch).
struct LinesReq {
    ld_lines_params lp;
    ld_segment *segs;   // [n][top_k][max_segments]
    int32_t *n_segs;    // [n][top_k]
    int32_t *support;   // nullable [n][top_k]
};

ld_status detect_impl(ld_ctx *ctx, const ld_frame *h_frames, int32_t n, const ld_params &p, ld_peak *d_peaks,
                      int32_t *d_n_peaks, int32_t *d_status, cudaStream_t s, const LinesReq *lines = nullptr,
                      const ld_canny_params *canny = nullptr);

ld_canny_params canny_defaults() {
    ld_canny_params q;
    q.t_low = 100;
    q.t_high = 200;
    q.reserved0 = q.reserved1 = 0;
    return q;
}

ld_status check_canny(const ld_canny_params &q) {
    if (q.t_low < 1 || q.t_low > 2040 || q.t_high < q.t_low || q.t_high > 2040)
        return fail(LD_ERR_INVALID, "Canny thresholds: need 1 <= t_low <= t_high <= 2040");
    if (q.reserved0 || q.reserved1) return fail(LD_ERR_INVALID, "ld_canny_params.reserved must be 0");
    return LD_OK;
}

// Canny scratch of px pixels: class map, strong marks, then the forest (4-byte aligned).
size_t canny_scratch_bytes(int64_t px) { return ((size_t)px * 2 + 15) / 16 * 16 + (size_t)px * 4; }
void canny_scratch(void *base, int64_t px_total, int64_t px_off, CannyFrame &F) {
    uint8_t *b = (uint8_t *)base;
    F.cls = b + px_off;
    F.strong = b + px_total + px_off;
    F.parent = (int32_t *)(b + ((size_t)px_total * 2 + 15) / 16 * 16) + px_off;
}

ld_lines_params lines_defaults() {
    ld_lines_params q;
    q.fill_gap = 20;
    q.min_length = 40;
    q.max_segments = 16;
    q.reserved = 0;
    return q;
}

ld_status check_lines(const ld_lines_params &q) {
    if (q.fill_gap < 0 || q.fill_gap > 65535 || q.min_length < 0 || q.min_length > 65535)
        return fail(LD_ERR_INVALID, "fill_gap and min_length must be in [0, 65535]");
    if (q.max_segments < 1 || q.max_segments > 4096)
        return fail(LD_ERR_INVALID, "max_segments must be in [1, 4096], got %d", q.max_segments);
    if (q.reserved != 0) return fail(LD_ERR_INVALID, "ld_lines_params.reserved must be 0");
    return LD_OK;
}

}  // namespace

// The parameters of a peak search on an n_theta-row accumulator, validated
// as ld_hough_peaks validates them (NULL: the defaults).
ld_status ld::peak_params(const ld_params *pp, int32_t n_theta, ld_params *out) {
    ld_params p = pp ? *pp : defaults();
    p.n_theta = (n_theta >= 2 && !(n_theta & 1)) ? n_theta : 2;   // n_theta of the table is unused here
    const ld_status st = check_params(&p);
    if (st == LD_OK) *out = p;
    return st;
}

extern "C" {

const char *ld_last_error(void) { return g_err.c_str(); }

ld_status ld_params_default(ld_params *p) {
    if (!p) return fail(LD_ERR_INVALID, "ld_params_default: NULL");
    *p = defaults();
    return LD_OK;
}

ld_status ld_ctx_create(ld_ctx **out, int device) {
    if (!out) return fail(LD_ERR_INVALID, "ld_ctx_create: NULL out");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(LD_ERR_INVALID, "device %d out of range (%d devices)", device, n);
    ld_ctx *c = new ld_ctx();
    c->device = device;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
        c->num_sms = sms;
    *out = c;
    return LD_OK;
}

ld_status ld_ctx_set_wait_limit(ld_ctx *ctx, int64_t polls) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_ctx_set_wait_limit: NULL ctx");
    if (polls > (int64_t)kSpinLimit)
        return fail(LD_ERR_INVALID, "ld_ctx_set_wait_limit: polls must be <= %u", kSpinLimit);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->wait_polls = polls < 0 ? kSpinLimit : (uint32_t)polls;
    return LD_OK;
}

ld_status ld_ctx_destroy(ld_ctx *ctx) {
    if (!ctx) return LD_OK;
    {
        DeviceGuard g(ctx->device);
        for (auto &kv : ctx->trig) cudaFree(kv.second);
        for (auto &e : ctx->ev) cudaEventDestroy(e);
        ctx->edges.release();
        ctx->small.release();
        ctx->cand.release();
        ctx->prop.release();
        ctx->part.release();
        ctx->canny.release();
        ctx->fused.release();
        if (ctx->hcopy) cudaStreamSynchronize(ctx->hcopy);   // uploads still in flight
        for (int b = 0; b < 2; ++b) {
            if (ctx->hev_free[b]) cudaEventSynchronize(ctx->hev_free[b]);
            ctx->stage[b].release();
            if (ctx->hev_copied[b]) cudaEventDestroy(ctx->hev_copied[b]);
            if (ctx->hev_free[b]) cudaEventDestroy(ctx->hev_free[b]);
        }
        if (ctx->hcopy) cudaStreamDestroy(ctx->hcopy);
    }
    delete ctx;
    return LD_OK;
}

ld_status ld_query_sizes(int32_t w, int32_t h, const ld_params *pp, size_t *acc_elems, size_t *edge_elems,
                         int32_t *D) {
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    std::vector<int32_t> t = make_trig(p.n_theta);
    st = check_size(w, h, p, &t);
    if (st != LD_OK) return st;
    const int64_t d = rho_max_of(w, h);
    if (acc_elems) *acc_elems = (size_t)p.n_theta * (size_t)(2 * d + 1);
    if (edge_elems) *edge_elems = (size_t)w * (size_t)h;
    if (D) *D = (int32_t)d;
    return LD_OK;
}

ld_status ld_ctx_reserve(ld_ctx *ctx, int64_t max_pixels, int32_t max_frames, int64_t max_acc_cells,
                         const ld_params *pp) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_ctx_reserve: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    if (max_pixels < 0 || max_frames < 0 || max_acc_cells < 0)
        return fail(LD_ERR_INVALID, "ld_ctx_reserve: negative size");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    const int32_t *dt;
    st = get_trig(ctx, p.n_theta, &dt, nullptr);
    if (st != LD_OK) return st;
    const int64_t groups_frames = max_frames < kMaxLaunchFrames ? max_frames : kMaxLaunchFrames;
    if (!ctx->edges.ensure((size_t)(max_pixels + 4 * (int64_t)groups_frames) * 4))
        return fail(LD_ERR_NOMEM, "scratch edges: %lld pixels", (long long)max_pixels);
    if (!ctx->small.ensure(kSmallInts * 4)) return fail(LD_ERR_NOMEM, "scratch counts");
    const int64_t per_frame = (int64_t)(p.n_theta / 2) * cand_m(p);
    const int64_t acc_chunks = (max_acc_cells + kSelectChunk - 1) / kSelectChunk;
    int64_t nc = groups_frames * per_frame;
    if (acc_chunks * cand_m(p) > nc) nc = acc_chunks * cand_m(p);
    if (!ctx->cand.ensure((size_t)nc * 8)) return fail(LD_ERR_NOMEM, "scratch candidates");
    if (max_frames > 0 && !ctx->part.ensure(split_scratch_bytes(ctx->num_sms, hough_cols_max_words())))
        return fail(LD_ERR_NOMEM, "scratch partial accumulators");
    return LD_OK;
}

constexpr int kMaxTimedCalls = 1024;

ld_status ld_ctx_enable_timing(ld_ctx *ctx, int enable) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_ctx_enable_timing: NULL ctx");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->timing = enable != 0;
    return LD_OK;
}

}  // extern "C"

namespace {
// Sum and reset the stage times of the calls timed so far (caller holds ctx->mu).
ld_status stage_sums(ld_ctx *ctx, float ms[3]) {
    ms[0] = ms[1] = 0.f;
    ms[2] = (float)ctx->timed_calls;
    for (int c = 0; c < ctx->timed_calls; ++c) {
        cudaEvent_t *e = &ctx->ev[3 * c];
        cudaError_t r = cudaEventSynchronize(e[2]);
        if (r != cudaSuccess) return cuda_fail(r, "cudaEventSynchronize");
        for (int i = 0; i < 2; ++i) {
            float t = 0.f;
            r = cudaEventElapsedTime(&t, e[i], e[i + 1]);
            if (r != cudaSuccess) return cuda_fail(r, "cudaEventElapsedTime");
            ms[i] += t;
        }
    }
    ctx->timed_calls = 0;
    return LD_OK;
}
}  // namespace

extern "C" {

ld_status ld_ctx_stage_ms(ld_ctx *ctx, float ms[3]) {
    if (!ctx || !ms) return fail(LD_ERR_INVALID, "ld_ctx_stage_ms: NULL argument");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    return stage_sums(ctx, ms);
}

ld_status ld_sobel_binarize(ld_ctx *ctx, const uint8_t *d_img, int32_t w, int32_t h, int32_t pitch,
                            const ld_params *pp, uint8_t *d_bin, uint32_t *d_edges, int32_t *d_edge_count,
                            void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_sobel_binarize: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    st = check_size(w, h, p, nullptr);
    if (st != LD_OK) return st;
    if (!d_img || !d_edges || !d_edge_count) return fail(LD_ERR_INVALID, "ld_sobel_binarize: NULL buffer");
    if (pitch < w || (pitch & 15) || !aligned16(d_img) || (d_bin && !aligned16(d_bin)))
        return fail(LD_ERR_INVALID, "pitch must be >= w and a multiple of 16, buffers 16-byte aligned");
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_edge_count, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(count)");
    SobelLaunch L;
    std::memset(&L, 0, sizeof L);
    L.n = 1;
    L.threshold = p.threshold;
    L.border = p.border;
    L.groups = pick_sobel_groups(sobel_frame_ctas(w, h, 1), ctx->num_sms);
    SobelFrame &F = L.f[0];
    F.img = d_img;
    F.bin = d_bin;
    F.edges = d_edges;
    F.count = d_edge_count;
    F.cap = p.edge_capacity > 0 ? p.edge_capacity : (int64_t)w * h;
    F.w = w;
    F.h = h;
    F.pitch = pitch;
    F.tile_begin = 0;
    F.tiles_x = sobel_strips(w);
    e = launch_sobel(L, sobel_frame_ctas(w, h, L.groups), s);
    if (e != cudaSuccess) return cuda_fail(e, "sobel launch");
    return LD_OK;
}

ld_status ld_sobel_hough_fused(ld_ctx *ctx, const uint8_t *d_img, int32_t w, int32_t h, int32_t pitch,
                               const ld_params *pp, int32_t *d_acc, void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_sobel_hough_fused: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    if (p.n_theta > kFusedMaxTheta) return fail(LD_ERR_INVALID, "fused path: n_theta must be <= %d", kFusedMaxTheta);
    if (!d_img || !d_acc) return fail(LD_ERR_INVALID, "ld_sobel_hough_fused: NULL buffer");
    if (pitch < w || (pitch & 15) || !aligned16(d_img))
        return fail(LD_ERR_INVALID, "pitch must be >= w and a multiple of 16, the image 16-byte aligned");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    const int32_t *dt;
    const std::vector<int32_t> *ht;
    st = get_trig(ctx, p.n_theta, &dt, &ht);
    if (st != LD_OK) return st;
    st = check_size(w, h, p, ht);
    if (st != LD_OK) return st;
    const int D = (int)rho_max_of(w, h), n_rho = 2 * D + 1;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_acc, 0, (size_t)p.n_theta * n_rho * 4, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(acc)");
    FusedLaunch FL;
    std::memset(&FL, 0, sizeof FL);
    FL.n = 1;
    FL.n_theta = p.n_theta;
    FL.threshold = p.threshold;
    FL.border = p.border;
    FL.trig = dt;
    FusedFrame &FF = FL.f[0];
    FF.img = d_img;
    FF.acc = d_acc;
    FF.w = w;
    FF.h = h;
    FF.pitch = pitch;
    FF.D = D;
    FF.n_rho = n_rho;
    FF.tiles_x = (w + kFusedBlock - 1) / kFusedBlock;
    e = launch_fused_vote(FL, fused_blocks(w, h), s);
    if (e != cudaSuccess) return cuda_fail(e, "fused launch");
    return LD_OK;
}

// The stage events of a timed call's first launch group (3 per call), or
// nullptr when timing is off, g0 is a later group or the record is full.
static ld_status stage_events(ld_ctx *ctx, int g0, cudaEvent_t **tev) {
    *tev = nullptr;
    if (!ctx->timing || g0 != 0 || ctx->timed_calls >= kMaxTimedCalls) return LD_OK;
    const size_t need = 3 * (size_t)(ctx->timed_calls + 1);
    while (ctx->ev.size() < need) {
        cudaEvent_t ne;
        cudaError_t r = cudaEventCreate(&ne);
        if (r != cudaSuccess) return cuda_fail(r, "cudaEventCreate");
        ctx->ev.push_back(ne);
    }
    *tev = &ctx->ev[3 * ctx->timed_calls];
    ++ctx->timed_calls;
    return LD_OK;
}

ld_status ld_detect_fused_batch(ld_ctx *ctx, const ld_frame *h_frames, int32_t n, const ld_params *pp,
                                ld_peak *d_peaks, int32_t *d_n_peaks, int32_t *d_status, void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_detect_fused_batch: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    if (p.n_theta > kFusedMaxTheta) return fail(LD_ERR_INVALID, "fused path: n_theta must be <= %d", kFusedMaxTheta);
    if (!h_frames || n < 1 || !d_peaks || !d_n_peaks || !d_status)
        return fail(LD_ERR_INVALID, "ld_detect_fused_batch: bad arguments");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    const int32_t *dt;
    const std::vector<int32_t> *ht;
    st = get_trig(ctx, p.n_theta, &dt, &ht);
    if (st != LD_OK) return st;
    for (int i = 0; i < n; ++i) {
        const ld_frame &f = h_frames[i];
        st = check_size(f.w, f.h, p, ht);
        if (st != LD_OK) return fail(st, "frame %d: %s", i, g_err.c_str());
        if (!f.img || f.pitch < f.w || (f.pitch & 15) || !aligned16(f.img) || f.reserved != 0)
            return fail(LD_ERR_INVALID, "frame %d: NULL image, bad pitch or alignment", i);
    }
    const int M = cand_m(p);
    cudaStream_t s = (cudaStream_t)stream;
    for (int g0 = 0; g0 < n; g0 += kMaxLaunchFrames) {
        const int g1 = std::min(n, g0 + kMaxLaunchFrames), gn = g1 - g0;
        // per-frame accumulators, then the candidates of their chunks
        std::vector<int64_t> aoff(gn), coff(gn);
        int64_t acells = 0, ccount = 0;
        int chunks = 0;
        for (int k = 0; k < gn; ++k) {
            const ld_frame &f = h_frames[g0 + k];
            const int64_t cells = (int64_t)p.n_theta * (2 * rho_max_of(f.w, f.h) + 1);
            aoff[k] = acells;
            acells += (cells + 3) / 4 * 4;
            coff[k] = ccount;
            const int nc = (int)((cells + kSelectChunk - 1) / kSelectChunk);
            ccount += (int64_t)nc * M;
            chunks += nc;
        }
        if (!ctx->fused.ensure((size_t)acells * 4)) return fail(LD_ERR_NOMEM, "scratch accumulators");
        if (!ctx->cand.ensure((size_t)ccount * 8)) return fail(LD_ERR_NOMEM, "scratch candidates");
        int32_t *acc = (int32_t *)ctx->fused.p;
        uint64_t *cand = (uint64_t *)ctx->cand.p;
        cudaEvent_t *tev = nullptr;
        st = stage_events(ctx, g0, &tev);
        if (st != LD_OK) return st;
        if (tev) cudaEventRecord(tev[0], s);
        cudaError_t e = cudaMemsetAsync(acc, 0, (size_t)acells * 4, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(acc)");
        FusedLaunch FL;
        std::memset(&FL, 0, sizeof FL);
        FL.n = gn;
        FL.n_theta = p.n_theta;
        FL.threshold = p.threshold;
        FL.border = p.border;
        FL.trig = dt;
        SelectLaunch SL;
        std::memset(&SL, 0, sizeof SL);
        SL.n = gn;
        SL.cand_m = M;
        SL.min_votes = p.min_votes;
        MergeLaunch ML;
        std::memset(&ML, 0, sizeof ML);
        ML.n = gn;
        ML.top_k = p.top_k;
        ML.nms_theta = p.nms_theta;
        ML.nms_rho = p.nms_rho;
        int blocks = 0, chunk_begin = 0;
        for (int k = 0; k < gn; ++k) {
            const ld_frame &f = h_frames[g0 + k];
            const int D = (int)rho_max_of(f.w, f.h), n_rho = 2 * D + 1;
            const int64_t cells = (int64_t)p.n_theta * n_rho;
            const int nc = (int)((cells + kSelectChunk - 1) / kSelectChunk);
            FusedFrame &FF = FL.f[k];
            FF.img = f.img;
            FF.acc = acc + aoff[k];
            FF.status_init = d_status + g0 + k;
            FF.npeaks_init = d_n_peaks + g0 + k;
            FF.w = f.w;
            FF.h = f.h;
            FF.pitch = f.pitch;
            FF.D = D;
            FF.n_rho = n_rho;
            FF.tile_begin = blocks;
            FF.tiles_x = (f.w + kFusedBlock - 1) / kFusedBlock;
            blocks += fused_blocks(f.w, f.h);
            SelectJob &J = SL.j[k];
            J.acc = FF.acc;
            J.cand = cand + coff[k];
            J.cells = cells;
            J.n_rho = n_rho;
            J.n_chunks = nc;
            J.chunk_begin = chunk_begin;
            chunk_begin += nc;
            MergeJob &MJ = ML.j[k];
            MJ.cand = cand + coff[k];
            MJ.n_cand = (int64_t)nc * M;
            MJ.peaks = d_peaks + (size_t)(g0 + k) * p.top_k;
            MJ.n_peaks = d_n_peaks + g0 + k;
            MJ.status = d_status + g0 + k;
        }
        e = launch_fused_vote(FL, blocks, s);
        if (e != cudaSuccess) return cuda_fail(e, "fused launch");
        if (tev) cudaEventRecord(tev[1], s);
        e = launch_select(SL, chunks, s);
        if (e != cudaSuccess) return cuda_fail(e, "select launch");
        e = launch_merge(ML, s);
        if (e != cudaSuccess) return cuda_fail(e, "merge launch");
        if (tev) cudaEventRecord(tev[2], s);
    }
    return LD_OK;
}

ld_status ld_canny_params_default(ld_canny_params *cp) {
    if (!cp) return fail(LD_ERR_INVALID, "ld_canny_params_default: NULL");
    *cp = canny_defaults();
    return LD_OK;
}

ld_status ld_canny(ld_ctx *ctx, const uint8_t *d_img, int32_t w, int32_t h, int32_t pitch, const ld_params *pp,
                   const ld_canny_params *cpp, uint8_t *d_bin, uint32_t *d_edges, int32_t *d_edge_count,
                   void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_canny: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    const ld_canny_params cp = cpp ? *cpp : canny_defaults();
    st = check_canny(cp);
    if (st != LD_OK) return st;
    st = check_size(w, h, p, nullptr);
    if (st != LD_OK) return st;
    if (!d_img || !d_edges || !d_edge_count) return fail(LD_ERR_INVALID, "ld_canny: NULL buffer");
    if (pitch < w || (pitch & 15) || !aligned16(d_img) || (d_bin && !aligned16(d_bin)))
        return fail(LD_ERR_INVALID, "pitch must be >= w and a multiple of 16, buffers 16-byte aligned");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    const int64_t px = (int64_t)w * h;
    if (!ctx->canny.ensure(canny_scratch_bytes(px))) return fail(LD_ERR_NOMEM, "scratch Canny");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_edge_count, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(count)");
    CannyLaunch CL;
    std::memset(&CL, 0, sizeof CL);
    CL.n = 1;
    CL.t_low = cp.t_low;
    CL.t_high = cp.t_high;
    CL.border = p.border;
    CL.total_px = px;
    CannyFrame &CF = CL.f[0];
    CF.img = d_img;
    CF.bin = d_bin;
    CF.edges = d_edges;
    CF.count = d_edge_count;
    canny_scratch(ctx->canny.p, px, 0, CF);
    CF.cap = p.edge_capacity > 0 ? p.edge_capacity : px;
    CF.w = w;
    CF.h = h;
    CF.pitch = pitch;
    e = launch_canny(CL, canny_tiles(w, h), s);
    if (e != cudaSuccess) return cuda_fail(e, "canny launch");
    return LD_OK;
}

ld_status ld_detect_canny_batch(ld_ctx *ctx, const ld_frame *h_frames, int32_t n, const ld_params *pp,
                                const ld_canny_params *cpp, ld_peak *d_peaks, int32_t *d_n_peaks, int32_t *d_status,
                                void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_detect_canny_batch: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    const ld_canny_params cp = cpp ? *cpp : canny_defaults();
    st = check_canny(cp);
    if (st != LD_OK) return st;
    if (!h_frames || n < 1 || !d_peaks || !d_n_peaks || !d_status)
        return fail(LD_ERR_INVALID, "ld_detect_canny_batch: bad arguments");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    return detect_impl(ctx, h_frames, n, p, d_peaks, d_n_peaks, d_status, (cudaStream_t)stream, nullptr, &cp);
}

ld_status ld_hough_vote(ld_ctx *ctx, const uint32_t *d_edges, const int32_t *d_edge_count, int32_t w,
                        int32_t h, const ld_params *pp, int32_t *d_acc, void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_hough_vote: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    if (!d_edges || !d_edge_count || !d_acc) return fail(LD_ERR_INVALID, "ld_hough_vote: NULL buffer");
    if (!aligned16(d_edges)) return fail(LD_ERR_INVALID, "d_edges must be 16-byte aligned");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    const int32_t *dt;
    const std::vector<int32_t> *ht;
    st = get_trig(ctx, p.n_theta, &dt, &ht);
    if (st != LD_OK) return st;
    st = check_size(w, h, p, ht);
    if (st != LD_OK) return st;
    const HoughPlan hp = plan_hough(w, h, p.n_theta);
    int ns = (ctx->num_sms + hp.n_tiles / 2) / hp.n_tiles;
    if (ns < 1) ns = 1;
    if (!ctx->small.ensure(kSmallInts * 4)) return fail(LD_ERR_NOMEM, "scratch counts");
    const Small sm = small_of(ctx->small.p);
    cudaStream_t s = (cudaStream_t)stream;
    if (ns > 1) {
        cudaError_t e = cudaMemsetAsync(d_acc, 0, (size_t)p.n_theta * hp.n_rho * sizeof(int32_t), s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(acc)");
    }
    cudaError_t e = cudaMemsetAsync(sm.queue, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(queue)");
    HoughLaunch L;
    std::memset(&L, 0, sizeof L);
    L.n = 1;
    L.n_theta = p.n_theta;
    L.mode = kHoughFullAcc;
    L.wait_polls = ctx->wait_polls;
    L.trig = dt;
    L.queue = sm.queue;
    L.total_units = hp.n_tiles * ns;
    HoughFrame &F = L.f[0];
    F.edges = d_edges;
    F.count = d_edge_count;
    F.cap = p.edge_capacity > 0 ? p.edge_capacity : (int64_t)w * h;
    F.acc = d_acc;
    F.w = w;
    F.h = h;
    F.D = hp.D;
    F.n_rho = hp.n_rho;
    F.unit_begin = 0;
    F.n_splits = ns;
    F.pairs_per_tile = hp.pairs;
    F.n_tiles = hp.n_tiles;
    const int n_ctas = L.total_units < ctx->num_sms ? L.total_units : ctx->num_sms;
    e = launch_hough(L, n_ctas, hp.pairs, (int64_t)hp.pairs * hp.n_rho, s);
    if (e != cudaSuccess) return cuda_fail(e, "hough launch");
    return LD_OK;
}

ld_status ld_hough_peaks(ld_ctx *ctx, const int32_t *d_acc, int32_t n_theta, int32_t n_rho,
                         const ld_params *pp, ld_peak *d_peaks, int32_t *d_n_peaks, void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_hough_peaks: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    p.n_theta = (n_theta >= 2 && !(n_theta & 1)) ? n_theta : 2;   // n_theta of the table is unused here
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    if (n_theta < 1 || n_theta > kMaxTheta || n_rho < 1 || n_rho > 65535)
        return fail(LD_ERR_INVALID, "accumulator %d x %d: need 1 <= n_theta <= %d, 1 <= n_rho <= 65535",
                    n_theta, n_rho, kMaxTheta);
    if (!d_acc || !d_peaks || !d_n_peaks) return fail(LD_ERR_INVALID, "ld_hough_peaks: NULL buffer");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    const int M = cand_m(p);
    const int64_t cells = (int64_t)n_theta * n_rho;
    const int n_chunks = (int)((cells + kSelectChunk - 1) / kSelectChunk);
    if (!ctx->cand.ensure((size_t)n_chunks * M * 8)) return fail(LD_ERR_NOMEM, "scratch candidates");
    uint64_t *cand = (uint64_t *)ctx->cand.p;
    cudaStream_t s = (cudaStream_t)stream;
    SelectLaunch SL;
    std::memset(&SL, 0, sizeof SL);
    SL.n = 1;
    SL.cand_m = M;
    SL.min_votes = p.min_votes;
    SL.j[0].acc = d_acc;
    SL.j[0].cand = cand;
    SL.j[0].cells = cells;
    SL.j[0].n_rho = n_rho;
    SL.j[0].n_chunks = n_chunks;
    SL.j[0].chunk_begin = 0;
    cudaError_t e = launch_select(SL, n_chunks, s);
    if (e != cudaSuccess) return cuda_fail(e, "select launch");
    MergeLaunch ML;
    std::memset(&ML, 0, sizeof ML);
    ML.n = 1;
    ML.top_k = p.top_k;
    ML.nms_theta = p.nms_theta;
    ML.nms_rho = p.nms_rho;
    ML.j[0].cand = cand;
    ML.j[0].n_cand = (int64_t)n_chunks * M;
    ML.j[0].peaks = d_peaks;
    ML.j[0].n_peaks = d_n_peaks;
    e = launch_merge(ML, s);
    if (e != cudaSuccess) return cuda_fail(e, "merge launch");
    return LD_OK;
}

ld_status ld_lines_params_default(ld_lines_params *lp) {
    if (!lp) return fail(LD_ERR_INVALID, "ld_lines_params_default: NULL");
    *lp = lines_defaults();
    return LD_OK;
}

ld_status ld_hough_lines(ld_ctx *ctx, const uint32_t *d_edges, const int32_t *d_edge_count, int32_t w, int32_t h,
                         const ld_params *pp, const ld_peak *d_peaks, const int32_t *d_n_peaks,
                         const ld_lines_params *lpp, ld_segment *d_segments, int32_t *d_n_segments,
                         int32_t *d_support, void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_hough_lines: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    const ld_lines_params lp = lpp ? *lpp : lines_defaults();
    st = check_lines(lp);
    if (st != LD_OK) return st;
    if (!d_edges || !aligned16(d_edges) || !d_edge_count || !d_peaks || !d_n_peaks || !d_segments || !d_n_segments)
        return fail(LD_ERR_INVALID, "ld_hough_lines: NULL or misaligned buffer");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    const int32_t *dt;
    const std::vector<int32_t> *ht;
    st = get_trig(ctx, p.n_theta, &dt, &ht);
    if (st != LD_OK) return st;
    st = check_size(w, h, p, ht);
    if (st != LD_OK) return st;
    if (w > kLinesMaxSide || h > kLinesMaxSide)
        return fail(LD_ERR_INVALID, "ld_hough_lines: max(w, h) must be <= %d", kLinesMaxSide);
    LinesLaunch LL;
    std::memset(&LL, 0, sizeof LL);
    LL.n = 1;
    LL.top_k = p.top_k;
    LL.n_theta = p.n_theta;
    LL.fill_gap = lp.fill_gap;
    LL.min_length = lp.min_length;
    LL.max_segments = lp.max_segments;
    LL.trig = dt;
    LinesFrame &LF = LL.f[0];
    LF.edges = d_edges;
    LF.count = d_edge_count;
    LF.cap = p.edge_capacity > 0 ? p.edge_capacity : (int64_t)w * h;
    LF.peaks = d_peaks;
    LF.n_peaks = d_n_peaks;
    LF.segs = d_segments;
    LF.n_segs = d_n_segments;
    LF.support = d_support;
    LF.w = w;
    LF.h = h;
    LF.D = (int32_t)rho_max_of(w, h);
    const cudaError_t e = launch_lines(LL, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "lines launch");
    return LD_OK;
}

ld_status ld_detect_lines_batch(ld_ctx *ctx, const ld_frame *h_frames, int32_t n, const ld_params *pp,
                                const ld_lines_params *lpp, ld_peak *d_peaks, int32_t *d_n_peaks, int32_t *d_status,
                                ld_segment *d_segments, int32_t *d_n_segments, int32_t *d_support, void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_detect_lines_batch: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    LinesReq req;
    req.lp = lpp ? *lpp : lines_defaults();
    st = check_lines(req.lp);
    if (st != LD_OK) return st;
    if (!h_frames || n < 1 || !d_peaks || !d_n_peaks || !d_status || !d_segments || !d_n_segments)
        return fail(LD_ERR_INVALID, "ld_detect_lines_batch: bad arguments");
    req.segs = d_segments;
    req.n_segs = d_n_segments;
    req.support = d_support;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    return detect_impl(ctx, h_frames, n, p, d_peaks, d_n_peaks, d_status, (cudaStream_t)stream, &req);
}

ld_status ld_detect_batch(ld_ctx *ctx, const ld_frame *h_frames, int32_t n, const ld_params *pp,
                          ld_peak *d_peaks, int32_t *d_n_peaks, int32_t *d_status, void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_detect_batch: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    if (!h_frames || n < 1) return fail(LD_ERR_INVALID, "ld_detect_batch: need n >= 1 frames");
    if (!d_peaks || !d_n_peaks || !d_status) return fail(LD_ERR_INVALID, "ld_detect_batch: NULL output");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    return detect_impl(ctx, h_frames, n, p, d_peaks, d_n_peaks, d_status, (cudaStream_t)stream);
}

ld_status ld_detect_batch_host(ld_ctx *ctx, const ld_frame *h_frames, int32_t n, const ld_params *pp,
                               ld_peak *h_peaks, int32_t *h_n_peaks, int32_t *h_status, void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_detect_batch_host: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    if (!h_frames || n < 1) return fail(LD_ERR_INVALID, "ld_detect_batch_host: need n >= 1 frames");
    if (!h_peaks || !h_n_peaks || !h_status) return fail(LD_ERR_INVALID, "ld_detect_batch_host: NULL output");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    const int32_t *dt;
    const std::vector<int32_t> *ht;
    st = get_trig(ctx, p.n_theta, &dt, &ht);
    if (st != LD_OK) return st;
    // the staging area: frame i at off[i] (16-byte aligned), then the outputs
    std::vector<size_t> off(n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        const ld_frame &f = h_frames[i];
        st = check_size(f.w, f.h, p, ht);
        if (st != LD_OK) return fail(st, "frame %d: %s", i, g_err.c_str());
        if (!f.img || f.pitch < f.w || (f.pitch & 15) || f.reserved != 0)
            return fail(LD_ERR_INVALID, "frame %d: NULL image or bad pitch", i);
        off[i] = total;
        total += ((size_t)f.pitch * f.h + 15) / 16 * 16;
    }
    const size_t pk_bytes = (size_t)n * p.top_k * sizeof(ld_peak);
    const size_t out_off = total, np_off = out_off + (pk_bytes + 15) / 16 * 16, st_off = np_off + (size_t)n * 4;
    const size_t need = st_off + (size_t)n * 4;
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx->hcopy) {
        cudaError_t e = cudaStreamCreateWithFlags(&ctx->hcopy, cudaStreamNonBlocking);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaEventCreateWithFlags(&ctx->hev_copied[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->hev_free[b], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) return cuda_fail(e, "copy stream / events");
    }
    const int b = (int)(ctx->host_calls & 1u);
    DevBuf &stg = ctx->stage[b];
    if (need > stg.bytes) {   // grow: the area's previous call must be done with it
        cudaError_t e = ctx->hev_used[b] ? cudaEventSynchronize(ctx->hev_free[b]) : cudaSuccess;
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->hcopy);   // uploads of a call that failed later
        if (e != cudaSuccess) return cuda_fail(e, "staging area in use");
        if (!stg.ensure(need)) return fail(LD_ERR_NOMEM, "staging area of %zu bytes", need);
    }
    uint8_t *base = (uint8_t *)stg.p;
    // frames: one copy per run of frames that are adjacent in host memory, on
    // the copy stream, after the area's previous outputs were read back
    cudaError_t e = cudaSuccess;
    if (ctx->hev_used[b]) e = cudaStreamWaitEvent(ctx->hcopy, ctx->hev_free[b], 0);
    for (int i = 0; i < n && e == cudaSuccess;) {
        const uint8_t *src = h_frames[i].img;
        size_t bytes = (size_t)h_frames[i].pitch * h_frames[i].h;
        int j = i + 1;
        while (j < n && h_frames[j].img == src + bytes && off[j] == off[i] + bytes) {
            bytes += (size_t)h_frames[j].pitch * h_frames[j].h;
            ++j;
        }
        e = cudaMemcpyAsync(base + off[i], src, bytes, cudaMemcpyHostToDevice, ctx->hcopy);
        i = j;
    }
    if (e == cudaSuccess) e = cudaEventRecord(ctx->hev_copied[b], ctx->hcopy);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->hev_copied[b], 0);
    if (e != cudaSuccess) return cuda_fail(e, "frame upload");
    std::vector<ld_frame> dev(h_frames, h_frames + n);
    for (int i = 0; i < n; ++i) dev[i].img = base + off[i];
    ld_peak *d_pk = (ld_peak *)(base + out_off);
    int32_t *d_np = (int32_t *)(base + np_off), *d_st = (int32_t *)(base + st_off);
    st = detect_impl(ctx, dev.data(), n, p, d_pk, d_np, d_st, s);
    if (st != LD_OK) return st;
    e = cudaMemcpyAsync(h_peaks, d_pk, pk_bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_n_peaks, d_np, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_status, d_st, (size_t)n * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->hev_free[b], s);
    if (e != cudaSuccess) return cuda_fail(e, "result download");
    ctx->hev_used[b] = true;
    ++ctx->host_calls;
    return LD_OK;
}

}  // extern "C"

namespace {

ld_status detect_impl(ld_ctx *ctx, const ld_frame *h_frames, int32_t n, const ld_params &p, ld_peak *d_peaks,
                      int32_t *d_n_peaks, int32_t *d_status, cudaStream_t s, const LinesReq *lines,
                      const ld_canny_params *canny) {
    ld_status st;
    const int32_t *dt;
    const std::vector<int32_t> *ht;
    st = get_trig(ctx, p.n_theta, &dt, &ht);
    if (st != LD_OK) return st;
    for (int i = 0; i < n; ++i) {
        const ld_frame &f = h_frames[i];
        st = check_size(f.w, f.h, p, ht);
        if (st != LD_OK) return fail(st, "frame %d: %s", i, g_err.c_str());
        if (!f.img || f.pitch < f.w || (f.pitch & 15) || !aligned16(f.img) || f.reserved != 0)
            return fail(LD_ERR_INVALID, "frame %d: NULL image, bad pitch or alignment", i);
        if (lines && (f.w > kLinesMaxSide || f.h > kLinesMaxSide))
            return fail(LD_ERR_INVALID, "frame %d: Hough lines need max(w, h) <= %d", i, kLinesMaxSide);
    }
    const int M = cand_m(p);
    // scratch for the largest group of frames
    int64_t max_edges = 0, max_cand = 0;
    for (int g0 = 0; g0 < n; g0 += kMaxLaunchFrames) {
        const int g1 = g0 + kMaxLaunchFrames < n ? g0 + kMaxLaunchFrames : n;
        int64_t ed = 0, ca = 0;
        for (int i = g0; i < g1; ++i) {
            ed += ((int64_t)h_frames[i].w * h_frames[i].h + 3) / 4 * 4;
            const int T0 = plan_for(ctx, h_frames[i].w, h_frames[i].h, p.n_theta, false).n_tiles;
            const int Tc = (p.n_theta / 2 + 7) / 8;   // interleaved tiles of 8 pairs at the most
            ca += (int64_t)std::max(Tc, std::min(p.n_theta / 2, T0 + (T0 + 3) / 4)) * M;   // room for balance_tiles
        }
        if (ed > max_edges) max_edges = ed;
        if (ca > max_cand) max_cand = ca;
    }
    if (!ctx->edges.ensure((size_t)max_edges * 4)) return fail(LD_ERR_NOMEM, "scratch edges");
    if (!ctx->small.ensure(kSmallInts * 4)) return fail(LD_ERR_NOMEM, "scratch counts");
    if (!ctx->cand.ensure((size_t)max_cand * 8)) return fail(LD_ERR_NOMEM, "scratch candidates");
    uint32_t *edges = (uint32_t *)ctx->edges.p;
    const Small sm = small_of(ctx->small.p);
    uint64_t *cand = (uint64_t *)ctx->cand.p;

    SobelLaunch SLn;
    HoughLaunch HLn, HLp;   // interleaved-column and packed-pair voting launches
    std::vector<int> order, sub_c, sub_p;
    std::vector<char> is_cols;
    std::vector<int64_t> eoffs, coffs;
    std::vector<HoughPlan> plans;

    for (int g0 = 0; g0 < n; g0 += kMaxLaunchFrames) {
        const int g1 = g0 + kMaxLaunchFrames < n ? g0 + kMaxLaunchFrames : n;
        const int gn = g1 - g0;
        cudaError_t e = cudaMemsetAsync(sm.counts, 0, kSmallInts * 4, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counts)");
        std::memset(&SLn, 0, sizeof SLn);
        std::memset(&HLn, 0, sizeof HLn);
        SLn.n = gn;
        SLn.threshold = p.threshold;
        SLn.border = p.border;
        SLn.groups = rows_for(ctx, h_frames, g0, g1, p.n_theta);
        // per-frame scratch offsets and plans (frame order)
        eoffs.assign(gn, 0);
        coffs.assign(gn, 0);
        plans.resize(gn);
        int64_t eoff = 0, coff = 0;
        // voting kernels: the interleaved-column kernel for the frames whose
        // plan allows it, the packed-pair kernel for the rest.  A group with
        // both kinds votes in two launches only if each part fills the GPU on
        // its own (else all frames take the packed-pair kernel in one launch,
        // so that small mixed batches keep one concurrent launch).
        is_cols.assign(gn, 0);
        int tiles_c = 0, tiles_p = 0;
        for (int k = 0; k < gn; ++k) {
            const ld_frame &fr = h_frames[g0 + k];
            if (p.min_votes >= 1) {
                const HoughPlan hc = plan_for(ctx, fr.w, fr.h, p.n_theta, true);
                if (hc.cols) {
                    plans[k] = hc;
                    is_cols[k] = 1;
                    tiles_c += hc.n_tiles;
                    continue;
                }
            }
            plans[k] = plan_for(ctx, fr.w, fr.h, p.n_theta, false);
            tiles_p += plans[k].n_tiles;
        }
        if (tiles_c > 0 && tiles_p > 0 && !two_launches(tiles_c, tiles_p, ctx->num_sms)) {
            for (int k = 0; k < gn; ++k)
                if (is_cols[k]) {
                    const ld_frame &fr = h_frames[g0 + k];
                    plans[k] = plan_for(ctx, fr.w, fr.h, p.n_theta, false);
                    is_cols[k] = 0;
                }
        }
        if (narrow_cols_tiles(tiles_c, ctx->num_sms)) {   // small launch: tiles of 8 pairs
            tiles_c = 0;
            for (int k = 0; k < gn; ++k)
                if (is_cols[k]) {
                    plans[k] = plan_cols_width(plans[k], p.n_theta, 8);
                    tiles_c += plans[k].n_tiles;
                }
        }
        {   // wave-filling tile counts for the packed-pair frames (equal plans only)
            std::vector<HoughPlan> pp;
            for (int k = 0; k < gn; ++k)
                if (!is_cols[k]) pp.push_back(plans[k]);
            if (!pp.empty()) {
                balance_tiles(pp, p.n_theta / 2, ctx->num_sms);
                for (int k = 0, i = 0; k < gn; ++k)
                    if (!is_cols[k]) plans[k] = pp[i++];
            }
        }
        for (int k = 0; k < gn; ++k) {
            const ld_frame &fr = h_frames[g0 + k];
            eoffs[k] = eoff;
            coffs[k] = coff;
            eoff += ((int64_t)fr.w * fr.h + 3) / 4 * 4;
            coff += (int64_t)plans[k].n_tiles * M;
        }
        int sob_ctas = 0;
        for (int k = 0; k < gn; ++k) {
            const ld_frame &fr = h_frames[g0 + k];
            SobelFrame &SF = SLn.f[k];
            SF.img = fr.img;
            SF.bin = nullptr;
            SF.edges = edges + eoffs[k];
            SF.count = sm.counts + k;
            SF.status_init = d_status + g0 + k;
            SF.npeaks_init = d_n_peaks + g0 + k;
            SF.cap = (int64_t)fr.w * fr.h;
            SF.w = fr.w;
            SF.h = fr.h;
            SF.pitch = fr.pitch;
            SF.tile_begin = sob_ctas;
            SF.tiles_x = sobel_strips(fr.w);
            sob_ctas += sobel_frame_ctas(fr.w, fr.h, SLn.groups);
        }
        // voting work units: frames with the most work (pixels x tile size)
        // first, so that the persistent CTAs end together (longest first)
        order.resize(gn);
        for (int k = 0; k < gn; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            const int64_t ca = (int64_t)h_frames[g0 + a].w * h_frames[g0 + a].h * plans[a].pairs;
            const int64_t cb = (int64_t)h_frames[g0 + b].w * h_frames[g0 + b].h * plans[b].pairs;
            return ca > cb;
        });
        // One voting launch over the frames sub (queue order) with one kernel.
        // Interleaved kernel: when the launch's last wave would be at most half
        // full, split each tile of the last frames in queue order (together
        // at least as many tiles as that wave holds) into ns edge ranges
        // (pieces, at most num_sms in all), which spread over the wave.  A
        // launch with fewer tiles than SMs (small batches: latency) splits
        // every tile, if its frames are large enough.
        struct Built {
            int units = 0, pmax = 1, words_cols = 16;   // words_cols: largest interleaved accumulator
            int64_t words_max = 0;
        };
        auto build_launch = [&](HoughLaunch &HL, bool cols, const std::vector<int> &sub, int32_t *queue,
                                Built &B) -> ld_status {
            const int gs = (int)sub.size();
            std::memset(&HL, 0, sizeof HL);
            int split_from = gs, ns_split = 1, split_tiles = 0;
            if (cols) {
                int64_t px_min = INT64_MAX;
                std::vector<int> tiles_q(gs);
                for (int q = 0; q < gs; ++q) {
                    const int k = sub[q];
                    tiles_q[q] = plans[k].n_tiles;
                    B.words_cols = std::max(B.words_cols, plans[k].rows * plans[k].width);
                    px_min = std::min(px_min, (int64_t)h_frames[g0 + k].w * h_frames[g0 + k].h);
                }
                const PieceSplit ps = plan_pieces(tiles_q.data(), gs, px_min, ctx->num_sms);
                split_from = ps.split_from;
                ns_split = ps.ns;
                split_tiles = ps.split_tiles;
                HL.col_chunk = hough_cols_chunk(B.words_cols);
                HL.part_stride = B.words_cols;
                if (split_tiles > 0) {
                    const size_t cnt_bytes = ((size_t)split_tiles * 4 + 255) / 256 * 256;
                    if (!ctx->part.ensure(split_scratch_bytes(split_tiles * ns_split, B.words_cols)))
                        return fail(LD_ERR_NOMEM, "scratch partial accumulators");
                    HL.tile_cnt = (int32_t *)ctx->part.p;
                    HL.part = (uint32_t *)((uint8_t *)ctx->part.p + cnt_bytes);
                    const cudaError_t r = cudaMemsetAsync(ctx->part.p, 0, (size_t)split_tiles * 4, s);
                    if (r != cudaSuccess) return cuda_fail(r, "cudaMemsetAsync(split counters)");
                }
            }
            HL.n = gs;
            HL.n_theta = p.n_theta;
            HL.mode = kHoughCandidates;
            HL.wait_polls = ctx->wait_polls;
            HL.cand_m = M;
            HL.min_votes = p.min_votes;
            HL.top_k = p.top_k;
            HL.nms_theta = p.nms_theta;
            HL.nms_rho = p.nms_rho;
            HL.trig = dt;
            HL.queue = queue;
            int split_base = 0;
            for (int q = 0; q < gs; ++q) {
                const int k = sub[q];
                const ld_frame &fr = h_frames[g0 + k];
                const HoughPlan &hp = plans[k];
                HoughFrame &HF = HL.f[q];
                HF.edges = edges + eoffs[k];
                HF.count = sm.counts + k;
                HF.cap = (int64_t)fr.w * fr.h;
                HF.acc = nullptr;
                HF.cand = cand + coffs[k];
                HF.flags = sm.flags + k;
                HF.done = sm.done + k;
                HF.peaks = d_peaks + (size_t)(g0 + k) * p.top_k;
                HF.n_peaks = d_n_peaks + g0 + k;
                HF.status = d_status + g0 + k;
                HF.w = fr.w;
                HF.h = fr.h;
                HF.D = hp.D;
                HF.n_rho = hp.n_rho;
                HF.unit_begin = B.units;
                HF.n_splits = q >= split_from ? ns_split : 1;
                HF.split_base = HF.n_splits > 1 ? split_base : 0;
                if (HF.n_splits > 1) split_base += hp.n_tiles;
                HF.pairs_per_tile = hp.pairs;
                HF.n_tiles = hp.n_tiles;
                HF.rows = hp.rows;
                HF.col_width = hp.width;
                B.units += hp.n_tiles * HF.n_splits;
                if (hp.pairs > B.pmax) B.pmax = hp.pairs;
                const int64_t wds = (int64_t)hp.pairs * hp.n_rho;
                if (wds > B.words_max) B.words_max = wds;
            }
            HL.total_units = B.units;
            return LD_OK;
        };
        sub_c.clear();
        sub_p.clear();
        for (int q = 0; q < gn; ++q) (is_cols[order[q]] ? sub_c : sub_p).push_back(order[q]);
        Built bc, bp;
        if (!sub_c.empty()) {
            st = build_launch(HLn, true, sub_c, sm.queue, bc);
            if (st != LD_OK) return st;
        }
        if (!sub_p.empty()) {
            st = build_launch(HLp, false, sub_p, sm.queue + 1, bp);
            if (st != LD_OK) return st;
        }
        cudaEvent_t *tev = nullptr;
        st = stage_events(ctx, g0, &tev);
        if (st != LD_OK) return st;
        if (tev) cudaEventRecord(tev[0], s);
        if (canny) {   // Canny edges in place of Steps 1-2, into the same lists
            int64_t px = 0;
            for (int k = 0; k < gn; ++k) px += (int64_t)h_frames[g0 + k].w * h_frames[g0 + k].h;
            if (!ctx->canny.ensure(canny_scratch_bytes(px))) return fail(LD_ERR_NOMEM, "scratch Canny");
            CannyLaunch CL;
            std::memset(&CL, 0, sizeof CL);
            CL.n = gn;
            CL.t_low = canny->t_low;
            CL.t_high = canny->t_high;
            CL.border = p.border;
            CL.total_px = px;
            int tiles = 0;
            int64_t off = 0;
            for (int k = 0; k < gn; ++k) {
                const ld_frame &fr = h_frames[g0 + k];
                CannyFrame &CF = CL.f[k];
                CF.img = fr.img;
                CF.bin = nullptr;
                CF.edges = edges + eoffs[k];
                CF.count = sm.counts + k;
                CF.status_init = d_status + g0 + k;
                CF.npeaks_init = d_n_peaks + g0 + k;
                canny_scratch(ctx->canny.p, px, off, CF);
                CF.cap = (int64_t)fr.w * fr.h;
                CF.px_begin = off;
                CF.w = fr.w;
                CF.h = fr.h;
                CF.pitch = fr.pitch;
                CF.tile_begin = tiles;
                tiles += canny_tiles(fr.w, fr.h);
                off += (int64_t)fr.w * fr.h;
            }
            e = launch_canny(CL, tiles, s);
            if (e != cudaSuccess) return cuda_fail(e, "canny launch");
        } else {
            e = launch_sobel(SLn, sob_ctas, s);
            if (e != cudaSuccess) return cuda_fail(e, "sobel launch");
        }
        if (tev) cudaEventRecord(tev[1], s);
        if (!sub_c.empty()) {
            e = launch_hough_cols(HLn, std::min(bc.units, ctx->num_sms), bc.words_cols, s);
            if (e != cudaSuccess) return cuda_fail(e, "hough launch");
        }
        if (!sub_p.empty()) {
            e = launch_hough(HLp, std::min(bp.units, ctx->num_sms), bp.pmax, bp.words_max, s);
            if (e != cudaSuccess) return cuda_fail(e, "hough launch");
        }
        if (tev) cudaEventRecord(tev[2], s);
        if (lines) {   // the group's edge lists and peaks are in place: its Hough lines
            LinesLaunch LL;
            std::memset(&LL, 0, sizeof LL);
            LL.n = gn;
            LL.top_k = p.top_k;
            LL.n_theta = p.n_theta;
            LL.fill_gap = lines->lp.fill_gap;
            LL.min_length = lines->lp.min_length;
            LL.max_segments = lines->lp.max_segments;
            LL.trig = dt;
            for (int k = 0; k < gn; ++k) {
                const ld_frame &fr = h_frames[g0 + k];
                const size_t fi = (size_t)(g0 + k);
                LinesFrame &LF = LL.f[k];
                LF.edges = edges + eoffs[k];
                LF.count = sm.counts + k;
                LF.cap = (int64_t)fr.w * fr.h;
                LF.peaks = d_peaks + fi * p.top_k;
                LF.n_peaks = d_n_peaks + fi;
                LF.segs = lines->segs + fi * p.top_k * lines->lp.max_segments;
                LF.n_segs = lines->n_segs + fi * p.top_k;
                LF.support = lines->support ? lines->support + fi * p.top_k : nullptr;
                LF.w = fr.w;
                LF.h = fr.h;
                LF.D = plans[k].D;
            }
            e = launch_lines(LL, s);
            if (e != cudaSuccess) return cuda_fail(e, "lines launch");
        }
    }
    return LD_OK;
}

}  // namespace

extern "C" {

ld_status ld_edge_pool_batch(ld_ctx *ctx, const ld_frame *h_frames, int32_t n, const ld_params *pp,
                             uint8_t *d_pool, void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_edge_pool_batch: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    if (!h_frames || n < 1 || !d_pool) return fail(LD_ERR_INVALID, "ld_edge_pool_batch: bad arguments");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    int64_t pool_bytes = 0, max_edges = 0;
    for (int i = 0; i < n; ++i) {
        const ld_frame &f = h_frames[i];
        st = check_size(f.w, f.h, p, nullptr);
        if (st != LD_OK) return fail(st, "frame %d: %s", i, g_err.c_str());
        if (!f.img || f.pitch < f.w || (f.pitch & 15) || !aligned16(f.img) || f.reserved != 0)
            return fail(LD_ERR_INVALID, "frame %d: NULL image, bad pitch or alignment", i);
        pool_bytes += (int64_t)((f.h + 7) / 8) * ((f.w + 7) / 8);
        max_edges += ((int64_t)f.w * f.h + 3) / 4 * 4;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_pool, 0, (size_t)pool_bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(pool)");
    if (!ctx->edges.ensure((size_t)std::min<int64_t>(max_edges, kMaxLaunchFrames * (int64_t)32767 * 32767 / 4) * 4))
        return fail(LD_ERR_NOMEM, "scratch edges");
    if (!ctx->small.ensure(kSmallInts * 4)) return fail(LD_ERR_NOMEM, "scratch counts");
    const Small sm = small_of(ctx->small.p);
    SobelLaunch SL;
    int64_t poff = 0;
    for (int g0 = 0; g0 < n; g0 += kMaxLaunchFrames) {
        const int g1 = std::min(n, g0 + kMaxLaunchFrames);
        std::memset(&SL, 0, sizeof SL);
        e = cudaMemsetAsync(sm.counts, 0, kMaxLaunchFrames * 4, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counts)");
        SL.n = g1 - g0;
        SL.threshold = p.threshold;
        SL.border = p.border;
        SL.groups = rows_for(ctx, h_frames, g0, g1, p.n_theta);
        int ctas = 0;
        int64_t eoff = 0;
        for (int i = g0; i < g1; ++i) {
            const ld_frame &fr = h_frames[i];
            SobelFrame &F = SL.f[i - g0];
            F.img = fr.img;
            F.edges = (uint32_t *)ctx->edges.p + eoff;
            F.count = sm.counts + (i - g0);
            F.pool = d_pool + poff;
            F.cap = (int64_t)fr.w * fr.h;
            F.w = fr.w;
            F.h = fr.h;
            F.pitch = fr.pitch;
            F.tile_begin = ctas;
            F.tiles_x = sobel_strips(fr.w);
            ctas += sobel_frame_ctas(fr.w, fr.h, SL.groups);
            eoff += ((int64_t)fr.w * fr.h + 3) / 4 * 4;
            poff += (int64_t)((fr.h + 7) / 8) * ((fr.w + 7) / 8);
        }
        e = launch_sobel(SL, ctas, s);
        if (e != cudaSuccess) return cuda_fail(e, "sobel launch");
    }
    return LD_OK;
}

}  // extern "C"

namespace {
// Layer sizes of the proposal network for an edge-count map ph x pw: conv1
// keeps the size, conv2-4 halve it (stride 2).  False if conv4's output is
// smaller than the 4 x 8 pooling grid.
bool net_sizes(int ph, int pw, int hs[5], int ws[5]) {
    hs[0] = hs[1] = ph;
    ws[0] = ws[1] = pw;
    for (int l = 2; l <= 4; ++l) {
        hs[l] = (hs[l - 1] - 1) / 2 + 1;
        ws[l] = (ws[l - 1] - 1) / 2 + 1;
    }
    return hs[4] >= 4 && ws[4] >= 8;
}

// The network's inference on n edge-count maps: conv1 fused into conv2 on the
// tensor cores (the same arithmetic as the separate layer calls, so the same
// bits), conv3, conv4 and pool + head -> logits [n][44].
ld_status net_infer(const uint8_t *pool, int n, const int hs[5], const int ws[5], const ld_proposal_net *net,
                    void *y2, void *y3, void *y4, float *feat, float *logits, cudaStream_t s) {
    const ConvTcGeom G2{n, hs[1], ws[1], hs[2], ws[2], 2};
    const cudaError_t e = launch_conv12_fused_tc(pool, G2, net->w[0], net->b[0], net->w[1], net->b[1], y2, s);
    if (e != cudaSuccess) return cuda_fail(e, "fused conv1-2");
    ld_status st = ld_conv3x3_forward(y2, n, hs[2], ws[2], 32, 32, 2, net->w[2], net->b[2], y3, s);
    if (st != LD_OK) return st;
    st = ld_conv3x3_forward(y3, n, hs[3], ws[3], 32, 32, 2, net->w[3], net->b[3], y4, s);
    if (st != LD_OK) return st;
    return ld_pool_head_forward(y4, n, hs[4], ws[4], net->wh, net->bh, feat, logits, s);
}
}  // namespace

extern "C" {

ld_status ld_proposal_logits(ld_ctx *ctx, const uint8_t *d_pool, int32_t n, int32_t ph, int32_t pw,
                             const ld_proposal_net *net, float *d_logits, void *stream) {
    if (!ctx || !d_pool || !d_logits || n < 1) return fail(LD_ERR_INVALID, "ld_proposal_logits: bad argument");
    if (!net || !net->wh || !net->bh) return fail(LD_ERR_INVALID, "ld_proposal_logits: NULL network");
    for (int i = 0; i < 4; ++i)
        if (!net->w[i] || !net->b[i]) return fail(LD_ERR_INVALID, "ld_proposal_logits: NULL network layer");
    int hs[5], ws[5];
    if (ph < 1 || pw < 2 || ph > 32767 || pw > 32767 || !net_sizes(ph, pw, hs, ws))
        return fail(LD_ERR_INVALID, "ld_proposal_logits: map %dx%d too small or too large", pw, ph);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    size_t off = 0;
    auto carve = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
    const size_t o_y2 = carve((size_t)n * hs[2] * ws[2] * 32 * 2);
    const size_t o_y3 = carve((size_t)n * hs[3] * ws[3] * 32 * 2);
    const size_t o_y4 = carve((size_t)n * hs[4] * ws[4] * 32 * 2);
    const size_t o_feat = carve((size_t)n * 1024 * 4);
    if (!ctx->prop.ensure(off)) return fail(LD_ERR_NOMEM, "scratch proposal");
    uint8_t *pb = (uint8_t *)ctx->prop.p;
    return net_infer(d_pool, n, hs, ws, net, pb + o_y2, pb + o_y3, pb + o_y4, (float *)(pb + o_feat), d_logits,
                     (cudaStream_t)stream);
}

ld_status ld_detect_batch_proposal(ld_ctx *ctx, const ld_frame *h_frames, int32_t n, const ld_params *pp,
                                   const ld_proposal_net *net, const ld_proposal_params *prp, ld_peak *d_peaks,
                                   int32_t *d_n_peaks, int32_t *d_status, int32_t *d_fallback,
                                   int32_t *d_active_pairs, void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_detect_batch_proposal: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    if (p.n_theta % 36 != 0) return fail(LD_ERR_INVALID, "ld_detect_batch_proposal: n_theta must be a multiple of 36");
    ld_proposal_params q = prp ? *prp : ld_proposal_params{0.2f, 0.5f, 2, 0};
    if (q.reserved != 0 || q.margin < 0 || !(q.p_band >= 0.f && q.p_band <= 1.f) ||
        !(q.p_fallback >= 0.f && q.p_fallback <= 1.f))
        return fail(LD_ERR_INVALID, "ld_detect_batch_proposal: bad proposal parameters");
    if (!h_frames || n < 1 || n > kMaxLaunchFrames)
        return fail(LD_ERR_INVALID, "ld_detect_batch_proposal: need 1 <= n <= %d frames", kMaxLaunchFrames);
    if (!d_peaks || !d_n_peaks || !d_status) return fail(LD_ERR_INVALID, "ld_detect_batch_proposal: NULL output");
    if (!net || !net->wh || !net->bh) return fail(LD_ERR_INVALID, "ld_detect_batch_proposal: NULL network");
    for (int i = 0; i < 4; ++i)
        if (!net->w[i] || !net->b[i]) return fail(LD_ERR_INVALID, "ld_detect_batch_proposal: NULL network layer");
    const int w = h_frames[0].w, h = h_frames[0].h;
    for (int i = 0; i < n; ++i)
        if (h_frames[i].w != w || h_frames[i].h != h)
            return fail(LD_ERR_INVALID, "ld_detect_batch_proposal: frames must share one size");
    const int ph = (h + 7) / 8, pw = (w + 7) / 8;
    int hs[5], ws[5];
    if (!net_sizes(ph, pw, hs, ws)) return fail(LD_ERR_INVALID, "ld_detect_batch_proposal: frame %dx%d too small", w, h);
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    const int32_t *dt;
    const std::vector<int32_t> *ht;
    st = get_trig(ctx, p.n_theta, &dt, &ht);
    if (st != LD_OK) return st;
    for (int i = 0; i < n; ++i) {
        const ld_frame &f = h_frames[i];
        st = check_size(f.w, f.h, p, ht);
        if (st != LD_OK) return fail(st, "frame %d: %s", i, g_err.c_str());
        if (!f.img || f.pitch < f.w || (f.pitch & 15) || !aligned16(f.img) || f.reserved != 0)
            return fail(LD_ERR_INVALID, "frame %d: NULL image, bad pitch or alignment", i);
    }
    const int M = cand_m(p);
    const HoughPlan hp = plan_for(ctx, w, h, p.n_theta, false);   // packed-pair plan
    // the interleaved-column kernel votes the kept pairs when the frame fits it
    // and min_votes >= 1 (its windows leave unvoted cells out); device plan
    const HoughPlan hc = plan_cols(ctx, w, h, p.n_theta);
    const bool cols = p.min_votes >= 1 && hc.cols && hc.width == kHoughColPairs;
    const int n_pairs = p.n_theta / 2;
    const int64_t epf = ((int64_t)w * h + 3) / 4 * 4;
    if (!ctx->edges.ensure((size_t)(n * epf) * 4)) return fail(LD_ERR_NOMEM, "scratch edges");
    if (!ctx->small.ensure(kSmallInts * 4)) return fail(LD_ERR_NOMEM, "scratch counts");
    // restricted-vote tiles per frame: up to twice the full vote's, so that
    // units can shrink to fill the persistent launch's last wave
    const int tile_cap = cols ? hc.n_tiles : std::min(n_pairs, 2 * hp.n_tiles);
    if (!ctx->cand.ensure((size_t)n * tile_cap * M * 8)) return fail(LD_ERR_NOMEM, "scratch candidates");
    if (cols && !ctx->part.ensure(split_scratch_bytes(ctx->num_sms, hc.rows * kHoughColPairs)))
        return fail(LD_ERR_NOMEM, "scratch partial accumulators");
    // proposal scratch, carved in 256-byte aligned pieces
    size_t off = 0;
    auto carve = [&](size_t bytes) { const size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
    const size_t o_pool = carve((size_t)n * ph * pw);
    const size_t o_y2 = carve((size_t)n * hs[2] * ws[2] * 32 * 2);
    const size_t o_y3 = carve((size_t)n * hs[3] * ws[3] * 32 * 2);
    const size_t o_y4 = carve((size_t)n * hs[4] * ws[4] * 32 * 2);
    const size_t o_feat = carve((size_t)n * 1024 * 4);
    const size_t o_logit = carve((size_t)n * 44 * 4);
    const size_t o_list = carve((size_t)n * n_pairs * 4);
    const size_t o_cnt = carve((size_t)n * 4);
    const size_t o_fb = carve((size_t)n * 4);
    const size_t o_tiles = carve((size_t)n * 4);
    const size_t o_ub = carve((size_t)(n + 1) * 4);
    const size_t o_cplan = carve((size_t)n * 3 * 4);
    if (!ctx->prop.ensure(off)) return fail(LD_ERR_NOMEM, "scratch proposal");
    uint8_t *pb = (uint8_t *)ctx->prop.p;
    uint8_t *pool = pb + o_pool;
    void *y[5] = {nullptr, nullptr, pb + o_y2, pb + o_y3, pb + o_y4};
    float *feat = (float *)(pb + o_feat), *logits = (float *)(pb + o_logit);
    int32_t *plist = (int32_t *)(pb + o_list), *pcnt = (int32_t *)(pb + o_cnt);
    int32_t *fb = d_fallback ? d_fallback : (int32_t *)(pb + o_fb);
    int32_t *tiles = (int32_t *)(pb + o_tiles), *ub = (int32_t *)(pb + o_ub);
    int32_t *cplan = (int32_t *)(pb + o_cplan);
    uint32_t *edges = (uint32_t *)ctx->edges.p;
    const Small sm = small_of(ctx->small.p);
    uint64_t *cand = (uint64_t *)ctx->cand.p;
    cudaStream_t s = (cudaStream_t)stream;

    cudaError_t e = cudaMemsetAsync(sm.counts, 0, kSmallInts * 4, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(counts)");
    // Steps 1-2 with the edge-count map
    SobelLaunch SL;
    std::memset(&SL, 0, sizeof SL);
    SL.n = n;
    SL.threshold = p.threshold;
    SL.border = p.border;
    SL.groups = rows_for(ctx, h_frames, 0, n, p.n_theta);
    const int per_frame_ctas = sobel_frame_ctas(w, h, SL.groups);
    for (int i = 0; i < n; ++i) {
        SobelFrame &F = SL.f[i];
        F.img = h_frames[i].img;
        F.edges = edges + i * epf;
        F.count = sm.counts + i;
        F.status_init = d_status + i;
        F.npeaks_init = d_n_peaks + i;
        F.pool = pool + (size_t)i * ph * pw;
        F.cap = (int64_t)w * h;
        F.w = w;
        F.h = h;
        F.pitch = h_frames[i].pitch;
        F.tile_begin = i * per_frame_ctas;
        F.tiles_x = sobel_strips(w);
    }
    e = launch_sobel(SL, n * per_frame_ctas, s);
    if (e != cudaSuccess) return cuda_fail(e, "sobel launch");
    // the network
    st = net_infer(pool, n, hs, ws, net, y[2], y[3], y[4], feat, logits, s);
    if (st != LD_OK) return st;
    // bands -> active pairs -> work units
    const size_t cnt_bytes = ((size_t)ctx->num_sms * 4 + 255) / 256 * 256;
    int32_t *tile_cnt = cols ? (int32_t *)ctx->part.p : nullptr;
    if (cols)
        e = launch_select_bands_cols(logits, n, p.n_theta, q.p_band, q.p_fallback, q.margin, ctx->num_sms,
                                     (int64_t)w * h >= kSplitFillPixels, plist, pcnt, fb, cplan, ub, tile_cnt, s);
    else
        e = launch_select_bands(logits, n, p.n_theta, q.p_band, q.p_fallback, q.margin, hp.pairs, tile_cap,
                                ctx->num_sms, plist, pcnt, fb, tiles, ub, s);
    if (e != cudaSuccess) return cuda_fail(e, "band selection");
    // Steps 3-4 on the kept pairs
    HoughLaunch HL;
    std::memset(&HL, 0, sizeof HL);
    HL.n = n;
    HL.n_theta = p.n_theta;
    HL.mode = kHoughCandidates;
    HL.wait_polls = ctx->wait_polls;
    HL.cand_m = M;
    HL.min_votes = p.min_votes;
    HL.top_k = p.top_k;
    HL.nms_theta = p.nms_theta;
    HL.nms_rho = p.nms_rho;
    HL.trig = dt;
    HL.queue = sm.queue;
    HL.unit_begin_dev = ub;
    if (cols) {
        HL.col_plan = cplan;
        HL.col_chunk = hough_cols_chunk(hc.rows * kHoughColPairs);
        HL.part_stride = hc.rows * kHoughColPairs;
        HL.tile_cnt = tile_cnt;
        HL.part = (uint32_t *)((uint8_t *)ctx->part.p + cnt_bytes);
    }
    for (int i = 0; i < n; ++i) {
        HoughFrame &HF = HL.f[i];
        HF.edges = edges + i * epf;
        HF.count = sm.counts + i;
        HF.cap = (int64_t)w * h;
        HF.cand = cand + (size_t)i * tile_cap * M;
        HF.flags = sm.flags + i;
        HF.done = sm.done + i;
        HF.peaks = d_peaks + (size_t)i * p.top_k;
        HF.n_peaks = d_n_peaks + i;
        HF.status = d_status + i;
        HF.pair_list = plist + (size_t)i * n_pairs;
        HF.pair_count = pcnt + i;
        HF.w = w;
        HF.h = h;
        HF.D = hp.D;
        HF.n_rho = hp.n_rho;
        HF.n_splits = 1;
        HF.pairs_per_tile = hp.pairs;
        HF.n_tiles = tile_cap;   // unused: the device plan gives each frame's tiles
        HF.rows = hc.rows;
        HF.col_width = kHoughColPairs;
    }
    const int max_units = n * tile_cap * (cols ? kMaxSplits : 1);
    const int ctas = max_units < ctx->num_sms ? max_units : ctx->num_sms;
    e = cols ? launch_hough_cols(HL, ctas, hc.rows * kHoughColPairs, s)
             : launch_hough(HL, ctas, hp.pairs, (int64_t)hp.pairs * hp.n_rho, s);
    if (e != cudaSuccess) return cuda_fail(e, "hough launch");
    if (d_active_pairs) {
        e = cudaMemcpyAsync(d_active_pairs, pcnt, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "active pairs copy");
    }
    return LD_OK;
}

ld_status ld_ctx_plan(ld_ctx *ctx, int32_t w, int32_t h, const ld_params *pp, int32_t *pairs_per_tile,
                      int32_t *sobel_rows) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_ctx_plan: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    st = check_size(w, h, p, nullptr);
    if (st != LD_OK) return st;
    std::lock_guard<std::mutex> lk(ctx->mu);
    const HoughPlan hp = plan_for(ctx, w, h, p.n_theta, p.min_votes >= 1);
    if (pairs_per_tile) *pairs_per_tile = hp.cols ? -hp.pairs : hp.pairs;
    if (sobel_rows) {
        const ld_frame f = {nullptr, w, h, w, 0};
        *sobel_rows = rows_for(ctx, &f, 0, 1, p.n_theta);
    }
    return LD_OK;
}

ld_status ld_autotune(ld_ctx *ctx, const ld_frame *h_frames, int32_t n, const ld_params *pp, int32_t iters,
                      void *stream) {
    if (!ctx) return fail(LD_ERR_INVALID, "ld_autotune: NULL ctx");
    ld_params p = pp ? *pp : defaults();
    ld_status st = check_params(&p);
    if (st != LD_OK) return st;
    if (!h_frames || n < 1 || iters < 1) return fail(LD_ERR_INVALID, "ld_autotune: need n >= 1 frames, iters >= 1");
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    if (!g.ok) return fail(LD_ERR_CUDA, "cannot select device %d", ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    // frames grouped by size
    std::map<std::pair<int, int>, std::vector<ld_frame>> groups;
    for (int i = 0; i < n; ++i) groups[{h_frames[i].w, h_frames[i].h}].push_back(h_frames[i]);
    size_t max_n = 0;
    for (auto &kv : groups) max_n = std::max(max_n, kv.second.size());
    void *outs = nullptr;
    cudaError_t e = cudaMalloc(&outs, max_n * (sizeof(ld_peak) * p.top_k + 2 * sizeof(int32_t)));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(autotune outputs)");
    ld_peak *d_peaks = (ld_peak *)outs;
    int32_t *d_np = (int32_t *)(d_peaks + max_n * p.top_k);
    int32_t *d_st = d_np + max_n;
    st = LD_OK;
    for (auto &kv : groups) {
        const int w = kv.first.first, h = kv.first.second;
        const std::vector<ld_frame> &fr = kv.second;
        const int n_rho = 2 * (int)rho_max_of(w, h) + 1;
        const int pmax = std::min(hough_max_pairs(n_rho), p.n_theta / 2);
        std::vector<int> pair_cands;
        // all compiled tile sizes down to 1/8 of what fits: small frames want
        // many small tiles (more CTAs), large batches few large ones
#define LD_CAND(P) if (P <= pmax && 8 * P >= pmax) pair_cands.push_back(P);
        LD_HOUGH_PAIR_SIZES(LD_CAND)
#undef LD_CAND
        if (pair_cands.empty()) pair_cands.push_back(std::max(1, pmax));
        if (p.min_votes >= 1 && plan_cols(ctx, w, h, p.n_theta).cols) pair_cands.push_back(-1);   // interleaved
        // the voting tile size by the voting stage's time, then the Sobel run
        // length by the Sobel stage's time (the two stages are independent)
        auto time_stage = [&](int P, int R, int stage, float *out) -> ld_status {
            ctx->force_pairs = P;
            ctx->force_rows = R;
            ld_status r = detect_impl(ctx, fr.data(), (int)fr.size(), p, d_peaks, d_np, d_st, s);   // warm-up
            if (r != LD_OK) return r;
            float junk[3];
            r = stage_sums(ctx, junk);   // drop earlier timed calls
            if (r != LD_OK) return r;
            ctx->timing = true;
            for (int it = 0; it < iters && r == LD_OK; ++it)
                r = detect_impl(ctx, fr.data(), (int)fr.size(), p, d_peaks, d_np, d_st, s);
            ctx->timing = false;
            if (r != LD_OK) return r;
            float ms[3];
            r = stage_sums(ctx, ms);
            *out = ms[stage];
            return r;
        };
        const bool timing_was = ctx->timing;
        const int r0 = rows_for(ctx, fr.data(), 0, 1, p.n_theta);
        float best_ms = 1e30f;
        int best_p = pair_cands[0], best_r = r0;
        for (int P : pair_cands) {
            float t = 0.f;
            st = time_stage(P, r0, 1, &t);
            if (st != LD_OK) break;
            if (t < best_ms) { best_ms = t; best_p = P; }
        }
        best_ms = 1e30f;
        for (int R : {1, 2, 4}) {
            if (st != LD_OK) break;
            float t = 0.f;
            st = time_stage(best_p, R, 0, &t);
            if (st != LD_OK) break;
            if (t < best_ms) { best_ms = t; best_r = R; }
        }
        ctx->timing = timing_was;
        ctx->force_pairs = 0;
        ctx->force_rows = 0;
        if (st != LD_OK) break;
        ctx->tuned[std::make_tuple(w, h, p.n_theta)] = {best_p, best_r};
    }
    ctx->force_pairs = 0;
    ctx->force_rows = 0;
    cudaFree(outs);
    return st;
}

}  // extern "C"
