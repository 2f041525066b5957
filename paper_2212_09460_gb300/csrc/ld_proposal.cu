// ld_proposal.cu -- the device steps around the learned proposal (the paper
// has no learned stage): turning the network's band logits into the list of
// theta pairs to vote, and turning a frame's Hough peaks into training targets.
#include <cmath>

#include "ld_internal.cuh"
#include "ld_plan.h"

namespace ld {
namespace {

constexpr int kBands = 36, kRowBands = 8, kOut = kBands + kRowBands;

// One CTA per frame.  Band b is kept if sigmoid(logit_b) >= p_band; the kept
// bands' theta bins, widened by `margin` bins on each side, are voted.  If no
// band reaches p_fallback, or none reaches p_band (possible when p_band >
// p_fallback), the frame votes every bin (full-vote fallback), so every
// frame votes at least one pair.  Pair j covers bins {j, n - j} (j = 0:
// {0, n/2}); the frame's list holds the pairs with an active bin, ascending.
__global__ void __launch_bounds__(256) select_bands_kernel(const float *logits, int n_theta, float p_band,
                                                          float p_fallback, int margin, int32_t *pair_list,
                                                          int32_t *pair_count, int32_t *fallback) {
    __shared__ float prob[kBands];
    __shared__ uint8_t bin_on[kMaxTheta];
    __shared__ int warp_cnt[8];
    __shared__ int fb_s;
    const int f = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < kBands) prob[tid] = 1.f / (1.f + expf(-logits[(int64_t)f * kOut + tid]));
    __syncthreads();
    if (tid == 0) {
        float mx = 0.f;
        for (int b = 0; b < kBands; ++b) mx = fmaxf(mx, prob[b]);
        fb_s = (mx < p_fallback || mx < p_band) ? 1 : 0;
    }
    __syncthreads();
    const int bpb = n_theta / kBands;
    for (int t = tid; t < n_theta; t += blockDim.x) {
        bool on = fb_s != 0;
        if (!on) {
            const int b_lo = max(0, (t - margin - bpb + 1) / bpb);   // a negative numerator gives <= 0
            const int b_hi = min(kBands - 1, (t + margin) / bpb);
            for (int b = b_lo; b <= b_hi && !on; ++b)
                on = prob[b] >= p_band && t >= b * bpb - margin && t <= (b + 1) * bpb - 1 + margin;
        }
        bin_on[t] = on ? 1 : 0;
    }
    __syncthreads();
    // ordered compaction of the active pairs
    const int n_pairs = n_theta / 2;
    int base = 0;
    for (int j0 = 0; j0 < n_pairs; j0 += blockDim.x) {
        const int j = j0 + tid;
        const bool act = j < n_pairs && (j == 0 ? (bin_on[0] || bin_on[n_theta / 2]) : (bin_on[j] || bin_on[n_theta - j]));
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, act);
        if (lane == 0) warp_cnt[warp] = __popc(bal);
        __syncthreads();
        int off = base;
        for (int w = 0; w < warp; ++w) off += warp_cnt[w];
        if (act) pair_list[(int64_t)f * n_pairs + off + __popc(bal & ((1u << lane) - 1u))] = j;
        int tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += warp_cnt[w];
        base += tot;
        __syncthreads();
    }
    if (tid == 0) {
        pair_count[f] = base;
        fallback[f] = fb_s;
    }
}

constexpr int kPlanThreads = kMaxLaunchFrames;   // one thread per frame

__device__ __forceinline__ int tiles_at(int c, int r, int tile_cap) {
    const int r_min = (c + tile_cap - 1) / tile_cap;   // at most tile_cap tiles per frame
    const int rr = r > r_min ? r : r_min;
    return (c + rr - 1) / rr;
}

// Work units of the restricted vote (one CTA).  Frame f's c_f active pairs
// are split evenly over T_f tiles.  The persistent vote runs `slots` CTAs, so
// U = sum T_f units take ceil(U / slots) waves, each as long as its largest
// unit.  With the largest tile pmax the batch needs at least
// k = ceil(sum ceil(c_f / pmax) / slots) waves; the plan keeps k and takes the
// smallest pairs per tile r whose units still fit k * slots: T_f =
// ceil(c_f / r) (never more than tile_cap tiles), so the last wave is full
// and every unit is as short as the wave count allows.  Writes tiles[f] and
// the prefix unit_begin [n + 1].
__global__ void __launch_bounds__(kPlanThreads) plan_units_kernel(const int32_t *pair_count, int n, int pmax,
                                                                  int tile_cap, int slots, int32_t *tiles,
                                                                  int32_t *unit_begin) {
    __shared__ int warp_sum[kPlanThreads / 32];
    __shared__ int r_s;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c = tid < n ? pair_count[tid] : 0;
    auto block_sum = [&](int v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        __syncthreads();
        if (lane == 0) warp_sum[warp] = v;
        __syncthreads();
        int t = 0;
        for (int i = 0; i < kPlanThreads / 32; ++i) t += warp_sum[i];
        return t;
    };
    const int u_min = block_sum(tid < n ? tiles_at(c, pmax, tile_cap) : 0);
    const int budget = (u_min + slots - 1) / slots * slots;
    if (tid == 0) r_s = pmax;
    for (int r = pmax - 1; r >= 1; --r) {   // block-uniform loop; U(r) grows as r falls
        const int u = block_sum(tid < n ? tiles_at(c, r, tile_cap) : 0);
        if (u > budget) break;
        if (tid == 0) r_s = r;
    }
    __syncthreads();
    const int t = tid < n ? tiles_at(c, r_s, tile_cap) : 0;
    // inclusive prefix over the frames (n <= kPlanThreads)
    int v = t;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, v, o);
        if (lane >= o) v += y;
    }
    __syncthreads();
    if (lane == 31) warp_sum[warp] = v;
    __syncthreads();
    for (int i = 0; i < warp; ++i) v += warp_sum[i];
    if (tid < n) {
        tiles[tid] = t;
        unit_begin[tid + 1] = v;
    }
    if (tid == 0) unit_begin[0] = 0;
}

// Work units of the restricted vote on the interleaved-column kernel (one
// CTA; thread f plans frame f).  Frame f votes c_f pairs in T_f =
// ceil(c_f / kHoughColPairs) tiles; a unit costs about the frame's edge count
// whatever its pairs, so tiles are as few as possible.  When the U = sum T_f
// units leave the persistent launch's last wave at most half full, the tiles
// of the last frames (together at least that wave's units) are split into
// ns = min(8, slots / their tiles) edge-range pieces, which fill it.  With
// fewer units than slots and `fill` (frames large enough), every tile splits
// into min(8, slots / U) pieces (latency of small batches).
__global__ void __launch_bounds__(kPlanThreads) plan_cols_units_kernel(const int32_t *pair_count, int n, int slots,
                                                                       int fill, int32_t *col_plan,
                                                                       int32_t *unit_begin, int32_t *tile_cnt) {
    __shared__ int tiles_s[kPlanThreads];
    const int tid = threadIdx.x;
    if (tid < n) {
        const int c = pair_count[tid] > 0 ? pair_count[tid] : 1;
        tiles_s[tid] = (c + kHoughColPairs - 1) / kHoughColPairs;
    }
    for (int i = tid; i < slots; i += blockDim.x) tile_cnt[i] = 0;
    __syncthreads();
    if (tid == 0) {
        // the host plan's rule (ld_plan.h), with fill standing for the frame size
        const PieceSplit ps = plan_pieces(tiles_s, n, fill ? kSplitFillPixels : 0, slots);
        const int split_from = ps.split_from, ns = ps.ns;
        int ub = 0, sb = 0;
        for (int f = 0; f < n; ++f) {
            const int t = tiles_s[f], k = f >= split_from ? ns : 1;
            col_plan[3 * f] = t;
            col_plan[3 * f + 1] = k;
            col_plan[3 * f + 2] = k > 1 ? sb : 0;
            if (k > 1) sb += t;
            unit_begin[f] = ub;
            ub += t * k;
        }
        unit_begin[n] = ub;
    }
}

// Training targets from a frame's peaks (one CTA per frame).  A peak counts
// if it is among the first `always_k` or has >= rel_votes times the first
// peak's votes.  Targets: the theta band of each counted peak, and every
// h/8-row band holding a row y at which the counted peak's line
// rho = x cos(theta) + y sin(theta) is inside the frame, 0 <= x <= w - 1
// (|cos theta| <= 1e-9: the row y = rho / sin theta).
__global__ void __launch_bounds__(256) targets_kernel(const ld_peak *peaks, const int32_t *n_peaks, int top_k, int w,
                                                     int h, int n_theta, int D, int always_k, float rel_votes,
                                                     float *targets) {
    __shared__ int on[kOut];
    const int f = blockIdx.x;
    if (threadIdx.x < kOut) on[threadIdx.x] = 0;
    __syncthreads();
    const int np = n_peaks[f];
    const float vmin = np > 0 ? rel_votes * (float)peaks[(int64_t)f * top_k].votes : 0.f;
    for (int q = threadIdx.x; q < np * h; q += blockDim.x) {
        const int k = q / h, y = q % h;
        const ld_peak pk = peaks[(int64_t)f * top_k + k];
        if (k >= always_k && (float)pk.votes < vmin) continue;
        if (y == 0) on[pk.theta_idx * kBands / n_theta] = 1;
        const double ang = M_PI * (double)pk.theta_idx / (double)n_theta;
        const double c = cos(ang), s = sin(ang), rho = (double)(pk.rho_idx - D);
        bool in;
        if (fabs(c) > 1e-9) {
            const double x = (rho - y * s) / c;
            in = x >= 0.0 && x <= (double)(w - 1);
        } else {
            const double y0 = rho / s;
            in = y0 >= 0.0 && y0 <= (double)(h - 1) && fabs((double)y - y0) <= 0.5;
        }
        if (in) on[kBands + min(y * kRowBands / h, kRowBands - 1)] = 1;
    }
    __syncthreads();
    if (threadIdx.x < kOut) targets[(int64_t)f * kOut + threadIdx.x] = on[threadIdx.x] ? 1.f : 0.f;
}

}  // namespace

cudaError_t launch_select_bands(const float *logits, int n, int n_theta, float p_band, float p_fallback, int margin,
                                int pmax, int tile_cap, int slots, int32_t *pair_list, int32_t *pair_count,
                                int32_t *fallback, int32_t *tiles, int32_t *unit_begin, cudaStream_t s) {
    if (n < 1 || n > kPlanThreads || pmax < 1 || tile_cap < 1 || slots < 1) return cudaErrorInvalidValue;
    select_bands_kernel<<<n, 256, 0, s>>>(logits, n_theta, p_band, p_fallback, margin, pair_list, pair_count,
                                          fallback);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    plan_units_kernel<<<1, kPlanThreads, 0, s>>>(pair_count, n, pmax, tile_cap, slots, tiles, unit_begin);
    return cudaGetLastError();
}

cudaError_t launch_select_bands_cols(const float *logits, int n, int n_theta, float p_band, float p_fallback,
                                     int margin, int slots, bool fill, int32_t *pair_list, int32_t *pair_count,
                                     int32_t *fallback, int32_t *col_plan, int32_t *unit_begin, int32_t *tile_cnt,
                                     cudaStream_t s) {
    if (n < 1 || n > kPlanThreads || slots < 1) return cudaErrorInvalidValue;
    select_bands_kernel<<<n, 256, 0, s>>>(logits, n_theta, p_band, p_fallback, margin, pair_list, pair_count,
                                          fallback);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    plan_cols_units_kernel<<<1, kPlanThreads, 0, s>>>(pair_count, n, slots, fill ? 1 : 0, col_plan, unit_begin,
                                                      tile_cnt);
    return cudaGetLastError();
}

}  // namespace ld

extern "C" ld_status ld_proposal_targets(const ld_peak *d_peaks, const int32_t *d_n_peaks, int32_t n, int32_t top_k,
                                        int32_t w, int32_t h, int32_t n_theta, int32_t always_k, float rel_votes,
                                        float *d_targets, void *stream) {
    if (!d_peaks || !d_n_peaks || !d_targets || n < 1 || top_k < 1 || w < 3 || h < 3 || n_theta < 36 ||
        n_theta % 36 != 0 || n_theta > ld::kMaxTheta || always_k < 0 || !(rel_votes >= 0.f)) {
        ld::set_last_error("ld_proposal_targets: bad argument (n_theta a multiple of 36)");
        return LD_ERR_INVALID;
    }
    const int64_t r2 = (int64_t)w * w + (int64_t)h * h;
    int64_t D = (int64_t)sqrt((double)r2);
    while (D * D < r2) ++D;
    while (D > 0 && (D - 1) * (D - 1) >= r2) --D;
    ld::targets_kernel<<<n, 256, 0, (cudaStream_t)stream>>>(d_peaks, d_n_peaks, top_k, w, h, n_theta, (int)D,
                                                            always_k, rel_votes, d_targets);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ld::set_last_error(cudaGetErrorString(e));
        return LD_ERR_CUDA;
    }
    return LD_OK;
}
