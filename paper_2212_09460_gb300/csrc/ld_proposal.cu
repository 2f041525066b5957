// ld_proposal.cu -- the device steps around the learned proposal (the paper
// has no learned stage): turning the network's band logits into the list of
// theta pairs to vote, and turning a frame's Hough peaks into training targets.
#include <cmath>

#include "ld_internal.cuh"

namespace ld {
namespace {

constexpr int kBands = 36, kRowBands = 8, kOut = kBands + kRowBands;

// One CTA per frame.  Band b is kept if sigmoid(logit_b) >= p_band; the kept
// bands' theta bins, widened by `margin` bins on each side, are voted.  If no
// band reaches p_fallback the frame votes every bin (full-vote fallback).
// Pair j covers bins {j, n - j} (j = 0: {0, n/2}); the frame's list holds the
// pairs with an active bin, ascending; tiles[f] = ceil(count / pairs_per_tile).
__global__ void __launch_bounds__(256) select_bands_kernel(const float *logits, int n_theta, float p_band,
                                                          float p_fallback, int margin, int pairs_per_tile,
                                                          int32_t *pair_list, int32_t *pair_count,
                                                          int32_t *fallback, int32_t *tiles) {
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
        fb_s = mx < p_fallback ? 1 : 0;
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
        tiles[f] = (base + pairs_per_tile - 1) / pairs_per_tile;
    }
}

// unit_begin[0] = 0, unit_begin[f + 1] = unit_begin[f] + tiles[f].
__global__ void prefix_kernel(const int32_t *tiles, int n, int32_t *unit_begin) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int s = 0;
        unit_begin[0] = 0;
        for (int f = 0; f < n; ++f) {
            s += tiles[f];
            unit_begin[f + 1] = s;
        }
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
                                int pairs_per_tile, int32_t *pair_list, int32_t *pair_count, int32_t *fallback,
                                int32_t *tiles, int32_t *unit_begin, cudaStream_t s) {
    select_bands_kernel<<<n, 256, 0, s>>>(logits, n_theta, p_band, p_fallback, margin, pairs_per_tile, pair_list,
                                          pair_count, fallback, tiles);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    prefix_kernel<<<1, 32, 0, s>>>(tiles, n, unit_begin);
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
