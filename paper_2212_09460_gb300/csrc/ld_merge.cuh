// ld_merge.cuh -- the greedy Hough-peak pick (Sec. 2.3 "Hough Peak") over a
// frame's candidate keys, as a block-level device function shared by the
// standalone merge kernel and the persistent voting kernel.
//
// Keys order like the peaks (votes desc, theta asc, rho asc), so each of the
// top_k rounds is a block-wide arg-max over the candidates that no earlier
// pick suppresses (window nms_theta x nms_rho, no theta wrap); empty slots
// hold key 0 and never win.
#pragma once

#include "ld_internal.cuh"

namespace ld {

struct MergeSmem {
    uint64_t picks[kMaxTopK];
    uint64_t red[32];
};

// Every thread of the block must call this.  Writes peaks[0..n), *n_peaks and,
// when status != nullptr, *status (LD_ERR_TIMEOUT if the frame's flags say a
// wait gave up, else LD_OK).
__device__ inline void block_merge(const uint64_t *cand, int64_t n_cand, int top_k, int nms_theta,
                                   int nms_rho, ld_peak *peaks, int32_t *n_peaks, int32_t *status,
                                   int32_t flags, MergeSmem &S) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int ht = nms_theta / 2, hr = nms_rho / 2;
    int n_picked = 0;
    for (int round = 0; round < top_k; ++round) {
        uint64_t best = 0;
        for (int64_t i = tid; i < n_cand; i += blockDim.x) {
            const uint64_t key = __ldcg(&cand[i]);   // written by other CTAs of this launch
            if (key <= best) continue;   // also skips empty (0) slots
            const int th = 0xFFFF - (int)((key >> 16) & 0xFFFFu);
            const int rh = 0xFFFF - (int)(key & 0xFFFFu);
            bool sup = false;
            for (int p = 0; p < n_picked; ++p) {
                const int pt = 0xFFFF - (int)((S.picks[p] >> 16) & 0xFFFFu);
                const int pr = 0xFFFF - (int)(S.picks[p] & 0xFFFFu);
                if (abs(th - pt) <= ht && abs(rh - pr) <= hr) { sup = true; break; }
            }
            if (!sup) best = key;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t v = __shfl_xor_sync(0xFFFFFFFFu, best, o);
            best = v > best ? v : best;
        }
        if (lane == 0) S.red[warp] = best;
        __syncthreads();
        if (tid == 0) {
            uint64_t b = 0;
            for (int w = 0; w < nw; ++w) b = S.red[w] > b ? S.red[w] : b;
            S.picks[round] = b;
        }
        __syncthreads();
        const bool none = S.picks[round] == 0ull;
        __syncthreads();
        if (none) break;
        ++n_picked;
    }
    if (tid < n_picked) {
        const uint64_t key = S.picks[tid];
        ld_peak pk;
        pk.theta_idx = 0xFFFF - (int)((key >> 16) & 0xFFFFu);
        pk.rho_idx = 0xFFFF - (int)(key & 0xFFFFu);
        pk.votes = (int32_t)((uint32_t)(key >> 32) ^ 0x80000000u);
        peaks[tid] = pk;
    }
    if (tid == 0) {
        *n_peaks = n_picked;
        if (status) *status = (flags & kFlagTimeout) ? LD_ERR_TIMEOUT : LD_OK;
    }
    __syncthreads();
}

}  // namespace ld
