// ld_select.cuh -- exact block-wide top-M selection used to cut the Hough
// peak search (Sec. 2.3 "Hough Peak") down to a few candidates per tile.
//
// Why it is exact: the greedy peak picker takes, at pick j, the first cell
// in the order (votes desc, theta asc, rho asc) that is not suppressed; each
// earlier pick suppresses at most nms_theta*nms_rho cells, so pick j has rank
// <= (nms_theta*nms_rho)*(j-1)+1 = M for j <= top_k.  Any partition of the
// accumulator into tiles whose local top-M (same order) are kept therefore
// keeps every cell the greedy can pick, and the greedy over that union gives
// the same peaks as over the whole accumulator.
//
// Selection: a most-significant-digit radix select with 4-bit digits on the
// order-preserving key u = votes ^ 0x80000000 finds u* (the M-th largest u
// among cells with votes >= min_votes) and how many cells equal to u* must be
// taken; the cells equal to u* are taken in (theta, rho) order.  Digit
// histograms are built with warp ballots (no shared atomics, so the many
// equal small counts of an accumulator cost nothing extra).
#pragma once

#include "ld_internal.cuh"

namespace ld {

struct SelectSmem {
    uint32_t hist[32][16];   // per-warp digit counts
    uint32_t digit_sum[16];
    uint32_t red[32];
    uint32_t prefix, pmask;
    int32_t rank;            // remaining rank inside the current prefix
    int32_t total;           // included cells
    int32_t out_n;           // emitted so far (cells > u*)
    int32_t tie_run;         // ties taken so far (ordered pass)
    int32_t surv;            // survivors compacted by the fast path
};

// Block-wide bitonic sort of buf[0..n) in shared memory, descending; n a
// power of two.  Every thread of the block must call it.
template <class T>
__device__ __forceinline__ void block_sort_desc(T *buf, int n) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const T a = buf[i], b = buf[ixj];
                    const bool desc = (i & k) == 0;
                    if (desc ? (a < b) : (a > b)) {
                        buf[i] = b;
                        buf[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
}


// The M-th largest of unsigned 32-bit values, one per thread; `has` says
// whether the thread holds one.  Returns false (no threshold) if fewer than M
// threads hold a value.  The threshold lies between the smallest and the
// largest value held (M of them reach it, all of them reach the smallest),
// so it shares the bits above their highest differing bit; those are taken
// as found, and the rest fixed bit by bit with block-wide counts.  One
// barrier pass gathers the count, the smallest and the largest (per-warp
// figures in S.hist, the block's in S.digit_sum), then one barrier per bit.
// Every thread of the block must call it; the caller writes S.hist and
// S.digit_sum again only after another barrier.
__device__ __forceinline__ bool block_mth_largest_u32(uint32_t u, bool has, int M, uint32_t &L, SelectSmem &S) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t wcnt = (uint32_t)__popc(__ballot_sync(0xFFFFFFFFu, has));
    const uint32_t wmax = __reduce_max_sync(0xFFFFFFFFu, has ? u : 0u);
    const uint32_t wmin = __reduce_min_sync(0xFFFFFFFFu, has ? u : 0xFFFFFFFFu);
    if (lane == 0) {
        S.hist[warp][0] = wcnt;
        S.hist[warp][1] = wmax;
        S.hist[warp][2] = wmin;
    }
    __syncthreads();
    if (warp == 0) {
        const uint32_t c = __reduce_add_sync(0xFFFFFFFFu, lane < nw ? S.hist[lane][0] : 0u);
        const uint32_t mx = __reduce_max_sync(0xFFFFFFFFu, lane < nw ? S.hist[lane][1] : 0u);
        const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, lane < nw ? S.hist[lane][2] : 0xFFFFFFFFu);
        if (lane == 0) {
            S.digit_sum[0] = c;
            S.digit_sum[1] = mx;
            S.digit_sum[2] = mn;
        }
    }
    __syncthreads();
    const int n_with = (int)S.digit_sum[0];
    const uint32_t umax = S.digit_sum[1], umin = S.digit_sum[2];
    if (n_with < M) return false;
    const uint32_t diff = umin ^ umax;
    if (diff == 0u) {   // every value held is the same
        L = umax;
        return true;
    }
    const int hb = 31 - __clz(diff);   // highest differing bit
    uint32_t lo = hb == 31 ? 0u : umax & (0xFFFFFFFFu << (hb + 1));
    for (int b = hb; b >= 0; --b) {
        const uint32_t cand = lo | (1u << b);
        if (__syncthreads_count(has && u >= cand) >= M) lo = cand;
    }
    L = lo;
    return true;
}

// Exact top-M of n unique keys in shared memory by rank (the number of larger
// keys): key i goes to out[rank_i] when rank_i < M, so out[0..min(n, M)) is
// written in descending order.  Threads take keys tid, tid + blockDim.x, ...
__device__ __forceinline__ void block_topm_by_rank(const uint64_t *keys, int n, int M, uint64_t *out) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const uint64_t k = keys[i];
        int r = 0;
        for (int j = 0; j < n; ++j) r += keys[j] > k ? 1 : 0;
        if (r < M) out[r] = k;
    }
}

// Add the ballot counts of one warp-step to this warp's 16 digit counters
// (kept by every lane in registers).
__device__ __forceinline__ void ballot_digits(uint32_t (&wh)[16], bool m, uint32_t dig) {
#pragma unroll
    for (int d = 0; d < 16; ++d) wh[d] += __popc(__ballot_sync(0xFFFFFFFFu, m && dig == (uint32_t)d));
}

// The M-th largest of one value per thread (a thread without a value passes
// -1): the largest L >= 0 with at least M threads holding a value >= L; -1 if
// fewer than M threads hold a value.  L is fixed bit by bit from the top with
// block-wide counts (the count of values >= L only falls as L grows), starting
// at the highest set bit of the block's largest value: a higher bit would
// give a candidate above every value, which no thread reaches.  One barrier
// pass gathers the count of values and the largest (per-warp figures in
// S.hist, the block's in S.digit_sum), then one barrier per bit.  Every
// thread of the block must call it; the caller writes S.hist and S.digit_sum
// again only after another barrier.
__device__ __forceinline__ int block_mth_largest(int v, int M, SelectSmem &S) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int wcnt = __popc(__ballot_sync(0xFFFFFFFFu, v >= 0));
    const int wmax = __reduce_max_sync(0xFFFFFFFFu, v);
    if (lane == 0) {
        S.hist[warp][0] = (uint32_t)wcnt;
        S.hist[warp][1] = (uint32_t)wmax;
    }
    __syncthreads();
    if (warp == 0) {
        const int c = __reduce_add_sync(0xFFFFFFFFu, lane < nw ? (int)S.hist[lane][0] : 0);
        const int m = __reduce_max_sync(0xFFFFFFFFu, lane < nw ? (int)S.hist[lane][1] : -1);
        if (lane == 0) {
            S.digit_sum[0] = (uint32_t)c;
            S.digit_sum[1] = (uint32_t)m;
        }
    }
    __syncthreads();
    const int n_with = (int)S.digit_sum[0], vmax = (int)S.digit_sum[1];
    if (n_with < M) return -1;
    int lo = 0;
    for (int b = 31 - __clz(vmax); b >= 0; --b) {   // vmax >= 0 here
        const int cand = lo | (1 << b);
        if (__syncthreads_count(v >= cand) >= M) lo = cand;
    }
    return lo;
}

// Block sum of a per-thread int.
__device__ __forceinline__ int block_sum(int v, SelectSmem &S) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    __syncthreads();
    if (lane == 0) S.red[warp] = (uint32_t)v;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < nw; ++w) t += (int)S.red[w];
    __syncthreads();
    return t;
}

// After every warp has stored its 16 counts into S.hist[warp], pick the digit
// holding rank S.rank (counting from the top), narrow the prefix.
__device__ __forceinline__ void select_digit(SelectSmem &S, int shift) {
    const int nw = blockDim.x >> 5;
    __syncthreads();
    if (threadIdx.x < 16) {
        uint32_t s = 0;
        for (int w = 0; w < nw; ++w) s += S.hist[w][threadIdx.x];
        S.digit_sum[threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int rank = S.rank, cum = 0, d = 15;
        for (; d > 0; --d) {
            int c = (int)S.digit_sum[d];
            if (cum + c >= rank) break;
            cum += c;
        }
        S.rank = rank - cum;
        S.prefix |= (uint32_t)d << shift;
        S.pmask |= 15u << shift;
    }
    __syncthreads();
}

}  // namespace ld
