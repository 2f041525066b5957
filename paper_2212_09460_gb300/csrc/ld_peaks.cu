// ld_peaks.cu -- Step 4, Hough peaks (Sec. 2.3 "Hough Peak"; done in MATLAB
// in the paper, Sec. 5): greedy non-maximum suppression in the order
// (votes desc, theta_idx asc, rho_idx asc), each pick suppressing an
// nms_theta x nms_rho window, clipped, without theta wrap.
//
// Two kernels.  select_kernel cuts a full int32 accumulator into chunks of
// contiguous (theta, rho) cells and keeps each chunk's exact top-M (the
// argument for exactness is in ld_select.cuh); the voting kernel emits the
// same per-tile candidates directly from shared memory in ld_detect_batch.
// merge_kernel then runs the greedy over one frame's candidates (ld_merge.cuh).
#include "ld_internal.cuh"
#include "ld_merge.cuh"
#include "ld_select.cuh"

namespace ld {
namespace {

__global__ void __launch_bounds__(kSelectThreads)
select_kernel(const __grid_constant__ SelectLaunch L) {
    __shared__ SelectSmem S;
    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (L.j[mid].chunk_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const SelectJob &J = L.j[lo];
    const int chunk = blockIdx.x - J.chunk_begin;
    const int64_t c0 = (int64_t)chunk * kSelectChunk;
    const int64_t c1 = (c0 + kSelectChunk < J.cells) ? c0 + kSelectChunk : J.cells;
    const int n = (int)(c1 - c0);
    const int32_t *a = J.acc + c0;
    const int M = L.cand_m;
    const int32_t mv = L.min_votes;
    uint64_t *out = J.cand + (size_t)chunk * M;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = kSelectThreads / 32;

    // pass 0: included count and the range of u = v ^ 0x80000000
    int cnt = 0;
    uint32_t umin = 0xFFFFFFFFu, umax = 0;
    for (int i = tid; i < n; i += kSelectThreads) {
        const int32_t v = a[i];
        if (v >= mv) {
            const uint32_t u = (uint32_t)v ^ 0x80000000u;
            ++cnt;
            umin = min(umin, u);
            umax = max(umax, u);
        }
    }
    // Fast path: L = the M-th largest of the per-thread maxima (M distinct
    // cells reach it, so every top-M cell does); the cells >= L, usually a few
    // hundred, are compacted as unique keys and the M largest taken by rank.
    // More survivors than the key buffer holds: the radix path below.
    {
        constexpr int kSurvKeys = 1024;
        __shared__ uint64_t skeys[kSurvKeys];
        __shared__ int n_surv;
        if (tid == 0) n_surv = 0;
        uint32_t Lu = 0;
        if (block_mth_largest_u32(umax, cnt > 0, M, Lu, S)) {   // block-uniform
            for (int i = tid; i < n; i += kSelectThreads) {
                const int32_t v = a[i];
                if (v >= mv && ((uint32_t)v ^ 0x80000000u) >= Lu) {
                    const int slot = atomicAdd(&n_surv, 1);
                    if (slot < kSurvKeys) {
                        const int64_t li = c0 + i;
                        const int th = (int)(li / J.n_rho), rh = (int)(li - (int64_t)th * J.n_rho);
                        skeys[slot] = peak_key(v, th, rh);
                    }
                }
            }
            __syncthreads();
            const int ns_ = n_surv;
            if (ns_ <= kSurvKeys) {   // block-uniform
                block_topm_by_rank(skeys, ns_, M, out);
                return;
            }
        }
        __syncthreads();
    }
    const int total = block_sum(cnt, S);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        umin = min(umin, __shfl_xor_sync(0xFFFFFFFFu, umin, o));
        umax = max(umax, __shfl_xor_sync(0xFFFFFFFFu, umax, o));
    }
    __shared__ uint32_t rmin[32], rmax[32];
    if (lane == 0) { rmin[warp] = umin; rmax[warp] = umax; }
    __syncthreads();
    uint32_t gmin = 0xFFFFFFFFu, gmax = 0;
    for (int w = 0; w < nw; ++w) { gmin = min(gmin, rmin[w]); gmax = max(gmax, rmax[w]); }

    const bool all_in = total <= M;
    // all included cells share the bits above the highest bit where the
    // smallest and the largest key differ; start the radix passes below them
    int top_shift = 28;
    uint32_t prefix = 0, pmask = 0;
    if (!all_in) {
        const uint32_t diff = gmin ^ gmax;
        top_shift = 0;
        for (int s = 28; s > 0; s -= 4)
            if (diff >> s) { top_shift = s; break; }
        if (top_shift < 28) {
            pmask = 0xFFFFFFFFu << (top_shift + 4);
            prefix = gmax & pmask;
        }
    }
    if (tid == 0) {
        S.prefix = prefix;
        S.pmask = pmask;
        S.rank = M;
        S.out_n = 0;
    }
    __syncthreads();
    if (!all_in) {
        for (int shift = top_shift; shift >= 0; shift -= 4) {
            uint32_t wh[16];
#pragma unroll
            for (int d = 0; d < 16; ++d) wh[d] = 0;
            const uint32_t pf = S.prefix, pm = S.pmask;
            for (int base = 0; base < n; base += kSelectThreads) {
                const int i = base + tid;
                const int32_t v = (i < n) ? a[i] : 0;
                const uint32_t u = (uint32_t)v ^ 0x80000000u;
                ballot_digits(wh, i < n && v >= mv && (u & pm) == pf, (u >> shift) & 15u);
            }
            if (lane == 0) {
#pragma unroll
                for (int d = 0; d < 16; ++d) S.hist[warp][d] = wh[d];
            }
            select_digit(S, shift);
        }
    }
    const uint32_t ustar = S.prefix;
    const int need = all_in ? 0 : S.rank;
    __syncthreads();

    // ordered emission over per-thread contiguous ranges
    const int r0 = (int)((int64_t)n * tid / kSelectThreads);
    const int r1 = (int)((int64_t)n * (tid + 1) / kSelectThreads);
    int ties = 0;
    if (!all_in)
        for (int i = r0; i < r1; ++i) {
            const int32_t v = a[i];
            ties += (v >= mv && ((uint32_t)v ^ 0x80000000u) == ustar);
        }
    int incl = ties;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) S.red[warp] = (uint32_t)incl;
    __syncthreads();
    int woff = 0;
    for (int w = 0; w < warp; ++w) woff += (int)S.red[w];
    int trank = woff + incl - ties;
    for (int i = r0; i < r1; ++i) {
        const int32_t v = a[i];
        if (v < mv) continue;
        const uint32_t u = (uint32_t)v ^ 0x80000000u;
        const int64_t li = c0 + i;
        const int th = (int)(li / J.n_rho), rh = (int)(li - (int64_t)th * J.n_rho);
        if (all_in || u > ustar) {
            const int slot = atomicAdd(&S.out_n, 1);
            if (slot < M) out[slot] = peak_key(v, th, rh);
        } else if (u == ustar) {
            if (trank < need) out[(M - need) + trank] = peak_key(v, th, rh);
            ++trank;
        }
    }
    __syncthreads();
    const int filled = all_in ? min(S.out_n, M) : M;
    for (int i = filled + tid; i < M; i += kSelectThreads) out[i] = 0ull;
}

__global__ void __launch_bounds__(kMergeThreads)
merge_kernel(const __grid_constant__ MergeLaunch L) {
    __shared__ MergeSmem S;
    const MergeJob &J = L.j[blockIdx.x];
    const int32_t fl = J.flags ? *J.flags : 0;
    block_merge(J.cand, J.n_cand, L.top_k, L.nms_theta, L.nms_rho, J.peaks, J.n_peaks, J.status, fl, S);
}

}  // namespace

cudaError_t launch_select(const SelectLaunch &L, int n_ctas, cudaStream_t s) {
    if (n_ctas <= 0) return cudaSuccess;
    select_kernel<<<n_ctas, kSelectThreads, 0, s>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_merge(const MergeLaunch &L, cudaStream_t s) {
    if (L.n <= 0) return cudaSuccess;
    merge_kernel<<<L.n, kMergeThreads, 0, s>>>(L);
    return cudaGetLastError();
}

}  // namespace ld
