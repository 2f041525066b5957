// ld_lines.cu -- Hough lines: the line segments behind each Hough peak (Step
// 4 of Sec. 1 without the drawing; the paper leaves it to MATLAB's "Hough
// lines", Sec. 5, Fig. 12).
//
// For peak (theta_k, rho index r) of a frame, the supporting pixels are the
// frame's edges whose Q16 rho at theta_k -- the vote's own rounding (Eq. 3,
// Eqs. 4-5) -- lands in cell r; there are exactly as many as the peak has
// votes.  They are ordered along the line (by x then y when |cos| <= |sin|,
// else by y then x), split where two consecutive pixels are more than
// fill_gap apart, and a piece is kept when its end pixels are at least
// min_length apart (squared Euclidean distances, exact integers).
//
// One CTA per (frame, peak):
//   1. streams the frame's edge list (16-byte loads) and appends the matching
//      pixels' sort keys to shared memory (warp ballot, one shared atomic per
//      warp);
//   2. sorts the keys (block bitonic sort; a key packs the pixel as
//      primary << 15 | secondary, so ascending keys are the line order);
//   3. marks segment starts (the gap test against the previous pixel),
//      numbers them with a block scan, tests each segment's length and writes
//      the kept ones in line order with a second scan.
// A ray of cells of width 1 holds at most 2 pixels per row (|cos| >= |sin|)
// or per column, so a peak has at most 2 max(w, h) supporting pixels: the
// host admits max(w, h) <= kLinesMaxSide so that they fit shared memory.
#include "ld_internal.cuh"
#include "ld_select.cuh"

namespace ld {
namespace {

constexpr int kLinesThreads = 1024;
constexpr int kLinesWarps = kLinesThreads / 32;

// Exclusive block-wide scan of one int per thread; *total = the sum.
__device__ __forceinline__ int block_excl_scan(int v, int *warp_sums, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int s = lane < kLinesWarps ? warp_sums[lane] : 0;
        int si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, si, o);
            if (lane >= o) si += t;
        }
        if (lane < kLinesWarps) warp_sums[lane] = si - s;   // exclusive warp offsets
        if (lane == 31) warp_sums[kLinesWarps] = si;
    }
    __syncthreads();
    const int r = warp_sums[warp] + incl - v;
    *total = warp_sums[kLinesWarps];
    __syncthreads();   // warp_sums is reused by the next scan
    return r;
}

__device__ __forceinline__ void key_xy(uint32_t key, bool by_x, int &x, int &y) {
    const int a = (int)(key >> 15), b = (int)(key & 0x7FFFu);
    x = by_x ? a : b;
    y = by_x ? b : a;
}

__device__ __forceinline__ int64_t dist2(int x0, int y0, int x1, int y1) {
    const int64_t dx = x1 - x0, dy = y1 - y0;
    return dx * dx + dy * dy;
}

__global__ void __launch_bounds__(kLinesThreads, 2) lines_kernel(const __grid_constant__ LinesLaunch L) {
    extern __shared__ __align__(16) uint32_t lsm[];
    const int cap = L.keys_cap;                             // >= 2 max(w, h), a power of two
    uint32_t *keys = lsm;                                   // [cap] sort keys
    int32_t *starts = reinterpret_cast<int32_t *>(lsm + cap);   // [cap] segment starts
    __shared__ int warp_sums[kLinesWarps + 1];
    __shared__ int n_sh;
    const int tid = threadIdx.x, lane = tid & 31;
    const int f = blockIdx.x / L.top_k, p = blockIdx.x % L.top_k;
    const LinesFrame &F = L.f[f];
    int32_t *nseg_out = F.n_segs + p;
    const int npk = *F.n_peaks;
    if (p >= npk) {   // block-uniform: no such peak
        if (tid == 0) {
            *nseg_out = 0;
            if (F.support) F.support[p] = 0;
        }
        return;
    }
    const ld_peak pk = F.peaks[p];
    const int k = pk.theta_idx, r = pk.rho_idx;
    if (k < 0 || k >= L.n_theta) {   // block-uniform: not a cell of this accumulator
        if (tid == 0) {
            *nseg_out = 0;
            if (F.support) F.support[p] = 0;
        }
        return;
    }
    const int half = L.n_theta / 2;
    const int kk = k <= half ? k : L.n_theta - k;
    const int32_t c = k <= half ? L.trig[2 * kk] : -L.trig[2 * kk];   // Eqs. 4-5
    const int32_t s = L.trig[2 * kk + 1];
    const bool by_x = abs(c) <= abs(s);
    // cell index = (x c + y s + 32768 + D 65536) >> 16, computed modulo 2^32
    // (its true value lies in [0, (2D + 1) 65536) for pixels of the image)
    const uint32_t kq = 32768u + (uint32_t)F.D * 65536u;
    const uint32_t W = (uint32_t)F.w, H = (uint32_t)F.h;
    if (tid == 0) n_sh = 0;
    __syncthreads();

    // 1. supporting pixels
    int64_t E = (int64_t)*F.count;
    if (E > F.cap) E = F.cap;
    if (E < 0) E = 0;
    auto test = [&](uint32_t e, bool valid) {
        const uint32_t x = e & 0xFFFFu, y = e >> 16;
        const bool m = valid && x < W && y < H && ((x * (uint32_t)c + y * (uint32_t)s + kq) >> 16) == (uint32_t)r;
        const uint32_t bal = __ballot_sync(0xFFFFFFFFu, m);
        if (bal) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&n_sh, __popc(bal));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            const int pos = base + __popc(bal & ((1u << lane) - 1u));
            if (m && pos < cap) keys[pos] = by_x ? (x << 15 | y) : (y << 15 | x);
        }
    };
    const int64_t E4 = E >> 2;
    const uint4 *e4 = reinterpret_cast<const uint4 *>(F.edges);
    for (int64_t base = 0; base < E4; base += kLinesThreads) {   // block-uniform trip count
        const int64_t i = base + tid;
        uint4 q = make_uint4(0u, 0u, 0u, 0u);
        const bool v = i < E4;
        if (v) q = __ldg(e4 + i);
        test(q.x, v);
        test(q.y, v);
        test(q.z, v);
        test(q.w, v);
    }
    {
        const int64_t i = (E4 << 2) + tid;   // the last E % 4 edges
        const bool v = tid < 32 && i < E;
        if (tid < 32) test(v ? F.edges[i] : 0u, v);
    }
    __syncthreads();
    const int n_all = n_sh;
    const int n = n_all < cap ? n_all : cap;   // distinct pixels never exceed it
    if (tid == 0 && F.support) F.support[p] = n_all;

    // 2. sort ascending (descending sort of the complemented keys; padding
    //    with complemented 0xFFFFFFFF = 0 sorts last)
    int n2 = 1;
    while (n2 < n) n2 <<= 1;
    for (int i = tid; i < n2; i += kLinesThreads) keys[i] = i < n ? ~keys[i] : 0u;
    __syncthreads();
    if (n > 1) block_sort_desc(keys, n2);
    for (int i = tid; i < n; i += kLinesThreads) keys[i] = ~keys[i];
    __syncthreads();

    // 3. segments: item i starts one when i == 0 or its gap to i - 1 exceeds fill_gap
    const int64_t gap2 = (int64_t)L.fill_gap * L.fill_gap, len2 = (int64_t)L.min_length * L.min_length;
    const int per = (n + kLinesThreads - 1) / kLinesThreads;
    const int i0 = min(n, tid * per), i1 = min(n, i0 + per);
    auto is_start = [&](int i) -> bool {
        if (i == 0) return true;
        int xa, ya, xb, yb;
        key_xy(keys[i - 1], by_x, xa, ya);
        key_xy(keys[i], by_x, xb, yb);
        return dist2(xa, ya, xb, yb) > gap2;
    };
    int my_starts = 0;
    for (int i = i0; i < i1; ++i) my_starts += is_start(i) ? 1 : 0;
    int nseg = 0;
    int sid = block_excl_scan(my_starts, warp_sums, &nseg);
    for (int i = i0; i < i1; ++i)
        if (is_start(i)) starts[sid++] = i;
    __syncthreads();
    // keep the long ones, in line order
    const int per2 = (nseg + kLinesThreads - 1) / kLinesThreads;
    const int j0 = min(nseg, tid * per2), j1 = min(nseg, j0 + per2);
    auto kept = [&](int j, int &xa, int &ya, int &xb, int &yb) -> bool {
        const int a = starts[j], b = (j + 1 < nseg ? starts[j + 1] : n) - 1;
        key_xy(keys[a], by_x, xa, ya);
        key_xy(keys[b], by_x, xb, yb);
        return dist2(xa, ya, xb, yb) >= len2;
    };
    int my_kept = 0;
    for (int j = j0; j < j1; ++j) {
        int xa, ya, xb, yb;
        my_kept += kept(j, xa, ya, xb, yb) ? 1 : 0;
    }
    int nkept = 0;
    int o = block_excl_scan(my_kept, warp_sums, &nkept);
    ld_segment *out = F.segs + (size_t)p * L.max_segments;
    for (int j = j0; j < j1; ++j) {
        int xa, ya, xb, yb;
        if (kept(j, xa, ya, xb, yb)) {
            if (o < L.max_segments) {
                ld_segment sg;
                sg.x1 = xa;
                sg.y1 = ya;
                sg.x2 = xb;
                sg.y2 = yb;
                sg.theta_idx = k;
                sg.rho_idx = r;
                out[o] = sg;
            }
            ++o;
        }
    }
    if (tid == 0) *nseg_out = nkept;
}

}  // namespace

cudaError_t launch_lines(const LinesLaunch &L0, cudaStream_t s) {
    if (L0.n <= 0) return cudaSuccess;
    // keys for the largest frame's 2 max(w, h) supporting pixels: smaller CTAs
    // let two of them share an SM (one wave for a 64-frame batch's peaks)
    LinesLaunch L = L0;
    int side = 1;
    for (int k = 0; k < L.n; ++k) side = max(side, max(L.f[k].w, L.f[k].h));
    if (side > kLinesMaxSide) return cudaErrorInvalidValue;
    int cap = 64;
    while (cap < 2 * side) cap <<= 1;
    L.keys_cap = cap;
    const size_t smem = (size_t)2 * cap * 4;
    static std::atomic<uint64_t> attr_done{0};
    const cudaError_t e = once_per_device(attr_done, [](int) {
        return cudaFuncSetAttribute(lines_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(2 * kLinesKeys * 4));
    });
    if (e != cudaSuccess) return e;
    lines_kernel<<<L.n * L.top_k, kLinesThreads, smem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace ld
