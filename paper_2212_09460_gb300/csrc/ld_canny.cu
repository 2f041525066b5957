// ld_canny.cu -- Canny edge detection in place of Steps 1-2 (the paper's
// future work, Sec. 7), writing the same 0/255 map and packed edge list the
// Hough vote reads (Sec. 4.3).  All arithmetic is integer, with zero outside
// the image at every stage (the padding of Sec. 3.1):
//   1. 5x5 binomial blur b b^T, b = (1 4 6 4 1): G = (sum K I + 128) >> 8;
//   2. Sobel on G (Step 1's kernels), M = |gx| + |gy| (Eq. 1, not saturated);
//   3. gradient sector from the Q16 tangents of 22.5 and 67.5 degrees;
//   4. non-maximum suppression: keep M > 0, M > M(n1), M >= M(n2), with n1
//      the neighbour of the sector's pair with the smaller y (smaller x along x);
//   5. hysteresis: kept pixels with M >= t_high are strong, t_low <= M <
//      t_high weak; the edges are the 8-connected components of kept pixels
//      with M >= t_low that hold a strong pixel.
//
// Kernels:
//   canny_nms_kernel     32 x 32 output tiles per CTA: the 40 x 40 input
//                        patch, the 36 x 36 blur, the 34 x 34 magnitudes and
//                        sectors live in shared memory; writes the class map
//                        (0, 1 weak, 2 strong), parent[i] = i and strong[i] = 0.
//   canny_union_kernel   one thread per pixel joins a candidate to its
//                        candidate neighbours above and to the left (each
//                        8-neighbour pair once) in a union-find forest: lock-free
//                        linking of the larger root under the smaller with
//                        atomicCAS (parent[i] <= i always, so finding a root
//                        ends; a failed CAS means another link succeeded).
//   canny_flatten_kernel every candidate points straight at its root; a strong
//                        pixel marks its root.
//   canny_emit_kernel    candidates whose root is marked become edges: the
//                        0/255 map and the compacted edge list (warp ballot,
//                        one atomic per warp on the frame's counter).
// The components, hence the edges, do not depend on the order of the links.
#include "ld_internal.cuh"

namespace ld {
namespace {

constexpr int kTile = 32;
constexpr int kCannyThreads = 256;
constexpr int kPxThreads = 256;

__device__ __forceinline__ int find_root(const int32_t *parent, int i) {
    int p = __ldcg(parent + i);
    while (p != i) {
        i = p;
        p = __ldcg(parent + i);
    }
    return i;
}

__device__ __forceinline__ void unite(int32_t *parent, int a, int b) {
    for (;;) {
        a = find_root(parent, a);
        b = find_root(parent, b);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        const int old = atomicCAS(parent + b, b, a);   // link root b under a < b
        if (old == b) return;
        b = old;   // b was linked meanwhile: continue from where it points
    }
}

__device__ __forceinline__ int frame_of_tile(const CannyLaunch &L, int t) {
    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.f[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int frame_of_px(const CannyLaunch &L, int64_t q) {
    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.f[mid].px_begin <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kCannyThreads) canny_nms_kernel(const __grid_constant__ CannyLaunch L) {
    constexpr int NI = kTile + 8, NG = kTile + 4, NM = kTile + 2;
    __shared__ uint8_t I_s[NI][NI];
    __shared__ int16_t H_s[NI][NG];   // horizontal binomial sums (<= 4080)
    __shared__ uint8_t G_s[NG][NG];
    __shared__ int16_t M_s[NM][NM];
    __shared__ uint8_t S_s[NM][NM];
    const int fi = frame_of_tile(L, blockIdx.x);
    const CannyFrame &F = L.f[fi];
    const int local = blockIdx.x - F.tile_begin;
    const int tiles_x = (F.w + kTile - 1) / kTile;
    const int X0 = (local % tiles_x) * kTile, Y0 = (local / tiles_x) * kTile;
    const int w = F.w, h = F.h, tid = threadIdx.x;
    if (local == 0 && tid == 0) {   // until the merge writes the frame's peaks
        if (F.status_init) *F.status_init = LD_ERR_TIMEOUT;
        if (F.npeaks_init) *F.npeaks_init = 0;
    }
    // input patch, zero outside the image
    for (int i = tid; i < NI * NI; i += kCannyThreads) {
        const int r = i / NI, c = i % NI;
        const int y = Y0 - 4 + r, x = X0 - 4 + c;
        I_s[r][c] = (x >= 0 && y >= 0 && x < w && y < h) ? F.img[(size_t)y * F.pitch + x] : 0;
    }
    __syncthreads();
    for (int i = tid; i < NI * NG; i += kCannyThreads) {
        const int r = i / NG, c = i % NG;
        const uint8_t *row = I_s[r] + c;
        H_s[r][c] = (int16_t)(row[0] + 4 * row[1] + 6 * row[2] + 4 * row[3] + row[4]);
    }
    __syncthreads();
    for (int i = tid; i < NG * NG; i += kCannyThreads) {
        const int r = i / NG, c = i % NG;
        const int y = Y0 - 2 + r, x = X0 - 2 + c;
        const int s = H_s[r][c] + 4 * H_s[r + 1][c] + 6 * H_s[r + 2][c] + 4 * H_s[r + 3][c] + H_s[r + 4][c];
        G_s[r][c] = (x >= 0 && y >= 0 && x < w && y < h) ? (uint8_t)((s + 128) >> 8) : 0;
    }
    __syncthreads();
    for (int i = tid; i < NM * NM; i += kCannyThreads) {
        const int r = i / NM, c = i % NM;
        const int y = Y0 - 1 + r, x = X0 - 1 + c;
        int m = 0, sc = 0;
        if (x >= 0 && y >= 0 && x < w && y < h) {
            const uint8_t *a = G_s[r] + c, *b = G_s[r + 1] + c, *d = G_s[r + 2] + c;   // rows y-1, y, y+1
            const int gx = (a[2] + 2 * b[2] + d[2]) - (a[0] + 2 * b[0] + d[0]);
            const int gy = (d[0] + 2 * d[1] + d[2]) - (a[0] + 2 * a[1] + a[2]);
            const int64_t ax = gx < 0 ? -gx : gx, ay = gy < 0 ? -gy : gy;
            m = (int)(ax + ay);
            if (ay * 65536 <= 27146 * ax) sc = 0;
            else if (ay * 65536 >= 158218 * ax) sc = 2;
            else sc = (gx > 0) == (gy > 0) ? 1 : 3;   // gx gy > 0 (neither is 0 here)
        }
        M_s[r][c] = (int16_t)m;
        S_s[r][c] = (uint8_t)sc;
    }
    __syncthreads();
    for (int i = tid; i < kTile * kTile; i += kCannyThreads) {
        const int r = i / kTile, c = i % kTile;
        const int y = Y0 + r, x = X0 + c;
        if (x >= w || y >= h) continue;
        const int sc = S_s[r + 1][c + 1], m = M_s[r + 1][c + 1];
        // (n1, n2) per sector: along x (x-1, x+1); (x-1,y-1), (x+1,y+1); along y; (x+1,y-1), (x-1,y+1)
        const int dx1 = sc == 0 ? -1 : sc == 1 ? -1 : sc == 2 ? 0 : 1;
        const int dy1 = sc == 0 ? 0 : -1;
        const int m1 = M_s[r + 1 + dy1][c + 1 + dx1], m2 = M_s[r + 1 - dy1][c + 1 - dx1];
        const bool keep = m > 0 && m > m1 && m >= m2;
        const uint8_t cls = !keep ? 0 : (m >= L.t_high ? 2 : (m >= L.t_low ? 1 : 0));
        const size_t p = (size_t)y * w + x;
        F.cls[p] = cls;
        F.parent[p] = (int32_t)p;
        F.strong[p] = 0;
    }
}

__global__ void __launch_bounds__(kPxThreads) canny_union_kernel(const __grid_constant__ CannyLaunch L) {
    const int64_t q = (int64_t)blockIdx.x * kPxThreads + threadIdx.x;
    if (q >= L.total_px) return;
    const CannyFrame &F = L.f[frame_of_px(L, q)];
    const int p = (int)(q - F.px_begin);
    if (!F.cls[p]) return;
    const int w = F.w, x = p % w, y = p / w;
    // the neighbours that come earlier in raster order: each 8-neighbour pair once
    if (x > 0 && F.cls[p - 1]) unite(F.parent, p, p - 1);
    if (y > 0) {
        const int u = p - w;
        if (x > 0 && F.cls[u - 1]) unite(F.parent, p, u - 1);
        if (F.cls[u]) unite(F.parent, p, u);
        if (x + 1 < w && F.cls[u + 1]) unite(F.parent, p, u + 1);
    }
}

__global__ void __launch_bounds__(kPxThreads) canny_flatten_kernel(const __grid_constant__ CannyLaunch L) {
    const int64_t q = (int64_t)blockIdx.x * kPxThreads + threadIdx.x;
    if (q >= L.total_px) return;
    const CannyFrame &F = L.f[frame_of_px(L, q)];
    const int p = (int)(q - F.px_begin);
    const uint8_t c = F.cls[p];
    if (!c) return;
    const int r = find_root(F.parent, p);
    F.parent[p] = r;
    if (c == 2) F.strong[r] = 1;
}

__global__ void __launch_bounds__(kPxThreads) canny_emit_kernel(const __grid_constant__ CannyLaunch L) {
    const int64_t q = (int64_t)blockIdx.x * kPxThreads + threadIdx.x;
    const int lane = threadIdx.x & 31;
    // frames are whole multiples of nothing in particular: a warp may straddle two
    // frames, so the ballot is per frame (lanes of another frame vote false)
    const bool in = q < L.total_px;
    const int fi = in ? frame_of_px(L, q) : 0;
    const CannyFrame &F = L.f[fi];
    const int p = in ? (int)(q - F.px_begin) : 0;
    bool edge = false;
    int x = 0, y = 0;
    if (in) {
        x = p % F.w;
        y = p / F.w;
        edge = F.cls[p] && F.strong[__ldcg(F.parent + p)];
        if (L.border == LD_BORDER_CLEAR && (x == 0 || y == 0 || x == F.w - 1 || y == F.h - 1)) edge = false;
        if (F.bin) F.bin[(size_t)y * F.pitch + x] = edge ? 255 : 0;
    }
    // one atomic per frame present in the warp
    uint32_t pending = __ballot_sync(0xFFFFFFFFu, edge);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int lf = __shfl_sync(0xFFFFFFFFu, fi, leader);
        const uint32_t mine = __ballot_sync(0xFFFFFFFFu, edge && fi == lf);
        int base = 0;
        if (lane == leader) base = atomicAdd(L.f[lf].count, __popc(mine));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (edge && fi == lf) {
            const int64_t pos = (int64_t)base + __popc(mine & ((1u << lane) - 1u));
            if (pos < F.cap) F.edges[pos] = ((uint32_t)y << 16) | (uint32_t)x;
        }
        pending &= ~mine;
    }
}

}  // namespace

cudaError_t launch_canny(const CannyLaunch &L, int n_tiles, cudaStream_t s) {
    if (L.n <= 0) return cudaSuccess;
    canny_nms_kernel<<<n_tiles, kCannyThreads, 0, s>>>(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t blocks = (L.total_px + kPxThreads - 1) / kPxThreads;
    if (blocks > 0x7FFFFFFF) return cudaErrorInvalidValue;
    canny_union_kernel<<<(int)blocks, kPxThreads, 0, s>>>(L);
    canny_flatten_kernel<<<(int)blocks, kPxThreads, 0, s>>>(L);
    canny_emit_kernel<<<(int)blocks, kPxThreads, 0, s>>>(L);
    return cudaGetLastError();
}

int canny_tiles(int w, int h) { return ((w + kTile - 1) / kTile) * ((h + kTile - 1) / kTile); }

}  // namespace ld
