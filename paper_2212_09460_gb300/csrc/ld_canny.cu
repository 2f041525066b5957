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
//   canny_nms_kernel     stages 1-4 in one pass down a strip of rows per CTA
//                        (one thread per column, a single barrier per row);
//                        writes the class map (0, 1 weak, 2 strong) and, for
//                        candidates only, parent[i] = i and strong[i] = 0.
//   canny_union_kernel   a thread per 16 pixels of a row (one 16-byte read of
//                        the classes) joins each candidate to its candidate
//                        neighbours above and to the left (each
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

constexpr int kPxThreads = 256;

// Root of i's tree, halving the path on the way: a node that is not a root
// is pointed at its grandparent.  A root is the smallest index of its tree
// (links put the larger root under the smaller), and the halving writes are
// minima with an ancestor, so a pointer only ever moves up its own tree and
// never past the root: concurrent links, halvings and the flatten's writes
// of roots all keep every node in its tree, and a root written by the
// flatten stays.
__device__ __forceinline__ int find_root(int32_t *parent, int i) {
    for (;;) {
        const int p = __ldcg(parent + i);
        if (p == i) return i;
        const int gp = __ldcg(parent + p);
        if (gp == p) return p;
        atomicMin(parent + i, gp);
        i = gp;
    }
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

// A CTA covers kRowsOut output columns and kStrip output rows of one frame
// with one thread per column of its kRowsW-wide input window (x = X0 - 4 + c)
// and walks down the rows.  Vertical neighbourhoods stay in registers (the
// last five horizontal blur sums, the last three blurred rows); horizontal
// ones go through shared memory rows.  The stages are skewed by one step so
// that a step needs a single barrier: at step t (input row yi = Y0 - 4 + t)
// a thread publishes the input pixel of row yi, the vertical Sobel parts of
// row yi - 4 and the magnitude of row yi - 5, then after the barrier reads
// them back to form the blur of row yi - 2 (-> Sobel parts of row yi - 3),
// the magnitude and sector of row yi - 4, and the suppression of row yi - 6.
// Shared rows are double-buffered (magnitudes: a ring of four) so that a
// step's writes never meet the previous step's reads.
constexpr int kRowsW = 128;
constexpr int kRowsOut = kRowsW - 8;
constexpr int kStrip = 64;

__device__ __forceinline__ int load_px(const CannyFrame &F, int x, bool xin, int y) {
    return (xin && y >= 0 && y < F.h) ? (int)F.img[(size_t)y * F.pitch + x] : 0;
}

__global__ void __launch_bounds__(kRowsW) canny_nms_kernel(const __grid_constant__ CannyLaunch L) {
    __shared__ uint8_t Is[2][kRowsW + 4];    // input row, column c at [2 + c]
    __shared__ uint32_t Vs[2][kRowsW + 2];   // Sobel parts, column c at [1 + c]
    __shared__ int16_t Ms[4][kRowsW + 2];    // magnitude rows y at [y & 3], column c at [1 + c]
    const int fi = frame_of_tile(L, blockIdx.x);
    const CannyFrame &F = L.f[fi];
    const int local = blockIdx.x - F.tile_begin;
    const int w = F.w, h = F.h;
    const int bxs = (w + kRowsOut - 1) / kRowsOut;
    const int X0 = (local % bxs) * kRowsOut, Y0 = (local / bxs) * kStrip;
    const int c = threadIdx.x, x = X0 - 4 + c;
    const bool xin = x >= 0 && x < w;
    const bool out_col = c >= 4 && c < kRowsW - 4 && x < w;
    if (local == 0 && c == 0) {   // until the merge writes the frame's peaks
        if (F.status_init) *F.status_init = LD_ERR_TIMEOUT;
        if (F.npeaks_init) *F.npeaks_init = 0;
    }
    for (int i = c; i < 2 * (kRowsW + 4); i += kRowsW) (&Is[0][0])[i] = 0;
    for (int i = c; i < 2 * (kRowsW + 2); i += kRowsW) (&Vs[0][0])[i] = 0;
    for (int i = c; i < 4 * (kRowsW + 2); i += kRowsW) (&Ms[0][0])[i] = 0;
    __syncthreads();
    const int yend = min(Y0 + kStrip, h);
    const int T = yend - Y0 + 10;   // the last step suppresses row yend - 1
    int h0 = 0, h1 = 0, h2 = 0, h3 = 0, h4 = 0;   // horizontal blur sums, rows yi-4 .. yi
    int g0 = 0, g1 = 0, g2 = 0;                    // blurred rows yi-4 .. yi-2
    uint32_t vpend = 0;                            // Sobel parts awaiting publication
    int mpend = 0, sc1 = 0, sc2 = 0;               // magnitude awaiting publication; sectors of the last two steps
    int pf0 = load_px(F, x, xin, Y0 - 4), pf1 = load_px(F, x, xin, Y0 - 3);
    for (int t = 0; t < T; ++t) {
        const int yi = Y0 - 4 + t, b = t & 1;
        const int cur = pf0;
        pf0 = pf1;
        pf1 = load_px(F, x, xin, yi + 2);
        Is[b][2 + c] = (uint8_t)cur;
        Vs[b][1 + c] = vpend;
        Ms[(yi - 5) & 3][1 + c] = (int16_t)mpend;
        __syncthreads();
        // 5x5 binomial blur: horizontal sum of row yi, vertical over the last five
        const uint8_t *q = Is[b] + c;   // columns c - 2 .. c + 2
        const int hn = q[0] + 4 * q[1] + 6 * q[2] + 4 * q[3] + q[4];
        h0 = h1; h1 = h2; h2 = h3; h3 = h4; h4 = hn;
        const int yg = yi - 2;
        int gn = (h0 + 4 * h1 + 6 * h2 + 4 * h3 + h4 + 128) >> 8;
        if (!xin || yg < 0 || yg >= h) gn = 0;
        g0 = g1; g1 = g2; g2 = gn;
        // Sobel parts of row yi - 3 at this column: smoothing G(y-1) + 2 G(y) + G(y+1)
        // (low half) and difference G(y+1) - G(y-1) + 256 (high half)
        vpend = (uint32_t)(g0 + 2 * g1 + g2) | ((uint32_t)(g2 - g0 + 256) << 16);
        // magnitude and sector of row yi - 4 from the parts published this step
        const uint32_t va = Vs[b][c], vb = Vs[b][c + 1], vc = Vs[b][c + 2];
        const int gx = (int)(vc & 0xFFFFu) - (int)(va & 0xFFFFu);
        const int gy = (int)(va >> 16) + 2 * (int)(vb >> 16) + (int)(vc >> 16) - 4 * 256;
        const int ym = yi - 4;
        int m = 0, sc = 0;
        if (xin && ym >= 0 && ym < h) {
            const int ax = abs(gx), ay = abs(gy);   // <= 1020: the products below fit 32 bits
            m = ax + ay;
            if (ay * 65536 <= 27146 * ax) sc = 0;
            else if (ay * 65536 >= 158218 * ax) sc = 2;
            else sc = (gx > 0) == (gy > 0) ? 1 : 3;   // gx gy > 0 (neither is 0 here)
        }
        mpend = m;
        // suppression of row yn = yi - 6 (sector from two steps ago), magnitude rows yn-1 .. yn+1
        const int yn = yi - 6, scn = sc2;
        sc2 = sc1;
        sc1 = sc;
        if (t >= 10 && out_col) {
            // (n1, n2) per sector: along x (x-1, x+1); (x-1,y-1), (x+1,y+1); along y; (x+1,y-1), (x-1,y+1)
            const int dx1 = scn == 0 ? -1 : scn == 1 ? -1 : scn == 2 ? 0 : 1;
            const int dy1 = scn == 0 ? 0 : -1;
            const int mc = Ms[yn & 3][1 + c];
            const int m1 = Ms[(yn + dy1) & 3][1 + c + dx1], m2 = Ms[(yn - dy1) & 3][1 + c - dx1];
            const bool keep = mc > 0 && mc > m1 && mc >= m2;
            const uint8_t cls = !keep ? 0 : (mc >= L.t_high ? 2 : (mc >= L.t_low ? 1 : 0));
            // the forest and the strong marks are initialised for candidates only
            // (nothing else reads them)
            const int p = yn * w + x;
            F.cls[p] = cls;
            if (cls) {
                F.parent[p] = p;
                F.strong[p] = 0;
            }
        }
    }
}

// Per-pixel kernels: a thread takes 16 consecutive pixels of a row (chunk
// q of the launch: the frame by its first chunk, then the row and column).
struct Chunk {
    const CannyFrame *F;
    int y, x0, n;   // pixels x0 .. x0 + n - 1 of row y
    bool ok;
};

__device__ __forceinline__ Chunk chunk_of(const CannyLaunch &L, int64_t q) {
    Chunk c;
    c.ok = false;
    if (q >= L.total_chunks) return c;
    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.f[mid].chunk_begin <= q) lo = mid; else hi = mid - 1;
    }
    c.F = &L.f[lo];
    const int cpr = (c.F->w + 15) >> 4;
    const int64_t local = q - c.F->chunk_begin;
    c.y = (int)(local / cpr);
    c.x0 = (int)(local - (int64_t)c.y * cpr) * 16;
    c.n = min(16, c.F->w - c.x0);
    c.ok = true;
    return c;
}

// The classes of a chunk's n <= 16 pixels as bit masks: bit i of *cand for a
// candidate (weak or strong), of *strong for a strong pixel.
__device__ __forceinline__ void load_cls16(const uint8_t *cls, int n, uint32_t *cand, uint32_t *strong) {
    uint32_t v[4];
    if (n == 16 && (reinterpret_cast<uintptr_t>(cls) & 15) == 0) {
        const uint4 q = __ldg(reinterpret_cast<const uint4 *>(cls));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t word = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b)
                if (4 * k + b < n) word |= (uint32_t)cls[4 * k + b] << (8 * b);
            v[k] = word;
        }
    }
    uint32_t c = 0, st = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint32_t byte = (v[k] >> (8 * b)) & 0xFFu;
            c |= (byte != 0 ? 1u : 0u) << (4 * k + b);
            st |= (byte == 2 ? 1u : 0u) << (4 * k + b);
        }
    *cand = c;
    *strong = st;
}

__global__ void __launch_bounds__(kPxThreads) canny_union_kernel(const __grid_constant__ CannyLaunch L) {
    const Chunk c = chunk_of(L, (int64_t)blockIdx.x * kPxThreads + threadIdx.x);
    if (!c.ok) return;
    const CannyFrame &F = *c.F;
    const int w = F.w;
    const uint8_t *row = F.cls + (size_t)c.y * w + c.x0;
    uint32_t cand, strong;
    load_cls16(row, c.n, &cand, &strong);
    // left neighbour of each pixel is a candidate (bit 0: the previous chunk's last pixel)
    const uint32_t left = (cand << 1) | ((c.x0 > 0 && row[-1]) ? 1u : 0u);
    uint32_t m = cand;
    while (m) {
        const int i = __ffs(m) - 1;
        m &= m - 1;
        const int x = c.x0 + i, p = c.y * w + x;
        // the neighbours that come earlier in raster order: each 8-neighbour pair once
        if ((left >> i) & 1u) unite(F.parent, p, p - 1);
        if (c.y > 0) {
            const int u = p - w;
            if (x > 0 && F.cls[u - 1]) unite(F.parent, p, u - 1);
            if (F.cls[u]) unite(F.parent, p, u);
            if (x + 1 < w && F.cls[u + 1]) unite(F.parent, p, u + 1);
        }
    }
}

__global__ void __launch_bounds__(kPxThreads) canny_flatten_kernel(const __grid_constant__ CannyLaunch L) {
    const Chunk c = chunk_of(L, (int64_t)blockIdx.x * kPxThreads + threadIdx.x);
    if (!c.ok) return;
    const CannyFrame &F = *c.F;
    uint32_t cand, strong;
    load_cls16(F.cls + (size_t)c.y * F.w + c.x0, c.n, &cand, &strong);
    uint32_t m = cand;
    while (m) {
        const int i = __ffs(m) - 1;
        m &= m - 1;
        const int p = c.y * F.w + c.x0 + i;
        const int r = find_root(F.parent, p);
        F.parent[p] = r;
        if ((strong >> i) & 1u) F.strong[r] = 1;
    }
}

__global__ void __launch_bounds__(kPxThreads) canny_emit_kernel(const __grid_constant__ CannyLaunch L) {
    const int lane = threadIdx.x & 31;
    const Chunk c = chunk_of(L, (int64_t)blockIdx.x * kPxThreads + threadIdx.x);
    uint32_t mask = 0;
    int fi = -1;
    if (c.ok) {
        const CannyFrame &F = *c.F;
        fi = (int)(c.F - L.f);
        uint32_t cand, strong;
        load_cls16(F.cls + (size_t)c.y * F.w + c.x0, c.n, &cand, &strong);
        while (cand) {
            const int i = __ffs(cand) - 1;
            cand &= cand - 1;
            const int p = c.y * F.w + c.x0 + i;
            if (F.strong[__ldcg(F.parent + p)]) mask |= 1u << i;
        }
        if (L.border == LD_BORDER_CLEAR) {
            if (c.y == 0 || c.y == F.h - 1) mask = 0;
            if (c.x0 == 0) mask &= ~1u;
            const int xr = F.w - 1 - c.x0;
            if (xr < 16) mask &= ~(1u << xr);
        }
        if (F.bin) {
            uint8_t *b = F.bin + (size_t)c.y * F.pitch + c.x0;
            if (c.n == 16) {   // a whole aligned chunk (pitch and buffer 16-byte aligned)
                uint32_t v4[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t nib = (mask >> (4 * k)) & 0xFu;
                    // spread the 4 bits to bytes of 0x00 / 0xFF
                    v4[k] = ((nib & 1u) ? 0xFFu : 0u) | ((nib & 2u) ? 0xFF00u : 0u) |
                            ((nib & 4u) ? 0xFF0000u : 0u) | ((nib & 8u) ? 0xFF000000u : 0u);
                }
                *reinterpret_cast<uint4 *>(b) = make_uint4(v4[0], v4[1], v4[2], v4[3]);
            } else {
                for (int i = 0; i < c.n; ++i) b[i] = (mask >> i) & 1u ? 255 : 0;
            }
        }
    }
    // one atomic per frame present in the warp, the lanes' edges in slot order
    uint32_t pending = __ballot_sync(0xFFFFFFFFu, mask != 0);
    while (pending) {
        const int leader = __ffs(pending) - 1;
        const int lf = __shfl_sync(0xFFFFFFFFu, fi, leader);
        const bool mine = mask != 0 && fi == lf;
        const int cnt = mine ? __popc(mask) : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += t;
        }
        const int tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
        int base = 0;
        if (lane == leader) base = atomicAdd(L.f[lf].count, tot);
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (mine) {
            const CannyFrame &F = L.f[lf];
            int64_t pos = (int64_t)base + incl - cnt;
            uint32_t m = mask;
            while (m) {
                const int i = __ffs(m) - 1;
                m &= m - 1;
                if (pos < F.cap) F.edges[pos] = ((uint32_t)c.y << 16) | (uint32_t)(c.x0 + i);
                ++pos;
            }
        }
        pending &= ~__ballot_sync(0xFFFFFFFFu, mine);
    }
}

}  // namespace

cudaError_t launch_canny(const CannyLaunch &L0, int n_tiles, cudaStream_t s) {
    if (L0.n <= 0) return cudaSuccess;
    CannyLaunch L = L0;
    int64_t chunks = 0;
    for (int k = 0; k < L.n; ++k) {
        L.f[k].chunk_begin = chunks;
        chunks += (int64_t)L.f[k].h * ((L.f[k].w + 15) / 16);
    }
    L.total_chunks = chunks;
    canny_nms_kernel<<<n_tiles, kRowsW, 0, s>>>(L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t blocks = (L.total_chunks + kPxThreads - 1) / kPxThreads;
    if (blocks > 0x7FFFFFFF) return cudaErrorInvalidValue;
    canny_union_kernel<<<(int)blocks, kPxThreads, 0, s>>>(L);
    canny_flatten_kernel<<<(int)blocks, kPxThreads, 0, s>>>(L);
    canny_emit_kernel<<<(int)blocks, kPxThreads, 0, s>>>(L);
    return cudaGetLastError();
}

int canny_tiles(int w, int h) { return ((w + kRowsOut - 1) / kRowsOut) * ((h + kStrip - 1) / kStrip); }

}  // namespace ld
