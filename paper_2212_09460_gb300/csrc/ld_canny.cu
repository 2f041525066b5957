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
//                        (two columns per thread as 16-bit lanes, a single
//                        barrier per row);
//                        writes the class map (0, 1 weak, 2 strong) and, for
//                        candidates only, parent[i] = i and strong[i] = 0.
//   canny_union_kernel   a thread per 16 pixels of a row (one 16-byte read of
//                        the classes) links the candidates run by run: along
//                        the run, to the left neighbour and to the runs above,
//                        so that every 8-neighbour pair joins one component of
//                        a union-find forest: lock-free linking of the larger
//                        root under the smaller with atomicCAS (parent[i] <= i
//                        always, so finding a root ends; a failed CAS means
//                        another link succeeded).
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

// A CTA of kRowsT threads covers kRowsOut output columns and kStrip output
// rows of one frame and walks down the rows.  Thread t holds columns
// x = X0 - 4 + 2t and x + 1 of the CTA's input window as the two 16-bit
// lanes of a word (low: x, high: x + 1).  The horizontal blur sums (<= 4080),
// the vertical blur sum with its rounding term (<= 65408), the Sobel
// smoothing (<= 1020) and the biased differences stay below 2^16 and never
// borrow, so one 32-bit add serves both columns.  Vertical neighbourhoods
// stay in registers (the last five horizontal sums, the last three blurred
// rows); horizontal ones go through shared-memory rows.  The stages are
// skewed by one step so that a step needs a single barrier: at step t (input
// row yi = Y0 - 4 + t) a thread publishes the input pair of row yi, the
// vertical Sobel parts of row yi - 4 and the magnitudes of row yi - 5, then
// after the barrier reads them back to form the blur of row yi - 2 (-> Sobel
// parts of row yi - 3), the magnitudes and sectors of row yi - 4, and the
// suppression of row yi - 6.  Shared rows are double-buffered (magnitudes: a
// ring of four) so that a step's writes never meet the previous step's reads.
constexpr int kRowsT = 128;
constexpr int kRowsOut = 2 * kRowsT - 8;
constexpr int kStrip = 64;

// Pixels (x, y) and (x + 1, y) as a 16-bit pair, zero outside the image (x
// even: 2-byte aligned, as the image and its pitch are 16-byte aligned).
__device__ __forceinline__ uint32_t load_pair(const CannyFrame &F, int x, int y) {
    if (y < 0 || y >= F.h || x < 0 || x >= F.w) return 0u;   // x even: x < 0 also puts x + 1 outside
    const uint8_t *q = F.img + (size_t)y * F.pitch + x;
    return x + 1 < F.w ? (uint32_t)*reinterpret_cast<const uint16_t *>(q) : (uint32_t)q[0];
}

// |gx| + |gy| from the biased Sobel sums (0 outside the image).
__device__ __forceinline__ int magnitude(uint32_t gxb, uint32_t gyb, bool inside) {
    return inside ? abs((int)gxb - 1024) + abs((int)gyb - 1024) : 0;
}

// Direction sector of a pixel from its biased Sobel sums: 0 along x, 2 along
// y, 1 and 3 the diagonals (gx gy > 0 and < 0).
__device__ __forceinline__ int sector(uint32_t gxb, uint32_t gyb) {
    const int gx = (int)gxb - 1024, gy = (int)gyb - 1024;
    const int ax = abs(gx), ay = abs(gy);   // <= 1020: the products below fit 32 bits
    if (ay * 65536 <= 27146 * ax) return 0;
    if (ay * 65536 >= 158218 * ax) return 2;
    return (gx > 0) == (gy > 0) ? 1 : 3;   // gx gy > 0 (neither is 0 here)
}

__global__ void __launch_bounds__(kRowsT) canny_nms_kernel(const __grid_constant__ CannyLaunch L) {
    __shared__ uint32_t Is[2][kRowsT + 2];    // input pairs, thread t at [1 + t]
    __shared__ uint32_t Vss[2][kRowsT + 2];   // smoothing pairs G(y-1) + 2 G(y) + G(y+1)
    __shared__ uint32_t Vds[2][kRowsT + 2];   // difference pairs G(y+1) - G(y-1) + 256
    __shared__ uint32_t Ms[4][kRowsT + 2];    // magnitude pairs of row y at [y & 3]
    const int fi = frame_of_tile(L, blockIdx.x);
    const CannyFrame &F = L.f[fi];
    const int local = blockIdx.x - F.tile_begin;
    const int w = F.w, h = F.h;
    const int bxs = (w + kRowsOut - 1) / kRowsOut;
    const int X0 = (local % bxs) * kRowsOut, Y0 = (local / bxs) * kStrip;
    const int t = threadIdx.x, x = X0 - 4 + 2 * t;
    const bool in0 = x >= 0 && x < w, in1 = x + 1 >= 0 && x + 1 < w;
    const uint32_t colmask = (in0 ? 0x0000FFFFu : 0u) | (in1 ? 0xFFFF0000u : 0u);
    // output columns: window columns 4 .. 2 kRowsT - 5, inside the image
    const bool out0 = t >= 2 && t < kRowsT - 2 && in0;
    const bool out1 = t >= 2 && t < kRowsT - 2 && in1;
    if (local == 0 && t == 0) {   // until the merge writes the frame's peaks
        if (F.status_init) *F.status_init = LD_ERR_TIMEOUT;
        if (F.npeaks_init) *F.npeaks_init = 0;
    }
    for (int i = t; i < 2 * (kRowsT + 2); i += kRowsT) {
        (&Is[0][0])[i] = 0u;
        (&Vss[0][0])[i] = 0u;
        (&Vds[0][0])[i] = 0u;
    }
    for (int i = t; i < 4 * (kRowsT + 2); i += kRowsT) (&Ms[0][0])[i] = 0u;
    __syncthreads();
    const int yend = min(Y0 + kStrip, h);
    const int T = yend - Y0 + 10;   // the last step suppresses row yend - 1
    uint32_t h0 = 0, h1 = 0, h2 = 0, h3 = 0, h4 = 0;   // horizontal blur pairs, rows yi-4 .. yi
    uint32_t g0 = 0, g1 = 0, g2 = 0;                    // blurred pairs, rows yi-4 .. yi-2
    uint32_t vs_pend = 0, vd_pend = 0, m_pend = 0;      // awaiting publication
    uint32_t gx1 = 0, gy1 = 0, gx2 = 0, gy2 = 0;        // biased Sobel sums of the last two steps
    uint32_t pf0 = load_pair(F, x, Y0 - 4), pf1 = load_pair(F, x, Y0 - 3);
    for (int s = 0; s < T; ++s) {
        const int yi = Y0 - 4 + s, b = s & 1;
        const uint32_t cur = pf0;
        pf0 = pf1;
        pf1 = load_pair(F, x, yi + 2);
        Is[b][1 + t] = cur;
        Vss[b][1 + t] = vs_pend;
        Vds[b][1 + t] = vd_pend;
        Ms[(yi - 5) & 3][1 + t] = m_pend;
        __syncthreads();
        // 5x5 binomial blur: horizontal sums of row yi from columns x-2 .. x+3
        const uint32_t xw = Is[b][t] | (Is[b][1 + t] << 16);   // I(x-2), I(x-1), I(x), I(x+1)
        const uint32_t rg = Is[b][2 + t];                        // I(x+2), I(x+3)
        const uint32_t A = __byte_perm(xw, 0u, 0x4140);   // [I(x-2), I(x-1)]
        const uint32_t B = __byte_perm(xw, 0u, 0x4241);   // [I(x-1), I(x)]
        const uint32_t C = __byte_perm(xw, 0u, 0x4342);   // [I(x),   I(x+1)]
        const uint32_t D = __byte_perm(xw, rg, 0x6463);   // [I(x+1), I(x+2)]
        const uint32_t E = __byte_perm(rg, 0u, 0x4140);   // [I(x+2), I(x+3)]
        h0 = h1; h1 = h2; h2 = h3; h3 = h4;
        h4 = A + E + 4u * (B + D) + 6u * C;
        const int yg = yi - 2;
        uint32_t g = ((h0 + h4 + 0x00800080u + 4u * (h1 + h3) + 6u * h2) >> 8) & 0x00FF00FFu;
        if (yg < 0 || yg >= h) g = 0u;
        g &= colmask;
        g0 = g1; g1 = g2; g2 = g;
        vs_pend = g0 + 2u * g1 + g2;
        vd_pend = g2 + 0x01000100u - g0;
        // magnitudes and sectors of row yi - 4 from the parts published this step
        const uint32_t so = Vss[b][1 + t], dd = Vds[b][1 + t];
        const uint32_t sr1 = __byte_perm(so, Vss[b][2 + t], 0x5432);   // [Vs(x+1), Vs(x+2)]
        const uint32_t sl1 = __byte_perm(Vss[b][t], so, 0x5432);       // [Vs(x-1), Vs(x)]
        const uint32_t dr1 = __byte_perm(dd, Vds[b][2 + t], 0x5432);
        const uint32_t dl1 = __byte_perm(Vds[b][t], dd, 0x5432);
        const uint32_t gxb = sr1 + 0x04000400u - sl1;   // gx + 1024 per lane
        const uint32_t gyb = dl1 + 2u * dd + dr1;      // gy + 1024 per lane (each part carries 256)
        const int ym = yi - 4;
        const bool yok = ym >= 0 && ym < h;
        m_pend = (uint32_t)magnitude(gxb & 0xFFFFu, gyb & 0xFFFFu, in0 && yok) |
                 ((uint32_t)magnitude(gxb >> 16, gyb >> 16, in1 && yok) << 16);
        // suppression of row yn = yi - 6 (its Sobel sums from two steps ago),
        // magnitude rows yn-1 .. yn+1; a pixel below t_low is never an edge
        const int yn = yi - 6;
        const uint32_t gxn = gx2, gyn = gy2;
        gx2 = gx1;
        gy2 = gy1;
        gx1 = gxb;
        gy1 = gyb;
        if (s >= 10) {
            const uint32_t mcp = Ms[yn & 3][1 + t];
            const size_t prow = (size_t)yn * w + x;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (!(k == 0 ? out0 : out1)) continue;
                const int mc = (int)((mcp >> (16 * k)) & 0xFFFFu);
                uint8_t cls = 0;
                if (mc >= L.t_low) {
                    const int sc = sector((gxn >> (16 * k)) & 0xFFFFu, (gyn >> (16 * k)) & 0xFFFFu);
                    const int col = 2 + 2 * t + k;   // 16-bit index in a row of Ms
                    // (n1, n2) per sector: along x (x-1, x+1); (x-1,y-1), (x+1,y+1); along y; (x+1,y-1), (x-1,y+1)
                    const int dx1 = sc == 0 ? -1 : sc == 1 ? -1 : sc == 2 ? 0 : 1;
                    const int dy1 = sc == 0 ? 0 : -1;
                    const int m1n = reinterpret_cast<const uint16_t *>(Ms[(yn + dy1) & 3])[col + dx1];
                    const int m2n = reinterpret_cast<const uint16_t *>(Ms[(yn - dy1) & 3])[col - dx1];
                    if (mc > m1n && mc >= m2n) cls = mc >= L.t_high ? 2 : 1;   // mc >= t_low >= 1 > 0
                }
                F.cls[prow + k] = cls;
                // the forest and the strong marks are initialised for candidates
                // only (nothing else reads them)
                if (cls) {
                    F.parent[prow + k] = (int32_t)(prow + k);
                    F.strong[prow + k] = 0;
                }
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

// Links by runs: in a chunk, a run of consecutive candidates is connected
// along the row, so each member is linked straight under the run's first
// pixel (independent compare-and-swaps, no root searches unless another link
// got there first); the first pixel then links to the left neighbour across
// the chunk border, and once to each run of candidates in the row above that
// touches the run's columns widened by one (any pixel of such a run is in
// its component).  Every 8-neighbour pair ends up in one component.
__global__ void __launch_bounds__(kPxThreads) canny_union_kernel(const __grid_constant__ CannyLaunch L) {
    const Chunk c = chunk_of(L, (int64_t)blockIdx.x * kPxThreads + threadIdx.x);
    if (!c.ok) return;
    const CannyFrame &F = *c.F;
    const int w = F.w;
    const uint8_t *row = F.cls + (size_t)c.y * w + c.x0;
    uint32_t cand, strong;
    load_cls16(row, c.n, &cand, &strong);
    if (!cand) return;
    const int p0 = c.y * w + c.x0;   // pixel of bit 0
    // the row above, columns x0 - 1 .. x0 + 16 as bits 0 .. 17
    uint32_t up = 0;
    if (c.y > 0) {
        const uint8_t *ur = row - w;
        uint32_t uc, us;
        load_cls16(ur, c.n, &uc, &us);
        up = uc << 1;
        if (c.x0 > 0 && ur[-1]) up |= 1u;
        if (c.n == 16 && c.x0 + 16 < w && ur[16]) up |= 1u << 17;
    }
    const int pu = p0 - w - 1;   // pixel of bit 0 of `up`
    uint32_t m = cand;
    while (m) {
        const int a = __ffs(m) - 1;
        const int len = __ffs(~(m >> a)) - 1;   // the run: bits a .. a + len - 1
        const int b = a + len - 1;
        m &= ~(((1u << len) - 1u) << a);
        const int s0 = p0 + a;
        for (int i = a + 1; i <= b; ++i) {
            const int q = p0 + i;
            if (atomicCAS(F.parent + q, q, s0) != q) unite(F.parent, q, s0);
        }
        if (a == 0 && c.x0 > 0 && row[-1]) unite(F.parent, s0, s0 - 1);
        uint32_t mu = up & ((1u << (b + 3)) - 1u) & ~((1u << a) - 1u);   // columns a - 1 .. b + 1
        while (mu) {
            const int j = __ffs(mu) - 1;
            const int lu = __ffs(~(mu >> j)) - 1;
            mu &= ~(((1u << lu) - 1u) << j);
            unite(F.parent, s0, pu + j);
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
    canny_nms_kernel<<<n_tiles, kRowsT, 0, s>>>(L);
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
