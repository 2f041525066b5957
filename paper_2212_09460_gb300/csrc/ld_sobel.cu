// ld_sobel.cu -- Steps 1-2 fused: Sobel |Gx|+|Gy| on the zero-padded image
// (Sec. 2.1 Eq. 1, Sec. 3.1, Sec. 4.1), binarization against the threshold
// (Sec. 2.2, Sec. 4.2), and compaction of the 255 pixels into the packed
// (y << 16) | x edge list the voting stage reads (Sec. 4.3).
//
// GB300 design (differs from the paper's 16x16-thread-block K80 kernel,
// Eq. 6): one warp covers 512 contiguous pixels of a row with one 16-byte
// load per lane, so every row is read with fully coalesced 512-byte warp
// transactions.  A warp issues the loads of all R + 2 rows of its strip
// (R output rows plus two halo rows) before computing, so that many bytes
// are in flight per SM, then slides the 3x3 window down in registers; the
// left/right neighbour bytes come from the adjacent lanes through shuffles,
// and zero padding is virtual (never materialised).  Edge bits are compacted with a
// block-wide prefix sum and one global atomic per CTA.
#include "ld_internal.cuh"

namespace ld {
namespace {

struct Row {
    uint32_t v[4];   // 16 pixels
    uint32_t l, r;   // pixel x0-1 and x0+16
};

__device__ __forceinline__ uint4 ldg_nc_v4(const void *p) {
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

// The 16 pixels of row y starting at x0 as one 16-byte vector; pixels
// outside the image (x >= w, y outside [0, h)) read as 0.
__device__ __forceinline__ uint4 load_vec(const SobelFrame &F, int x0, int y) {
    uint4 q = make_uint4(0, 0, 0, 0);
    if (y >= 0 && y < F.h && x0 < F.w) {
        q = ldg_nc_v4(F.img + (size_t)y * F.pitch + x0);
        const int nvalid = F.w - x0;
        if (nvalid < 16) {
            uint32_t *v = reinterpret_cast<uint32_t *>(&q);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int k = nvalid - 4 * i;
                v[i] &= k >= 4 ? 0xFFFFFFFFu : (k <= 0 ? 0u : ((1u << (8 * k)) - 1u));
            }
        }
    }
    return q;
}

// Pixel x0-1 (lane 0) or x0+16 (lane 31) of row y, 0 outside the image.
__device__ __forceinline__ uint32_t load_edge_byte(const SobelFrame &F, int x, int y) {
    return (y >= 0 && y < F.h && x >= 0 && x < F.w) ? (uint32_t)F.img[(size_t)y * F.pitch + x] : 0u;
}

// Assemble a row from its vector and the neighbour bytes, which come from
// the adjacent lanes (lanes 0 and 31 use the bytes they loaded themselves).
// All 32 lanes of the warp must call this (shuffles).
__device__ __forceinline__ Row make_row(uint4 q, uint32_t own_l, uint32_t own_r, int lane) {
    Row R;
    R.v[0] = q.x; R.v[1] = q.y; R.v[2] = q.z; R.v[3] = q.w;
    uint32_t left = __shfl_up_sync(0xFFFFFFFFu, q.w >> 24, 1);
    uint32_t right = __shfl_down_sync(0xFFFFFFFFu, q.x & 0xFFu, 1);
    R.l = (lane == 0) ? own_l : left;
    R.r = (lane == 31) ? own_r : right;
    return R;
}

// A row in 16-bit lanes: E[k] = pixels (4k, 4k+2), O[k] = pixels (4k+1, 4k+3)
// of the lane's 16, plus the neighbour pixels x0-1 (l) and x0+16 (r).
struct URow {
    uint32_t E[4], O[4];
    uint32_t l, r;
};

__device__ __forceinline__ URow unpack(const Row &R) {
    URow U;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        U.E[k] = __byte_perm(R.v[k], 0u, 0x4240);   // bytes 0, 2 -> lanes 0, 1
        U.O[k] = __byte_perm(R.v[k], 0u, 0x4341);   // bytes 1, 3
    }
    U.l = R.l;
    U.r = R.r;
    return U;
}

// Eq. 1 and the threshold for the 16 pixels of the middle row, two pixels per
// 32-bit operation (16-bit lanes, every lane kept non-negative by a bias so
// no borrow crosses lanes):
//   S = T + 2M + B (vertical smoothing), D = B - T + 255,
//   gx(x) = S(x+1) - S(x-1),  gy(x) = D(x-1) + 2D(x) + D(x+1) - 1020,
//   |gx| + |gy| = max(|gx + gy|, |gx - gy|), tested against thr with four
//   compares whose result lands in bit 15 of each lane.
// Returns bit i set iff |Gx| + |Gy| >= thr at pixel x0 + i.
__device__ __forceinline__ uint32_t sobel16(const URow &T, const URow &M, const URow &B, uint32_t thr) {
    uint32_t SE[5], SO[5], DE[5], DO[5];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        SE[k] = T.E[k] + B.E[k] + 2u * M.E[k];
        SO[k] = T.O[k] + B.O[k] + 2u * M.O[k];
        DE[k] = B.E[k] + 0x00FF00FFu - T.E[k];
        DO[k] = B.O[k] + 0x00FF00FFu - T.O[k];
    }
    // neighbours: S(-1), D(-1) in the high lane of index "-1" (stored at [4] of
    // the odd arrays), S(16), D(16) in the low lane of index 4 of the even arrays
    const uint32_t sl = T.l + B.l + 2u * M.l, dl = B.l + 255u - T.l;
    const uint32_t sr = T.r + B.r + 2u * M.r, dr = B.r + 255u - T.r;
    SE[4] = sr;
    DE[4] = dr;
    SO[4] = sl << 16;
    DO[4] = dl << 16;
    const uint32_t K1 = (0x8000u - 2040u - thr) * 0x10001u;
    const uint32_t K2 = (0x8000u + 2040u - thr) * 0x10001u;
    uint32_t bits = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t sOm = __funnelshift_l(SO[k == 0 ? 4 : k - 1], SO[k], 16);   // S(4k-1), S(4k+1)
        const uint32_t dOm = __funnelshift_l(DO[k == 0 ? 4 : k - 1], DO[k], 16);
        const uint32_t sEp = __funnelshift_r(SE[k], SE[k + 1], 16);               // S(4k+2), S(4k+4)
        const uint32_t dEp = __funnelshift_r(DE[k], DE[k + 1], 16);
        // biased by 1020 per lane, in [0, 2040]
        const uint32_t gxE = SO[k] + 0x03FC03FCu - sOm;   // pixels 4k, 4k+2
        const uint32_t gxO = sEp + 0x03FC03FCu - SE[k];   // pixels 4k+1, 4k+3
        const uint32_t gyE = dOm + 2u * DE[k] + DO[k];
        const uint32_t gyO = DE[k] + 2u * DO[k] + dEp;
        uint32_t t[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t G = h ? gxO : gxE, Hh = h ? gyO : gyE;
            const uint32_t s1 = G + Hh;                     // gx + gy + 2040
            const uint32_t s2 = G + 0x07F807F8u - Hh;       // gx - gy + 2040
            t[h] = ((s1 + K1) | (K2 - s1) | (s2 + K1) | (K2 - s2)) & 0x80008000u;
        }
        // bit 14: pixel 4k, 15: 4k+1, 30: 4k+2, 31: 4k+3
        const uint32_t w = (t[0] >> 1) | t[1];
        bits |= ((w >> 14) & 3u) << (4 * k);
        bits |= ((w >> 28) & 12u) << (4 * k);
    }
    return bits;
}

// 4 mask bits -> 4 bytes of 0x00 / 0xFF.
__device__ __forceinline__ uint32_t spread4(uint32_t nib) {
    return ((nib * 0x00204081u) & 0x01010101u) * 0xFFu;
}

template <int R>
__global__ void __launch_bounds__(kSobelThreads)
sobel_bin_edges_kernel(const __grid_constant__ SobelLaunch L) {
    // frame of this CTA (binary search over tile_begin)
    const int t = blockIdx.x;
    int lo = 0, hi = L.n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (L.f[mid].tile_begin <= t) lo = mid; else hi = mid - 1;
    }
    const SobelFrame &F = L.f[lo];
    const int local = t - F.tile_begin;
    if (local == 0 && threadIdx.x == 0) {   // until the merge writes the frame's peaks
        if (F.status_init) *F.status_init = LD_ERR_TIMEOUT;
        if (F.npeaks_init) *F.npeaks_init = 0;
    }
    const int tx = local % F.tiles_x, ty = local / F.tiles_x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = tx * kSobelTileW + lane * 16;
    const int ya = ty * (R * (kSobelThreads / 32)) + warp * R;

    // valid-column mask of this lane's 16 pixels
    uint32_t colmask = 0;
    if (x0 < F.w) colmask = (F.w - x0 >= 16) ? 0xFFFFu : ((1u << (F.w - x0)) - 1u);
    if (L.border == LD_BORDER_CLEAR) {
        if (x0 == 0) colmask &= ~1u;
        int xr = F.w - 1 - x0;
        if (xr >= 0 && xr < 16) colmask &= ~(1u << xr);
    }

    uint32_t masks[R];
#pragma unroll
    for (int r = 0; r < R; ++r) masks[r] = 0;

    if (ya < F.h) {   // warp-uniform
        // issue every load of the strip first (R + 2 rows), then compute
        uint4 raw[R + 2];
        uint32_t eb[R + 2];
#pragma unroll
        for (int j = 0; j < R + 2; ++j) raw[j] = load_vec(F, x0, ya - 1 + j);
#pragma unroll
        for (int j = 0; j < R + 2; ++j)
            eb[j] = (lane == 0) ? load_edge_byte(F, x0 - 1, ya - 1 + j)
                                : ((lane == 31) ? load_edge_byte(F, x0 + 16, ya - 1 + j) : 0u);
        URow top = unpack(make_row(raw[0], eb[0], eb[0], lane));
        URow mid = unpack(make_row(raw[1], eb[1], eb[1], lane));
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = ya + r;
            URow bot = unpack(make_row(raw[r + 2], eb[r + 2], eb[r + 2], lane));
            uint32_t bits = (y < F.h) ? (sobel16(top, mid, bot, (uint32_t)L.threshold) & colmask) : 0u;
            if (L.border == LD_BORDER_CLEAR && (y == 0 || y == F.h - 1)) bits = 0;
            masks[r] = bits;
            if (F.bin != nullptr && x0 < F.pitch && y < F.h) {
                uint4 o;
                o.x = spread4(bits & 0xF);
                o.y = spread4((bits >> 4) & 0xF);
                o.z = spread4((bits >> 8) & 0xF);
                o.w = spread4((bits >> 12) & 0xF);
                *reinterpret_cast<uint4 *>(F.bin + (size_t)y * F.pitch + x0) = o;
            }
            top = mid;
            mid = bot;
        }
    }

    // 8x8 edge-count pool: the CTA's tile (512 px x 8R rows) is a whole number
    // of 8x8 blocks, so each block is counted in this CTA's shared memory and
    // written once.  A warp's R rows lie in one 8-row block (ya is a multiple of
    // R, R divides 8); a lane's 16 pixels are 2 blocks.
    __shared__ uint32_t pool_s[R][kSobelTileW / 8];
    if (F.pool != nullptr) {
        for (int i = threadIdx.x; i < R * (kSobelTileW / 8); i += kSobelThreads) (&pool_s[0][0])[i] = 0;
        __syncthreads();
        if (ya < F.h && x0 < F.w) {
            uint32_t c0 = 0, c1 = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                c0 += __popc(masks[r] & 0xFFu);
                c1 += __popc(masks[r] >> 8);
            }
            const int br = (warp * R) >> 3;
            if (c0) atomicAdd(&pool_s[br][lane * 2], c0);
            if (c1) atomicAdd(&pool_s[br][lane * 2 + 1], c1);
        }
        __syncthreads();
        const int pw = (F.w + 7) >> 3, ph = (F.h + 7) >> 3;
        const int bx0 = tx * (kSobelTileW / 8), by0 = (ty * R * (kSobelThreads / 32)) >> 3;
        for (int i = threadIdx.x; i < R * (kSobelTileW / 8); i += kSobelThreads) {
            const int br = i / (kSobelTileW / 8), bc = i % (kSobelTileW / 8);
            if (by0 + br < ph && bx0 + bc < pw) F.pool[(size_t)(by0 + br) * pw + bx0 + bc] = (uint8_t)pool_s[br][bc];
        }
    }

    // block-wide exclusive prefix of the edge counts, one atomic per CTA
    int cnt = 0;
#pragma unroll
    for (int r = 0; r < R; ++r) cnt += __popc(masks[r]);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    __shared__ int warp_tot[kSobelThreads / 32];
    __shared__ int cta_base;
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < kSobelThreads / 32; ++w) {
            int v = warp_tot[w];
            warp_tot[w] = tot;
            tot += v;
        }
        cta_base = tot ? atomicAdd(F.count, tot) : 0;
    }
    __syncthreads();
    int64_t pos = (int64_t)cta_base + warp_tot[warp] + (incl - cnt);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        uint32_t bits = masks[r];
        const uint32_t yy = (uint32_t)(ya + r) << 16;
        while (bits) {
            int i = __ffs(bits) - 1;
            bits &= bits - 1;
            if (pos < F.cap) F.edges[pos] = yy | (uint32_t)(x0 + i);
            ++pos;
        }
    }
}

}  // namespace

cudaError_t launch_sobel(const SobelLaunch &L, int n_ctas, cudaStream_t s) {
    if (n_ctas <= 0) return cudaSuccess;
    switch (L.rows_per_warp) {
        case 2: sobel_bin_edges_kernel<2><<<n_ctas, kSobelThreads, 0, s>>>(L); break;
        case 4: sobel_bin_edges_kernel<4><<<n_ctas, kSobelThreads, 0, s>>>(L); break;
        case 8: sobel_bin_edges_kernel<8><<<n_ctas, kSobelThreads, 0, s>>>(L); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace ld
