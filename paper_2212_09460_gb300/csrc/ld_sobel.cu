// ld_sobel.cu -- Steps 1-2 fused: Sobel |Gx|+|Gy| on the zero-padded image
// (Sec. 2.1 Eq. 1, Sec. 3.1, Sec. 4.1), binarization against the threshold
// (Sec. 2.2, Sec. 4.2), and compaction of the 255 pixels into the packed
// (y << 16) | x edge list the voting stage reads (Sec. 4.3).
//
// Arithmetic.  With T, M, B the rows above, at and below the pixel, let
// P = M + B and Q = T + M per column, and SP(x) = P(x) + P(x+1), SQ(x) =
// Q(x) + Q(x+1) their horizontal pair sums.  The Sobel components are
// gx = (P+Q)(x+1) - (P+Q)(x-1) and gy = (B-T)(x-1) + 2(B-T)(x) + (B-T)(x+1),
// and with B - T = P - Q:
//   gx + gy = 2 [SP(x) - SQ(x-1)] = 2u,
//   gy - gx = 2 [SP(x-1) - SQ(x)] = 2w,
// so |Gx| + |Gy| = max(|gx + gy|, |gx - gy|) = 2 max(|u|, |w|), and for a
// threshold T in [1, 255] the saturated magnitude min(|Gx|+|Gy|, 255) >= T
// exactly when max(|u|, |w|) >= ceil(T/2).  Q of a row is P of the row above,
// so SQ is the previous row's SP: a row costs one P, one SP, u and w.
//
// Every quantity is an integer of magnitude < 2048, computed exactly in
// fp16x2 in units of 2^-24: the fp16 numbers k * 2^-24 for |k| < 2048 are
// exactly the subnormals and the lowest normal binade, spaced 2^-24 apart,
// and the bit pattern of k * 2^-24 (k >= 0) is k itself.  So a pixel byte
// placed in the low byte of a half is its value, sums and differences are
// exact (no flush to zero: the instructions carry no .ftz), and the edge
// flags are accumulated into bit masks by fused multiply-adds with weights
// 2^j units.  Two pixels per instruction, on the fp16 pipe.
//
// Layout.  A lane holds 16 pixels of a row; its 32-bit word j (j = 0..7)
// holds pixels (j, j + 8) as a half pair, so the x+1 and x-1 neighbours of
// word j are the words j+1 and j-1, and only the words at the lane's ends
// need the adjacent lanes (one shuffle each way per row).  A warp loads 512
// contiguous bytes per row (16-byte copies, fully coalesced) and produces the
// middle 480 pixels: lanes 0 and 31 only supply the left and right halo.  A
// warp slides down a run of 8*G rows, prefetching 6 rows ahead into shared
// memory (cp.async).  Zero padding is virtual: loads outside the image read 0.
//
// Compaction.  Every 8 rows a lane holds its edge flags as four 32-bit words
// (bits 0-15: pixels 0-15 of rows 2k, bits 16-31: of rows 2k+1).  Edges
// cluster (the 3x3 ring around a salt pixel, the sides of a lane stripe), so a
// lane that extracted its own pixels' edges would leave the rest of the warp
// waiting.  Instead each 32 x 32 bit matrix of a word across the warp is
// transposed with five shuffle-xor steps: lane l then holds pixel l % 16 of
// rows 2k + l / 16 of all 32 lanes' segments, which spreads every cluster over
// several lanes.  A warp prefix sum and one atomic on the frame's counter give
// each lane its slots; the lanes write their edges into per-warp staging slots
// that the warp copies out with coalesced stores.
#include <algorithm>

#include "ld_internal.cuh"

namespace ld {
namespace {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr int kStage = 1024;   // edge staging slots per warp (one 8-row group)

__device__ __forceinline__ uint32_t h2_add(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t h2_sub(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
// acc + (max(|u|, |w|) >= tau ? wt : 0), per half.
__device__ __forceinline__ uint32_t h2_edge_acc(uint32_t u, uint32_t w, uint32_t tau, uint32_t wt, uint32_t acc) {
    uint32_t au, aw, m, c, d;
    asm("abs.f16x2 %0, %1;" : "=r"(au) : "r"(u));
    asm("abs.f16x2 %0, %1;" : "=r"(aw) : "r"(w));
    asm("max.f16x2 %0, %1, %2;" : "=r"(m) : "r"(au), "r"(aw));
    asm("set.ge.f16x2.f16x2 %0, %1, %2;" : "=r"(c) : "r"(m), "r"(tau));   // 1.0 or 0.0
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(c), "r"(wt), "r"(acc));
    return d;
}

// Row prefetch through shared memory: each lane copies its own 16 bytes of
// a row with cp.async (zero-filled beyond the image: rows outside [0, h),
// columns outside [0, w)), so rows wait in shared memory rather than in
// registers.  A lane only ever reads back its own bytes, after its own
// cp.async.wait_group, so no barrier is needed.
constexpr int kRing = 8;       // row slots per warp
constexpr int kAhead = 6;      // rows in flight ahead of the one being used
// dynamic shared memory: the row rings and the staging slots (64 KB)
constexpr int kSobelSmem = kSobelWarps * (kRing * 512 + kStage * 4);
static_assert(kAhead <= kRing - 2, "a fetch must not overwrite a row still to be read");

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, int nbytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(nbytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint4 lds128(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}

// Position of the highest set bit of m (m != 0).
__device__ __forceinline__ uint32_t bfind32(uint32_t m) {
    uint32_t d;
    asm("bfind.u32 %0, %1;" : "=r"(d) : "r"(m));
    return d;
}

// 16 bytes -> 8 half pairs (p_j, p_{j+8}) in units of 2^-24.
__device__ __forceinline__ void to_halves(const uint4 q, uint32_t (&Bb)[8]) {
    const uint32_t t0 = __byte_perm(q.x, q.z, 0x5140);   // p0 p8 p1 p9
    const uint32_t t1 = __byte_perm(q.x, q.z, 0x7362);   // p2 p10 p3 p11
    const uint32_t t2 = __byte_perm(q.y, q.w, 0x5140);   // p4 p12 p5 p13
    const uint32_t t3 = __byte_perm(q.y, q.w, 0x7362);   // p6 p14 p7 p15
    Bb[0] = __byte_perm(t0, 0u, 0x4140);
    Bb[1] = __byte_perm(t0, 0u, 0x4342);
    Bb[2] = __byte_perm(t1, 0u, 0x4140);
    Bb[3] = __byte_perm(t1, 0u, 0x4342);
    Bb[4] = __byte_perm(t2, 0u, 0x4140);
    Bb[5] = __byte_perm(t2, 0u, 0x4342);
    Bb[6] = __byte_perm(t3, 0u, 0x4140);
    Bb[7] = __byte_perm(t3, 0u, 0x4342);
}

// Sliding state of a lane: the centre row M as halves, and SQ = SP of the
// previous output row, with SQm0 = SQ at (x-1) for word 0 (shifted in from
// the previous lane).
struct Window {
    uint32_t M[8], SQ[8];
    uint32_t SQm0;
};

// Advance the window by one row (the new bottom row q) and, if EMIT, return
// the edge mask of the middle row: bit i set iff pixel i of the lane's 16 is
// an edge.  All 32 lanes of the warp must call this (shuffles).
template <bool EMIT>
__device__ __forceinline__ uint32_t step(Window &S, const uint4 q, uint32_t tau) {
    uint32_t B[8], P[8], SP[8];
    to_halves(q, B);
#pragma unroll
    for (int j = 0; j < 8; ++j) P[j] = h2_add(S.M[j], B[j]);   // M + B
    const uint32_t nx = __shfl_down_sync(kFull, P[0], 1);   // next lane's pixels (16, 24)
    const uint32_t Pp7 = __byte_perm(P[0], nx, 0x5432);     // P at (8, 16): x+1 of word 7
#pragma unroll
    for (int j = 0; j < 8; ++j) SP[j] = h2_add(P[j], j < 7 ? P[j + 1] : Pp7);
    const uint32_t pv = __shfl_up_sync(kFull, SP[7], 1);    // previous lane's SP at (-9, -1)
    const uint32_t SPm0 = __byte_perm(SP[7], pv, 0x1076);   // SP at (-1, 7): x-1 of word 0
    uint32_t acc = 0;
    if (EMIT) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t u = h2_sub(SP[j], j > 0 ? S.SQ[j - 1] : S.SQm0);   // SP(x) - SQ(x-1)
            const uint32_t w = h2_sub(j > 0 ? SP[j - 1] : SPm0, S.SQ[j]);     // SP(x-1) - SQ(x)
            acc = h2_edge_acc(u, w, tau, 0x00010001u << j, acc);   // + 2^j units per edge
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        S.M[j] = B[j];
        S.SQ[j] = SP[j];
    }
    S.SQm0 = SPm0;
    return __byte_perm(acc, 0u, 0x4420);   // bits 0-7: pixels 0-7, bits 8-15: pixels 8-15
}

// 4 mask bits -> 4 bytes of 0x00 / 0xFF.
__device__ __forceinline__ uint32_t spread4(uint32_t nib) {
    return ((nib * 0x00204081u) & 0x01010101u) * 0xFFu;
}

// One run of a warp: output rows [y0, y_last) (y0 a multiple of 8) of column
// strip sx of frame F.
template <bool BIN, bool POOL>
__device__ __forceinline__ void sobel_run(const SobelLaunch &L, const SobelFrame &F, int sx, int y0, int y_last,
                                          int warp, int lane, uint8_t *smem_dyn) {
    const uint8_t *const img = F.img;
    const int w = F.w, h = F.h, pitch = F.pitch;
    const int xl = sx * kSobelStripW - 16 + 16 * lane;   // first pixel held by this lane
    const int nb_lane = xl < 0 ? 0 : min(16, max(0, w - xl));   // bytes of a row this lane reads

    // output pixels of this lane: lanes 1..30, inside the image
    uint32_t colmask = 0;
    if (lane >= 1 && lane <= 30 && nb_lane > 0) colmask = (1u << nb_lane) - 1u;
    const bool clear = L.border == LD_BORDER_CLEAR;
    if (clear) {
        if (xl == 0) colmask &= ~1u;
        const int xr = w - 1 - xl;
        if (xr >= 0 && xr < 16) colmask &= ~(1u << xr);
    }
    const uint32_t tau_u = (uint32_t)(L.threshold + 1) >> 1;   // ceil(T / 2), T in [1, 255]
    const uint32_t tau = tau_u | (tau_u << 16);                  // in units of 2^-24

    // this lane's row slots ring_s[warp][k % kRing][lane * 16]: relative row k
    // is image row y0 - 1 + k; output row y0 + 8g + r needs k = 8g + r .. + 2
    uint8_t(*ring_s)[kRing][512] = reinterpret_cast<uint8_t(*)[kRing][512]>(smem_dyn);
    uint32_t *const stage = reinterpret_cast<uint32_t *>(smem_dyn + kSobelWarps * kRing * 512) + warp * kStage;
    const uint32_t slot0 = (uint32_t)__cvta_generic_to_shared(&ring_s[warp][0][lane * 16]);
    // the next row to fetch is image row yf, at pf; rows up to y_last (the last
    // output row's lower neighbour) that lie inside the image are read, the rest
    // of the slot (and rows outside the image) is zero-filled
    const unsigned y_lim = (unsigned)min(h, y_last + 1);
    int yf = y0 - 1;
    const uint8_t *pf = img + (nb_lane > 0 ? xl : 0) + (ptrdiff_t)(y0 - 1) * pitch;
    auto fetch = [&](int slot) {
        const int nb = ((unsigned)yf < y_lim) ? nb_lane : 0;
        cp_async16(slot0 + (uint32_t)slot * 512u, nb ? pf : img, nb);
        cp_async_commit();   // one group per row, possibly empty
        ++yf;
        pf += pitch;
    };
#pragma unroll
    for (int k = 0; k < kAhead; ++k) fetch(k);

    // window primed with rows y0-1 and y0 (the first step only builds SP)
    Window S;
    cp_async_wait<kAhead - 1>();
    to_halves(lds128(slot0), S.M);
#pragma unroll
    for (int j = 0; j < 8; ++j) S.SQ[j] = 0u;
    S.SQm0 = 0u;
    fetch(kAhead % kRing);
    cp_async_wait<kAhead - 1>();
    step<false>(S, lds128(slot0 + 512u), tau);
    fetch((kAhead + 1) % kRing);

    for (int yg = y0; yg < y_last; yg += 8) {   // warp-uniform
        const int nr = y_last - yg;              // output rows in this group (1..8)
        uint32_t m2[4];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int y = yg + r;
            cp_async_wait<kAhead - 1>();
            const uint4 q = lds128(slot0 + (uint32_t)((r + 2) % kRing) * 512u);   // bottom row of y
            fetch((r + 2 + kAhead) % kRing);
            uint32_t mk = step<true>(S, q, tau) & colmask;
            if (r >= nr || (clear && (y == 0 || y == h - 1))) mk = 0;
            if (r & 1) m2[r >> 1] = __byte_perm(m2[r >> 1], mk, 0x5410); else m2[r >> 1] = mk;
            if (BIN && r < nr && lane >= 1 && lane <= 30 && xl < pitch) {
                uint4 o;
                o.x = spread4(mk & 0xF);
                o.y = spread4((mk >> 4) & 0xF);
                o.z = spread4((mk >> 8) & 0xF);
                o.w = spread4((mk >> 12) & 0xF);
                *reinterpret_cast<uint4 *>(F.bin + (size_t)y * pitch + xl) = o;
            }
        }

        // 8x8 edge counts: this lane's two blocks of the 8-row group
        if (POOL && lane >= 1 && lane <= 30) {
            uint32_t c0 = 0, c1 = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                c0 += __popc(m2[k] & 0x00FF00FFu);
                c1 += __popc(m2[k] & 0xFF00FF00u);
            }
            const int pw = (w + 7) >> 3;
            const int bx = xl >> 3;
            uint8_t *row = F.pool + (size_t)(yg >> 3) * pw;
            if (bx < pw) row[bx] = (uint8_t)c0;
            if (bx + 1 < pw) row[bx + 1] = (uint8_t)c1;
        }

        // transpose the four 32 x 32 bit matrices (word k of every lane): lane l
        // ends with bit l of each lane's word, i.e. bit s of T[k] is pixel
        // x0 + 16 s + l % 16 of row yg + 2k + l / 16, x0 = the strip's first column
        uint32_t T[4] = {m2[0], m2[1], m2[2], m2[3]};
#pragma unroll
        for (int j = 16; j >= 1; j >>= 1) {
            const uint32_t mlo = j == 16 ? 0x0000FFFFu : j == 8 ? 0x00FF00FFu : j == 4 ? 0x0F0F0F0Fu
                                 : j == 2 ? 0x33333333u : 0x55555555u;   // bit positions b with b & j == 0
            const bool up = (lane & j) == 0;
            const uint32_t keep = up ? mlo : ~mlo;
            const uint32_t rot = up ? (uint32_t)j : (uint32_t)(32 - j);   // rotate left by j / right by j
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t y = __shfl_xor_sync(kFull, T[k], j);
                T[k] = (T[k] & keep) | (__funnelshift_l(y, y, rot) & ~keep);
            }
        }

        // the group's edges: warp prefix sum, one atomic on the frame's counter
        const int cnt = __popc(T[0]) + __popc(T[1]) + __popc(T[2]) + __popc(T[3]);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        const int tot = __shfl_sync(kFull, incl, 31);
        if (tot == 0) continue;   // warp-uniform
        int base = 0;
        if (lane == 31) base = atomicAdd(F.count, tot);
        base = __shfl_sync(kFull, base, 31);
        const uint32_t b0 = ((uint32_t)(yg + (lane >> 4)) << 16) + (uint32_t)(sx * kSobelStripW - 16 + (lane & 15));
        if (tot <= kStage && (int64_t)base + tot <= F.cap) {   // warp-uniform
            uint32_t *st = stage + (incl - cnt);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t m = T[k];
                const uint32_t bk = b0 + ((uint32_t)(2 * k) << 16);
                while (m) {   // two edges per trip
                    const uint32_t sb = bfind32(m);
                    m ^= 1u << sb;
                    st[0] = bk + 16u * sb;
                    if (m) {
                        const uint32_t sc = bfind32(m);
                        m ^= 1u << sc;
                        st[1] = bk + 16u * sc;
                        st += 2;
                    } else {
                        st += 1;
                    }
                }
            }
            __syncwarp();
            uint32_t *dst = F.edges + base;
            for (int i = lane; i < tot; i += 32) dst[i] = stage[i];
            __syncwarp();
        } else {   // a group denser than the staging slots, or a list that overflows
            int64_t pos = (int64_t)base + (incl - cnt);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t m = T[k];
                const uint32_t bk = b0 + ((uint32_t)(2 * k) << 16);
                while (m) {
                    const uint32_t sb = bfind32(m);
                    m &= ~(1u << sb);
                    if (pos < F.cap) F.edges[pos] = bk + 16u * sb;
                    ++pos;
                }
            }
        }
    }
}

// Persistent warps: the launch's 8-row groups, ordered (frame, column strip,
// group), are cut into one contiguous range per warp of the grid, so every
// warp gets the same number of groups (to one) whatever the frame sizes; a
// range runs down a strip and continues in the next strip or frame.
template <bool BIN, bool POOL>
__global__ void __launch_bounds__(kSobelThreads, 3)
sobel_bin_edges_kernel(const __grid_constant__ SobelLaunch L) {
    extern __shared__ __align__(16) uint8_t smem_dyn[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * kSobelWarps, wid = (int64_t)blockIdx.x * kSobelWarps + warp;
    int64_t r = L.total_groups * wid / nw;
    const int64_t r1 = L.total_groups * (wid + 1) / nw;
    while (r < r1) {   // warp-uniform
        int lo = 0, hi = L.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (L.f[mid].group_begin <= r) lo = mid; else hi = mid - 1;
        }
        const SobelFrame &F = L.f[lo];
        const int gps = (F.h + 7) >> 3;   // groups per strip
        const int64_t local = r - F.group_begin;
        const int sx = (int)(local / gps), g = (int)(local - (int64_t)sx * gps);
        const int64_t left = r1 - r;
        const int n = left < (int64_t)(gps - g) ? (int)left : gps - g;
        if (local == 0 && lane == 0) {   // until the merge writes the frame's peaks
            if (F.status_init) *F.status_init = LD_ERR_TIMEOUT;
            if (F.npeaks_init) *F.npeaks_init = 0;
        }
        sobel_run<BIN, POOL>(L, F, sx, 8 * g, min(F.h, 8 * (g + n)), warp, lane, smem_dyn);
        r += n;
    }
}

}  // namespace

cudaError_t launch_sobel(const SobelLaunch &Lin, int n_ctas, cudaStream_t s) {
    if (n_ctas <= 0) return cudaSuccess;
    if (Lin.groups < 1 || Lin.groups > 64) return cudaErrorInvalidValue;
    SobelLaunch L = Lin;   // the launch's group ranges (n_ctas, from the run length, caps the grid)
    int64_t groups = 0;
    for (int i = 0; i < L.n; ++i) {
        L.f[i].group_begin = groups;
        groups += (int64_t)sobel_strips(L.f[i].w) * ((L.f[i].h + 7) / 8);
    }
    L.total_groups = groups;
    int dev = 0, sms = 0;
    cudaError_t e0 = cudaGetDevice(&dev);
    if (e0 == cudaSuccess) e0 = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e0 != cudaSuccess) return e0;
    const int64_t resident = (int64_t)sms * 3;                       // 3 CTAs of 8 warps per SM
    const int64_t need = (groups + kSobelWarps - 1) / kSobelWarps;   // at least one group per warp
    n_ctas = (int)std::min<int64_t>(std::min<int64_t>(need, resident), n_ctas);
    if (n_ctas <= 0) return cudaSuccess;
    // the optional outputs are uniform over a launch (all frames or none)
    const bool bin = L.f[0].bin != nullptr, pool = L.f[0].pool != nullptr;
    for (int i = 1; i < L.n; ++i)
        if ((L.f[i].bin != nullptr) != bin || (L.f[i].pool != nullptr) != pool) return cudaErrorInvalidValue;
    auto kern = bin ? (pool ? sobel_bin_edges_kernel<true, true> : sobel_bin_edges_kernel<true, false>)
                    : (pool ? sobel_bin_edges_kernel<false, true> : sobel_bin_edges_kernel<false, false>);
    static std::atomic<uint64_t> attr_done[4];   // per template instance, one bit per device
    cudaError_t e = once_per_device(attr_done[(bin ? 2 : 0) + (pool ? 1 : 0)], [&](int) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSobelSmem);
    });
    if (e != cudaSuccess) return e;
    kern<<<n_ctas, kSobelThreads, kSobelSmem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace ld
