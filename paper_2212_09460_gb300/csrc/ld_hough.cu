// ld_hough.cu -- Step 3, Hough voting r = x cos(theta) + y sin(theta)
// (Sec. 2.3 Eq. 3, Sec. 4.3), with the sin/cos symmetry of Sec. 3.3
// (Eqs. 4-5), and the per-tile candidate emission for Step 4.
//
// GB300 design.  As in the paper's GPU kernel (Sec. 4.3) every CTA owns a
// slice of the theta axis in shared memory and counts the votes of all edge
// pixels with shared-memory atomics; unlike it, a CTA owns a tile of theta
// *pairs* {k, n_theta-k} (Eqs. 4-5: sin equal, cos opposite), so one
// y*s_k product serves both angles, and the two counts of a pair share one
// 32-bit word (low half theta_k, high half theta_{n-k}).  A count never
// exceeds 2*max(w, h) <= 65528 for a list of distinct pixels (a rho strip of
// width 1 holds at most 2 pixels per row or per column), so 16 bits are
// exact and the tile holds twice as many angles.  rho comes from the integer
// Q16 table: idx = (y*s + 32768 + D*65536 +/- x*c) >> 16, computed modulo
// 2^32 (its true value lies in [0, (2D+1)*65536)).
//
// The edge list is streamed through shared memory in chunks by the bulk-copy
// engine (cp.async.bulk, completion on an mbarrier, 3 stages).  Lane l of
// every warp reads edges l*S + o with S odd, so the 32 lanes hit 32 distinct
// banks and sit far apart in the row-major list, which keeps lanes of a warp
// from voting into the same cell at once (that serialises shared atomics).
// Every mbarrier wait is bounded; a wait that gives up sets the frame's
// timeout flag and the CTA leaves after draining its own copies.
#include "ld_internal.cuh"
#include "ld_merge.cuh"
#include "ld_plan.h"
#include "ld_select.cuh"

namespace ld {
namespace {

constexpr int kRingBytes = kStages * kChunkEdges * 4;   // 30336 bytes
constexpr int kRingBytesPad = (kRingBytes + 127) / 128 * 128;
// static shared memory of the kernel (barriers, select and merge scratch)
constexpr int kStaticSmemReserve = (int)(sizeof(SelectSmem) + sizeof(MergeSmem)) + 512;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Shared-memory reduction without a returned value.
__device__ __forceinline__ void red_add_shared(uint32_t *addr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(smem_u32(addr)), "r"(v) : "memory");
}
// The same at a 32-bit shared-window address.
__device__ __forceinline__ void red_add_shared_at(uint32_t saddr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: true if the phase completed, false if it gave up after
// `limit` polls (0: at once).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit = kSpinLimit) {
    for (uint32_t it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// theta of the low / high half of pair slot p (tj: the tile's pair indices).
__device__ __forceinline__ int theta_lo(const int *tj, int p) { return tj[p]; }
__device__ __forceinline__ int theta_hi(const int *tj, int p, int n_theta) {
    const int j = tj[p];
    return j == 0 ? n_theta / 2 : n_theta - j;
}

// Ordered column q of a tile (theta ascending) -> (slot, half).
// The tile's pair indices ascend, so low halves carry ascending theta < n/2
// and high halves theta > n/2 descending in the slot, except pair 0, whose
// high half is theta = n/2.
__device__ __forceinline__ void ordered_col(int q, int np, bool has0, int &slot, int &half) {
    if (q < np) { slot = q; half = 0; return; }
    int q2 = q - np;
    half = 1;
    if (has0) slot = (q2 == 0) ? 0 : np - q2;
    else slot = np - 1 - q2;
}

// Accumulator layouts of a tile, for the candidate selection.  A tile holds
// np theta pairs (slots); each 32-bit word packs two 16-bit counts, the low
// half for theta_lo(slot) and the high half for theta_hi(slot).
//
// PairRowLayout: slot p's words are p * n_rho + rho (rho index of both halves).
struct PairRowLayout {
    int n_rho;
    // word i -> its slot and the rho index of its low / high count
    __device__ __forceinline__ void cells(int i, int &slot, int &rho_lo, int &rho_hi) const {
        slot = i / n_rho;
        rho_lo = rho_hi = i - slot * n_rho;
    }
    __device__ __forceinline__ int col_len() const { return n_rho; }   // rows of one theta column
    __device__ __forceinline__ int word(int slot, int row) const { return slot * n_rho + row; }
    __device__ __forceinline__ int rho(int slot, int half, int row) const { return row; }
};

// InterleavedLayout<W>: word row * W + slot (W = 16 or 8 slots); row r of
// slot p holds the count of theta_lo(p) at rho index r + lo[p] and of
// theta_hi(p) at r + hi[p] (each theta's rho window starts at its own minimum
// over the image).
constexpr int kCols = kHoughColPairs;   // the widest tile
template <int W>
struct InterleavedLayout {
    const int *lo, *hi;   // shared memory: rho index of row 0 per slot and half
    int rows;
    __device__ __forceinline__ void cells(int i, int &slot, int &rho_lo, int &rho_hi) const {
        slot = i % W;
        const int row = i / W;
        rho_lo = row + lo[slot];
        rho_hi = row + hi[slot];
    }
    __device__ __forceinline__ int col_len() const { return rows; }
    __device__ __forceinline__ int word(int slot, int row) const { return row * W + slot; }
    __device__ __forceinline__ int rho(int slot, int half, int row) const { return row + (half ? hi[slot] : lo[slot]); }
};

// Exact local top-M (order: votes desc, theta asc, rho asc) of a tile's
// `words` accumulator words, written as keys to out[0..M) (unused slots 0).
// Every cell of a theta column that the layout does not hold must have 0 votes
// and min_votes >= 1, or be held.  The edge ring is free and serves as scratch
// (at least 4 * blockDim.x + 8 * 2048 bytes).  Every thread calls it.
template <class Lay>
__device__ void select_tile(const HoughLaunch &L, uint64_t *out, const uint32_t *acc, int words, int np, bool has0,
                            const int *tj, const Lay &lay, SelectSmem &S, uint32_t *ring) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthr = blockDim.x, nwarps = nthr >> 5;
    const int n_theta = L.n_theta;
    const int M = L.cand_m;
    const int32_t mv = L.min_votes;

    // Fast path.  Each thread's largest count over its words (one packed
    // 16-bit max per word); L = the M-th largest of these maxima among the
    // threads whose maximum is >= min_votes.  M distinct cells have votes
    // >= L, so every top-M cell does too.  The cells with votes >= L
    // ("survivors", a few hundred at most on road frames) are compacted as
    // keys, which are unique and ordered like the peaks, and the M largest
    // keys are exactly the tile's top-M: picked by rank (up to one survivor
    // per thread) or by a descending sort.  No threshold (fewer than M
    // threads hold a cell >= min_votes) or too many survivors: the general
    // path below.
    constexpr int kMaxSurv = 2048;
    if (M <= nthr) {
        uint32_t m2 = 0u;
        for (int i = tid; i < words; i += nthr) {
            const uint32_t wv = acc[i];
            asm("max.u16x2 %0, %1, %2;" : "=r"(m2) : "r"(m2), "r"(wv));
        }
        int tmax = max((int)(m2 & 0xFFFFu), (int)(m2 >> 16));
        if (tmax < mv) tmax = -1;
        uint64_t *keys = reinterpret_cast<uint64_t *>(ring + nthr);
        if (tid == 0) S.surv = 0;
        const int Lth = block_mth_largest(tmax, M, S);
        if (Lth >= 0) {   // block-uniform
            // a word holds a survivor iff max(lo, hi) >= L, i.e. the packed
            // max with (L-1, L-1) differs from (L-1, L-1)
            const uint32_t t2 = Lth >= 1 ? (uint32_t)(Lth - 1) * 0x10001u : 0u;
            for (int i = tid; i < words; i += nthr) {
                const uint32_t wv = acc[i];
                uint32_t mx;
                asm("max.u16x2 %0, %1, %2;" : "=r"(mx) : "r"(wv), "r"(t2));
                if (Lth == 0 || mx != t2) {
                    const int32_t a = (int32_t)(wv & 0xFFFFu), b = (int32_t)(wv >> 16);
                    int p, ra, rb;
                    lay.cells(i, p, ra, rb);
                    if (a >= Lth) {
                        const int slot = atomicAdd(&S.surv, 1);
                        if (slot < kMaxSurv) keys[slot] = peak_key(a, theta_lo(tj, p), ra);
                    }
                    if (b >= Lth) {
                        const int slot = atomicAdd(&S.surv, 1);
                        if (slot < kMaxSurv) keys[slot] = peak_key(b, theta_hi(tj, p, n_theta), rb);
                    }
                }
            }
            __syncthreads();
            const int ns_ = S.surv;
            if (ns_ <= nthr) {   // block-uniform
                block_topm_by_rank(keys, ns_, M, out);
                return;
            }
            if (ns_ <= kMaxSurv) {   // block-uniform
                int n2 = 1;
                while (n2 < ns_) n2 <<= 1;
                for (int i = ns_ + tid; i < n2; i += nthr) keys[i] = 0ull;
                __syncthreads();
                block_sort_desc(keys, n2);
                for (int i = tid; i < M; i += nthr) out[i] = keys[i];
                return;
            }
        }
        __syncthreads();
    }

    // General path.  Pass 0: included count and overall maximum.
    int cnt = 0;
    int tmax = -1;
    for (int i = tid; i < words; i += nthr) {
        const uint32_t wv = acc[i];
        const int32_t a = (int32_t)(wv & 0xFFFFu), b = (int32_t)(wv >> 16);
        if (a >= mv) { ++cnt; tmax = max(tmax, a); }
        if (b >= mv) { ++cnt; tmax = max(tmax, b); }
    }
    const int total = block_sum(cnt, S);
    uint32_t vmax = tmax < 0 ? 0u : (uint32_t)tmax;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) vmax = max(vmax, __shfl_xor_sync(0xFFFFFFFFu, vmax, o));
    if (lane == 0) S.red[warp] = vmax;
    __syncthreads();
    uint32_t gmax = 0;
    for (int w = 0; w < nwarps; ++w) gmax = max(gmax, S.red[w]);
    __syncthreads();

    const bool all_in = total <= M;
    if (tid == 0) {
        S.prefix = 0x80000000u;
        S.pmask = 0xFFFF0000u;
        S.rank = M;
        S.out_n = 0;
    }
    __syncthreads();
    if (!all_in) {
        int top_shift = 0;   // highest nibble holding a set bit of the max count
        for (int s = 12; s > 0; s -= 4)
            if (gmax >> s) { top_shift = s; break; }
        for (int shift = top_shift; shift >= 0; shift -= 4) {
            uint32_t wh[16];
#pragma unroll
            for (int d = 0; d < 16; ++d) wh[d] = 0;
            const uint32_t prefix = S.prefix, pmask = S.pmask;
            for (int base = 0; base < words; base += nthr) {
                const int i = base + tid;
                const uint32_t wv = (i < words) ? acc[i] : 0u;
                const int32_t a = (int32_t)(wv & 0xFFFFu), b = (int32_t)(wv >> 16);
                const uint32_t ua = (uint32_t)a ^ 0x80000000u, ub = (uint32_t)b ^ 0x80000000u;
                ballot_digits(wh, i < words && a >= mv && (ua & pmask) == prefix, (ua >> shift) & 15u);
                ballot_digits(wh, i < words && b >= mv && (ub & pmask) == prefix, (ub >> shift) & 15u);
            }
            if (lane == 0) {
#pragma unroll
                for (int d = 0; d < 16; ++d) S.hist[warp][d] = wh[d];
            }
            select_digit(S, shift);
        }
    }
    const uint32_t ustar = S.prefix;
    const int need = all_in ? 0 : S.rank;   // cells equal to u* to take, in order
    __syncthreads();

    // ordered emission over per-thread contiguous ranges of the ordered cells
    // (theta columns ascending, rho ascending inside a column)
    const int clen = lay.col_len();
    const int64_t ncell = 2 * (int64_t)np * clen;
    const int64_t r0 = ncell * tid / nthr, r1 = ncell * (tid + 1) / nthr;
    auto cell_at = [&](int64_t li, int &theta, int &rho) -> int32_t {
        const int q = (int)(li / clen);
        const int row = (int)(li - (int64_t)q * clen);
        int slot, half;
        ordered_col(q, np, has0, slot, half);
        theta = half ? theta_hi(tj, slot, n_theta) : theta_lo(tj, slot);
        rho = lay.rho(slot, half, row);
        const uint32_t wv = acc[lay.word(slot, row)];
        return (int32_t)(half ? (wv >> 16) : (wv & 0xFFFFu));
    };
    int ties = 0;
    if (!all_in) {
        for (int64_t li = r0; li < r1; ++li) {
            int th, rh;
            const int32_t v = cell_at(li, th, rh);
            ties += (v >= mv && ((uint32_t)v ^ 0x80000000u) == ustar);
        }
    }
    // exclusive block scan of the tie counts
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
    for (int64_t li = r0; li < r1; ++li) {
        int th, rh;
        const int32_t v = cell_at(li, th, rh);
        if (v < mv) continue;
        const uint32_t u = (uint32_t)v ^ 0x80000000u;
        if (all_in || u > ustar) {
            const int slot = atomicAdd(&S.out_n, 1);
            if (slot < M) out[slot] = peak_key(v, th, rh);
        } else if (u == ustar) {
            if (trank < need) out[(M - need) + trank] = peak_key(v, th, rh);
            ++trank;
        }
    }
    __syncthreads();
    // unused slots (fewer included cells than M) are empty keys
    const int filled = all_in ? min(S.out_n, M) : M;
    for (int i = filled + tid; i < M; i += nthr) out[i] = 0ull;
}

// Votes of one edge pixel (x, y) into the tile's packed accumulator.  For
// slot p (theta pair {j, n-j}), kq[p] = 32768 + (D + p*n_rho)*65536 folds the
// Q16 rounding constant, the rho offset D and the slot's word offset, so
//   v1 = x*c + y*s + kq  and  v2 = 2*(y*s + kq) - v1 = -x*c + y*s + kq
// give, after >> 16, the accumulator word of the vote for theta_j (low half)
// and theta_{n-j} (high half) (Eqs. 3-5).  HAS0: slot 0 is the pair
// {0, n/2}, whose rho is x and y.  RAGGED: only the first np slots are used.
template <int P, bool HAS0, bool RAGGED>
__device__ __forceinline__ void vote_edge(uint32_t x, uint32_t y, const uint32_t (&cq)[P],
                                          const uint32_t (&sq)[P], const uint32_t (&kq)[P], uint32_t *acc,
                                          uint32_t D, int np) {
    if (HAS0) {   // theta = 0 (rho = x) and theta = 90 deg (rho = y)
        red_add_shared(acc + (x + D), 1u);
        red_add_shared(acc + (y + D), 0x10000u);
    }
#pragma unroll
    for (int p = HAS0 ? 1 : 0; p < P; ++p) {
        if (RAGGED && p >= np) break;
        const uint32_t A = y * sq[p] + kq[p];
        const uint32_t v1 = x * cq[p] + A;
        const uint32_t v2 = 2u * A - v1;
        red_add_shared(acc + (v1 >> 16), 1u);         // theta_j
        red_add_shared(acc + (v2 >> 16), 0x10000u);   // theta_{n-j}
    }
}

// One streamed chunk of n_c edges: lane l of warp w takes edges l*S + o for
// o = w, w + 16, ... (S odd: 32 distinct banks, lanes far apart in the list).
template <int P, bool HAS0, bool RAGGED>
__device__ __forceinline__ void vote_chunk(const uint32_t *buf, const uint32_t *gedges, int n_c, int lane,
                                           int warp, const uint32_t (&cq)[P], const uint32_t (&sq)[P],
                                           const uint32_t (&kq)[P], uint32_t *acc, uint32_t W, uint32_t H,
                                           uint32_t D, int np) {
    const int n4 = n_c & ~3;
    for (int o = warp; o < kChunkSeg; o += kHoughWarps) {
        const int idx = lane * kChunkSeg + o;
        if (idx < n_c) {
            const uint32_t e = (idx < n4) ? buf[idx] : gedges[idx];
            const uint32_t x = e & 0xFFFFu, y = e >> 16;
            if (x < W && y < H) vote_edge<P, HAS0, RAGGED>(x, y, cq, sq, kq, acc, D, np);
        }
    }
}

// One work unit: theta tile `local / n_splits` of frame F over edge range
// `local % n_splits`.  seq counts the chunks this CTA streamed before (it
// fixes the stage and phase of every mbarrier).  Returns false if a bounded
// wait gave up (the frame is flagged; the CTA must stop).
template <int PMAX>
__device__ __forceinline__ bool hough_unit(const HoughLaunch &L, const HoughFrame &F, int local, int n_tiles,
                                           uint32_t &seq, uint8_t *smem_raw, uint64_t *bars, SelectSmem &S,
                                           int &abort_flag, int *tj) {
    const int ns = F.n_splits;
    const int tile = local / ns, split = local % ns;
    const int n_theta = L.n_theta;
    // pairs of this tile: the frame's pairs (all n_theta/2, or the active-pair
    // list of a restricted vote) split as evenly as possible over its n_tiles
    // tiles, the first n_avail % n_tiles tiles taking one more (<= PMAX)
    const int n_avail = F.pair_list ? *F.pair_count : n_theta / 2;
    const int base = n_avail / n_tiles, extra = n_avail % n_tiles;
    const int np = base + (tile < extra ? 1 : 0);
    const int j0 = tile * base + min(tile, extra);
    if (threadIdx.x < PMAX) tj[threadIdx.x] = (threadIdx.x < np) ? (F.pair_list ? F.pair_list[j0 + threadIdx.x]
                                                                                 : j0 + (int)threadIdx.x)
                                                                  : 0;
    __syncthreads();
    const bool has0 = (tj[0] == 0);
    const int n_rho = F.n_rho;
    const uint32_t W = (uint32_t)F.w, H = (uint32_t)F.h;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    uint32_t *ring = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem_raw + kRingBytesPad);
    const int words = np * n_rho;

    // ---- Q16 (c, s) of the tile's pairs and their folded constants in registers
    uint32_t cq[PMAX], sq[PMAX], kq[PMAX];
#pragma unroll
    for (int p = 0; p < PMAX; ++p) {
        cq[p] = 0; sq[p] = 0; kq[p] = 0;
        if (p < np) {
            cq[p] = (uint32_t)L.trig[2 * tj[p]];
            sq[p] = (uint32_t)L.trig[2 * tj[p] + 1];
            kq[p] = 32768u + ((uint32_t)F.D + (uint32_t)(p * n_rho)) * 65536u;
        }
    }

    // ---- zero the accumulator tile
    for (int i = tid; i < words; i += kHoughThreads) acc[i] = 0u;
    __syncthreads();

    // ---- this CTA's edge range (split boundaries are multiples of 4 edges)
    int64_t E = (int64_t)*F.count;
    if (E > F.cap) E = F.cap;
    if (E < 0) E = 0;
    const int64_t e0 = (E * split / ns) & ~int64_t(3);
    const int64_t e1 = (split + 1 == ns) ? E : ((E * (split + 1) / ns) & ~int64_t(3));
    const int64_t n_chunks = (e1 > e0) ? (e1 - e0 + kChunkEdges - 1) / kChunkEdges : 0;

    auto issue = [&](int64_t c) {
        const int st = (int)((seq + (uint32_t)c) % kStages);
        const int64_t start = e0 + c * kChunkEdges;
        const int n_c = (int)((e1 - start) < kChunkEdges ? (e1 - start) : kChunkEdges);
        const int n4 = n_c & ~3;
        if (n4 > 0) {
            mbar_arrive_expect_tx(&bars[st], (uint32_t)n4 * 4u);
            bulk_g2s(ring + st * kChunkEdges, F.edges + start, (uint32_t)n4 * 4u, &bars[st]);
        } else {
            mbar_arrive(&bars[st]);
        }
    };
    if (tid == 0) {
        fence_proxy_async();   // the ring was last written by generic stores
        for (int64_t c = 0; c < n_chunks && c < kStages; ++c) issue(c);
    }

    int64_t c = 0;
    for (; c < n_chunks; ++c) {
        const uint32_t g = seq + (uint32_t)c;
        const int st = (int)(g % kStages);
        const uint32_t par = (g / kStages) & 1u;
        const bool ok = mbar_wait_bounded(&bars[st], par, L.wait_polls);
        if (!ok) abort_flag = 1;
        if (ok) {
            const uint32_t *buf = ring + st * kChunkEdges;
            const int64_t start = e0 + c * kChunkEdges;
            const int n_c = (int)((e1 - start) < kChunkEdges ? (e1 - start) : kChunkEdges);
            const uint32_t *ge = F.edges + start;
            const uint32_t D = (uint32_t)F.D;
            if (np == PMAX) {
                if (has0) vote_chunk<PMAX, true, false>(buf, ge, n_c, lane, warp, cq, sq, kq, acc, W, H, D, np);
                else vote_chunk<PMAX, false, false>(buf, ge, n_c, lane, warp, cq, sq, kq, acc, W, H, D, np);
            } else {
                if (has0) vote_chunk<PMAX, true, true>(buf, ge, n_c, lane, warp, cq, sq, kq, acc, W, H, D, np);
                else vote_chunk<PMAX, false, true>(buf, ge, n_c, lane, warp, cq, sq, kq, acc, W, H, D, np);
            }
        }
        __syncthreads();
        if (abort_flag) break;
        if (tid == 0 && c + kStages < n_chunks) {
            fence_proxy_async();
            issue(c + kStages);
        }
    }

    if (abort_flag) {
        // drain this CTA's own copies still in flight (bounded), flag the frame
        if (tid == 0) {
            for (int64_t k = c; k < n_chunks && k < c + kStages; ++k) {
                const uint32_t g = seq + (uint32_t)k;
                (void)mbar_wait_bounded(&bars[g % kStages], (g / kStages) & 1u);
            }
            if (F.flags) atomicOr(F.flags, kFlagTimeout);
        }
        return false;
    }
    seq += (uint32_t)n_chunks;
    __syncthreads();

    if (L.mode == kHoughFullAcc) {
        for (int p = 0; p < np; ++p) {
            const int ta = theta_lo(tj, p), tb = theta_hi(tj, p, n_theta);
            int32_t *ga = F.acc + (size_t)ta * n_rho;
            int32_t *gb = F.acc + (size_t)tb * n_rho;
            for (int r = tid; r < n_rho; r += kHoughThreads) {
                const uint32_t wv = acc[p * n_rho + r];
                const int32_t a = (int32_t)(wv & 0xFFFFu), b = (int32_t)(wv >> 16);
                if (ns == 1) {
                    ga[r] = a;
                    gb[r] = b;
                } else {
                    if (a) atomicAdd(ga + r, a);
                    if (b) atomicAdd(gb + r, b);
                }
            }
        }
        return true;
    }

    // ---- candidate mode: exact local top-M of this tile (see ld_select.cuh)
    select_tile(L, F.cand + (size_t)tile * L.cand_m, acc, words, np, has0, tj, PairRowLayout{n_rho}, S, ring);
    return true;
}

// Persistent voting kernel: each CTA (one per SM) takes work units from the
// launch's queue until it is empty.  In candidate mode the CTA that finishes
// the last theta tile of a frame also runs that frame's greedy peak merge
// (ld_merge.cuh), so Steps 3-4 take one launch.
template <int PMAX>
__global__ void __launch_bounds__(kHoughThreads, 1)
hough_kernel(const __grid_constant__ HoughLaunch L) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ uint64_t bars[kStages];
    __shared__ SelectSmem S;
    __shared__ MergeSmem MS;
    __shared__ int abort_flag, unit_s, last_s;
    __shared__ int tile_j[PMAX];
    const int tid = threadIdx.x;
    const int total_units = L.unit_begin_dev ? L.unit_begin_dev[L.n] : L.total_units;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();
    uint32_t seq = 0;
    for (;;) {
        if (tid == 0) unit_s = atomicAdd(L.queue, 1);
        __syncthreads();
        const int u = unit_s;
        if (u >= total_units) break;   // block-uniform
        const int32_t *ub = L.unit_begin_dev;
        int lo = 0, hi = L.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((ub ? ub[mid] : L.f[mid].unit_begin) <= u) lo = mid; else hi = mid - 1;
        }
        const HoughFrame &F = L.f[lo];
        const int begin = ub ? ub[lo] : F.unit_begin;
        const int n_tiles = ub ? ub[lo + 1] - ub[lo] : F.n_tiles;
        if (!hough_unit<PMAX>(L, F, u - begin, n_tiles, seq, smem_raw, bars, S, abort_flag, tile_j)) break;
        if (L.mode == kHoughCandidates) {
            __syncthreads();   // this tile's candidates are written
            if (tid == 0) {
                __threadfence();
                last_s = (atomicAdd(F.done, 1) == n_tiles - 1) ? 1 : 0;
            }
            __syncthreads();
            if (last_s) {   // block-uniform
                __threadfence();
                const int32_t fl = F.flags ? __ldcg(F.flags) : 0;
                block_merge(F.cand, (int64_t)n_tiles * L.cand_m, L.top_k, L.nms_theta, L.nms_rho, F.peaks,
                            F.n_peaks, F.status, fl, MS);
            }
        }
        __syncthreads();   // before unit_s is overwritten
    }
}


// ---------------------------------------------------------------- interleaved columns
//
// Second voting kernel, for the detection paths (candidate mode, min_votes
// >= 1): the full vote of ld_detect_batch and the restricted vote of the
// proposal path.
//
// Banks.  Each 32-lane red.shared of the kernel above hits 32 random words,
// which fall on about 3.5 distinct-bank wavefronts.  Here lane l of a warp
// owns slot l % 16 of a tile of up to 16 theta pairs, and the tile's words
// are interleaved (word = row * 16 + slot), so slot l lives in banks l and
// l + 16 only.  The two half-warps vote two different edges into the same 16
// slots, so one red.shared costs at most 2 wavefronts (2 when any slot's two
// rows agree in parity, i.e. almost always).
//
// Rows.  Each theta's rho window starts at its own minimum over the image
// corners, so a column needs only the frame's widest window (at most D + 1
// rows) instead of 2D + 1: 16 pairs of a 1080p frame take 141 KB.  Cells
// outside a window have no votes, which min_votes >= 1 keeps out of the peaks.
//
// Vote.  Each lane holds the (cos, sin) of both thetas of its pair, so the
// pair {0, n/2} needs no special case.  The vote has no per-edge branch (the
// kernel is issue-bound once the bank conflicts are gone): one min.u16x2
// clamps (y, x) into the image, x is folded into the multiply (e = y * 65536
// + x, so e c + y (s - 65536 c) = x c + y s mod 2^32), addresses are 32-bit
// shared-window offsets, and the lanes of unused slots vote into their own
// spare columns, which are cleared before the selection.  The clamp is a
// memory guard only: the edge lists come from the Sobel kernel, whose entries
// are always inside the image.
//
// Edges.  The edge list streams through a 2-stage ring of 8192-edge chunks
// (4096 when the accumulator leaves less room; fewer, larger chunks measured
// faster) without block barriers.  Each half-warp reads a 16-byte group of 4
// edges per loop step (a broadcast load).  The first half of each chunk goes to
// half-warp 0 and the second to half-warp 1, so the two edges voted together
// lie far apart in the row-major list (far-apart edges seldom share a cell).
//
// Pieces.  A launch whose last wave would be poorly filled, or a small launch
// with fewer tiles than SMs, splits tiles into edge-range pieces.  Their
// partial accumulators meet in global memory, and the last piece of a tile
// adds them up and selects.
constexpr int kColThreads = 1024;
constexpr int kColWarps = kColThreads / 32;
constexpr int kColStages = 2;                 // edge ring stages of L.col_chunk edges
constexpr int kColChunkMin = 4096, kColChunkMax = 8192;
constexpr int kColRingMin = kColStages * kColChunkMin * 4;   // 32 KB
static_assert(kColRingMin >= 4 * kColThreads + 8 * 2048, "ring too small for the selection scratch");

// floor(v / 65536) of a signed value
__device__ __forceinline__ int32_t floor_q16(int64_t v) {
    return (int32_t)(v >= 0 ? v / 65536 : -((-v + 65535) / 65536));
}
// Smallest floor((x c + y s + 32768) / 65536) over the image (a corner).
__device__ __forceinline__ int32_t window_min(int32_t c, int32_t s, int W, int H) {
    const int64_t xm = c < 0 ? (int64_t)(W - 1) * c : 0;
    const int64_t ym = s < 0 ? (int64_t)(H - 1) * s : 0;
    return floor_q16(xm + ym + 32768);
}
// A bounded wait (`limit` polls) that also gives up once *abort is set (by
// another warp that gave up).
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity, const volatile int *abort,
                                                   uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && *abort) return false;
    }
    return false;
}

// Ring state of a CTA of the interleaved kernel (shared memory).
struct ColRing {
    uint64_t bars[kColStages];   // full barriers (bytes landed)
    uint32_t rel[kColStages];    // warps done with a stage, counted over the kernel
    int issued_hi;               // chunks [0, issued_hi) of the current unit were issued
};

enum ColResult { kColAbort = -1, kColPiece = 0, kColTile = 1 };

// One work unit of frame F: tile `tile` of n_tiles, edge range `split` of
// ns (chunk-aligned).  The frame's pairs are all n_theta/2, or its ascending
// active-pair list (restricted vote), split evenly over its tiles (at most
// kCols pairs each).  A split tile's pieces store their partial accumulators
// in L.part (tile index split_base + tile); the last piece to finish adds
// the others' and selects.  Returns kColTile if this unit finished its tile
// (candidates written), kColPiece if another piece will, kColAbort if a
// bounded wait gave up (the frame is flagged; the CTA must stop).
template <int NC>
__device__ __forceinline__ int cols_unit(const HoughLaunch &L, const HoughFrame &F, int tile, int split,
                                         int n_tiles, int ns, int split_base, uint32_t &seq, uint8_t *smem_raw,
                                         ColRing &R, SelectSmem &S, int &abort_flag, int &last_s, int *tj,
                                         int *wlo, int *whi) {
    const int n_theta = L.n_theta, chunk = L.col_chunk;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_avail = F.pair_list ? *F.pair_count : n_theta / 2;
    const int base = n_avail / n_tiles, extra = n_avail % n_tiles;
    const int np = base + (tile < extra ? 1 : 0);   // <= NC (plan)
    const int j0 = tile * base + min(tile, extra);
    const bool has0 = (F.pair_list ? F.pair_list[j0] : j0) == 0;
    const int W = F.w, H = F.h, D = F.D, rows = F.rows;

    // per-lane constants: (c, s) and Q16 offset of both thetas of the lane's pair
    // lane -> (slot, part): NC = 16 slots: two half-warps, NC = 8: four
    // quarter-warps, each voting its own edge into all NC slots
    constexpr int kParts = 32 / NC;
    const int slot = lane % NC, half = lane / NC;
    const int j = slot < np ? (F.pair_list ? F.pair_list[j0 + slot] : j0 + slot) : 0;   // unused: a spare column
    const int32_t cl = L.trig[2 * j], sl = L.trig[2 * j + 1];
    const int32_t ch = j == 0 ? L.trig[2 * (n_theta / 2)] : -cl;
    const int32_t sh = j == 0 ? L.trig[2 * (n_theta / 2) + 1] : sl;
    const int32_t ml = window_min(cl, sl, W, H), mh = window_min(ch, sh, W, H);
    // v = x c + y s + kq; v >> 16 = floor((x c + y s + 32768) / 65536) - m, the row
    const uint32_t kql = 32768u - (uint32_t)ml * 65536u, kqh = 32768u - (uint32_t)mh * 65536u;
    // e = y * 65536 + x, so e c + y (s - 65536 c) = x c + y s (mod 2^32)
    const uint32_t sl2 = (uint32_t)sl - ((uint32_t)cl << 16), sh2 = (uint32_t)sh - ((uint32_t)ch << 16);
    const uint32_t lim = ((uint32_t)(H - 1) << 16) | (uint32_t)(W - 1);   // clamp of (y, x)
    if (warp == 0 && half == 0) {   // lanes 0 .. NC-1
        tj[slot] = j;
        wlo[slot] = ml + D;   // rho index of row 0
        whi[slot] = mh + D;
    }

    uint32_t *ring = reinterpret_cast<uint32_t *>(smem_raw);
    uint32_t *acc = reinterpret_cast<uint32_t *>(smem_raw + (size_t)kColStages * chunk * 4);
    const int words = rows * NC;
    const uint32_t acc_slot = smem_u32(acc) + (uint32_t)slot * 4u;

    // ---- zero the accumulator
    {
        uint4 *a4 = reinterpret_cast<uint4 *>(acc);
        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
        for (int i = tid; i < words / 4; i += kColThreads) a4[i] = z;   // words is a multiple of 8
    }
    __syncthreads();

    // ---- this unit's edges: range `split` of ns, boundaries at multiples of 4
    //      edges (16 bytes, for the bulk copies), streamed in chunks
    int64_t E = (int64_t)*F.count;
    if (E > F.cap) E = F.cap;
    if (E < 0) E = 0;
    const int64_t e0 = (E * split / ns) & ~int64_t(3);
    const int64_t e1 = (split + 1 == ns) ? E : ((E * (split + 1) / ns) & ~int64_t(3));
    const int n_chunks = e1 > e0 ? (int)((e1 - e0 + chunk - 1) / chunk) : 0;

    auto issue = [&](int c) {   // local chunk c: edges e0 + c * chunk ..
        const int st = (int)((seq + (uint32_t)c) % kColStages);
        const int64_t start = e0 + (int64_t)c * chunk;
        const int n_c = (int)((e1 - start) < chunk ? (e1 - start) : chunk);
        const int n4 = n_c & ~3;
        if (n4 > 0) {
            mbar_arrive_expect_tx(&R.bars[st], (uint32_t)n4 * 4u);
            bulk_g2s(ring + st * chunk, F.edges + start, (uint32_t)n4 * 4u, &R.bars[st]);
        } else {
            mbar_arrive(&R.bars[st]);
        }
    };
    if (tid == 0) {
        fence_proxy_async();   // the ring was last written by generic stores
        const int k0 = n_chunks < kColStages ? n_chunks : kColStages;
        for (int c = 0; c < k0; ++c) issue(c);
        R.issued_hi = k0;
    }

    auto vote = [&](uint32_t e) {
        uint32_t ec;
        asm("min.u16x2 %0, %1, %2;" : "=r"(ec) : "r"(e), "r"(lim));
        const uint32_t y = ec >> 16;
        const uint32_t v1 = ec * (uint32_t)cl + y * sl2 + kql;   // = x c + y s + kq
        const uint32_t v2 = ec * (uint32_t)ch + y * sh2 + kqh;
        red_add_shared_at(acc_slot + (v1 >> 16) * (NC * 4), 1u);         // theta_lo
        red_add_shared_at(acc_slot + (v2 >> 16) * (NC * 4), 0x10000u);   // theta_hi
    };

    // Warps stream the chunks without block barriers: lane 0 of each warp waits
    // for a chunk's bytes, and the last warp to finish with a ring stage (its
    // release count reaching a multiple of kColWarps; the counts only grow)
    // issues the copy of the chunk kColStages ahead into it.  Copies are issued
    // in chunk order, so the chunks issued so far are [0, R.issued_hi).
    int c = 0;
    for (; c < n_chunks; ++c) {
        const uint32_t g = seq + (uint32_t)c;
        const int st = (int)(g % kColStages);
        uint32_t ok = 1u;
        if (lane == 0)
            ok = mbar_wait_or_abort(&R.bars[st], (g / kColStages) & 1u, &abort_flag, L.wait_polls) ? 1u : 0u;
        ok = __shfl_sync(0xFFFFFFFFu, ok, 0);
        __syncwarp();   // lane 0's wait orders the chunk's bytes for the whole warp
        if (!ok) {
            if (lane == 0) atomicExch(&abort_flag, 1);
            break;
        }
        const int64_t start = e0 + (int64_t)c * chunk;
        const int n_c = (int)((e1 - start) < chunk ? (e1 - start) : chunk);
        const int n4 = n_c & ~3;
        // the chunk's 4-edge groups: part `half` of warp w takes groups
        // half + kParts (w + kColWarps i), so the parts of a warp read adjacent
        // groups (a pointer loop unrolled by four: no per-group bound test)
        const uint4 *buf4 = reinterpret_cast<const uint4 *>(ring + st * chunk);
        const uint4 *const g_end = buf4 + (n4 >> 2);
#pragma unroll 4
        for (const uint4 *gp = buf4 + half + kParts * warp; gp < g_end; gp += kParts * kColWarps) {
            const uint4 q = *gp;   // the part's 4 edges (a broadcast load)
            vote(q.x);
            vote(q.y);
            vote(q.z);
            vote(q.w);
        }
        if (warp == kColWarps - 1 && half == 0)   // the last n_c % 4 edges (the frame's last chunk)
            for (int i = n4; i < n_c; ++i) vote(F.edges[start + i]);
        __syncwarp();
        if (lane == 0) {
            __threadfence_block();   // this warp's reads of the stage come first
            const uint32_t last = (g / kColStages + 1u) * kColWarps - 1u;
            if (atomicAdd(&R.rel[st], 1u) == last && c + kColStages < n_chunks) {
                __threadfence_block();
                fence_proxy_async();
                issue(c + kColStages);
                atomicMax(&R.issued_hi, c + kColStages + 1);
            }
        }
    }
    __syncthreads();

    if (abort_flag) {
        // drain this CTA's copies that may still be in flight (bounded), flag the frame
        if (tid == 0) {
            const int hi = R.issued_hi;
            for (int k = hi - kColStages < 0 ? 0 : hi - kColStages; k < hi; ++k) {
                const uint32_t g = seq + (uint32_t)k;
                (void)mbar_wait_bounded(&R.bars[g % kColStages], (g / kColStages) & 1u);
            }
            if (F.flags) atomicOr(F.flags, kFlagTimeout);
        }
        return kColAbort;
    }
    seq += (uint32_t)n_chunks;
    if (np < NC) {   // clear the spare columns (votes of the unused slots' lanes)
        const int spare = NC - np;
        for (int i = tid; i < rows * spare; i += kColThreads) acc[(i / spare) * NC + np + i % spare] = 0u;
        __syncthreads();
    }

    if (ns > 1) {
        // a piece of a split tile: publish the partial accumulator; the last
        // piece adds the others' (each cell's total fits its 16 bits, so the
        // halves add without carries) and selects
        const size_t tile_ix = (size_t)split_base + tile;
        uint4 *mine = reinterpret_cast<uint4 *>(L.part + (tile_ix * ns + split) * L.part_stride);
        const uint4 *a4 = reinterpret_cast<const uint4 *>(acc);
        for (int i = tid; i < words / 4; i += kColThreads) mine[i] = a4[i];
        __threadfence();
        __syncthreads();
        if (tid == 0) last_s = (atomicAdd(L.tile_cnt + tile_ix, 1) == ns - 1) ? 1 : 0;
        __syncthreads();
        if (!last_s) return kColPiece;   // block-uniform
        __threadfence();
        // every 16-byte group gathers the other pieces' words in one pass (the
        // loads are independent, so their latencies overlap)
        uint4 *acc4 = reinterpret_cast<uint4 *>(acc);
        const uint4 *part4 = reinterpret_cast<const uint4 *>(L.part + tile_ix * ns * L.part_stride);
        const int stride4 = L.part_stride / 4;
        for (int i = tid; i < words / 4; i += kColThreads) {
            uint4 a = acc4[i];
#pragma unroll
            for (int o = 0; o < kMaxSplits; ++o) {
                if (o < ns && o != split) {
                    const uint4 b = __ldcg(part4 + (size_t)o * stride4 + i);
                    a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
                }
            }
            acc4[i] = a;
        }
        __syncthreads();
    }

    select_tile(L, F.cand + (size_t)tile * L.cand_m, acc, words, np, has0, tj, InterleavedLayout<NC>{wlo, whi, rows},
                S, ring);
    return kColTile;
}

__global__ void __launch_bounds__(kColThreads, 1) hough_cols_kernel(const __grid_constant__ HoughLaunch L) {
    extern __shared__ __align__(128) uint8_t smem_raw[];
    __shared__ ColRing R;
    __shared__ SelectSmem S;
    __shared__ MergeSmem MS;
    __shared__ int abort_flag, unit_s, last_s, piece_s;
    __shared__ int tile_j[kCols], win_lo[kCols], win_hi[kCols];
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < kColStages; ++s) {
            mbar_init(&R.bars[s], 1);
            R.rel[s] = 0u;
        }
        fence_mbar_init();
        abort_flag = 0;
    }
    __syncthreads();
    uint32_t seq = 0;
    const int32_t *ub = L.unit_begin_dev;   // restricted vote: device plan
    const int total_units = ub ? ub[L.n] : L.total_units;
    for (;;) {
        if (tid == 0) unit_s = atomicAdd(L.queue, 1);
        __syncthreads();
        const int u = unit_s;
        if (u >= total_units) break;   // block-uniform
        int lo = 0, hi = L.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((ub ? ub[mid] : L.f[mid].unit_begin) <= u) lo = mid; else hi = mid - 1;
        }
        const HoughFrame &F = L.f[lo];
        const int local = u - (ub ? ub[lo] : F.unit_begin);
        const int n_tiles = ub ? L.col_plan[3 * lo] : F.n_tiles;
        const int ns = ub ? L.col_plan[3 * lo + 1] : F.n_splits;
        const int sb = ub ? L.col_plan[3 * lo + 2] : F.split_base;
        const int r = F.col_width == 8
                          ? cols_unit<8>(L, F, local / ns, local % ns, n_tiles, ns, sb, seq, smem_raw, R, S,
                                         abort_flag, piece_s, tile_j, win_lo, win_hi)
                          : cols_unit<kCols>(L, F, local / ns, local % ns, n_tiles, ns, sb, seq, smem_raw, R, S,
                                             abort_flag, piece_s, tile_j, win_lo, win_hi);
        if (r == kColAbort) break;
        if (r == kColTile) {
            __syncthreads();   // this tile's candidates are written
            if (tid == 0) {
                __threadfence();
                last_s = (atomicAdd(F.done, 1) == n_tiles - 1) ? 1 : 0;
            }
            __syncthreads();
            if (last_s) {   // block-uniform
                __threadfence();
                const int32_t fl = F.flags ? __ldcg(F.flags) : 0;
                block_merge(F.cand, (int64_t)n_tiles * L.cand_m, L.top_k, L.nms_theta, L.nms_rho, F.peaks,
                            F.n_peaks, F.status, fl, MS);
            }
        }
        __syncthreads();   // before unit_s and the tile's shared arrays are overwritten
    }
}

template <int PMAX>
cudaError_t launch_p(const HoughLaunch &L, int n_ctas, size_t smem, cudaStream_t s) {
    static std::atomic<uint64_t> attr_done{0};
    const cudaError_t e = once_per_device(attr_done, [](int) {
        return cudaFuncSetAttribute(hough_kernel<PMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kSmemLimit - kStaticSmemReserve);
    });
    if (e != cudaSuccess) return e;
    hough_kernel<PMAX><<<n_ctas, kHoughThreads, smem, s>>>(L);
    return cudaGetLastError();
}

}  // namespace

int hough_max_pairs(int n_rho) {
    const int avail = kSmemLimit - kStaticSmemReserve - kRingBytesPad;
    int p = avail / (n_rho * 4);
    return p < 30 ? p : 30;   // registers: 3 per pair, 128 per thread
}

cudaError_t launch_hough(const HoughLaunch &L, int n_ctas, int pairs_max, int64_t acc_words_max,
                         cudaStream_t s) {
    if (n_ctas <= 0) return cudaSuccess;
    const size_t smem = (size_t)kRingBytesPad + (size_t)acc_words_max * 4;
    switch (hough_template_pairs(pairs_max)) {
#define LD_CASE(P) case P: return launch_p<P>(L, n_ctas, smem, s);
        LD_HOUGH_PAIR_SIZES(LD_CASE)
#undef LD_CASE
        default: return cudaErrorInvalidValue;
    }
}

int hough_cols_max_words() {
    const int avail = kSmemLimit - kStaticSmemReserve - kColRingMin;
    return avail / 4 / kCols * kCols;
}

int hough_cols_max_rows(int width) { return hough_cols_max_words() / width; }

int hough_cols_chunk(int words_max) {
    const int avail = kSmemLimit - kStaticSmemReserve - words_max * 4;
    return avail >= kColStages * kColChunkMax * 4 ? kColChunkMax : kColChunkMin;
}

cudaError_t launch_hough_cols(const HoughLaunch &L, int n_ctas, int words_max, cudaStream_t s) {
    if (n_ctas <= 0) return cudaSuccess;
    if (words_max < 1 || words_max > hough_cols_max_words() ||
        (L.col_chunk != kColChunkMin && L.col_chunk != kColChunkMax))
        return cudaErrorInvalidValue;
    for (int i = 0; i < L.n; ++i)
        if (L.f[i].col_width != 8 && L.f[i].col_width != kCols) return cudaErrorInvalidValue;
    const size_t smem = (size_t)kColStages * L.col_chunk * 4 + (size_t)words_max * 4;
    if (smem > (size_t)(kSmemLimit - kStaticSmemReserve)) return cudaErrorInvalidValue;
    static std::atomic<uint64_t> attr_done{0};
    const cudaError_t e = once_per_device(attr_done, [](int) {
        return cudaFuncSetAttribute(hough_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kSmemLimit - kStaticSmemReserve);
    });
    if (e != cudaSuccess) return e;
    hough_cols_kernel<<<n_ctas, kColThreads, smem, s>>>(L);
    return cudaGetLastError();
}

int hough_template_pairs(int pairs) {
    int best = 0;
#define LD_PICK(P) if (P >= pairs && (best == 0 || P < best)) best = P;
    LD_HOUGH_PAIR_SIZES(LD_PICK)
#undef LD_PICK
    return best;
}

}  // namespace ld
