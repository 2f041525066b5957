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
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: true if the phase completed, false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < kSpinLimit; ++it)
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
        const bool ok = mbar_wait_bounded(&bars[st], par);
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
    const int M = L.cand_m;
    const int32_t mv = L.min_votes;
    uint64_t *out = F.cand + (size_t)tile * M;

    // pass 0: included count, per-thread maximum, overall maximum
    int cnt = 0;
    int tmax = -1;
    for (int i = tid; i < words; i += kHoughThreads) {
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
    for (int w = 0; w < kHoughWarps; ++w) gmax = max(gmax, S.red[w]);
    __syncthreads();

    // Fast path.  L = the M-th largest of the per-thread maxima: M distinct
    // cells have votes >= L, so every top-M cell does too.  The cells with
    // votes >= L ("survivors", usually a few hundred) are compacted as keys,
    // which are unique and ordered like the peaks, and the first M keys of
    // their descending sort are exactly the tile's top-M.  The edge ring is
    // free now and holds the scratch.  Too many survivors: the general path.
    constexpr int kMaxSurv = 2048;
    if (total > M && M <= kHoughThreads) {
        int *tm = reinterpret_cast<int *>(ring);
        uint64_t *keys = reinterpret_cast<uint64_t *>(ring + kHoughThreads);
        tm[tid] = tmax;
        if (tid == 0) S.surv = 0;
        __syncthreads();
        block_sort_desc(tm, kHoughThreads);
        const int Lth = tm[M - 1];
        if (Lth >= 0) {   // block-uniform
            for (int i = tid; i < words; i += kHoughThreads) {
                const uint32_t wv = acc[i];
                const int32_t a = (int32_t)(wv & 0xFFFFu), b = (int32_t)(wv >> 16);
                if (a >= Lth || b >= Lth) {
                    const int p = i / n_rho, r = i - p * n_rho;
                    if (a >= Lth) {
                        const int slot = atomicAdd(&S.surv, 1);
                        if (slot < kMaxSurv) keys[slot] = peak_key(a, theta_lo(tj, p), r);
                    }
                    if (b >= Lth) {
                        const int slot = atomicAdd(&S.surv, 1);
                        if (slot < kMaxSurv) keys[slot] = peak_key(b, theta_hi(tj, p, n_theta), r);
                    }
                }
            }
            __syncthreads();
            const int ns_ = S.surv;
            if (ns_ <= kMaxSurv) {   // block-uniform
                int n2 = 1;
                while (n2 < ns_) n2 <<= 1;
                for (int i = ns_ + tid; i < n2; i += kHoughThreads) keys[i] = 0ull;
                __syncthreads();
                block_sort_desc(keys, n2);
                for (int i = tid; i < M; i += kHoughThreads) out[i] = keys[i];
                return true;
            }
        }
        __syncthreads();
    }

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
            for (int base = 0; base < words; base += kHoughThreads) {
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
    const int64_t ncell = 2 * (int64_t)words;
    const int64_t r0 = ncell * tid / kHoughThreads, r1 = ncell * (tid + 1) / kHoughThreads;
    auto cell_at = [&](int64_t li, int &theta, int &rho) -> int32_t {
        const int q = (int)(li / n_rho);
        rho = (int)(li - (int64_t)q * n_rho);
        int slot, half;
        ordered_col(q, np, has0, slot, half);
        theta = half ? theta_hi(tj, slot, n_theta) : theta_lo(tj, slot);
        const uint32_t wv = acc[slot * n_rho + rho];
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
    for (int i = filled + tid; i < M; i += kHoughThreads) out[i] = 0ull;
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

template <int PMAX>
cudaError_t launch_p(const HoughLaunch &L, int n_ctas, size_t smem, cudaStream_t s) {
    static uint64_t attr_set = 0;   // devices 0..63 whose attribute is set
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !(attr_set >> dev & 1u)) {
        e = cudaFuncSetAttribute(hough_kernel<PMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemLimit - kStaticSmemReserve);
        if (e != cudaSuccess) return e;
        if (dev < 64) attr_set |= uint64_t(1) << dev;
    }
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

int hough_template_pairs(int pairs) {
    int best = 0;
#define LD_PICK(P) if (P >= pairs && (best == 0 || P < best)) best = P;
    LD_HOUGH_PAIR_SIZES(LD_PICK)
#undef LD_PICK
    return best;
}

}  // namespace ld
