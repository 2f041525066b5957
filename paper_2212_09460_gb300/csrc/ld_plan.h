// ld_plan.h -- the host-side arithmetic of launch planning: the rho range of a
// frame (Sec. 2.3), the Q16 cos/sin table (Sec. 3.3), the rows of the
// interleaved voting accumulator, tile balancing and the split of tiles into
// edge-range pieces.  Plain C++ with no CUDA dependency (plan_pieces is also
// compiled for the device), so that it can be tested on a host without a GPU.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#if defined(__CUDACC__)
#define LD_PLAN_HD __host__ __device__
#else
#define LD_PLAN_HD
#endif

namespace ld {

// Interleaved voting kernel: theta pairs per tile (one per half-warp lane).
constexpr int kPlanColPairs = 16;
// Split pieces: at most this many per tile, and at most one per SM in all.
constexpr int kMaxSplits = 8;
// A launch with fewer tiles than SMs splits every tile (to fill the GPU) only
// when its frames have at least this many pixels: below it a tile's edge
// stream is too short to pay for a piece's partial store and merge.
constexpr int64_t kSplitFillPixels = 1 << 17;

// D = ceil(sqrt(w^2 + h^2)): every rho of a w x h frame lies in [-D, D].
inline int64_t rho_max_of(int64_t w, int64_t h) {
    const int64_t r2 = w * w + h * h;
    int64_t d = (int64_t)std::sqrt((double)r2);
    while (d * d < r2) ++d;
    while (d > 0 && (d - 1) * (d - 1) >= r2) --d;
    return d;
}

// Q16 table over k = 0..n_theta/2 (Eqs. 4-5 supply the rest on the device):
// t[2k] = round(65536 cos(k pi / n_theta)), t[2k + 1] likewise for sin.
inline std::vector<int32_t> make_trig(int n_theta) {
    std::vector<int32_t> t(2 * (n_theta / 2 + 1));
    for (int k = 0; k <= n_theta / 2; ++k) {
        const double a = (double)k * M_PI / (double)n_theta;
        t[2 * k] = (int32_t)std::llround(std::cos(a) * 65536.0);
        t[2 * k + 1] = (int32_t)std::llround(std::sin(a) * 65536.0);
    }
    return t;
}

// Rows of the interleaved voting accumulator for w x h frames: the widest
// theta window, max - min + 1 over the image of floor((x c + y s + 32768) /
// 65536), over the thetas the kernel votes ((c_k, s_k) for k <= n/2 from the
// table t, (-c_k, s_k) for n/2 < n - k < n).  The expression is linear in
// (x, y), so its extremes are at the corners.
inline int window_rows(int w, int h, int n_theta, const std::vector<int32_t> &t) {
    const int half = n_theta / 2;
    auto fl = [](int64_t v) { return v >= 0 ? v / 65536 : -((-v + 65535) / 65536); };
    int64_t rows = 1;
    for (int k = 0; k < n_theta; ++k) {
        const int kk = k <= half ? k : n_theta - k;
        const int64_t c = k <= half ? t[2 * kk] : -t[2 * kk];
        const int64_t s = t[2 * kk + 1];
        const int64_t xlo = c < 0 ? (w - 1) * c : 0, xhi = c < 0 ? 0 : (w - 1) * c;
        const int64_t ylo = s < 0 ? (h - 1) * s : 0, yhi = s < 0 ? 0 : (h - 1) * s;
        rows = std::max(rows, fl(xhi + yhi + 32768) - fl(xlo + ylo + 32768) + 1);
    }
    return (int)std::min<int64_t>(rows, 1 << 30);
}

struct HoughPlan {
    int n_rho = 0, D = 0, pairs = 0, n_tiles = 0;
    bool cols = false;   // interleaved-column kernel (tiles of <= width pairs)
    int rows = 0;        // its accumulator rows
    int width = kPlanColPairs;   // its slots per tile: 16, or 8 when 16 x rows does not fit
};

// Fraction of the persistent CTAs' slots that `units` equal work units fill.
inline double wave_fill(int64_t units, int num_sms) {
    const int64_t waves = (units + num_sms - 1) / num_sms;
    return waves > 0 ? (double)units / (double)(waves * num_sms) : 1.0;
}

// For a launch group whose frames share one packed-pair plan: the tile count
// in [T, 1.25 T] (and at least 2 pairs per tile) whose units fill the last
// wave of the persistent launch best; more tiles only when that gains > 2% of
// fill.  Plans that differ, or an empty list, are left as they are.
inline void balance_tiles(std::vector<HoughPlan> &plans, int n_pairs, int num_sms) {
    const int gn = (int)plans.size();
    if (gn == 0) return;
    for (int k = 1; k < gn; ++k)
        if (plans[k].n_tiles != plans[0].n_tiles || plans[k].n_rho != plans[0].n_rho) return;
    const int T0 = plans[0].n_tiles;
    if ((int64_t)gn * T0 < num_sms) return;
    int best = T0;
    double best_fill = wave_fill((int64_t)gn * T0, num_sms);
    for (int T = T0 + 1; T <= T0 + (T0 + 3) / 4 && 2 * T <= n_pairs; ++T) {
        const double f = wave_fill((int64_t)gn * T, num_sms);
        if (f > best_fill + 0.02) {
            best = T;
            best_fill = f;
        }
    }
    if (best == T0) return;
    for (HoughPlan &hp : plans) {
        hp.n_tiles = best;
        hp.pairs = (n_pairs + best - 1) / best;
    }
}

// Split of an interleaved-kernel launch's tiles into edge-range pieces:
// frames at queue positions >= split_from have each tile in ns pieces
// (split_tiles tiles in all); ns == 1: no split.
struct PieceSplit {
    int split_from, ns, split_tiles;
};

// tiles[q]: tiles of the frame at queue position q (n frames); px_min: the
// fewest pixels of a frame; slots: persistent CTAs.  When the launch's last
// wave would be at most half full, the tiles of the last frames (together at
// least that wave's tiles) split into min(kMaxSplits, slots / their tiles)
// pieces, which spread over the wave.  A launch with fewer tiles than slots
// splits every tile into min(kMaxSplits, slots / tiles) pieces if px_min >=
// kSplitFillPixels (latency of small batches).  Splits into fewer than 2
// pieces are not made.  Pieces never exceed slots.
LD_PLAN_HD inline PieceSplit plan_pieces(const int *tiles, int n, int64_t px_min, int slots) {
    PieceSplit r{n, 1, 0};
    int u0 = 0;
    for (int q = 0; q < n; ++q) u0 += tiles[q];
    if (n <= 0 || u0 <= 0 || slots <= 0) return r;
    const int tail = u0 % slots;
    if (u0 < slots && px_min >= kSplitFillPixels) {
        const int ns = slots / u0 < kMaxSplits ? slots / u0 : kMaxSplits;
        if (ns >= 2) r = PieceSplit{0, ns, u0};
    } else if (u0 > slots && tail > 0 && 2 * tail <= slots) {
        int q = n, units = 0;
        while (q > 0 && units < tail) units += tiles[--q];
        const int ns = slots / units < kMaxSplits ? slots / units : kMaxSplits;
        if (ns >= 2) r = PieceSplit{q, ns, units};
    }
    return r;
}

// A launch whose interleaved-kernel tiles of 16 pairs would occupy at most
// half the SMs (small batches: latency) votes in tiles of 8 pairs instead:
// twice the tiles, so the per-tile work (clearing, selection, the merge of a
// split tile's pieces) runs on twice the SMs.
inline bool narrow_cols_tiles(int tiles16, int slots) { return tiles16 > 0 && 2 * tiles16 <= slots; }

// A launch group with tiles_c interleaved-kernel tiles and tiles_p
// packed-pair tiles votes in two launches only if each part fills the slots.
inline bool two_launches(int tiles_c, int tiles_p, int slots) {
    return tiles_c >= slots && tiles_p >= slots && tiles_c > 0 && tiles_p > 0;
}

}  // namespace ld
