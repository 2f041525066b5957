// Host checks of the launch-planning arithmetic (csrc/ld_plan.h), compiled
// with the host compiler alone: no GPU, no CUDA.  Each check prints a line;
// the process exits non-zero if any fails.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../paper_2212_09460_gb300/csrc/ld_plan.h"

using namespace ld;

static int failures = 0;
#define CHECK(cond)                                                      \
    do {                                                                 \
        if (!(cond)) {                                                   \
            std::printf("FAIL %s:%d: %s\n", __FILE__, __LINE__, #cond);  \
            ++failures;                                                  \
        }                                                                \
    } while (0)

// Rows by brute force: every pixel, every voted theta (the kernel's thetas:
// table k <= n/2, mirrored (-c, s) for the rest), max - min + 1 of the Q16 rho
// index; the corner argument of window_rows must give the same number.
static int rows_brute(int w, int h, int n_theta, const std::vector<int32_t> &t) {
    int64_t best = 1;
    const int half = n_theta / 2;
    for (int k = 0; k < n_theta; ++k) {
        const int kk = k <= half ? k : n_theta - k;
        const int64_t c = k <= half ? t[2 * kk] : -t[2 * kk], s = t[2 * kk + 1];
        int64_t lo = INT64_MAX, hi = INT64_MIN;
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; ++x) {
                const int64_t v = x * c + y * s + 32768;
                const int64_t r = v >= 0 ? v / 65536 : -((-v + 65535) / 65536);
                lo = std::min(lo, r);
                hi = std::max(hi, r);
            }
        best = std::max(best, hi - lo + 1);
    }
    return (int)best;
}

static PieceSplit pieces(const std::vector<int> &tiles, int64_t px_min, int slots = 152) {
    return plan_pieces(tiles.data(), (int)tiles.size(), px_min, slots);
}

int main() {
    // D = ceil(sqrt(w^2 + h^2)) at the workloads' sizes
    CHECK(rho_max_of(1920, 1080) == 2203);
    CHECK(rho_max_of(640, 480) == 800);
    CHECK(rho_max_of(1280, 720) == 1469);
    CHECK(rho_max_of(3840, 2160) == 4406);
    CHECK(rho_max_of(512, 512) == 725);
    CHECK(rho_max_of(3, 4) == 5);   // exact square: no rounding up

    // Q16 table: end points, unit circle within rounding, monotone
    for (int n : {2, 8, 180, 360, 4096}) {
        const std::vector<int32_t> t = make_trig(n);
        CHECK(t.size() == (size_t)(2 * (n / 2 + 1)));
        CHECK(t[0] == 65536 && t[1] == 0);
        CHECK(t[2 * (n / 2)] == 0 && t[2 * (n / 2) + 1] == 65536);
        for (int k = 0; k <= n / 2; ++k) {
            const int64_t c = t[2 * k], s = t[2 * k + 1];
            CHECK(std::llabs(c * c + s * s - (int64_t)65536 * 65536) <= 2 * 65536);
            if (k > 0) CHECK(c <= t[2 * k - 2] && s >= t[2 * k - 1]);
        }
    }

    // window rows: the corner formula against brute force on small frames
    for (int n : {2, 8, 30, 180}) {
        const std::vector<int32_t> t = make_trig(n);
        for (auto wh : {std::pair<int, int>{3, 3}, {17, 5}, {5, 17}, {40, 23}, {64, 64}}) {
            const int got = window_rows(wh.first, wh.second, n, t), want = rows_brute(wh.first, wh.second, n, t);
            if (got != want) std::printf("rows %dx%d n=%d: %d vs %d\n", wh.first, wh.second, n, got, want);
            CHECK(got == want);
        }
    }
    // and the large sizes: at most D + 1 rows
    for (auto wh : {std::pair<int, int>{1920, 1080}, {2560, 1440}, {3840, 2160}, {640, 480}}) {
        const int r = window_rows(wh.first, wh.second, 360, make_trig(360));
        CHECK(r >= 1 && r <= rho_max_of(wh.first, wh.second) + 1);
    }
    CHECK(window_rows(1920, 1080, 360, make_trig(360)) == 2203);

    // tile balancing: nothing to do on an empty list; 64 frames of 18 tiles
    // on 152 SMs move to 19 tiles (1216 units = 8 full waves)
    std::vector<HoughPlan> none;
    balance_tiles(none, 180, 152);
    CHECK(none.empty());
    std::vector<HoughPlan> b(64);
    for (HoughPlan &hp : b) {
        hp.n_tiles = 18;
        hp.pairs = 10;
        hp.n_rho = 4407;
    }
    balance_tiles(b, 180, 152);
    CHECK(b[0].n_tiles == 19 && b[63].n_tiles == 19 && b[0].pairs == 10);
    CHECK(wave_fill(1216, 152) == 1.0);

    // pieces (152 slots)
    PieceSplit p;
    p = pieces(std::vector<int>(64, 12), 2073600);   // 768 tiles: last wave 8 -> the last frame in eighths
    CHECK(p.split_from == 63 && p.ns == 8 && p.split_tiles == 12);
    p = pieces(std::vector<int>(13, 12), 2073600);   // 156 tiles: tail 4
    CHECK(p.split_from == 12 && p.ns == 8 && p.split_tiles == 12);
    p = pieces(std::vector<int>(60, 3), 307200);     // 180 tiles: tail 28 -> 10 frames, 5 pieces
    CHECK(p.split_from == 50 && p.ns == 5 && p.split_tiles == 30);
    p = pieces(std::vector<int>(1, 12), 2073600);    // one 1080p frame: fill the GPU
    CHECK(p.split_from == 0 && p.ns == 8 && p.split_tiles == 12);
    p = pieces(std::vector<int>(3, 12), 921600);     // three 720p frames: 36 tiles, 4 pieces
    CHECK(p.split_from == 0 && p.ns == 4 && p.split_tiles == 36);
    p = pieces(std::vector<int>(1, 6), 307200);      // one 640x480 frame: 6 tiles in eighths
    CHECK(p.split_from == 0 && p.ns == 8 && p.split_tiles == 6);
    p = pieces(std::vector<int>(1, 6), 97 * 61);     // a tiny frame: no split
    CHECK(p.ns == 1 && p.split_from == 1 && p.split_tiles == 0);
    p = pieces(std::vector<int>(152, 1), 2073600);   // exactly one wave
    CHECK(p.ns == 1);
    p = pieces(std::vector<int>(76, 3), 2073600);    // tail 76 = half: the frames' tiles exceed half the slots
    CHECK(p.ns == 1);
    p = pieces(std::vector<int>(), 2073600);         // empty launch
    CHECK(p.ns == 1 && p.split_tiles == 0);
    for (int n = 1; n <= 128; ++n)                   // pieces never exceed the slots
        for (int t : {1, 3, 12, 15, 36}) {
            const PieceSplit q = pieces(std::vector<int>(n, t), 4000000);
            CHECK(q.ns == 1 || q.split_tiles * q.ns <= 152);
            CHECK(q.ns >= 1 && q.ns <= kMaxSplits);
        }

    // two voting launches only when both parts fill the GPU
    CHECK(two_launches(168, 180, 152));
    CHECK(!two_launches(72, 864, 152));
    CHECK(!two_launches(864, 0, 152));
    // small launches vote in tiles of 8 pairs: one 640x480 frame (6 tiles of
    // 16 pairs at 180 theta), one 1080p frame (12 tiles), not a 64-frame batch
    CHECK(narrow_cols_tiles(6, 152));
    CHECK(narrow_cols_tiles(12, 152));
    CHECK(narrow_cols_tiles(76, 152));
    CHECK(!narrow_cols_tiles(77, 152));
    CHECK(!narrow_cols_tiles(768, 152));
    CHECK(!narrow_cols_tiles(0, 152));

    std::printf(failures ? "plan checks: %d FAILED\n" : "plan checks: all passed%.0d\n", failures);
    return failures ? 1 : 0;
}
